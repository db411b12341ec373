// batch_kernel.cuh — the persistent batch kernel (device code). Included by
// mprk_kernels.cu only: the FP64 tile body is a non-inlined template, and
// a translation unit compiles its own copy of each instantiation it uses.
// With the batch kernel in the same unit as the single-instance stage
// kernel, both call one compiled copy, so an instance gives bitwise the
// same result alone and in a batch (two copies were seen to contract
// floating-point operations differently with the general bases).
//
// Work items (instance, stage, a run of consecutive tiles) are listed
// stage-major; see mprk_batch.cu for the list, the dependencies and the
// bounded waits.
#pragma once

#include <cuda/atomic>

#include "batch_types.h"
#include "stage_tile.cuh"
#include "stage_tile_mixed.cuh"

namespace mprk {

__device__ __forceinline__ bool wait_for(const BatchArgs& A, int ctr, int need) {
  // one thread waits with acquire semantics; returns false after an abort or timeout
  cuda::atomic_ref<int, cuda::thread_scope_device> c(A.counters[ctr]);
  cuda::atomic_ref<int, cuda::thread_scope_device> ab(*A.abort_flag);
  const long long t0 = clock64();
  while (c.load(cuda::memory_order_acquire) < need) {
    if (ab.load(cuda::memory_order_relaxed)) return false;
    if (clock64() - t0 > A.wait_cycles) {
      atomicOr(A.status, ST_TIMEOUT);
      ab.store(1, cuda::memory_order_relaxed);
      return false;
    }
    __nanosleep(256);
  }
  return true;
}

__device__ __forceinline__ void finalize_chunk(const Geom& g, const Bufs& b, int chunk) {
  const int m_odd = g.m & 1;
  const bool mixed = b.dA != nullptr;
  const int rows = (m_odd || mixed) ? g.nz : g.n1_r;
  const long long per_c = (long long)rows * g.nx;  // elements of one component (< 2^31)
  const long long total = 4LL * per_c;
  for (long long e = (long long)chunk * FIN_CHUNK + threadIdx.x; e < total && e < (long long)(chunk + 1) * FIN_CHUNK;
       e += blockDim.x) {
    const int c = (e >= per_c) + (e >= 2 * per_c) + (e >= 3 * per_c);
    const int rem = (int)(e - c * per_c);
    const int k = rem / g.nx, i = rem - k * g.nx;
    const size_t o = ((size_t)c * g.nz + k) * g.pitch + i;
    double v;
    if (k < g.nS_r) v = b.accS[((size_t)c * g.nS_r + k) * g.pitch + i];
    else if (k < g.n1_r) v = b.accB[((size_t)c * (g.n1_r - g.nS_r) + (k - g.nS_r)) * g.pitch + i];
    else v = m_odd ? b.qB[o] : b.qA[o];
    if (k < g.n1_r || m_odd) b.qA[o] = v;  // F rows after an even m hold q_{n+1} already
    if (mixed) b.dA[o] = narrow(v - (double)b.rowc[4 * k + c]);
  }
}

// The FP32-flux tile of a work item, compiled as a function of its own: the
// tile reads its arguments from shared memory (not from the constant bank
// as the single-instance kernel does), and allocated apart from the
// persistent loop it spills less than inlined there.
template <int PAR>
__device__ __noinline__ void batch_tile_mixed(const StageArgs& a, int tile, MixedTileSmem& S) {
  stage_tile_mixed<PAR>(a, tile, S);
}

// three CTAs per SM in both precisions (80 and 72 registers; the FP32-flux
// form spills some, and still runs faster than at two CTAs). ROWS: rows of
// the FP64 tile, TZ (one thread per cell) or TZ / 2 (two threads per cell);
// the block size stays the same.
template <int PREC, int ROWS = TZ>
__global__ void __launch_bounds__(batch_threads(PREC), 3) batch_kernel(const BatchArgs A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the current and the next claimed item: thread 0 claims the next one
  // while the CTA works on the current, so the atomic's latency is hidden.
  // Items depend only on items before them in the list, and each CTA runs
  // its claims in order, so claiming ahead cannot deadlock.
  __shared__ int s_item[2];
  __shared__ int s_ok;
  // the item's stage arguments, one copy for the CTA: the tile reads its
  // launch constants from shared memory instead of a per-thread local copy
  __shared__ __align__(16) StageArgs s_a;
  cuda::atomic_ref<int, cuda::thread_scope_device> nxt(*A.next);
  if (threadIdx.x == 0) s_item[0] = nxt.fetch_add(1, cuda::memory_order_relaxed);
  __syncthreads();
  for (int cur = 0;; cur ^= 1) {
    const int it = s_item[cur];
    if (it >= A.n_items) break;
    const BatchItem item = A.items[it];
    const BatchInst& I = A.insts[item.inst];
    const bool stage_item = item.stage < I.g.s * I.g.m;
    if (threadIdx.x == 0) {
      s_item[cur ^ 1] = nxt.fetch_add(1, cuda::memory_order_relaxed);
      s_ok = 1;
      if (item.need > 0) s_ok = wait_for(A, I.counter_base + item.stage - 1, item.need) ? 1 : 0;
      else if (*(volatile int*)A.abort_flag) s_ok = 0;
      if (!s_ok) atomicOr(I.status, ST_TIMEOUT);  // this instance's step is incomplete
    } else if (stage_item && (int)threadIdx.x <= ARGS_WORDS) {
      // meanwhile the next threads copy the stage's arguments
      const int w = threadIdx.x - 1;
      reinterpret_cast<int4*>(&s_a)[w] = reinterpret_cast<const int4*>(A.args + I.args_base + item.stage)[w];
    }
    __syncthreads();
    if (s_ok) {
      if (stage_item) {
        for (int t = 0; t < item.count; t++) {
          if (t > 0) __syncthreads();  // the previous tile is done with shared memory
          if (PREC == 0 && s_a.g.gen)  // a general s-stage base (RK3, RK4)
            stage_tile<double, double, true, NTHREADS, ROWS>(s_a, item.tile + t,
                                                             *reinterpret_cast<TileSmem<double, ROWS>*>(smem_raw));
          else if (PREC == 0)
            stage_tile<double, double, false, NTHREADS, ROWS>(s_a, item.tile + t,
                                                              *reinterpret_cast<TileSmem<double, ROWS>*>(smem_raw));
          else if (s_a.stage & 1)  // the FP32-flux tile compiled per stage parity
            batch_tile_mixed<1>(s_a, item.tile + t, *reinterpret_cast<MixedTileSmem*>(smem_raw));
          else
            batch_tile_mixed<0>(s_a, item.tile + t, *reinterpret_cast<MixedTileSmem*>(smem_raw));
        }
      } else {
        for (int t = 0; t < item.count; t++) finalize_chunk(I.g, I.b, item.tile + t);
      }
    }
    __syncthreads();  // the tile's writes are done; shared memory is free again
    if (threadIdx.x == 0 && s_ok &&
        !(item.inst == A.withhold_inst && item.stage == A.withhold_stage)) {
      cuda::atomic_ref<int, cuda::thread_scope_device> c(A.counters[I.counter_base + item.stage]);
      c.fetch_add(1, cuda::memory_order_release);
    }
  }
}

// ---- the per-stage form ----------------------------------------------------
// One launch per stage index covers every instance that has that stage: one
// CTA per (stage arguments, tile) pair of the launch's work list. Stream
// order between the launches takes the place of the persistent kernel's
// waits. With no persistent loop around it, the FP32-flux tile fits its
// registers without spilling while it reads its arguments from the table in
// global memory.
// single >= 0: every CTA of the launch takes stage arguments `single` and
// tile blockIdx.x (a launch over one instance: no work-list load).
template <int PAR>
__global__ void __launch_bounds__(MIXED_THREADS, 3)
    wave_stage_mixed(const StageArgs* __restrict__ tab, const StageWork* __restrict__ work, int single) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const StageWork w = single >= 0 ? StageWork{single, (int)blockIdx.x} : work[blockIdx.x];
  const StageArgs& a = tab[w.args];
  const int tzi = w.tile / a.tiles_x, txi = w.tile - tzi * a.tiles_x;
  (void)stage_tile_mixed<PAR>(a, a.row0 + tzi * MTZ, txi * TX, *reinterpret_cast<MixedTileSmem*>(smem_raw),
                              nullptr, nullptr);
}

// Step completion of rows r0 .. r0 + fin_rows(nx) - 1 of component c of one
// 2-D instance (the rows the single-instance completion covers): q_{n+1}
// of S and B rows (and of F rows after an odd m) into the state buffer,
// and in FP32-flux mode the float shadow of every row. The threads walk the
// rows' cells two at a time, with 16-byte accesses where the buffers allow.
__device__ __forceinline__ int fin_rows(int nx) { return max(1, FIN_CHUNK / nx); }
__device__ __forceinline__ void finalize_rows(const Geom& g, const Bufs& b, int c, int r0) {
  const bool m_odd = g.m & 1;
  const bool mixed = b.dA != nullptr;
  const int k_hi = min(r0 + fin_rows(g.nx), (m_odd || mixed) ? g.nz : g.n1_r);
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool vec = (g.pitch % 2 == 0) && a16(b.qA) && a16(b.qB) && a16(b.accS) && a16(b.accB) &&
                   (!mixed || (reinterpret_cast<uintptr_t>(b.dA) & 7u) == 0);
  const int hx = (g.nx + 1) / 2;  // cell pairs per row
  for (int e = threadIdx.x; e < (k_hi - r0) * hx; e += blockDim.x) {
    const int k = r0 + e / hx, i = 2 * (e - (k - r0) * hx);
    const size_t o = ((size_t)c * g.nz + k) * g.pitch;
    const double* src;
    if (k < g.nS_r) src = b.accS + ((size_t)c * g.nS_r + k) * g.pitch;
    else if (k < g.n1_r) src = b.accB + ((size_t)c * (g.n1_r - g.nS_r) + (k - g.nS_r)) * g.pitch;
    else src = (m_odd ? b.qB : b.qA) + o;
    const bool store_q = k < g.n1_r || m_odd;
    const double ref = mixed ? (double)b.rowc[4 * k + c] : 0.0;
    if (vec && i + 1 < g.nx) {
      const double2 v = *reinterpret_cast<const double2*>(src + i);
      if (store_q) *reinterpret_cast<double2*>(b.qA + o + i) = v;
      if (mixed) *reinterpret_cast<float2*>(b.dA + o + i) = make_float2(narrow(v.x - ref), narrow(v.y - ref));
    } else {
      for (int j = i; j < i + 2 && j < g.nx; j++) {
        const double v = src[j];
        if (store_q) b.qA[o + j] = v;
        if (mixed) b.dA[o + j] = narrow(v - ref);
      }
    }
  }
}

// The step completions of the per-stage form: one CTA per (instance, band of
// rows of one component); tile = 4 r0 + c.
__global__ void __launch_bounds__(NTHREADS) wave_finalize(const BatchInst* __restrict__ insts,
                                                          const StageWork* __restrict__ work) {
  const StageWork w = work[blockIdx.x];
  const BatchInst& I = insts[w.args];
  finalize_rows(I.g, I.b, w.tile & 3, w.tile >> 2);
}

}  // namespace mprk
