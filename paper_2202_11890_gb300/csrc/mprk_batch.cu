// mprk_batch.cu — many independent instances advanced together: one
// persistent launch per slow step covers every instance's stage tiles and
// step completions (mprk_step_batch).
//
// Work items (instance, stage, tile) are listed stage-major: all first-stage
// tiles of all instances, then all second-stage tiles, and so on, with each
// instance's completion items after its last stage. CTAs take items in list
// order from one atomic counter. An item of stage s of instance I first waits
// until every tile of stage s-1 of I has finished (a per-instance counter).
// Since items are taken in list order, every item an item waits on was taken
// earlier by a CTA that is already running, so the waits always end. Waits
// are bounded all the same: after a fixed number of clock cycles a CTA sets
// the status word's timeout bit and an abort flag, and every CTA then drains
// without touching the states (no trap, no hang).
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mprk.h"
#include "mprk_internal.h"
#include "stage_tile.cuh"
#include "stage_tile_mixed.cuh"

namespace mprk {

struct BatchInst {
  Geom g;
  Bufs b;
  unsigned* status;  // the instance's status word
  int counter_base;  // first counter of this instance: one per stage, then completion
  int precision;
};

struct BatchItem {
  int inst;
  int stage;  // 0 .. 2m-1, or 2m for a completion item
  int tile;   // first tile of the stage, or first chunk of the completion
  int count;  // consecutive tiles (chunks) the item covers
  int need;   // items of the previous stage this one waits for (0: none)
};

// Tiles per work item. An FP32-flux tile takes a few microseconds, about
// what an item's scheduling costs (counter, wait, barriers, argument copy),
// so four tiles share one item; FP64 tiles take an item each.
constexpr int batch_group(int prec) { return prec == 0 ? 2 : 8; }

struct BatchArgs {
  const BatchInst* insts;
  const BatchItem* items;
  int n_items;
  int* next;           // work counter
  int* counters;       // per-instance stage completion counters
  int* abort_flag;
  unsigned* status;
  long long wait_cycles;
  int withhold_inst;   // test hook: this instance's withhold_stage tiles never report done
  int withhold_stage;
};

constexpr int FIN_CHUNK = NTHREADS * 8;  // cells per completion item

// block size of the batch kernel per precision (the tile's own block size)
constexpr int batch_threads(int prec) { return prec == 0 ? NTHREADS : MIXED_THREADS; }

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
  const long long total = 4LL * rows * g.nx;
  for (long long e = (long long)chunk * FIN_CHUNK + threadIdx.x; e < total && e < (long long)(chunk + 1) * FIN_CHUNK;
       e += blockDim.x) {
    const int c = (int)(e / ((long long)rows * g.nx));
    const int rem = (int)(e - (long long)c * rows * g.nx);
    const int k = rem / g.nx, i = rem - k * g.nx;
    const size_t o = ((size_t)c * g.nz + k) * g.pitch + i;
    double v;
    if (k < g.nS_r) v = b.accS[((size_t)c * g.nS_r + k) * g.pitch + i];
    else if (k < g.n1_r) v = b.accB[((size_t)c * (g.n1_r - g.nS_r) + (k - g.nS_r)) * g.pitch + i];
    else v = m_odd ? b.qB[o] : b.qA[o];
    b.qA[o] = v;
    if (mixed) b.dA[o] = narrow(v - (double)b.rowc[4 * k + c]);
  }
}

// three CTAs per SM in both precisions (80 and 72 registers; the FP32-flux
// form spills some, and still runs faster than at two CTAs)
template <int PREC>
__global__ void __launch_bounds__(batch_threads(PREC), 3) batch_kernel(const BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ int s_ok;
  // the item's stage arguments, one copy for the CTA: the tile reads its
  // launch constants from shared memory instead of a per-thread local copy
  __shared__ StageArgs s_a;
  cuda::atomic_ref<int, cuda::thread_scope_device> nxt(*A.next);
  for (;;) {
    if (threadIdx.x == 0) s_item = nxt.fetch_add(1, cuda::memory_order_relaxed);
    __syncthreads();
    const int it = s_item;
    if (it >= A.n_items) break;
    const BatchItem item = A.items[it];
    const BatchInst& I = A.insts[item.inst];
    if (threadIdx.x == 0) {
      s_ok = 1;
      if (item.need > 0) s_ok = wait_for(A, I.counter_base + item.stage - 1, item.need) ? 1 : 0;
      else if (*(volatile int*)A.abort_flag) s_ok = 0;
      if (!s_ok) atomicOr(I.status, ST_TIMEOUT);  // this instance's step is incomplete
      else if (item.stage < 2 * I.g.m) s_a = stage_args(I.g, I.b, item.stage);
    }
    __syncthreads();
    if (s_ok) {
      if (item.stage < 2 * I.g.m) {
        for (int t = 0; t < item.count; t++) {
          if (t > 0) __syncthreads();  // the previous tile is done with shared memory
          if (PREC == 0)
            stage_tile<double, double>(s_a, item.tile + t, *reinterpret_cast<TileSmem<double>*>(smem_raw));
          else
            stage_tile_mixed(s_a, item.tile + t, *reinterpret_cast<MixedTileSmem*>(smem_raw));
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

}  // namespace mprk

using namespace mprk;

// ---------------------------------------------------------------------------
// Host side: a plan per set of instances (cached), captured in a CUDA graph.
// ---------------------------------------------------------------------------
namespace {

struct Plan {
  std::vector<const void*> key;
  int precision = 0;
  int n_items = 0;
  int n_counters = 0;
  int grid = 0;
  long long cell_stages = 0;
  BatchInst* d_insts = nullptr;
  BatchItem* d_items = nullptr;
  int* d_ctr = nullptr;  // [0] next, [1] abort, [2..] counters
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  long long wait_cycles = 0;
  int withhold_inst = -1, withhold_stage = -1;
};

std::mutex g_batch_mu;
std::vector<Plan*> g_plans;

int bfail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

void free_plan(Plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  cudaFree(p->d_insts);
  cudaFree(p->d_items);
  cudaFree(p->d_ctr);
  delete p;
}

}  // namespace


namespace {

// The stage-major work list: all first-stage items of all instances, then
// all second-stage items, ...; each instance's completion items follow its
// last stage. Items group batch_group(precision) consecutive tiles.
void build_items(const std::vector<BatchInst>& hinst, int precision, std::vector<BatchItem>& items,
                 long long* cell_stages) {
  const int G = batch_group(precision);
  int max_stages = 0;
  for (const BatchInst& bi : hinst) max_stages = std::max(max_stages, 2 * bi.g.m);
  long long cs = 0;
  items.clear();
  for (int st = 0; st <= max_stages; st++) {
    for (int j = 0; j < (int)hinst.size(); j++) {
      const Geom& g = hinst[j].g;
      const int ms = 2 * g.m;
      if (st > ms) continue;
      auto ntiles = [&](int s) {
        if (s < ms) return stage_tiles(stage_args(g, hinst[j].b, s));
        const int rows = ((g.m & 1) || hinst[j].b.dA) ? g.nz : g.n1_r;
        const long long total = 4LL * rows * g.nx;
        return (int)((total + FIN_CHUNK - 1) / FIN_CHUNK);
      };
      const int nt = ntiles(st);
      const int need = st == 0 ? 0 : (ntiles(st - 1) + G - 1) / G;
      for (int t = 0; t < nt; t += G) items.push_back({j, st, t, std::min(G, nt - t), need});
      if (st < ms) cs += (long long)(g.nz - stage_args(g, hinst[j].b, st).row0) * g.nx;
    }
  }
  *cell_stages = cs;
}

int build_plan(mprk_instance* const* insts, int count, long long wait_cycles, int wi, int ws,
               cudaStream_t stream, Plan** out) {
  Plan* p = new Plan();
  p->wait_cycles = wait_cycles;
  p->withhold_inst = wi;
  p->withhold_stage = ws;
  std::vector<BatchInst> hinst(count);
  unsigned* status = nullptr;
  for (int j = 0; j < count; j++) {
    cudaStream_t s;
    unsigned* st;
    int prec;
    int rc = instance_view(insts[j], &hinst[j].g, &hinst[j].b, &prec, &s, &st);
    if (rc) { free_plan(p); return rc; }
    if (hinst[j].g.ny > 1 || hinst[j].g.gen) {
      free_plan(p);
      return bfail(MPRK_EINVAL, "batches take 2-D instances with the Heun base only");
    }
    hinst[j].status = st;
    if (j == 0) {
      p->precision = prec;
      p->stream = stream ? stream : s;
      status = st;
    } else if (prec != p->precision) {
      free_plan(p);
      return bfail(MPRK_EINVAL, "all instances of a batch need the same precision");
    }
    hinst[j].precision = prec;
    hinst[j].counter_base = p->n_counters;
    p->n_counters += 2 * hinst[j].g.m + 1;
    p->key.push_back(insts[j]);
  }
  std::vector<BatchItem> items;
  build_items(hinst, p->precision, items, &p->cell_stages);
  p->n_items = (int)items.size();
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_insts, sizeof(BatchInst) * count)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_items, sizeof(BatchItem) * items.size())) != cudaSuccess ||
      (e = cudaMalloc(&p->d_ctr, sizeof(int) * (2 + p->n_counters))) != cudaSuccess) {
    free_plan(p);
    return bfail(MPRK_ENOMEM, std::string("batch plan allocation: ") + cudaGetErrorString(e));
  }
  cudaMemcpy(p->d_insts, hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(p->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  // grid: every CTA resident (persistent kernel)
  const size_t smem = stage_smem_bytes(p->precision);
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // dynamic shared memory above 48 KB needs the kernel attribute first
  if (p->precision == 0) {
    e = cudaFuncSetAttribute(batch_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<0>, batch_threads(0), smem);
  } else {
    e = cudaFuncSetAttribute(batch_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<1>, batch_threads(1), smem);
  }
  if (e != cudaSuccess || per_sm < 1) {
    free_plan(p);
    return bfail(MPRK_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e) + ", " +
                                 std::to_string(per_sm) + " blocks per SM");
  }
  p->grid = std::min(per_sm * sms, p->n_items);
  // capture: reset the counters, then the persistent launch
  BatchArgs A;
  A.insts = p->d_insts;
  A.items = p->d_items;
  A.n_items = p->n_items;
  A.next = p->d_ctr;
  A.abort_flag = p->d_ctr + 1;
  A.counters = p->d_ctr + 2;
  A.status = status;
  A.wait_cycles = p->wait_cycles;
  A.withhold_inst = p->withhold_inst;
  A.withhold_stage = p->withhold_stage;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(p->d_ctr, 0, sizeof(int) * (2 + p->n_counters), p->stream);
    if (p->precision == 0) batch_kernel<0><<<p->grid, batch_threads(0), smem, p->stream>>>(A);
    else batch_kernel<1><<<p->grid, batch_threads(1), smem, p->stream>>>(A);
    cudaError_t el = cudaGetLastError();
    e = cudaStreamEndCapture(p->stream, &graph);
    if (el != cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    free_plan(p);
    return bfail(MPRK_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  *out = p;
  return MPRK_OK;
}

Plan* find_plan(mprk_instance* const* insts, int count, long long wait_cycles, int wi, int ws,
                cudaStream_t stream) {
  for (Plan* p : g_plans) {
    if ((int)p->key.size() != count || p->wait_cycles != wait_cycles || p->withhold_inst != wi ||
        p->withhold_stage != ws || (stream && p->stream != stream))
      continue;
    bool same = true;
    for (int j = 0; j < count && same; j++) same = p->key[j] == insts[j];
    if (same) return p;
  }
  return nullptr;
}

int step_batch(mprk_instance* const* insts, int count, int n, long long wait_cycles, int wi, int ws,
               cudaStream_t stream, long long* cell_stages) {
  if (!insts || count <= 0) return bfail(MPRK_EINVAL, "empty batch");
  if (n < 0) return bfail(MPRK_EINVAL, "negative step count");
  for (int j = 0; j < count; j++)
    if (!insts[j]) return bfail(MPRK_EINVAL, "NULL instance in batch");
  std::lock_guard<std::mutex> lk(g_batch_mu);
  Plan* p = find_plan(insts, count, wait_cycles, wi, ws, stream);
  if (!p) {
    int rc = build_plan(insts, count, wait_cycles, wi, ws, stream, &p);
    if (rc) return rc;
    if (g_plans.size() >= 64) {
      free_plan(g_plans.front());
      g_plans.erase(g_plans.begin());
    }
    g_plans.push_back(p);
  }
  if (cell_stages) *cell_stages = p->cell_stages;
  // order: the batch stream waits for every instance's queued work, and every
  // instance stream waits for the batch before its own later work
  std::vector<cudaStream_t> others;
  for (int j = 0; j < count; j++) {
    cudaStream_t s = instance_stream(insts[j]);
    if (s != p->stream && std::find(others.begin(), others.end(), s) == others.end()) others.push_back(s);
  }
  cudaEvent_t ev = nullptr;
  if (!others.empty()) {
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("event: ") + cudaGetErrorString(e));
    for (cudaStream_t s : others) {
      cudaEventRecord(ev, s);
      cudaStreamWaitEvent(p->stream, ev, 0);
    }
  }
  for (int s = 0; s < n; s++) {
    cudaError_t e = cudaGraphLaunch(p->exec, p->stream);
    if (e != cudaSuccess) {
      if (ev) cudaEventDestroy(ev);
      return bfail(MPRK_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    }
  }
  if (ev) {
    cudaEventRecord(ev, p->stream);
    for (cudaStream_t s : others) cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
  }
  for (int j = 0; j < count; j++) instance_count_steps(insts[j], n);
  return MPRK_OK;
}

}  // namespace

namespace mprk {

// ---------------------------------------------------------------------------
// BatchRunner: the same persistent launch without a graph, for a resident set
// that changes between slow steps (the server). The work list is rebuilt and
// uploaded only when the set changes; device buffers grow stream-ordered.
// ---------------------------------------------------------------------------
struct BatchRunner {
  int precision = 0;
  cudaStream_t stream = nullptr;
  std::vector<const void*> key;
  BatchInst* d_insts = nullptr;
  BatchItem* d_items = nullptr;
  int* d_ctr = nullptr;
  size_t cap_insts = 0, cap_items = 0, cap_ctr = 0;
  int n_items = 0, n_counters = 0, grid = 0, per_sm = 0;
  long long cell_stages = 0;
  unsigned* status = nullptr;
};

BatchRunner* runner_create(int precision, cudaStream_t stream) {
  BatchRunner* r = new BatchRunner();
  r->precision = precision;
  r->stream = stream;
  return r;
}

void runner_destroy(BatchRunner* r) {
  if (!r) return;
  if (r->d_insts) cudaFreeAsync(r->d_insts, r->stream);
  if (r->d_items) cudaFreeAsync(r->d_items, r->stream);
  if (r->d_ctr) cudaFreeAsync(r->d_ctr, r->stream);
  delete r;
}

template <typename T>
static cudaError_t grow(T** p, size_t* cap, size_t need, cudaStream_t s) {
  if (need <= *cap) return cudaSuccess;
  size_t c = std::max(need, *cap * 2);
  if (*p) cudaFreeAsync(*p, s);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMallocAsync((void**)p, c * sizeof(T), s);
  if (e == cudaSuccess) *cap = c;
  return e;
}

void runner_invalidate(BatchRunner* r) {
  if (r) r->key.clear();
}

int runner_step(BatchRunner* r, mprk_instance* const* insts, int count, long long* cell_stages) {
  if (count <= 0) return MPRK_OK;
  bool same = (int)r->key.size() == count;
  for (int j = 0; j < count && same; j++) same = r->key[j] == insts[j];
  if (!same) {
    std::vector<BatchInst> hinst(count);
    int n_counters = 0;
    for (int j = 0; j < count; j++) {
      cudaStream_t s;
      unsigned* st;
      int prec;
      int rc = instance_view(insts[j], &hinst[j].g, &hinst[j].b, &prec, &s, &st);
      if (rc) return rc;
      if (prec != r->precision) return bfail(MPRK_EINVAL, "batch runner: precision mismatch");
      if (hinst[j].g.ny > 1 || hinst[j].g.gen)
        return bfail(MPRK_EINVAL, "batch runner: 2-D instances with the Heun base only");
      hinst[j].status = st;
      hinst[j].precision = prec;
      hinst[j].counter_base = n_counters;
      n_counters += 2 * hinst[j].g.m + 1;
      if (j == 0) r->status = st;
    }
    std::vector<BatchItem> items;
    long long cs = 0;
    build_items(hinst, r->precision, items, &cs);
    cudaError_t e = grow(&r->d_insts, &r->cap_insts, (size_t)count, r->stream);
    if (e == cudaSuccess) e = grow(&r->d_items, &r->cap_items, items.size(), r->stream);
    if (e == cudaSuccess) e = grow(&r->d_ctr, &r->cap_ctr, (size_t)(2 + n_counters), r->stream);
    if (e != cudaSuccess) return bfail(MPRK_ENOMEM, std::string("batch runner: ") + cudaGetErrorString(e));
    // pageable sources: the copies are staged before the calls return
    e = cudaMemcpyAsync(r->d_insts, hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                          r->stream);
    if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("batch runner upload: ") + cudaGetErrorString(e));
    r->key.assign(insts, insts + count);
    r->n_items = (int)items.size();
    r->n_counters = n_counters;
    r->cell_stages = cs;
    if (r->per_sm == 0) {
      const size_t smem = stage_smem_bytes(r->precision);
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (r->precision == 0) {
        e = cudaFuncSetAttribute(batch_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r->per_sm, batch_kernel<0>, batch_threads(0), smem);
      } else {
        e = cudaFuncSetAttribute(batch_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r->per_sm, batch_kernel<1>, batch_threads(1), smem);
      }
      if (e != cudaSuccess || r->per_sm < 1) return bfail(MPRK_ECUDA, "batch runner: occupancy query failed");
      r->grid = r->per_sm * sms;
    }
  }
  BatchArgs A;
  A.insts = r->d_insts;
  A.items = r->d_items;
  A.n_items = r->n_items;
  A.next = r->d_ctr;
  A.abort_flag = r->d_ctr + 1;
  A.counters = r->d_ctr + 2;
  A.status = r->status;
  A.wait_cycles = 2000000000LL;
  A.withhold_inst = -1;
  A.withhold_stage = -1;
  cudaError_t e = cudaMemsetAsync(r->d_ctr, 0, sizeof(int) * (2 + r->n_counters), r->stream);
  if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("batch runner: ") + cudaGetErrorString(e));
  const size_t smem = stage_smem_bytes(r->precision);
  const int grid = std::min(r->grid, r->n_items);
  if (r->precision == 0) batch_kernel<0><<<grid, batch_threads(0), smem, r->stream>>>(A);
  else batch_kernel<1><<<grid, batch_threads(1), smem, r->stream>>>(A);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(MPRK_ECUDA, std::string("batch runner launch: ") + cudaGetErrorString(e));
  for (int j = 0; j < count; j++) instance_count_steps(insts[j], 1);
  if (cell_stages) *cell_stages = r->cell_stages;
  return MPRK_OK;
}

int batch_step_on(mprk_instance* const* insts, int count, int n, cudaStream_t stream, long long* cell_stages) {
  return step_batch(insts, count, n, 2000000000LL, -1, -1, stream, cell_stages);
}

// Drop cached plans that mention an instance about to be destroyed.
void batch_forget(const void* inst) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t j = 0; j < g_plans.size();) {
    Plan* p = g_plans[j];
    if (std::find(p->key.begin(), p->key.end(), inst) != p->key.end()) {
      if (p->stream) cudaStreamSynchronize(p->stream);
      free_plan(p);
      g_plans.erase(g_plans.begin() + j);
    } else {
      j++;
    }
  }
}
}  // namespace mprk

extern "C" {

int mprk_step_batch(mprk_instance* const* insts, int count, int n_slow_steps) {
  // about one second at 2 GHz per wait
  return step_batch(insts, count, n_slow_steps, 2000000000LL, -1, -1, nullptr, nullptr);
}

int mprk_batch_test_withhold(mprk_instance* const* insts, int count, int inst_index, int stage,
                             long long wait_cycles) {
  if (inst_index < 0 || inst_index >= count || stage < 0) return bfail(MPRK_EINVAL, "bad withhold target");
  return step_batch(insts, count, 1, wait_cycles, inst_index, stage, nullptr, nullptr);
}

}  // extern "C"
