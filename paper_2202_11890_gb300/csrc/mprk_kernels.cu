// mprk_kernels.cu — CUDA kernels of one MPRK2 slow step for sm_103a:
//   stage_kernel    fused RHS + stage combination over the rows of one stage
//   finalize_kernel moves q_{n+1} of the S and B rows (and of F rows after an
//                   odd number of substeps) into the state buffer
//   diag_*          deterministic monitoring reductions (Sec. 5.1 mass and
//                   energy; Courant numbers; non-finite count)
#include "mprk_internal.h"
#include "stage_tile.cuh"

namespace mprk {

template <typename Real, typename Store>
__global__ void __launch_bounds__(NTHREADS, (sizeof(Real) == 8 ? 2 : 3))
    stage_kernel(const StageArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileSmem<Real>& S = *reinterpret_cast<TileSmem<Real>*>(smem_raw);
  stage_tile<Real, Store>(a, blockIdx.x, S);
}

size_t stage_smem_bytes(int precision) {
  return precision == 0 ? sizeof(TileSmem<double>) : sizeof(TileSmem<float>);
}

cudaError_t prepare_kernels() {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<double, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TileSmem<double>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(stage_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(TileSmem<float>));
}

cudaError_t launch_stage(const StageArgs& a, int precision, int n_tiles, cudaStream_t stream) {
  if (n_tiles <= 0) return cudaSuccess;
  if (precision == 0) {
    stage_kernel<double, double><<<n_tiles, NTHREADS, sizeof(TileSmem<double>), stream>>>(a);
  } else {
    stage_kernel<float, float><<<n_tiles, NTHREADS, sizeof(TileSmem<float>), stream>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Step completion: S and B rows from accS / accB; F rows from qB when the
// fast state ended in qB (odd m). One thread per (component, row, column).
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const Geom g, const Bufs b, int m_odd) {
  const int rows = m_odd ? g.nz : g.n1_r;
  const long long total = 4LL * rows * g.nx;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / ((long long)rows * g.nx));
    const int rem = (int)(e - (long long)c * rows * g.nx);
    const int k = rem / g.nx, i = rem - k * g.nx;
    const size_t o = ((size_t)c * g.nz + k) * g.pitch + i;
    double v;
    if (k < g.nS_r) v = b.accS[((size_t)c * g.nS_r + k) * g.pitch + i];
    else if (k < g.n1_r) v = b.accB[((size_t)c * (g.n1_r - g.nS_r) + (k - g.nS_r)) * g.pitch + i];
    else v = b.qB[o];
    b.qA[o] = v;
  }
}

cudaError_t launch_finalize(const Geom& g, const Bufs& b, int m_odd, cudaStream_t stream) {
  const int rows = m_odd ? g.nz : g.n1_r;
  if (rows == 0) return cudaSuccess;
  const long long total = 4LL * rows * g.nx;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  finalize_kernel<<<blocks, 256, 0, stream>>>(g, b, m_odd);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Monitoring. Pass 1: each block reduces a fixed, strided set of cells into
// 16 partials (fixed order: per-thread sequential, then shuffle trees, then
// warps in order). Pass 2: one block reduces the partials block by block.
// Slots: 0-3 sums over fluid 1 (rho, rho u, rho w, rho E), 4-7 over fluid 2,
// 8-10 max wave speed in S, B, F, 11 non-finite entries, 12 min rho, 13 min p.
// ---------------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;

int diag_blocks(const Geom& g) {
  long long cells = (long long)g.nz * g.nx;
  long long b = (cells + DIAG_THREADS * 8 - 1) / (DIAG_THREADS * 8);
  if (b < 1) b = 1;
  if (b > 1024) b = 1024;
  return (int)b;
}

__device__ __forceinline__ void combine16(double* d, const double* s) {
#pragma unroll
  for (int j = 0; j < 8; j++) d[j] += s[j];
#pragma unroll
  for (int j = 8; j < 11; j++) d[j] = fmax(d[j], s[j]);
  d[11] += s[11];
  d[12] = fmin(d[12], s[12]);
  d[13] = fmin(d[13], s[13]);
}

__global__ void diag_partial_kernel(const Geom g, const double* __restrict__ q, double* partials) {
  double acc[16];
#pragma unroll
  for (int j = 0; j < 16; j++) acc[j] = 0.0;
  acc[12] = INFINITY;
  acc[13] = INFINITY;
  const long long cells = (long long)g.nz * g.nx;
  const size_t plane = (size_t)g.nz * g.pitch;
  for (long long e = blockIdx.x * (long long)DIAG_THREADS + threadIdx.x; e < cells;
       e += (long long)gridDim.x * DIAG_THREADS) {
    const int k = (int)(e / g.nx), i = (int)(e - (long long)k * g.nx);
    const size_t o = (size_t)k * g.pitch + i;
    const double r = q[o], mu = q[plane + o], mw = q[2 * plane + o], E = q[3 * plane + o];
    const int f = k < g.n1 ? 0 : 4;
    acc[f + 0] += r;
    acc[f + 1] += mu;
    acc[f + 2] += mw;
    acc[f + 3] += E;
    const double bad = (double)(!isfinite(r)) + (double)(!isfinite(mu)) + (double)(!isfinite(mw)) +
                       (double)(!isfinite(E));
    acc[11] += bad;
    const double u = mu / r, w = mw / r;
    const double p = g.gm1 * (E - 0.5 * (mu * u + mw * w));
    const double c = sqrt(g.gamma * p / r);
    const double ws = fmax(fabs(u), fabs(w)) + c;
    const int band = (k < g.nS_g) ? 8 : (k < g.n1 ? 9 : 10);  // S, B, F bands of the grid
    if (ws == ws) acc[band] = fmax(acc[band], ws);
    acc[12] = fmin(acc[12], r);
    acc[13] = fmin(acc[13], p);
  }
  // warp tree (fixed order)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    double o[16];
#pragma unroll
    for (int j = 0; j < 16; j++) o[j] = __shfl_down_sync(0xffffffffu, acc[j], off);
    combine16(acc, o);
  }
  __shared__ double warp_part[DIAG_THREADS / 32][16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < 16; j++) warp_part[wid][j] = acc[j];
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    const int j = threadIdx.x;
    double v = warp_part[0][j];
    for (int w = 1; w < DIAG_THREADS / 32; w++) {
      const double s = warp_part[w][j];
      if (j < 8 || j == 11) v += s;
      else if (j < 11) v = fmax(v, s);
      else v = fmin(v, s);
    }
    partials[(size_t)blockIdx.x * 16 + j] = v;
  }
}

__global__ void diag_final_kernel(const Geom g, const double* partials, int nblocks, double* out,
                                  unsigned* status, double cfl_limit) {
  __shared__ double res[16];
  const int j = threadIdx.x;
  if (j < 16) {
    double v = partials[j];
    for (int b = 1; b < nblocks; b++) {
      const double s = partials[(size_t)b * 16 + j];
      if (j < 8 || j == 11) v += s;
      else if (j < 11) v = fmax(v, s);
      else if (j < 14) v = fmin(v, s);
    }
    res[j] = v;
  }
  __syncthreads();
  if (j == 0) {
    const double a1 = 1.0 / (g.inv_dx * g.inv_dz1), a2 = 1.0 / (g.inv_dx * g.inv_dz2);
    double o[16];
    for (int c = 0; c < 4; c++) {
      o[c] = res[c] * a1;
      o[4 + c] = res[4 + c] * a2;
    }
    const double dx = 1.0 / g.inv_dx, dz1 = 1.0 / g.inv_dz1, dz2 = 1.0 / g.inv_dz2;
    const double dtS = (g.n1_r > 0) ? g.dt : g.dt / g.m;
    o[8] = dtS * res[8] / fmin(dx, dz1);
    o[9] = dtS * res[9] / fmin(dx, dz1);
    o[10] = (g.dt / g.m) * res[10] / fmin(dx, dz2);
    o[11] = res[11];
    o[12] = res[12];
    o[13] = res[13];
    o[14] = 0.0;  // slow steps taken: filled in by the host
    o[15] = g.dt;
    for (int c = 0; c < 16; c++) out[c] = o[c];
    unsigned st = 0;
    if (o[11] > 0.0 || !(o[12] > 0.0) || !(o[13] > 0.0)) st |= ST_NONFINITE;
    if (cfl_limit > 0.0 && (o[8] > cfl_limit || o[9] > cfl_limit || o[10] > cfl_limit)) st |= ST_CFL;
    if (st) atomicOr(status, st);
  }
}

cudaError_t launch_diag(const Geom& g, const double* q, double* partials, int nblocks, double* out,
                        unsigned* status, double cfl_limit, cudaStream_t stream) {
  diag_partial_kernel<<<nblocks, DIAG_THREADS, 0, stream>>>(g, q, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, 32, 0, stream>>>(g, partials, nblocks, out, status, cfl_limit);
  return cudaGetLastError();
}

}  // namespace mprk
