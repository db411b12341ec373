// mprk_kernels.cu — CUDA kernels of one MPRK2 slow step for sm_103a:
//   stage_kernel    fused RHS + stage combination over the rows of one stage
//   finalize_kernel moves q_{n+1} of the S and B rows (and of F rows after an
//                   odd number of substeps) into the state buffer
//   diag_*          deterministic monitoring reductions (Sec. 5.1 mass and
//                   energy; Courant numbers; non-finite count)
#include <cudaTypedefs.h>

#include <cstring>

#include "mprk_internal.h"
#include "stage_tile.cuh"
#include "stage_tile_mixed.cuh"

namespace mprk {

template <typename Real, typename Store>
__global__ void __launch_bounds__(NTHREADS, 2)
    stage_kernel(const StageArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TileSmem<Real>& S = *reinterpret_cast<TileSmem<Real>*>(smem_raw);
  stage_tile<Real, Store>(a, blockIdx.x, S);
}

// FP32-flux stage kernel: one CTA per tile, blockIdx = (tile column, tile
// row). An interior tile away from the x wrap has its float planes
// tensor-copied (TMA) into shared memory: one thread issues the copies at
// the start, and the row constants are fetched while they fly.
__global__ void __launch_bounds__(MIXED_THREADS, 3)
    stage_kernel_mixed(const StageArgs a, const __grid_constant__ CUtensorMap tm_sb,
                       const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_ra) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  MixedKernelSmem& S = *reinterpret_cast<MixedKernelSmem*>(smem_raw);
  const int k0 = a.row0 + blockIdx.y * MTZ, i0 = blockIdx.x * TX;
  const bool staged = tile_bulk_ok(a, k0, i0);
  if (staged && threadIdx.x == MIXED_THREADS - 32) {
    mbar_init(&S.bar);
    stage_issue(a, k0, i0, S.stg, &S.bar, &tm_sb, &tm_f, &tm_ra);
  }
  if (staged) __syncthreads();  // the mbarrier is initialised before anyone waits on it
  if (!stage_tile_mixed(a, k0, i0, S.work, staged ? &S.stg : nullptr, &S.bar)) {
    // a tensor copy never completed within the bound: flag it, give the
    // copies one more bounded wait, and leave
    if (threadIdx.x == 0 && a.status) atomicOr(a.status, ST_TIMEOUT);
    (void)mbar_wait(&S.bar, 0);
  }
}

size_t stage_smem_bytes(int precision) {
  return precision == 0 ? sizeof(TileSmem<double>) : sizeof(MixedTileSmem);
}

cudaError_t prepare_kernels() {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<double, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TileSmem<double>));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(stage_kernel_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(MixedKernelSmem));
}

namespace {
// cuTensorMapEncodeTiled, looked up once through the runtime (no link-time
// dependency on the driver library); null if the driver lacks it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}
}  // namespace

cudaError_t make_stage_maps(const Geom& g, const Bufs& b, StageMaps* out) {
  out->valid = false;
  if (!b.dA || g.pitch % 4 != 0 || g.nx < SCOLS || g.nz < SROWS) return cudaSuccess;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaSuccess;
  // [4][nz][pitch] float: x = column (nx of pitch used), y = row, z = component
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.nz, 4};
  const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.nz * g.pitch * 4};
  const cuuint32_t box[3] = {SCOLS, SROWS, 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  void* planes[3] = {b.dA, b.dB, b.Ra};
  CUtensorMap* maps[3] = {&out->dA, &out->dB, &out->Ra};
  for (int j = 0; j < 3; j++) {
    if (((unsigned long long)planes[j] & 15ull) != 0) return cudaSuccess;
    const CUresult r = enc(maps[j], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, planes[j], dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  out->valid = true;
  return cudaSuccess;
}

cudaError_t launch_stage(const StageArgs& a, int precision, int n_tiles, cudaStream_t stream,
                         const StageMaps* maps) {
  if (n_tiles <= 0) return cudaSuccess;
  if (precision == 0) {
    stage_kernel<double, double><<<n_tiles, NTHREADS, sizeof(TileSmem<double>), stream>>>(a);
  } else {
    StageArgs s = a;
    CUtensorMap none;
    memset(&none, 0, sizeof(none));
    const bool staged = maps && maps->valid;
    s.bulk = staged ? 1 : 0;
    const CUtensorMap& sb = staged ? maps->dA : none;
    const CUtensorMap& f = staged ? (a.dF == a.b.dA ? maps->dA : maps->dB) : none;
    const CUtensorMap& ra = staged ? maps->Ra : none;
    const dim3 grid(a.tiles_x, n_tiles / a.tiles_x);
    stage_kernel_mixed<<<grid, MIXED_THREADS, mixed_kernel_smem(a.stage & 1), stream>>>(s, sb, f, ra);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32-flux mode set-up. Row means of q give the reference q_ref(k), rounded
// to float; its derived constants are formed in double from the rounded
// values and stored as float (layout in stage_tile_mixed.cuh).
// ---------------------------------------------------------------------------
__global__ void row_mean_kernel(const Geom g, const double* __restrict__ q, double* refd) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.nz) return;
  const size_t plane = (size_t)g.nz * g.pitch;
  for (int c = 0; c < 4; c++) {
    double s = 0.0;
    const double* row = q + (size_t)c * plane + (size_t)k * g.pitch;
    for (int i = 0; i < g.nx; i++) s += row[i];
    refd[c * g.nz + k] = (double)(float)(s / g.nx);
  }
}

__device__ __forceinline__ double ref_pressure(const Geom& g, const double* refd, int k, double* ke) {
  const double r = refd[k], mu = refd[g.nz + k], mw = refd[2 * g.nz + k], E = refd[3 * g.nz + k];
  const double kk = 0.5 * (mu * mu + mw * mw) / r;
  if (ke) *ke = kk;
  return g.gm1 * (E - kk);
}

__global__ void row_const_kernel(const Geom g, const double* __restrict__ refd, float4* rowc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.nz) return;
  const int nz = g.nz, n1 = g.n1;
  const bool up_in = (k + 1 < nz) && ((k + 1 < n1) == (k < n1));
  const bool dn_in = (k - 1 >= 0) && ((k - 1 < n1) == (k < n1));
  float a[4], b[4], c[4];
  for (int j = 0; j < 4; j++) {
    const double own = refd[j * nz + k];
    const double mir = (j == 2) ? -own : own;
    const double up = up_in ? refd[j * nz + k + 1] : mir;
    const double dn = dn_in ? refd[j * nz + k - 1] : mir;
    a[j] = (float)own;
    b[j] = (float)(0.25 * (up - dn));
    c[j] = (k + 1 < nz) ? (float)(own - refd[j * nz + k + 1]) : 0.f;
  }
  double ke;
  const double p = ref_pressure(g, refd, k, &ke);
  // reference pressure carried by the faces below and above row k: a wall
  // or the interface carries the row's own p_ref, an interior face the mean
  const bool wall_dn = (k == 0) || (k == n1), wall_up = (k == nz - 1) || (k == n1 - 1);
  const double p_dn = wall_dn ? p : 0.5 * (p + ref_pressure(g, refd, k - 1, nullptr));
  const double p_up = wall_up ? p : 0.5 * (p + ref_pressure(g, refd, k + 1, nullptr));
  const double inv_dz = k < n1 ? g.inv_dz1 : g.inv_dz2;
  rowc[k] = make_float4(a[0], a[1], a[2], a[3]);
  rowc[nz + k] = make_float4(b[0], b[1], b[2], b[3]);
  rowc[2 * nz + k] = make_float4(c[0], c[1], c[2], c[3]);
  rowc[3 * nz + k] =
      make_float4((float)ke, (float)((p_dn - p_up) * inv_dz - refd[k] * g.G), (float)p, 0.f);
}

// The paired copies of the row constants for the pair path: rows (k, k + TZ)
// side by side (groups RC_PAIR .. 11; zero where k + TZ is outside the grid).
__global__ void row_pair_kernel(const Geom g, float4* rowc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.nz) return;
  const int nz = g.nz;
  const bool in = k + TZ < nz;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  float4* P = rowc + RC_PAIR * nz;
  for (int j = 0; j < 3; j++) {
    const float4 a = rowc[j * nz + k], b = in ? rowc[j * nz + k + TZ] : z;
    P[(2 * j) * nz + k] = make_float4(a.x, b.x, a.y, b.y);
    P[(2 * j + 1) * nz + k] = make_float4(a.z, b.z, a.w, b.w);
  }
  const float4 d = rowc[3 * nz + k], e = in ? rowc[3 * nz + k + TZ] : z;
  P[6 * nz + k] = make_float4(d.x, e.x, d.z, e.z);
  P[7 * nz + k] = make_float4(d.y, e.y, 0.f, 0.f);
}

cudaError_t launch_reference(const Geom& g, const double* q, double* refd, float* rowc,
                             cudaStream_t stream) {
  const int b = (g.nz + 127) / 128;
  row_mean_kernel<<<b, 128, 0, stream>>>(g, q, refd);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  row_const_kernel<<<b, 128, 0, stream>>>(g, refd, reinterpret_cast<float4*>(rowc));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  row_pair_kernel<<<b, 128, 0, stream>>>(g, reinterpret_cast<float4*>(rowc));
  return cudaGetLastError();
}

__global__ void shadow_kernel(const Geom g, const double* __restrict__ q, const float* __restrict__ rowc,
                              float* d) {
  const long long total = 4LL * g.nz * g.nx;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / ((long long)g.nz * g.nx));
    const int rem = (int)(e - (long long)c * g.nz * g.nx);
    const int k = rem / g.nx, i = rem - k * g.nx;
    const size_t o = ((size_t)c * g.nz + k) * g.pitch + i;
    d[o] = narrow(q[o] - (double)rowc[4 * k + c]);
  }
}

cudaError_t launch_shadow(const Geom& g, const double* q, const float* rowc, float* d,
                          cudaStream_t stream) {
  const long long total = 4LL * g.nz * g.nx;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  shadow_kernel<<<blocks, 256, 0, stream>>>(g, q, rowc, d);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Step completion: S and B rows from accS / accB; F rows from qB when the
// fast state ended in qB (odd m). In the FP32-flux mode every row's float
// shadow is also resynchronised to the new double state. One thread per
// (component, row, column).
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(const Geom g, const Bufs b, int m_odd) {
  const bool mixed = b.dA != nullptr;
  const int rows = (m_odd || mixed) ? g.nz : g.n1_r;
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
    else v = m_odd ? b.qB[o] : b.qA[o];
    b.qA[o] = v;
    if (mixed) b.dA[o] = narrow(v - (double)b.rowc[4 * k + c]);
  }
}

cudaError_t launch_finalize(const Geom& g, const Bufs& b, int m_odd, cudaStream_t stream) {
  const int rows = (m_odd || b.dA != nullptr) ? g.nz : g.n1_r;
  if (rows == 0) return cudaSuccess;
  const long long total = 4LL * rows * g.nx;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  finalize_kernel<<<blocks, 256, 0, stream>>>(g, b, m_odd);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Test hook: the bit-operation conversions of the FP32-flux mode next to the
// hardware conversions, for the same inputs.
// ---------------------------------------------------------------------------
__global__ void convert_check_kernel(const double* in, int n, float* nar, float* nar_hw, double* wid,
                                     double* wid_hw) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double x = in[j];
  nar[j] = narrow(x);
  nar_hw[j] = (float)x;
  const float f = (float)x;
  wid[j] = widen(f);
  wid_hw[j] = (double)f;
}

cudaError_t launch_convert_check(const double* in, int n, float* nar, float* nar_hw, double* wid,
                                 double* wid_hw, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  convert_check_kernel<<<(n + 255) / 256, 256, 0, stream>>>(in, n, nar, nar_hw, wid, wid_hw);
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
