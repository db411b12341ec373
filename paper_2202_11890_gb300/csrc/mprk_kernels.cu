// mprk_kernels.cu — CUDA kernels of one MPRK2 slow step for sm_103a:
//   stage_kernel        FP64 fused RHS + stage combination over the rows of
//                       one stage (one thread per cell, or two in launches
//                       with fewer tiles than SMs; Heun or a general base)
//   stage_kernel_mixed  the FP32-flux form, one instantiation per stage parity
//   yface3_kernel, stage3_kernel  the 3-D model (App. B)
//   finalize_kernel     moves q_{n+1} of the S and B rows (and of F rows after
//                       an odd number of substeps) into the state buffer
//   diag_*              deterministic monitoring reductions (Sec. 5.1 mass
//                       and energy; Courant numbers; non-finite count)
#include <cudaTypedefs.h>

#include <cstring>

#include <algorithm>

#include "mprk_internal.h"
#include "stage_tile.cuh"
#include "stage_tile3d.cuh"
#include "stage_tile_mixed.cuh"
#include "batch_kernel.cuh"

namespace mprk {

// GEN: the general s-stage base (RK3, RK4) in place of Heun's low-storage
// combination. TZR: tile rows (TZ; 4 or 2 for launches of few tiles). One
// thread per cell: 80 registers, a few spilled in the tile (three 32 x 8
// CTAs per SM). NT = 2 TX TZR: two threads per cell for launches with no
// more tiles than SMs.
template <typename Real, typename Store, bool GEN = false, int NT = NTHREADS, int TZR = TZ>
__global__ void __launch_bounds__(NT, NT == TX * TZR ? 3 * NTHREADS / NT : 1)
    stage_kernel(const StageArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TileSmem<Real, TZR>& S = *reinterpret_cast<TileSmem<Real, TZR>*>(smem_raw);
  stage_tile<Real, Store, GEN, NT, TZR>(a, blockIdx.x, S);
}

// FP32-flux stage kernel: one CTA per tile, blockIdx = (tile column, tile
// row). An interior tile away from the x wrap has its float planes
// tensor-copied (TMA) into shared memory: one thread issues the copies at
// the start, and the row constants are fetched while they fly.
template <int PAR>
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
  if (!stage_tile_mixed<PAR>(a, k0, i0, S.work, staged ? &S.stg : nullptr, &S.bar)) {
    // a tensor copy never completed within the bound: flag it, give the
    // copies one more bounded wait, and leave
    if (threadIdx.x == 0 && a.status) atomicOr(a.status, ST_TIMEOUT);
    (void)mbar_wait(&S.bar, 0);
  }
}

// 3-D stage (App. B in full): the y faces of a plane pair, then the x and z
// faces, the divergence and the combination of a plane; one CTA per TX x TZ
// tile of an x-z plane, blockIdx = (tile column, tile row, plane).
__global__ void __launch_bounds__(NTHREADS, 2) yface3_kernel(const StageArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  yface_tile(a, a.row0 + blockIdx.y * TZ, blockIdx.x * TX, blockIdx.z, *reinterpret_cast<YfaceSmem*>(smem_raw));
}

__global__ void __launch_bounds__(NTHREADS, 2) stage3_kernel(const StageArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  stage_tile3(a, a.row0 + blockIdx.y * TZ, blockIdx.x * TX, blockIdx.z, *reinterpret_cast<Tile3Smem*>(smem_raw));
}

cudaError_t launch_stage3(const StageArgs& a, cudaStream_t stream) {
  const int hi = a.rhs_only ? a.rhs_hi : a.g.nz;
  const int tz = (hi - a.row0 + TZ - 1) / TZ;
  if (tz <= 0) return cudaSuccess;
  const dim3 grid(a.tiles_x, tz, a.g.ny);
  yface3_kernel<<<grid, NTHREADS, sizeof(YfaceSmem), stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stage3_kernel<<<grid, NTHREADS, sizeof(Tile3Smem), stream>>>(a);
  return cudaGetLastError();
}

size_t stage_smem_bytes(int precision) {
  return precision == 0 ? sizeof(TileSmem<double>) : sizeof(MixedTileSmem);
}

cudaError_t prepare_kernels() {
  cudaError_t e = cudaFuncSetAttribute(stage_kernel<double, double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TileSmem<double>));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(stage_kernel<double, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(TileSmem<double>));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(stage_kernel<double, double, false, 2 * NTHREADS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem<double>));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(stage_kernel<double, double, true, 2 * NTHREADS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem<double>));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(yface3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(YfaceSmem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(stage3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Tile3Smem));
  if (e != cudaSuccess) return e;
  // one FP32-flux kernel per stage parity, and one that reads it (and the
  // right-hand-side hook) from its arguments
  for (auto k : {stage_kernel_mixed<0>, stage_kernel_mixed<1>, stage_kernel_mixed<PAR_RT>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MixedKernelSmem));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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

namespace {
// SMs of the current device (queried once per device)
int sm_count() {
  static int counts[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (counts[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    counts[dev] = n;
  }
  return counts[dev];
}
}  // namespace

namespace {
// One FP64 stage launch with TZR-row tiles; wide: two threads per cell.
template <int TZR>
void launch_fp64(const StageArgs& a, int n_tiles, bool wide, cudaStream_t stream) {
  constexpr int NT1 = TX * TZR, NT2 = 2 * TX * TZR;
  const size_t smem = sizeof(TileSmem<double, TZR>);
  if (wide && a.g.gen)
    stage_kernel<double, double, true, NT2, TZR><<<n_tiles, NT2, smem, stream>>>(a);
  else if (wide)
    stage_kernel<double, double, false, NT2, TZR><<<n_tiles, NT2, smem, stream>>>(a);
  else if (a.g.gen)
    stage_kernel<double, double, true, NT1, TZR><<<n_tiles, NT1, smem, stream>>>(a);
  else
    stage_kernel<double, double, false, NT1, TZR><<<n_tiles, NT1, smem, stream>>>(a);
}
}  // namespace

TileShape default_tile_shape(const StageArgs& a) {
  // One SM completes two FP64 operations per clock, so a launch of fewer
  // tiles than SMs is bound by the FP64 work of one tile.
  const int sms = sm_count();
  StageArgs s = a;
  int n = 0;
  for (const int t : {TZ / 4, TZ / 2, TZ}) {
    s.tz = t;
    n = stage_tiles(s);
    if (n <= sms) break;
  }
  return TileShape{s.tz, n <= sms ? 2 : 1};
}

cudaError_t launch_stage(const StageArgs& a, int precision, int n_tiles, cudaStream_t stream,
                         const StageMaps* maps, const TileShape* shape) {
  if (n_tiles <= 0) return cudaSuccess;
  if (precision == 0) {
    // FP64: the shape given, else the tuned one for the launch's size
    // bucket (mprk_tile_tune), else the default rule
    TileShape ts;
    if (shape && tile_shape_valid(*shape)) {
      ts = *shape;
    } else {
      const int hi = a.rhs_only ? a.rhs_hi : a.g.nz;
      if (!tuned_tile_shape((long long)(hi - a.row0) * a.g.nx, &ts)) ts = default_tile_shape(a);
    }
    StageArgs s = a;
    s.tz = ts.rows;
    const int n = stage_tiles(s);
    const bool wide = ts.tpc == 2;
    if (s.tz == TZ) launch_fp64<TZ>(s, n, wide, stream);
    else if (s.tz == TZ / 2) launch_fp64<TZ / 2>(s, n, wide, stream);
    else launch_fp64<TZ / 4>(s, n, wide, stream);
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
    const size_t smem = mixed_kernel_smem(a.stage & 1);
    if (a.rhs_only) {
      stage_kernel_mixed<PAR_RT><<<grid, MIXED_THREADS, smem, stream>>>(s, sb, f, ra);
    } else if (a.stage & 1) {
      stage_kernel_mixed<1><<<grid, MIXED_THREADS, smem, stream>>>(s, sb, f, ra);
    } else {
      stage_kernel_mixed<0><<<grid, MIXED_THREADS, smem, stream>>>(s, sb, f, ra);
    }
  }
  return cudaGetLastError();
}

// The persistent batch kernel: shared-memory limit, occupancy and launch
// (declared in batch_types.h).
cudaError_t batch_prepare(int prec, int rows, size_t smem, int* per_sm) {
  cudaError_t e;
  if (prec == 1) {
    e = cudaFuncSetAttribute(batch_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<1>, batch_threads(1), smem);
  } else if (rows == TZ / 2) {
    e = cudaFuncSetAttribute(batch_kernel<0, TZ / 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<0, TZ / 2>, batch_threads(0), smem);
  } else {
    e = cudaFuncSetAttribute(batch_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<0>, batch_threads(0), smem);
  }
  return e;
}
cudaError_t wave_prepare() {
  static const cudaError_t e = [] {
    cudaError_t r = cudaFuncSetAttribute(wave_stage_mixed<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(MixedTileSmem));
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(wave_stage_mixed<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)sizeof(MixedTileSmem));
    return r;
  }();
  return e;
}

void wave_launch_stage(int parity, int grid, const StageArgs* tab, const StageWork* work, int single,
                       cudaStream_t s) {
  if (grid <= 0) return;
  if (parity) wave_stage_mixed<1><<<grid, MIXED_THREADS, sizeof(MixedTileSmem), s>>>(tab, work, single);
  else wave_stage_mixed<0><<<grid, MIXED_THREADS, sizeof(MixedTileSmem), s>>>(tab, work, single);
}

void wave_launch_finalize(int grid, const BatchInst* insts, const StageWork* work, cudaStream_t s) {
  if (grid > 0) wave_finalize<<<grid, NTHREADS, 0, s>>>(insts, work);
}

void batch_launch(int prec, int rows, int grid, size_t smem, cudaStream_t s, const BatchArgs& A) {
  if (prec == 1) batch_kernel<1><<<grid, batch_threads(1), smem, s>>>(A);
  else if (rows == TZ / 2) batch_kernel<0, TZ / 2><<<grid, batch_threads(0), smem, s>>>(A);
  else batch_kernel<0><<<grid, batch_threads(0), smem, s>>>(A);
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
// shadow is also resynchronised to the new double state.
// ---------------------------------------------------------------------------
// An x-row r of a component is (k, j) with r = k ny + j (ny = 1 in 2-D);
// the buffers' rows of the S and B bands are numbered the same way.
// One row of one component per block row: blockIdx.z the component,
// rows r = blockIdx.y + n gridDim.y (r = k ny + j, k the z row), threads
// over x, two consecutive cells per thread. vec: every row starts on a
// 16-byte boundary (an even pitch and 16-byte aligned buffers, as
// mprk_create's padded layout always has), so the pairs move as 16-byte
// loads and stores; otherwise (mprk_step_static's unpadded rows) one cell
// at a time. F rows after an even m already hold q_{n+1} in qA and only
// refresh the float shadow (which the last stage leaves to this kernel).
// Rows k_lo <= k < k_hi (x-rows r = k ny + j).
__global__ void finalize_kernel(const Geom g, const Bufs b, int m_odd, int vec, int k_lo, int k_hi) {
  const bool mixed = b.dA != nullptr;
  const int c = blockIdx.z;
  for (int r = k_lo * g.ny + blockIdx.y; r < k_hi * g.ny; r += gridDim.y) {
    const int k = r / g.ny;
    const size_t o = ((size_t)c * g.nz * g.ny + r) * g.pitch;
    const double* src;
    if (k < g.nS_r) src = b.accS + ((size_t)c * g.nS_r * g.ny + r) * g.pitch;
    else if (k < g.n1_r) src = b.accB + ((size_t)c * (g.n1_r - g.nS_r) * g.ny + (r - (size_t)g.nS_r * g.ny)) * g.pitch;
    else src = (m_odd ? b.qB : b.qA) + o;
    const bool store_q = k < g.n1_r || m_odd;
    const double ref = mixed ? (double)b.rowc[4 * k + c] : 0.0;
    for (int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x); i < g.nx; i += 2 * gridDim.x * blockDim.x) {
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
}

cudaError_t launch_finalize(const Geom& g, const Bufs& b, int m_odd, cudaStream_t stream) {
  const int k_lo = 0;
  const int k_hi = (m_odd || b.dA) ? g.nz : g.n1_r;  // rows it completes
  const int rows = k_hi - k_lo;
  if (rows <= 0) return cudaSuccess;
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const int vec = (g.pitch % 2 == 0 && a16(b.qA) && a16(b.qB) && a16(b.accS) && a16(b.accB) &&
                   (!b.dA || (reinterpret_cast<uintptr_t>(b.dA) & 7u) == 0))
                      ? 1
                      : 0;
  const dim3 grid((g.nx + 511) / 512, (unsigned)std::min(rows * g.ny, 65535), (unsigned)g.nc);
  finalize_kernel<<<grid, 256, 0, stream>>>(g, b, m_odd, vec, k_lo, k_hi);
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
  long long cells = (long long)g.nz * g.ny * g.nx;
  long long b = (cells + DIAG_THREADS * 8 - 1) / (DIAG_THREADS * 8);
  if (b < 1) b = 1;
  if (b > 1024) b = 1024;
  return (int)b;
}

// Monitoring slots for NC components: sums over fluid 1 [0, NC), fluid 2
// [NC, 2NC), the maximal wave speed of the S, B, F bands [2NC, 2NC+3), the
// non-finite count 2NC+3, the minimum density 2NC+4 and pressure 2NC+5
// (NC = 4: the 2-D layout; NC = 5: the 3-D one).
template <int NC>
__device__ __forceinline__ void combine_diag(double* d, const double* s) {
#pragma unroll
  for (int j = 0; j < 2 * NC; j++) d[j] += s[j];
#pragma unroll
  for (int j = 2 * NC; j < 2 * NC + 3; j++) d[j] = fmax(d[j], s[j]);
  d[2 * NC + 3] += s[2 * NC + 3];
  d[2 * NC + 4] = fmin(d[2 * NC + 4], s[2 * NC + 4]);
  d[2 * NC + 5] = fmin(d[2 * NC + 5], s[2 * NC + 5]);
}

template <int NC>
__global__ void diag_partial_kernel(const Geom g, const double* __restrict__ q, double* partials) {
  constexpr int NS = 2 * NC + 6;
  double acc[NS];
#pragma unroll
  for (int j = 0; j < NS; j++) acc[j] = 0.0;
  acc[2 * NC + 4] = INFINITY;
  acc[2 * NC + 5] = INFINITY;
  const long long xrows = (long long)g.nz * g.ny;
  const long long cells = xrows * g.nx;
  const size_t plane = (size_t)xrows * g.pitch;
  for (long long e = blockIdx.x * (long long)DIAG_THREADS + threadIdx.x; e < cells;
       e += (long long)gridDim.x * DIAG_THREADS) {
    const int r = (int)(e / g.nx), i = (int)(e - (long long)r * g.nx);
    const int k = r / g.ny;
    const size_t o = (size_t)r * g.pitch + i;
    double v[NC];
#pragma unroll
    for (int c = 0; c < NC; c++) v[c] = q[c * plane + o];
    const int f = k < g.n1 ? 0 : NC;
    double bad = 0.0;
#pragma unroll
    for (int c = 0; c < NC; c++) {
      acc[f + c] += v[c];
      bad += (double)(!isfinite(v[c]));
    }
    acc[2 * NC + 3] += bad;
    const double rho = v[0], E = v[NC - 1];
    double ke = 0.0, umax = 0.0;
#pragma unroll
    for (int c = 1; c < NC - 1; c++) {
      const double u = v[c] / rho;
      ke += v[c] * u;
      umax = fmax(umax, fabs(u));
    }
    const double p = g.gm1 * (E - 0.5 * ke);
    const double ws = umax + sqrt(g.gamma * p / rho);
    const int band = 2 * NC + ((k < g.nS_g) ? 0 : (k < g.n1 ? 1 : 2));  // S, B, F bands of the grid
    if (ws == ws) acc[band] = fmax(acc[band], ws);
    acc[2 * NC + 4] = fmin(acc[2 * NC + 4], rho);
    acc[2 * NC + 5] = fmin(acc[2 * NC + 5], p);
  }
  // warp tree (fixed order)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    double o[NS];
#pragma unroll
    for (int j = 0; j < NS; j++) o[j] = __shfl_down_sync(0xffffffffu, acc[j], off);
    combine_diag<NC>(acc, o);
  }
  __shared__ double warp_part[DIAG_THREADS / 32][NS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < NS; j++) warp_part[wid][j] = acc[j];
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    const int j = threadIdx.x;
    double v = warp_part[0][j];
    for (int w = 1; w < DIAG_THREADS / 32; w++) {
      const double s = warp_part[w][j];
      if (j < 2 * NC || j == 2 * NC + 3) v += s;
      else if (j < 2 * NC + 3) v = fmax(v, s);
      else v = fmin(v, s);
    }
    partials[(size_t)blockIdx.x * 16 + j] = v;
  }
}

// Final combination and scaling. 2-D: out = the 14 slots scaled to sums
// times the cell area and Courant numbers, then out[14] = 0 (steps, filled
// by the host) and out[15] = dt. 3-D: the 16 slots, sums times the cell
// volume.
template <int NC>
__global__ void diag_final_kernel(const Geom g, const double* partials, int nblocks, double* out,
                                  unsigned* status, double cfl_limit) {
  constexpr int NS = 2 * NC + 6;
  __shared__ double res[NS];
  const int j = threadIdx.x;
  if (j < NS) {
    double v = partials[j];
    for (int b = 1; b < nblocks; b++) {
      const double s = partials[(size_t)b * 16 + j];
      if (j < 2 * NC || j == 2 * NC + 3) v += s;
      else if (j < 2 * NC + 3) v = fmax(v, s);
      else v = fmin(v, s);
    }
    res[j] = v;
  }
  __syncthreads();
  if (j == 0) {
    const double dx = 1.0 / g.inv_dx, dz1 = 1.0 / g.inv_dz1, dz2 = 1.0 / g.inv_dz2;
    const double dy = NC == 5 ? 1.0 / g.inv_dy : 1.0;
    const double a1 = dx * dy * dz1, a2 = dx * dy * dz2;
    const double h = NC == 5 ? fmin(dx, dy) : dx;
    double o[16];
    for (int c = 0; c < NC; c++) {
      o[c] = res[c] * a1;
      o[NC + c] = res[NC + c] * a2;
    }
    const double dtS = (g.n1_r > 0) ? g.dt : g.dt / g.m;
    o[2 * NC] = dtS * res[2 * NC] / fmin(h, dz1);
    o[2 * NC + 1] = dtS * res[2 * NC + 1] / fmin(h, dz1);
    o[2 * NC + 2] = (g.dt / g.m) * res[2 * NC + 2] / fmin(h, dz2);
    o[2 * NC + 3] = res[2 * NC + 3];
    o[2 * NC + 4] = res[2 * NC + 4];
    o[2 * NC + 5] = res[2 * NC + 5];
    if (NC == 4) {
      o[14] = 0.0;  // slow steps taken: filled in by the host
      o[15] = g.dt;
    }
    for (int c = 0; c < 16; c++) out[c] = o[c];
    unsigned st = 0;
    if (o[2 * NC + 3] > 0.0 || !(o[2 * NC + 4] > 0.0) || !(o[2 * NC + 5] > 0.0)) st |= ST_NONFINITE;
    if (cfl_limit > 0.0 &&
        (o[2 * NC] > cfl_limit || o[2 * NC + 1] > cfl_limit || o[2 * NC + 2] > cfl_limit))
      st |= ST_CFL;
    if (st) atomicOr(status, st);
  }
}

cudaError_t launch_diag(const Geom& g, const double* q, double* partials, int nblocks, double* out,
                        unsigned* status, double cfl_limit, cudaStream_t stream) {
  if (g.nc == 5) {
    diag_partial_kernel<5><<<nblocks, DIAG_THREADS, 0, stream>>>(g, q, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<5><<<1, 32, 0, stream>>>(g, partials, nblocks, out, status, cfl_limit);
    return cudaGetLastError();
  }
  diag_partial_kernel<4><<<nblocks, DIAG_THREADS, 0, stream>>>(g, q, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<4><<<1, 32, 0, stream>>>(g, partials, nblocks, out, status, cfl_limit);
  return cudaGetLastError();
}

}  // namespace mprk
