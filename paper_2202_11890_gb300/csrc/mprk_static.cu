// mprk_static.cu — the allocation-free entry point mprk_step_static.
//
// Some callers cannot call cudaMalloc. Examples are code running inside
// another framework's memory pool or a custom allocator, a process whose
// device memory is already reserved up front, and real-time loops where an
// allocation could block or fail at the wrong moment. For them this file
// advances a state that the caller already holds on the device. It keeps
// its scratch (the odd-substep fast state, the stage-one right-hand side and
// the buffer and slow accumulators) in one file-scope __device__ array of
// fixed size. Every GPU that loads the library holds that array until the
// process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "mprk.h"
#include "mprk_internal.h"

using namespace mprk;

namespace {

constexpr size_t kStaticScratchBytes = MPRK_STATIC_SCRATCH_BYTES;

// Scratch shared by every call on a device. In host code this name is only a
// host-side stand-in for the symbol, not a device address: device pointers
// come from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mu;
// Device address of g_scratch per device, valid for the CUDA context it was
// looked up in: a cudaDeviceReset makes a new primary context, which loads
// the module again at another address.
void* g_scratch_ptr[64] = {nullptr};
CUcontext g_scratch_ctx[64] = {nullptr};

int sfail(int code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

// cuCtxGetCurrent, looked up once through the runtime (no link-time
// dependency on the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

// Once per device and context, with that device current: look up the
// array's device address and set the kernels' shared-memory limits.
int setup_device(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return sfail(MPRK_ECUDA, "device ordinal out of range");
  const CtxGetCurrentFn get = ctx_get_current();
  if (!get) return sfail(MPRK_ECUDA, "cuCtxGetCurrent not found in the driver");
  // null until the runtime has made its context current on this thread
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  if (!g_scratch_ptr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);  // makes the context current if needed
    if (e != cudaSuccess || !p)
      return sfail(MPRK_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = prepare_kernels();
    if (e != cudaSuccess)
      return sfail(MPRK_ECUDA, std::string("kernel setup: ") + cudaGetErrorString(e));
    if (get(&ctx) != CUDA_SUCCESS || !ctx) return sfail(MPRK_ECUDA, "no current CUDA context");
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return MPRK_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Scratch bytes a configuration needs: qB | Ra | accB | accS, and in the
// FP32-flux mode also dA | dB | rowc | refd; pitch = nx.
size_t scratch_bytes(const mprk_config* c) {
  if (!c || c->nx <= 0 || c->nz_S < 0 || c->nz_B < 0 || c->nz_F < 0) return 0;
  const size_t nz = (size_t)c->nz_S + c->nz_B + c->nz_F;
  const size_t plane = nz * (size_t)c->nx;
  const bool fp64 = c->precision == MPRK_FP64;
  const size_t rsz = fp64 ? 8 : 4;
  const bool mprk2 = c->scheme == MPRK_SCHEME_MPRK2;
  const size_t nB = mprk2 ? (size_t)c->nz_B : 0, nS = mprk2 ? (size_t)c->nz_S : 0;
  size_t b = align256(4 * plane * 8) + align256(4 * plane * rsz) + align256(4 * nB * c->nx * 8) +
             align256(4 * nS * c->nx * 8);
  if (!fp64) b += 2 * align256(4 * plane * 4) + align256(NROWC * nz * 4) + align256(4 * nz * 8);
  return b;
}

}  // namespace

extern "C" {

int mprk_step_static(const mprk_config* cfg, double* q_dev, int n_slow_steps, void* cuda_stream) {
  if (!cfg || !q_dev) return sfail(MPRK_EINVAL, "NULL argument");
  if (n_slow_steps < 0) return sfail(MPRK_EINVAL, "negative step count");
  if (cfg->ny != 1) return sfail(MPRK_EINVAL, "mprk_step_static is 2-D only (ny = 1)");
  if (cfg->base != MPRK_BASE_RK2) return sfail(MPRK_EINVAL, "mprk_step_static takes the Heun base only");
  if (cfg->nx < 4 || cfg->nz_S < 2 || cfg->nz_B < 4 || cfg->nz_F < 2 || cfg->m < 1 ||
      cfg->m > 64 || (cfg->x_walls != MPRK_X_PERIODIC && cfg->x_walls != MPRK_X_WALLS))
    return sfail(MPRK_EINVAL, "invalid grid, buffer width (>= 4), rate ratio or x boundary");
  if (cfg->precision != MPRK_FP64 && cfg->precision != MPRK_FP32FLUX)
    return sfail(MPRK_EINVAL, "unknown precision");
  if (cfg->scheme != MPRK_SCHEME_MPRK2 && cfg->scheme != MPRK_SCHEME_SR_RK2)
    return sfail(MPRK_EINVAL, "unknown scheme");
  if (cfg->wall != MPRK_WALL_NOSLIP && cfg->wall != MPRK_WALL_SLIP)
    return sfail(MPRK_EINVAL, "unknown wall type");
  if (!(cfg->dt > 0.0))
    return sfail(MPRK_EINVAL, "mprk_step_static needs an explicit dt > 0");
  // The FP32-flux tiles tensor-copy the float rows of interior tiles and the
  // completion moves pairs of cells with 16-byte accesses; this entry point
  // accepts the unpadded layouts on which those paths were tested (every row
  // of the caller's state starting on a 256-byte boundary): nx a multiple of
  // 32 and q_dev itself 256-byte aligned.
  if (cfg->precision == MPRK_FP32FLUX && (cfg->nx % 32 != 0 || (reinterpret_cast<uintptr_t>(q_dev) & 255u) != 0))
    return sfail(MPRK_EINVAL,
                 "the FP32-flux mode of mprk_step_static needs nx a multiple of 32 and q_dev 256-byte aligned");
  if (!(cfg->dx > 0) || !(cfg->dz1 > 0) || !(cfg->dz2 > 0) || !(cfg->gamma > 1.0) ||
      !(cfg->Pr > 0.0) || !(cfg->mu1 > 0.0) || !(cfg->mu2 > 0.0) || !(cfg->G >= 0.0))
    return sfail(MPRK_EINVAL, "invalid physical parameters");
  const size_t need = scratch_bytes(cfg);
  if (need > kStaticScratchBytes)
    return sfail(MPRK_EINVAL, "grid needs " + std::to_string(need) +
                                  " bytes of scratch, more than the static maximum of " +
                                  std::to_string(kStaticScratchBytes) + " bytes");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sfail(MPRK_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  void* base = nullptr;
  int rc = setup_device(dev, &base);
  if (rc) return rc;

  // geometry: the caller's state is the home buffer, unpadded (pitch = nx)
  Geom g;
  geom_from_config(*cfg, cfg->nx, &g);

  // carve the scratch: qB | Ra | accB | accS (each 256-byte aligned)
  const size_t plane = (size_t)g.nz * g.pitch;
  const size_t rsz = cfg->precision == MPRK_FP64 ? 8 : 4;
  unsigned char* p = static_cast<unsigned char*>(base);
  Bufs b;
  b.qA = q_dev;
  b.qB = reinterpret_cast<double*>(p);
  p += align256(4 * plane * 8);
  b.Ra = p;
  p += align256(4 * plane * rsz);
  b.accB = reinterpret_cast<double*>(p);
  p += align256(4 * (size_t)(g.n1_r - g.nS_r) * g.nx * 8);
  b.accS = reinterpret_cast<double*>(p);
  p += align256(4 * (size_t)g.nS_r * g.nx * 8);
  b.dA = nullptr;
  b.dB = nullptr;
  b.rowc = nullptr;
  double* refd = nullptr;
  if (cfg->precision != MPRK_FP64) {
    b.dA = reinterpret_cast<float*>(p);
    p += align256(4 * plane * 4);
    b.dB = reinterpret_cast<float*>(p);
    p += align256(4 * plane * 4);
    b.rowc = reinterpret_cast<float*>(p);
    p += align256((size_t)NROWC * g.nz * 4);
    refd = reinterpret_cast<double*>(p);
  }

  // Nothing in the scratch needs clearing: every entry a step reads was
  // written earlier in the same call (stage 1 writes R_a and the buffer sum
  // on every row, stage 2 writes the fast state of substep 1 and the slow
  // result, the FP32-flux reference rows and shadow are rebuilt from q_dev
  // below, and padding does not exist because the pitch is nx).
  cudaStream_t s = (cudaStream_t)cuda_stream;
  StageMaps maps;
  maps.valid = false;
  if (b.dA) {
    e = launch_reference(g, q_dev, refd, b.rowc, s);
    if (e == cudaSuccess) e = launch_shadow(g, q_dev, b.rowc, b.dA, s);
    if (e == cudaSuccess) e = make_stage_maps(g, b, &maps);  // host-side encoding, no allocation
    if (e != cudaSuccess) return sfail(MPRK_ECUDA, std::string("reference set-up: ") + cudaGetErrorString(e));
  }
  for (int step = 0; step < n_slow_steps; step++) {
    for (int st = 0; st < 2 * g.m; st++) {
      const StageArgs a = stage_args(g, b, st);
      e = launch_stage(a, cfg->precision, stage_tiles(a), s, &maps);
      if (e != cudaSuccess) return sfail(MPRK_ECUDA, std::string("stage launch: ") + cudaGetErrorString(e));
    }
    e = launch_finalize(g, b, g.m & 1, s);
    if (e != cudaSuccess) return sfail(MPRK_ECUDA, std::string("completion launch: ") + cudaGetErrorString(e));
  }
  return MPRK_OK;
}

}  // extern "C"
