// mprk_runtime.cu — host runtime behind the C ABI of include/mprk.h: instance
// buffers, the slow step captured as a CUDA graph, state I/O (with a row-copy
// kernel for device-to-device copies), monitoring and the right-hand-side
// test hook. No code path computes on the CPU.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "mprk.h"
#include "mprk_internal.h"

using namespace mprk;

namespace {
thread_local std::string g_err;
}  // namespace

void mprk::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

// rows x width doubles from src (row stride spitch) to dst (row stride
// dpitch), on the SMs: a copy-engine 2-D copy between device buffers runs
// well below HBM bandwidth. x over columns, y over rows (grid-stride).
__global__ void copy_rows_kernel(double* __restrict__ dst, size_t dpitch, const double* __restrict__ src,
                                 size_t spitch, int width, long long rows) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= width) return;
  for (long long r = blockIdx.y; r < rows; r += gridDim.y) dst[r * dpitch + c] = src[r * spitch + c];
}

cudaError_t copy_rows(double* dst, size_t dpitch, const double* src, size_t spitch, int width, long long rows,
                      cudaStream_t s) {
  if (width <= 0 || rows <= 0) return cudaSuccess;
  const dim3 block(256);
  const dim3 grid((unsigned)((width + 255) / 256), (unsigned)(rows < 32768 ? rows : 32768));
  copy_rows_kernel<<<grid, block, 0, s>>>(dst, dpitch, src, spitch, width, rows);
  return cudaGetLastError();
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(MPRK_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                 \
  } while (0)

std::mutex g_prep_mu;
bool g_prepared[64] = {false};

int prepare_device(int dev) {
  std::lock_guard<std::mutex> lk(g_prep_mu);
  if (dev < 0 || dev >= 64) return fail(MPRK_ECUDA, "device ordinal %d out of range", dev);
  if (!g_prepared[dev]) {
    CU(prepare_kernels());
    g_prepared[dev] = true;
  }
  return MPRK_OK;
}

}  // namespace

struct mprk_instance {
  mprk_config cfg;
  Geom g;
  Bufs b;
  int precision;
  int device;
  cudaStream_t stream;
  bool own_stream;
  double* partials;
  double* diag_dev;
  unsigned* status_dev;
  int diag_nblocks;
  double* rhs_in;   // lazily allocated padded buffers for mprk_rhs
  double* rhs_out;
  double* refd;     // FP32-flux mode: row means scratch [4][nz]
  cudaGraphExec_t exec;       // one slow step
  cudaGraphExec_t exec_diag;  // one slow step followed by monitoring
  long long steps_done;
  long long bytes;
  bool stream_ordered;  // buffers from cudaMallocAsync on `stream` (server instances)
  StageMaps maps;       // FP32-flux mode: tensor maps of the float planes
  double* gy;           // 3-D: y-face fluxes of the current stage
  // mprk_step_io (allocated on its first call): staging copies of one
  // state in the caller's layout, two copy streams and their events
  double* io_in;
  double* io_out;
  cudaStream_t s_up, s_down;
  cudaEvent_t ev_up, ev_in_free, ev_out_ready, ev_out_free;
};

namespace {

}  // namespace

int mprk::validate_config(const mprk_config* c) {
  if (!c) return fail(MPRK_EINVAL, "config is NULL");
  if (c->nx < 4) return fail(MPRK_EINVAL, "nx = %d: need at least 4 columns", c->nx);
  if (c->nz_S < 2) return fail(MPRK_EINVAL, "nz_S = %d: need at least 2 slow rows", c->nz_S);
  if (c->nz_B < 4)
    return fail(MPRK_EINVAL,
                "nz_B = %d: the buffer needs at least 4 rows for the buffer condition", c->nz_B);
  if (c->nz_F < 2) return fail(MPRK_EINVAL, "nz_F = %d: need at least 2 fast rows", c->nz_F);
  if (c->m < 1 || c->m > 64) return fail(MPRK_EINVAL, "m = %d: need 1 <= m <= 64", c->m);
  if (c->precision != MPRK_FP64 && c->precision != MPRK_FP32FLUX)
    return fail(MPRK_EINVAL, "unknown precision %d", c->precision);
  if (c->scheme != MPRK_SCHEME_MPRK2 && c->scheme != MPRK_SCHEME_SR_RK2)
    return fail(MPRK_EINVAL, "unknown scheme %d", c->scheme);
  if (c->wall != MPRK_WALL_NOSLIP && c->wall != MPRK_WALL_SLIP)
    return fail(MPRK_EINVAL, "unknown wall type %d", c->wall);
  if (c->diag_every < 0) return fail(MPRK_EINVAL, "diag_every must be >= 0");
  if (c->x_walls != MPRK_X_PERIODIC && c->x_walls != MPRK_X_WALLS)
    return fail(MPRK_EINVAL, "unknown x boundary %d", c->x_walls);
  if (!(c->dt >= 0.0) || !std::isfinite(c->dt)) return fail(MPRK_EINVAL, "dt must be >= 0");
  if (!(c->cfl >= 0.0) || c->cfl > 10.0) return fail(MPRK_EINVAL, "cfl out of range");
  if (!(c->dx > 0) || !(c->dz1 > 0) || !(c->dz2 > 0))
    return fail(MPRK_EINVAL, "cell sizes must be positive");
  if (!(c->gamma > 1.0) || !(c->Pr > 0.0)) return fail(MPRK_EINVAL, "need gamma > 1 and Pr > 0");
  if (!(c->mu1 > 0.0) || !(c->mu2 > 0.0)) return fail(MPRK_EINVAL, "viscosities must be positive");
  if (!(c->G >= 0.0)) return fail(MPRK_EINVAL, "G must be >= 0");
  if (c->ny < 1) return fail(MPRK_EINVAL, "ny = %d: need ny >= 1", c->ny);
  if (c->base < MPRK_BASE_RK2 || c->base > MPRK_BASE_RK4)
    return fail(MPRK_EINVAL, "unknown base method %d", c->base);
  if (c->base != MPRK_BASE_RK2 && (c->precision != MPRK_FP64 || c->ny > 1))
    return fail(MPRK_EINVAL, "the RK3 and RK4 bases run in FP64 on the 2-D model only");
  if (c->ny > 1) {
    if (c->ny < 4) return fail(MPRK_EINVAL, "ny = %d: a 3-D grid needs at least 4 columns in y", c->ny);
    if (c->precision != MPRK_FP64) return fail(MPRK_EINVAL, "the 3-D model runs in FP64 only");
    if (c->x_walls != MPRK_X_PERIODIC) return fail(MPRK_EINVAL, "the 3-D model is periodic in x and y");
    if (!(c->dy > 0)) return fail(MPRK_EINVAL, "dy must be positive");
  }
  long long cells = (long long)c->nx * c->ny * (c->nz_S + c->nz_B + c->nz_F);
  if (cells > (1LL << 31)) return fail(MPRK_EINVAL, "grid too large");
  return MPRK_OK;
}

namespace {

void fill_geom(mprk_instance* I) { geom_from_config(I->cfg, (I->cfg.nx + 31) / 32 * 32, &I->g); }

// mprk_step_io's staging buffers, copy streams and events: released
// together (after their queued work) and reset, so a later call starts over.
void release_io(mprk_instance* I) {
  for (cudaStream_t* s : {&I->s_up, &I->s_down})
    if (*s) {
      cudaStreamSynchronize(*s);
      cudaStreamDestroy(*s);
      *s = nullptr;
    }
  for (cudaEvent_t* ev : {&I->ev_up, &I->ev_in_free, &I->ev_out_ready, &I->ev_out_free})
    if (*ev) {
      cudaEventDestroy(*ev);
      *ev = nullptr;
    }
  for (double** b : {&I->io_in, &I->io_out})
    if (*b) {
      cudaFree(*b);
      *b = nullptr;
    }
}

void free_instance(mprk_instance* I) {
  if (!I) return;
  if (I->stream && !I->stream_ordered) cudaStreamSynchronize(I->stream);
  release_io(I);
  if (I->exec) cudaGraphExecDestroy(I->exec);
  if (I->exec_diag) cudaGraphExecDestroy(I->exec_diag);
  void* bufs[] = {I->b.qA,     I->b.qB,     I->b.Ra,     I->b.accB, I->b.accS, I->partials, I->diag_dev,
                  I->status_dev, I->rhs_in, I->rhs_out, I->b.dA,   I->b.dB,   I->b.rowc,   I->refd,
                  I->gy};
  for (void* p : bufs) {
    if (!p) continue;
    // stream-ordered buffers go back to the pool after the stream's queued work
    if (I->stream_ordered) cudaFreeAsync(p, I->stream);
    else cudaFree(p);
  }
  if (I->own_stream && I->stream) cudaStreamDestroy(I->stream);
  delete I;
}

// Enqueue the stage launches and the completion of one slow step.
// after_launch(j), when given, runs after launch j on s (0-based, stages
// first, the completion last): the profiling hook records events there.
template <typename F>
int enqueue_step_with(mprk_instance* I, cudaStream_t s, F after_launch) {
  const Geom& g = I->g;
  for (int st = 0; st < g.s * g.m; st++) {
    StageArgs a = stage_args(g, I->b, st);
    a.status = I->status_dev;
    a.gy = I->gy;
    CU(g.ny > 1 ? launch_stage3(a, s) : launch_stage(a, I->precision, stage_tiles(a), s, &I->maps));
    CU(after_launch(st));
  }
  CU(launch_finalize(g, I->b, g.m & 1, s));
  CU(after_launch(g.s * g.m));
  return MPRK_OK;
}

int enqueue_step(mprk_instance* I, cudaStream_t s) {
  return enqueue_step_with(I, s, [](int) { return cudaSuccess; });
}

int capture(mprk_instance* I, bool with_diag, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  CU(cudaStreamBeginCapture(I->stream, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_step(I, I->stream);
  if (rc == MPRK_OK && with_diag) {
    cudaError_t e = launch_diag(I->g, I->b.qA, I->partials, I->diag_nblocks, I->diag_dev,
                                I->status_dev, 0.0, I->stream);
    if (e != cudaSuccess) rc = fail(MPRK_ECUDA, "monitoring launch: %s", cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamEndCapture(I->stream, &graph);
  if (rc != MPRK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(MPRK_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(MPRK_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return MPRK_OK;
}

int copy_state_in(mprk_instance* I, const double* q, int loc) {
  const Geom& g = I->g;
  const long long rows = (long long)g.nc * g.nz * g.ny;
  if (loc == MPRK_DEVICE)
    CU(copy_rows(I->b.qA, (size_t)g.pitch, q, (size_t)g.nx, g.nx, rows, I->stream));
  else
    CU(cudaMemcpy2DAsync(I->b.qA, (size_t)g.pitch * 8, q, (size_t)g.nx * 8, (size_t)g.nx * 8, (size_t)rows,
                         cudaMemcpyHostToDevice, I->stream));
  if (I->b.dA && I->b.rowc) CU(launch_shadow(g, I->b.qA, I->b.rowc, I->b.dA, I->stream));
  return MPRK_OK;
}

// Run the monitoring kernels now and read the 16 results (synchronises).
int run_diag(mprk_instance* I, double out[16]) {
  CU(launch_diag(I->g, I->b.qA, I->partials, I->diag_nblocks, I->diag_dev, I->status_dev, 0.0,
                 I->stream));
  CU(cudaMemcpyAsync(out, I->diag_dev, 16 * sizeof(double), cudaMemcpyDeviceToHost, I->stream));
  CU(cudaStreamSynchronize(I->stream));
  if (I->g.nc == 4) out[14] = (double)I->steps_done;
  return MPRK_OK;
}

}  // namespace

int mprk::instance_view(const mprk_instance* I, Geom* g, Bufs* b, int* precision, cudaStream_t* stream,
                        unsigned** status) {
  if (!I) return fail(MPRK_EINVAL, "NULL instance");
  *g = I->g;
  *b = I->b;
  *precision = I->precision;
  *stream = I->stream;
  *status = I->status_dev;
  return MPRK_OK;
}

cudaStream_t mprk::instance_stream(const mprk_instance* I) { return I->stream; }

long long mprk::instance_steps(const mprk_instance* I) { return I->steps_done; }

long long mprk::instance_device_bytes(const mprk_instance* I) { return I->bytes; }

void mprk::destroy_instance(mprk_instance* I) {
  batch_forget(I);
  free_instance(I);
}

// The base tableau (A, b) of Sec. 3's remark. Heun keeps gen = 0: its
// low-storage path needs no tableau.
static void set_base(int base, Geom* g) {
  for (int p = 0; p < 4; p++) {
    g->bb[p] = 0.0;
    for (int q = 0; q < 4; q++) g->bA[p][q] = 0.0;
  }
  if (base == MPRK_BASE_RK3) {
    // three-stage SSP: stages at 0, 1 and 1/2 of the step
    g->s = 3;
    g->bA[1][0] = 1.0;
    g->bA[2][0] = 0.25;
    g->bA[2][1] = 0.25;
    g->bb[0] = 1.0 / 6.0;
    g->bb[1] = 1.0 / 6.0;
    g->bb[2] = 2.0 / 3.0;
  } else if (base == MPRK_BASE_RK4) {
    // classical RK4: stages at 0, 1/2, 1/2 and 1
    g->s = 4;
    g->bA[1][0] = 0.5;
    g->bA[2][1] = 0.5;
    g->bA[3][2] = 1.0;
    g->bb[0] = 1.0 / 6.0;
    g->bb[1] = 1.0 / 3.0;
    g->bb[2] = 1.0 / 3.0;
    g->bb[3] = 1.0 / 6.0;
  } else {
    g->s = 2;
    g->bA[1][0] = 1.0;
    g->bb[0] = 0.5;
    g->bb[1] = 0.5;
  }
  g->gen = base != MPRK_BASE_RK2;
}

void mprk::geom_from_config(const mprk_config& c, int pitch, Geom* gp) {
  Geom& g = *gp;
  memset(&g, 0, sizeof g);
  g.nx = c.nx;
  g.pitch = pitch;
  g.nz = c.nz_S + c.nz_B + c.nz_F;
  g.n1 = c.nz_S + c.nz_B;
  if (c.scheme == MPRK_SCHEME_MPRK2) {
    g.nS_r = c.nz_S;
    g.n1_r = g.n1;
  } else {
    g.nS_r = 0;
    g.n1_r = 0;
  }
  g.nS_g = c.nz_S;
  g.m = c.m;
  g.wall = c.wall;
  g.xwall = c.x_walls;
  g.dt = c.dt;
  g.inv_dx = 1.0 / c.dx;
  g.inv_dz1 = 1.0 / c.dz1;
  g.inv_dz2 = 1.0 / c.dz2;
  g.gamma = c.gamma;
  g.gm1 = c.gamma - 1.0;
  g.mu1 = c.mu1;
  g.mu2 = c.mu2;
  const double cp = 1.0 / (c.gamma - 1.0);  // c~_p of App. A
  g.kap1 = cp * c.mu1 / c.Pr;
  g.kap2 = cp * c.mu2 / c.Pr;
  g.G = c.G;
  // bulk coefficients of App. B: 2 k1 k2 / (dz2 k1 + dz1 k2)
  g.bu = 2.0 * c.mu1 * c.mu2 / (c.dz2 * c.mu1 + c.dz1 * c.mu2);
  g.bT = 2.0 * g.kap1 * g.kap2 / (c.dz2 * g.kap1 + c.dz1 * g.kap2);
  g.cu1 = c.dz1 / (2.0 * c.mu1);
  g.cT1 = c.dz1 / (2.0 * g.kap1);
  g.cu2 = c.dz2 / (2.0 * c.mu2);
  g.cT2 = c.dz2 / (2.0 * g.kap2);
  g.ny = c.ny > 1 ? c.ny : 1;
  g.nc = c.ny > 1 ? 5 : 4;
  g.inv_dy = c.ny > 1 ? 1.0 / c.dy : 0.0;
  set_base(c.base, &g);
  g.hF = c.dt / c.m;
  g.h2 = c.dt / (2.0 * c.m);
  g.hdt = 0.5 * c.dt;
  g.gammaf = (float)g.gamma;
  g.gm1f = (float)g.gm1;
  g.mu1f = (float)g.mu1;
  g.mu2f = (float)g.mu2;
  g.kap1f = (float)g.kap1;
  g.kap2f = (float)g.kap2;
  g.Gf = (float)g.G;
  g.inv_dxf = (float)g.inv_dx;
  g.inv_dz1f = (float)g.inv_dz1;
  g.inv_dz2f = (float)g.inv_dz2;
  g.dtf = (float)g.dt;
  g.hFf = (float)g.hF;
  g.h2f = (float)g.h2;
}

void mprk::instance_count_steps(mprk_instance* I, int n) { I->steps_done += n; }

long long mprk::instance_bytes(const mprk_config& c) {
  auto r16 = [](long long b) { return b == 0 ? 16LL : b; };
  const long long pitch = (c.nx + 31) / 32 * 32;
  const long long nz = (long long)c.nz_S + c.nz_B + c.nz_F;
  const long long ny = c.ny > 1 ? c.ny : 1, nc = c.ny > 1 ? 5 : 4;
  const long long plane = nz * ny * pitch;
  const bool mprk2 = c.scheme == MPRK_SCHEME_MPRK2;
  const long long nB = mprk2 ? c.nz_B : 0, nS = mprk2 ? c.nz_S : 0;
  const long long rsz = c.precision == MPRK_FP64 ? 8 : 4;
  const long long ra_slots = c.base == MPRK_BASE_RK4 ? 3 : c.base == MPRK_BASE_RK3 ? 2 : 1;
  long long b = 2 * nc * plane * 8 + ra_slots * nc * plane * rsz + r16(nc * nB * ny * pitch * 8) +
                r16(nc * nS * ny * pitch * 8);
  if (ny > 1) b += nc * plane * 8;  // y-face fluxes
  b += 1024 * 16 * 8 + 16 * 8 + 16;  // monitoring partials (upper bound), results, status
  if (c.precision != MPRK_FP64) b += 2 * 4 * plane * 4 + NROWC * nz * 4 + 4 * nz * 8;
  return b;
}

extern "C" {

int mprk_config_default(mprk_config* cfg, int nx, int nz_S, int nz_B, int nz_F, int m) {
  if (!cfg) return fail(MPRK_EINVAL, "config is NULL");
  if (nx <= 0) return fail(MPRK_EINVAL, "nx must be positive");
  memset(cfg, 0, sizeof *cfg);
  cfg->nx = nx;
  cfg->nz_S = nz_S;
  cfg->nz_B = nz_B;
  cfg->nz_F = nz_F;
  cfg->m = m;
  cfg->precision = MPRK_FP64;
  cfg->scheme = MPRK_SCHEME_MPRK2;
  cfg->wall = MPRK_WALL_NOSLIP;
  cfg->diag_every = 0;
  cfg->dt = 0.0;
  cfg->cfl = 0.4;
  cfg->dx = 10.0 / nx;
  cfg->dz1 = cfg->dx;
  cfg->dz2 = cfg->dx;
  cfg->gamma = 1.4;
  cfg->Pr = 0.72;
  cfg->mu1 = 1.0 / 20000.0;
  cfg->mu2 = 1.0 / 5000.0;
  cfg->G = 0.008140864714;
  cfg->ny = 1;
  cfg->dy = cfg->dx;
  return MPRK_OK;
}

}  // extern "C"

int mprk::instance_step_alone(mprk_instance* I, cudaStream_t s, long long* cell_stages) {
  const int rc = enqueue_step(I, s);
  if (rc) return rc;
  I->steps_done++;
  return mprk_info(I, nullptr, cell_stages, nullptr, nullptr);
}

long long mprk::instance_cells(const mprk_instance* I) {
  return (long long)I->g.nx * I->g.ny * I->g.nz;
}

int mprk::create_instance(const mprk_config* cfg, const double* q0, int q0_location, void* cuda_stream,
                          bool stream_ordered, mprk_instance** out) {
  if (!out) return fail(MPRK_EINVAL, "out is NULL");
  if (stream_ordered && !cuda_stream) return fail(MPRK_EINVAL, "stream-ordered instances need a stream");
  *out = nullptr;
  int rc = validate_config(cfg);
  if (rc) return rc;
  if (!q0) return fail(MPRK_EINVAL, "q0 is NULL");
  if (q0_location != MPRK_HOST && q0_location != MPRK_DEVICE)
    return fail(MPRK_EINVAL, "q0_location must be MPRK_HOST or MPRK_DEVICE");
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if ((rc = prepare_device(dev))) return rc;

  mprk_instance* I = new (std::nothrow) mprk_instance();
  if (!I) return fail(MPRK_ENOMEM, "host allocation failed");
  memset(I, 0, sizeof *I);
  I->cfg = *cfg;
  if (I->cfg.cfl == 0.0) I->cfg.cfl = 0.4;
  I->precision = cfg->precision;
  I->device = dev;
  fill_geom(I);
  const Geom& g = I->g;

  I->stream_ordered = stream_ordered;
  if (cuda_stream) {
    I->stream = (cudaStream_t)cuda_stream;
    I->own_stream = false;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&I->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      free_instance(I);
      return fail(MPRK_ECUDA, "stream create: %s", cudaGetErrorString(e));
    }
    I->own_stream = true;
  }
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (bytes == 0) bytes = 16;
    cudaError_t e = stream_ordered ? cudaMallocAsync(p, bytes, I->stream) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MPRK_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    I->bytes += (long long)bytes;
    return MPRK_OK;
  };
  const size_t plane = (size_t)g.nz * g.ny * g.pitch;  // elements of one component
  const size_t nc = g.nc;
  const size_t rsz = I->precision == MPRK_FP64 ? sizeof(double) : sizeof(float);
  I->diag_nblocks = diag_blocks(g);
  if ((rc = alloc((void**)&I->b.qA, nc * plane * 8)) || (rc = alloc((void**)&I->b.qB, nc * plane * 8)) ||
      (rc = alloc(&I->b.Ra, (size_t)(g.s - 1) * nc * plane * rsz)) ||
      (rc = alloc((void**)&I->b.accB, nc * (size_t)(g.n1_r - g.nS_r) * g.ny * g.pitch * 8)) ||
      (rc = alloc((void**)&I->b.accS, nc * (size_t)g.nS_r * g.ny * g.pitch * 8)) ||
      (g.ny > 1 && (rc = alloc((void**)&I->gy, nc * plane * 8))) ||
      (rc = alloc((void**)&I->partials, (size_t)I->diag_nblocks * 16 * 8)) ||
      (rc = alloc((void**)&I->diag_dev, 16 * 8)) || (rc = alloc((void**)&I->status_dev, 16))) {
    free_instance(I);
    return rc;
  }
  if (I->precision == MPRK_FP32FLUX &&
      ((rc = alloc((void**)&I->b.dA, 4 * plane * 4)) || (rc = alloc((void**)&I->b.dB, 4 * plane * 4)) ||
       (rc = alloc((void**)&I->b.rowc, (size_t)NROWC * g.nz * 4)) ||
       (rc = alloc((void**)&I->refd, (size_t)4 * g.nz * 8)))) {
    free_instance(I);
    return rc;
  }
  auto fin = [&](int code) {
    free_instance(I);
    return code;
  };
  if (cudaMemsetAsync(I->b.qA, 0, nc * plane * 8, I->stream) != cudaSuccess ||
      cudaMemsetAsync(I->b.qB, 0, nc * plane * 8, I->stream) != cudaSuccess ||
      cudaMemsetAsync(I->b.Ra, 0, (size_t)(g.s - 1) * nc * plane * rsz, I->stream) != cudaSuccess ||
      cudaMemsetAsync(I->status_dev, 0, 16, I->stream) != cudaSuccess)
    return fin(fail(MPRK_ECUDA, "memset failed"));
  if (I->b.dA &&
      (cudaMemsetAsync(I->b.dA, 0, 4 * plane * 4, I->stream) != cudaSuccess ||
       cudaMemsetAsync(I->b.dB, 0, 4 * plane * 4, I->stream) != cudaSuccess))
    return fin(fail(MPRK_ECUDA, "memset failed"));
  if ((rc = copy_state_in(I, q0, q0_location))) return fin(rc);
  if (I->b.dA) {
    // reference rows from the initial state, then the shadow of qA
    cudaError_t e = launch_reference(g, I->b.qA, I->refd, I->b.rowc, I->stream);
    if (e == cudaSuccess) e = launch_shadow(g, I->b.qA, I->b.rowc, I->b.dA, I->stream);
    if (e == cudaSuccess) e = make_stage_maps(g, I->b, &I->maps);
    if (e != cudaSuccess) return fin(fail(MPRK_ECUDA, "reference set-up: %s", cudaGetErrorString(e)));
  }

  // check the initial state and pick dt
  double d[16];
  I->g.dt = 1.0;  // placeholder for the Courant numbers of the check
  if ((rc = run_diag(I, d))) return fin(rc);
  const int o = 2 * g.nc;  // first Courant slot (8 in 2-D, 10 in 3-D)
  if (d[o + 3] > 0.0 || !(d[o + 4] > 0.0) || !(d[o + 5] > 0.0))
    return fin(fail(MPRK_ENONFINITE, "q0 has %g non-finite entries, min rho %g, min p %g", d[o + 3],
                    d[o + 4], d[o + 5]));
  if (cudaMemsetAsync(I->status_dev, 0, 16, I->stream) != cudaSuccess)
    return fin(fail(MPRK_ECUDA, "memset failed"));
  double dt = cfg->dt;
  if (dt == 0.0) {
    // wave speeds: d[8..10] hold max(|u|,|w|)+a per band times dt/min(dx,dz)
    // with dt = 1 (S, B at dt, F at dt/m)
    const double sr = cfg->scheme == MPRK_SCHEME_MPRK2 ? 1.0 : (double)cfg->m;
    const double h = g.ny > 1 ? fmin(cfg->dx, cfg->dy) : cfg->dx;
    const double c1 = fmax(d[o], d[o + 1]) * sr * fmin(h, cfg->dz1);
    const double c2 = d[o + 2] * cfg->m * fmin(h, cfg->dz2);
    const double cfl = I->cfg.cfl;
    const double d1 = cfl * fmin(h, cfg->dz1) / c1;
    const double d2 = cfg->m * cfl * fmin(h, cfg->dz2) / c2;
    dt = cfg->scheme == MPRK_SCHEME_MPRK2 ? fmin(d1, d2) : cfg->m * fmin(d1, d2 / cfg->m);
  }
  I->cfg.dt = dt;
  geom_from_config(I->cfg, I->g.pitch, &I->g);
  if (!stream_ordered) {  // stream-ordered (server) instances advance only in batches
    if ((rc = capture(I, false, &I->exec))) return fin(rc);
    if (I->cfg.diag_every > 0 && (rc = capture(I, true, &I->exec_diag))) return fin(rc);
  }
  cudaError_t e = cudaStreamSynchronize(I->stream);
  if (e != cudaSuccess) return fin(fail(MPRK_ECUDA, "create: %s", cudaGetErrorString(e)));
  *out = I;
  return MPRK_OK;
}

extern "C" {

int mprk_create(const mprk_config* cfg, const double* q0, int q0_location, void* cuda_stream,
                mprk_instance** out) {
  return create_instance(cfg, q0, q0_location, cuda_stream, false, out);
}

int mprk_destroy(mprk_instance* inst) {
  if (!inst) return fail(MPRK_EINVAL, "instance is NULL");
  batch_forget(inst);
  free_instance(inst);
  return MPRK_OK;
}

int mprk_step(mprk_instance* I, int n) {
  if (!I) return fail(MPRK_EINVAL, "instance is NULL");
  if (n < 0) return fail(MPRK_EINVAL, "negative step count");
  if (!I->exec) return fail(MPRK_EINVAL, "this instance advances only in batches");
  for (int s = 0; s < n; s++) {
    const bool diag = I->cfg.diag_every > 0 && ((I->steps_done + 1) % I->cfg.diag_every) == 0;
    CU(cudaGraphLaunch(diag ? I->exec_diag : I->exec, I->stream));
    I->steps_done++;
  }
  return MPRK_OK;
}

int mprk_get_state(mprk_instance* I, double* q_out, int location) {
  if (!I || !q_out) return fail(MPRK_EINVAL, "NULL argument");
  if (location != MPRK_HOST && location != MPRK_DEVICE) return fail(MPRK_EINVAL, "bad location");
  const Geom& g = I->g;
  const long long rows = (long long)g.nc * g.nz * g.ny;
  if (location == MPRK_DEVICE)
    CU(copy_rows(q_out, (size_t)g.nx, I->b.qA, (size_t)g.pitch, g.nx, rows, I->stream));
  else
    CU(cudaMemcpy2DAsync(q_out, (size_t)g.nx * 8, I->b.qA, (size_t)g.pitch * 8, (size_t)g.nx * 8, (size_t)rows,
                         cudaMemcpyDeviceToHost, I->stream));
  CU(cudaStreamSynchronize(I->stream));
  return MPRK_OK;
}

namespace {

// Allocates mprk_step_io's staging buffers, streams and events on first use:
// all of them or none.
int io_setup(mprk_instance* I, size_t bytes) {
  if (I->io_in) return MPRK_OK;
  cudaError_t e = cudaMalloc(&I->io_in, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&I->io_out, bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&I->s_up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&I->s_down, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&I->ev_up, &I->ev_in_free, &I->ev_out_ready, &I->ev_out_free})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release_io(I);
    return fail(MPRK_ECUDA, "mprk_step_io set-up: %s", cudaGetErrorString(e));
  }
  return MPRK_OK;
}

// Enqueues the pipelined copies and steps of mprk_step_io; returns at the
// first failure (the caller drains the streams either way).
int io_enqueue(mprk_instance* I, const double* const* q_in, double* const* q_out, int count) {
  const Geom& g = I->g;
  const size_t rows = (size_t)g.nc * g.nz * g.ny, bytes = (size_t)g.nx * 8 * rows;
  // everything queued on the instance stream so far comes first
  CU(cudaEventRecord(I->ev_in_free, I->stream));
  CU(cudaStreamWaitEvent(I->s_up, I->ev_in_free, 0));
  CU(cudaStreamWaitEvent(I->s_down, I->ev_in_free, 0));
  CU(cudaMemcpyAsync(I->io_in, q_in[0], bytes, cudaMemcpyHostToDevice, I->s_up));
  CU(cudaEventRecord(I->ev_up, I->s_up));
  for (int j = 0; j < count; j++) {
    // state j from the staging copy (and the float shadow in FP32-flux mode)
    CU(cudaStreamWaitEvent(I->stream, I->ev_up, 0));
    int rc = copy_state_in(I, I->io_in, MPRK_DEVICE);
    if (rc) return rc;
    CU(cudaEventRecord(I->ev_in_free, I->stream));
    // input j+1 uploads while step j runs
    if (j + 1 < count) {
      CU(cudaStreamWaitEvent(I->s_up, I->ev_in_free, 0));
      CU(cudaMemcpyAsync(I->io_in, q_in[j + 1], bytes, cudaMemcpyHostToDevice, I->s_up));
      CU(cudaEventRecord(I->ev_up, I->s_up));
    }
    if ((rc = mprk_step(I, 1))) return rc;
    // result j to the output staging copy once result j-1 has left it, then
    // down to the host while step j+1 runs
    if (j > 0) CU(cudaStreamWaitEvent(I->stream, I->ev_out_free, 0));
    CU(copy_rows(I->io_out, (size_t)g.nx, I->b.qA, (size_t)g.pitch, g.nx, (long long)rows, I->stream));
    CU(cudaEventRecord(I->ev_out_ready, I->stream));
    CU(cudaStreamWaitEvent(I->s_down, I->ev_out_ready, 0));
    CU(cudaMemcpyAsync(q_out[j], I->io_out, bytes, cudaMemcpyDeviceToHost, I->s_down));
    CU(cudaEventRecord(I->ev_out_free, I->s_down));
  }
  return MPRK_OK;
}

}  // namespace

int mprk_step_io(mprk_instance* I, const double* const* q_in, double* const* q_out, int count) {
  if (!I || !q_in || !q_out) return fail(MPRK_EINVAL, "NULL argument");
  if (count < 0) return fail(MPRK_EINVAL, "negative count");
  if (!I->exec) return fail(MPRK_EINVAL, "this instance advances only in batches");
  for (int j = 0; j < count; j++)
    if (!q_in[j] || !q_out[j]) return fail(MPRK_EINVAL, "q_in[%d] or q_out[%d] is NULL", j, j);
  if (count == 0) return MPRK_OK;
  const Geom& g = I->g;
  int rc = io_setup(I, (size_t)g.nx * 8 * g.nc * g.nz * g.ny);
  if (rc) return rc;
  rc = io_enqueue(I, q_in, q_out, count);
  // whatever was queued finishes before the caller's buffers are released,
  // also after a failure part way
  const cudaError_t e_up = cudaStreamSynchronize(I->s_up), e_down = cudaStreamSynchronize(I->s_down),
                    e_st = cudaStreamSynchronize(I->stream);
  if (rc) return rc;
  for (cudaError_t e : {e_up, e_down, e_st})
    if (e != cudaSuccess) return fail(MPRK_ECUDA, "mprk_step_io: %s", cudaGetErrorString(e));
  return MPRK_OK;
}

int mprk_set_state(mprk_instance* I, const double* q, int location) {
  if (!I || !q) return fail(MPRK_EINVAL, "NULL argument");
  if (location != MPRK_HOST && location != MPRK_DEVICE) return fail(MPRK_EINVAL, "bad location");
  int rc = copy_state_in(I, q, location);
  if (rc) return rc;
  CU(cudaStreamSynchronize(I->stream));
  return MPRK_OK;
}

int mprk_diagnostics(mprk_instance* I, double out[16]) {
  if (!I || !out) return fail(MPRK_EINVAL, "NULL argument");
  return run_diag(I, out);
}

int mprk_sync(mprk_instance* I) {
  if (!I) return fail(MPRK_EINVAL, "instance is NULL");
  CU(cudaStreamSynchronize(I->stream));
  return MPRK_OK;
}

int mprk_status(mprk_instance* I) {
  if (!I) return fail(MPRK_EINVAL, "instance is NULL");
  unsigned st = 0;
  CU(cudaMemcpyAsync(&st, I->status_dev, sizeof st, cudaMemcpyDeviceToHost, I->stream));
  CU(cudaStreamSynchronize(I->stream));
  if (st & ST_NONFINITE) return MPRK_ENONFINITE;
  if (st & ST_TIMEOUT) return MPRK_ETIMEOUT;
  if (st & ST_CFL) return MPRK_ECFL;
  return MPRK_OK;
}

int mprk_info(const mprk_instance* I, double* dt, long long* cell_stages, long long* bytes,
              void** stream) {
  if (!I) return fail(MPRK_EINVAL, "instance is NULL");
  const mprk_config& c = I->cfg;
  if (dt) *dt = I->g.dt;
  if (cell_stages) {
    const long long nz = c.nz_S + c.nz_B + c.nz_F;
    const long long cols = (long long)c.nx * (c.ny > 1 ? c.ny : 1);
    const long long s = I->g.s;
    *cell_stages = c.scheme == MPRK_SCHEME_MPRK2 ? cols * (s * c.nz_S + s * c.m * (c.nz_B + c.nz_F))
                                                 : cols * s * c.m * nz;
  }
  if (bytes) *bytes = I->bytes;
  if (stream) *stream = (void*)I->stream;
  return MPRK_OK;
}

int mprk_rhs(mprk_instance* I, const double* W_dev, double* R_dev, int k_lo, int k_hi) {
  if (!I || !W_dev || !R_dev) return fail(MPRK_EINVAL, "NULL argument");
  const Geom& g = I->g;
  if (k_lo < 0 || k_hi > g.nz || k_lo >= k_hi) return fail(MPRK_EINVAL, "bad row range");
  const size_t plane = (size_t)g.nz * g.ny * g.pitch;
  const size_t nc = g.nc;
  if (!I->rhs_in) {
    CU(cudaMalloc((void**)&I->rhs_in, nc * plane * 8));
    CU(cudaMalloc((void**)&I->rhs_out, nc * plane * 8));
    CU(cudaMemsetAsync(I->rhs_in, 0, nc * plane * 8, I->stream));
  }
  CU(cudaMemcpy2DAsync(I->rhs_in, (size_t)g.pitch * 8, W_dev, (size_t)g.nx * 8, (size_t)g.nx * 8,
                       nc * g.nz * g.ny, cudaMemcpyDeviceToDevice, I->stream));
  StageArgs a = stage_args(g, I->b, 0);
  a.row0 = k_lo;
  a.rhs_only = 1;
  a.rhs_out = I->rhs_out;
  a.rhs_hi = k_hi;
  a.rhs_in = I->rhs_in;
  a.status = I->status_dev;
  if (g.ny > 1) {
    a.gy = I->gy;
    CU(launch_stage3(a, I->stream));
  } else {
    CU(launch_stage(a, I->precision, stage_tiles(a), I->stream));
  }
  for (size_t c = 0; c < nc; c++) {
    CU(cudaMemcpy2DAsync(R_dev + ((size_t)c * g.nz + k_lo) * g.ny * g.nx, (size_t)g.nx * 8,
                         I->rhs_out + c * plane + (size_t)k_lo * g.ny * g.pitch, (size_t)g.pitch * 8,
                         (size_t)g.nx * 8, (size_t)(k_hi - k_lo) * g.ny, cudaMemcpyDeviceToDevice, I->stream));
  }
  return MPRK_OK;
}

int mprk_profile_step(mprk_instance* I, double* launch_ms, long long* launch_cells, int cap) {
  if (!I) return fail(MPRK_EINVAL, "instance is NULL");
  const Geom& g = I->g;
  const int n = g.s * g.m + 1;
  // The step is captured exactly as the one mprk_step replays, with an
  // event record node before the first launch and after
  // each launch on the instance stream, and runs as a graph: each duration
  // is then the kernel as the step graph runs it.
  cudaEvent_t ev[4 * 64 + 2];
  int made = 0;
  int rc = MPRK_OK;
  for (; made <= n; made++)
    if (cudaEventCreate(&ev[made]) != cudaSuccess) {
      rc = fail(MPRK_ECUDA, "event create failed");
      break;
    }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (rc == MPRK_OK) {
    cudaError_t e = cudaStreamBeginCapture(I->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = fail(MPRK_ECUDA, "profile capture: %s", cudaGetErrorString(e));
  }
  if (rc == MPRK_OK) {
    cudaError_t e = cudaEventRecordWithFlags(ev[0], I->stream, cudaEventRecordExternal);
    if (e == cudaSuccess)
      rc = enqueue_step_with(I, I->stream, [&](int j) {
        return cudaEventRecordWithFlags(ev[j + 1], I->stream, cudaEventRecordExternal);
      });
    const cudaError_t e2 = cudaStreamEndCapture(I->stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (rc == MPRK_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (rc == MPRK_OK && e == cudaSuccess) e = cudaGraphUpload(exec, I->stream);
    if (rc == MPRK_OK && e == cudaSuccess) e = cudaGraphLaunch(exec, I->stream);
    if (rc == MPRK_OK && e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
    if (rc == MPRK_OK && e != cudaSuccess) rc = fail(MPRK_ECUDA, "profile: %s", cudaGetErrorString(e));
  }
  if (rc == MPRK_OK) {
    for (int j = 0; j < n && j < cap; j++) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[j], ev[j + 1]);
      if (launch_ms) launch_ms[j] = ms;
      if (launch_cells) {
        if (j < n - 1) {
          const StageArgs a = stage_args(g, I->b, j);
          launch_cells[j] = (long long)(g.nz - a.row0) * g.ny * g.nx;
        } else {
          launch_cells[j] = 0;
        }
      }
    }
    I->steps_done++;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (int j = 0; j < made; j++) cudaEventDestroy(ev[j]);
  return rc == MPRK_OK ? n : rc;
}

int mprk_selftest_convert(const double* in_dev, int n, float* narrow_dev, float* narrow_hw_dev,
                          double* widen_dev, double* widen_hw_dev) {
  if (!in_dev || !narrow_dev || !narrow_hw_dev || !widen_dev || !widen_hw_dev || n < 0)
    return fail(MPRK_EINVAL, "bad argument");
  CU(launch_convert_check(in_dev, n, narrow_dev, narrow_hw_dev, widen_dev, widen_hw_dev, 0));
  CU(cudaStreamSynchronize(0));
  return MPRK_OK;
}

const char* mprk_last_error(void) { return g_err.c_str(); }

}  // extern "C"
