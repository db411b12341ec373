// mprk_internal.h — structures shared by the CUDA kernels and the host runtime.
//
// Device layout of one instance (all planes row-major with a padded pitch):
//   qA   [4][nz][pitch] double   the state q_n (S, B rows) and the fast state
//                                at even fast substeps (F rows)
//   qB   [4][nz][pitch] double   the fast state at odd fast substeps (F rows)
//   Ra   [4][nz][pitch] double   (FP64) or float (FP32FLUX): the right-hand
//                                side of the first stage of the current fast
//                                substep (and of stage 1 on S rows)
//   accB [4][nB][pitch] double   running sum of the buffer right-hand sides,
//                                then q_{n+1} on B rows
//   accS [4][nS][pitch] double   q_{n+1} on S rows until the step ends
// FP32-flux mode only:
//   dA, dB [4][nz][pitch] float  deviations q - q_ref of qA, qB (float shadows)
//   rowc [NROWC][nz] float       per-row reference constants (stage_tile_mixed.cuh)
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder is looked up at run time)
#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "mprk.h"

namespace mprk {

// Tile of the stage kernel: TX columns by TZ rows, one thread per cell.
constexpr int TX = 32;
constexpr int TZ = 8;
constexpr int NTHREADS = TX * TZ;
// The FP32-flux kernel's tile is TX x 2*TZ cells; each thread of its fast
// path carries two cells of one column, rows k and k + TZ.
constexpr int MTZ = 2 * TZ;
// Floats of per-row constants in the FP32-flux mode (layout in stage_tile_mixed.cuh).
constexpr int NROWC = 48;
// Threads of the FP32-flux tile: nine warps. Warps 0-7 own the TX x TZ cell
// pairs, warp 8 computes the faces on the tile's top edge (one pass) and
// right edge (one pass), so every warp makes two face passes.
constexpr int MIXED_THREADS = NTHREADS + 32;

// Status bits written by device code.
constexpr unsigned ST_NONFINITE = 1u;
constexpr unsigned ST_CFL = 2u;
constexpr unsigned ST_TIMEOUT = 4u;

// Physics and grid of one instance, constant over its life.
struct Geom {
  int nx, pitch, nz;
  int n1;          // rows of fluid 1 (S and B): the interface lies below row n1
  int nS_r, n1_r;  // region bounds used by the stage combination: rows < nS_r are
                   // S, rows < n1_r are B, the rest F (single rate: 0 and 0)
  int nS_g;        // rows of the slow band of the grid (Courant numbers per band)
  int m;           // fast substeps per slow step
  int wall;        // 0 no-slip, 1 slip
  int xwall;       // 0 periodic x, 1 walls (of kind `wall`) at both x ends
  double dt;
  double inv_dx, inv_dz1, inv_dz2;
  double gamma, gm1;
  double mu1, mu2, kap1, kap2;
  double G;
  double bu, bT;       // interface bulk coefficients (App. B)
  double cu1, cT1;     // dz1/(2 mu1), dz1/(2 kappa1): wall states from fluid 1
  double cu2, cT2;     // dz2/(2 mu2), dz2/(2 kappa2): wall states from fluid 2
  int ny;              // columns in y: 1 in 2-D
  int nc;              // conserved components: 4 (2-D) or 5 (3-D)
  double inv_dy;       // 3-D only
  // base method of the MPRK framework (Sec. 3 remark): s stages, A, b.
  // gen = 0 for Heun (Table 1), which runs the dedicated RK2 low-storage
  // path; otherwise the general s-stage path with s R_a slots.
  int s, gen;
  double bA[4][4], bb[4];
  double hF;           // dt / m
  double h2;           // dt / (2 m)
  double hdt;          // dt / 2
  // the same constants rounded to float once on the host, so that float
  // kernels never convert (conversions run at the FP64 rate on this GPU)
  float gammaf, gm1f, mu1f, mu2f, kap1f, kap2f, Gf;
  float inv_dxf, inv_dz1f, inv_dz2f;
  float dtf, hFf, h2f;
};


// Buffers of one instance.
struct Bufs {
  double* qA;
  double* qB;
  void* Ra;
  double* accB;
  double* accS;
  float* dA;    // FP32-flux mode only (else null)
  float* dB;
  float* rowc;
};

// One launch of the stage kernel over rows [row0, nz) of one instance.
struct StageArgs {
  Geom g;
  Bufs b;
  const double* qF;   // base state of F rows this substep (qA or qB)
  double* qF_next;    // F rows of the next substep (the other one)
  const float* dF;    // FP32-flux mode: shadows matching qF and qF_next
  float* dF_next;
  int stage;          // 0-based stage index i in [0, 2m)
  int row0;           // first row of the launch (0 at stages 0, 1; nS_r later)
  int tiles_x;        // tiles across x
  int tz;             // tile rows: TZ (FP64) or MTZ (FP32-flux)
  int rhs_only;       // test hook: write R to rhs_out instead of combining
  double* rhs_out;    // [4][nz][pitch] when rhs_only
  int rhs_hi;         // last row (exclusive) when rhs_only
  const double* rhs_in;  // full stage state when rhs_only
  double* gy;         // 3-D: y-face fluxes [5][nz][ny][pitch] (face j+1/2 at j)
  int bulk;           // FP32-flux: interior tiles stage their float planes by
                      // tensor copies (set by launch_stage when maps exist)
  unsigned* status;   // status word for device-side errors, or null
};

// Arguments of stage st of one slow step: F rows ping-pong between the A and
// B buffers at every fast substep.
__host__ __device__ inline StageArgs stage_args(const Geom& g, const Bufs& b, int st) {
  StageArgs a{};
  a.g = g;
  a.b = b;
  const bool even_sub = ((st / g.s) % 2) == 0;
  a.qF = even_sub ? b.qA : b.qB;
  a.qF_next = even_sub ? b.qB : b.qA;
  a.dF = even_sub ? b.dA : b.dB;
  a.dF_next = even_sub ? b.dB : b.dA;
  a.stage = st;
  a.row0 = st < g.s ? 0 : g.nS_r;  // S rows only during the first substep
  a.tiles_x = (g.nx + TX - 1) / TX;
  a.tz = b.dA ? MTZ : TZ;  // float shadows exist only in the FP32-flux mode
  return a;
}
__host__ __device__ inline int stage_tiles(const StageArgs& a) {
  const int hi = a.rhs_only ? a.rhs_hi : a.g.nz;
  return a.tiles_x * ((hi - a.row0 + a.tz - 1) / a.tz);
}

// Tensor maps of the FP32-flux float planes ([4][nz][pitch] float each) for
// the bulk tensor copies of the stage kernel (mprk_kernels.cu).
struct StageMaps {
  CUtensorMap dA, dB, Ra;
  bool valid;
};
// Encodes the maps of b's float planes. Sets valid = false (and returns
// cudaSuccess) where the planes cannot be tensor-copied (pitch not a
// multiple of 4 floats, or no encoder in the driver); tiles then load
// directly.
cudaError_t make_stage_maps(const Geom& g, const Bufs& b, StageMaps* out);

// Shape of the FP64 stage tile: rows per tile (TZ, TZ/2 or TZ/4, with TX
// columns) and threads per cell (1 or 2). Every shape computes the same
// arithmetic in the same order, so results do not depend on it.
struct TileShape {
  int rows, tpc;
};
inline bool tile_shape_valid(const TileShape& t) {
  return (t.rows == TZ || t.rows == TZ / 2 || t.rows == TZ / 4) && (t.tpc == 1 || t.tpc == 2);
}
// The tuned shape of single-instance FP64 stage launches of `cells` cells,
// when the tuning table has one for their size bucket (mprk_batch.cu).
bool tuned_tile_shape(long long cells, TileShape* out);
// The shape launch_stage takes without a tuned one: the shortest tile whose
// launch fits in one wave (n tiles <= SMs), with two threads per cell; a
// launch that does not fit even with TZ rows keeps them, one thread per cell.
TileShape default_tile_shape(const StageArgs& a);

// Launchers (mprk_kernels.cu). All enqueue on `stream` and return the launch error.
// maps (FP32-flux only, may be null) enables the staged tiles. shape (FP64
// only, may be null) overrides the tuned and the default tile shape.
cudaError_t launch_stage(const StageArgs& a, int precision, int n_tiles, cudaStream_t stream,
                         const StageMaps* maps = nullptr, const TileShape* shape = nullptr);
cudaError_t launch_finalize(const Geom& g, const Bufs& b, int m_odd, cudaStream_t stream);
// 3-D (g.ny > 1): the y-face launch and the stage launch of one stage; a.gy
// must point at a state-sized buffer.
cudaError_t launch_stage3(const StageArgs& a, cudaStream_t stream);
// FP32-flux mode: per-row reference of q (row means, refd [4][nz] scratch)
// and the float shadow dA = q - q_ref of qA.
cudaError_t launch_reference(const Geom& g, const double* q, double* refd, float* rowc,
                             cudaStream_t stream);
cudaError_t launch_shadow(const Geom& g, const double* q, const float* rowc, float* d,
                          cudaStream_t stream);
cudaError_t launch_diag(const Geom& g, const double* q, double* partials, int nblocks,
                        double* out, unsigned* status, double cfl_limit, cudaStream_t stream);
int diag_blocks(const Geom& g);
cudaError_t launch_convert_check(const double* in, int n, float* nar, float* nar_hw, double* wid,
                                 double* wid_hw, cudaStream_t stream);
cudaError_t prepare_kernels();  // one-time attribute setup (dynamic shared memory)
size_t stage_smem_bytes(int precision);

// Fills g from a configuration; pitch is the row pitch of the buffers
// (mprk_runtime.cu).
void geom_from_config(const mprk_config& c, int pitch, Geom* g);

// Sets the calling thread's message for mprk_last_error (mprk_runtime.cu).
void set_last_error(const std::string& msg);

}  // namespace mprk

struct mprk_instance;

namespace mprk {
// Instance internals the batch path uses (mprk_runtime.cu).
int instance_view(const mprk_instance* inst, Geom* g, Bufs* b, int* precision, cudaStream_t* stream,
                  unsigned** status);
cudaStream_t instance_stream(const mprk_instance* inst);
void instance_count_steps(mprk_instance* inst, int n);
// One slow step of an instance by its own stage launches on stream s (the
// kernels mprk_step's graph replays), counted in its steps; cell_stages gets
// the step's cell-stages (mprk_runtime.cu).
int instance_step_alone(mprk_instance* inst, cudaStream_t s, long long* cell_stages);
// Cells of an instance (nx ny nz).
long long instance_cells(const mprk_instance* inst);
// Drops cached batch plans that mention inst (mprk_batch.cu).
void batch_forget(const void* inst);
// One batched launch per slow step on an explicit stream (mprk_batch.cu).
int batch_step_on(mprk_instance* const* insts, int count, int n, cudaStream_t stream, long long* cell_stages);
// A persistent batch launcher for a resident set that changes between slow
// steps (mprk_batch.cu); one launch per call, no graph.
struct BatchRunner;
BatchRunner* runner_create(int precision, cudaStream_t stream);
void runner_destroy(BatchRunner* r);
int runner_step(BatchRunner* r, mprk_instance* const* insts, int count, long long* cell_stages);
// Forget the cached work list (the resident set changed; an address may be reused).
void runner_invalidate(BatchRunner* r);
// Device bytes mprk_create allocates for a configuration (mprk_runtime.cu).
long long instance_bytes(const mprk_config& c);
// Configuration check of mprk_create (sets the error message).
int validate_config(const mprk_config* c);
// mprk_create with an option: stream_ordered instances allocate with
// cudaMallocAsync on cuda_stream, free with cudaFreeAsync, capture no graph
// and advance only through batches (the server's instances).
int create_instance(const mprk_config* cfg, const double* q0, int q0_location, void* cuda_stream,
                    bool stream_ordered, mprk_instance** out);
long long instance_steps(const mprk_instance* inst);
long long instance_device_bytes(const mprk_instance* inst);
void destroy_instance(mprk_instance* inst);

}  // namespace mprk
