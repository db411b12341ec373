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
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

namespace mprk {

// Tile of the stage kernel: TX columns by TZ rows, one thread per cell.
constexpr int TX = 32;
constexpr int TZ = 8;
constexpr int NTHREADS = TX * TZ;

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
  double dt;
  double inv_dx, inv_dz1, inv_dz2;
  double gamma, gm1;
  double mu1, mu2, kap1, kap2;
  double G;
  double bu, bT;       // interface bulk coefficients (App. B)
  double cu1, cT1;     // dz1/(2 mu1), dz1/(2 kappa1): wall states from fluid 1
};

// Buffers of one instance.
struct Bufs {
  double* qA;
  double* qB;
  void* Ra;
  double* accB;
  double* accS;
};

// One launch of the stage kernel over rows [row0, nz) of one instance.
struct StageArgs {
  Geom g;
  Bufs b;
  const double* qF;   // base state of F rows this substep (qA or qB)
  double* qF_next;    // F rows of the next substep (the other one)
  int stage;          // 0-based stage index i in [0, 2m)
  int row0;           // first row of the launch (0 at stages 0, 1; nS_r later)
  int tiles_x;        // tiles across x
  int rhs_only;       // test hook: write R to rhs_out instead of combining
  double* rhs_out;    // [4][nz][pitch] when rhs_only
  int rhs_hi;         // last row (exclusive) when rhs_only
  const double* rhs_in;  // full stage state when rhs_only
};

// Launchers (mprk_kernels.cu). All enqueue on `stream` and return the launch error.
cudaError_t launch_stage(const StageArgs& a, int precision, int n_tiles, cudaStream_t stream);
cudaError_t launch_finalize(const Geom& g, const Bufs& b, int m_odd, cudaStream_t stream);
cudaError_t launch_diag(const Geom& g, const double* q, double* partials, int nblocks,
                        double* out, unsigned* status, double cfl_limit, cudaStream_t stream);
int diag_blocks(const Geom& g);
cudaError_t prepare_kernels();  // one-time attribute setup (dynamic shared memory)
size_t stage_smem_bytes(int precision);

// Sets the calling thread's message for mprk_last_error (mprk_runtime.cu).
void set_last_error(const std::string& msg);

}  // namespace mprk
