/*
 * mprk.h — C ABI of the GB300 (sm_103a) library for one slow step of the
 * multirate partitioned Runge–Kutta method MPRK2 applied to two coupled
 * compressible Navier–Stokes fluids (Kang, Dener, Hamilton, Zhang,
 * Constantinescu, Jacob, arXiv 2202.11890).
 *
 * The problem (Sec. 3, Eq. semi-discretized-coupled-model): a structured x–z
 * grid, periodic in x, split in z, bottom to top, into a slow band S, a slow
 * buffer band B and a fast band F. S and B hold fluid 1 (the ocean), F holds
 * fluid 2 (the atmosphere), and the rigid-lid interface Gamma separates them
 * (App. B). One slow step of size dt advances S and B with the base RK2 and F
 * with m RK2 substeps of dt/m, coupled as in Eq. MRK2, Table 1 (generalised
 * to any m) and Algorithm 1. The right-hand side is the cell-centred
 * finite-volume scheme of Sec. 2.1 and App. B (Lax–Friedrichs inviscid flux,
 * linear reconstruction, common-gradient viscous flux, bulk interface fluxes).
 *
 * State layout on every host or device buffer that crosses this ABI:
 * structure of arrays [4][nz][nx] of double, contiguous, nz = nz_S + nz_B +
 * nz_F, components (rho, rho*u, rho*w, rho*E), rows bottom to top.
 *
 * Three dimensions (ny > 1 in the configuration; App. B in full): the same
 * x-z rows with y added, periodic in x and y, FP64 only. Every state buffer
 * is then [5][nz][ny][nx] of double with components (rho, rho*u, rho*v,
 * rho*w, rho*E). Every single-instance call below takes that layout where
 * the 2-D text says [4][nz][nx]. The batch, server and static entry points
 * are 2-D only.
 *
 * Conventions. Every call returns 0 (MPRK_OK) or a negative MPRK_E* code, and
 * on error mprk_last_error() returns a message for the calling thread.
 * Nothing runs on the CPU: without a usable CUDA device every compute call
 * fails with MPRK_ECUDA. Pointers passed in stay owned by the caller; the
 * library copies what it needs. All instance work runs asynchronously on the
 * instance's CUDA stream unless a call says it synchronises.
 */
#ifndef MPRK_H
#define MPRK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define MPRK_OK 0
#define MPRK_EINVAL (-1)     /* invalid argument or configuration          */
#define MPRK_ENOMEM (-2)     /* device or host allocation failed           */
#define MPRK_EBUDGET (-3)    /* the request can never fit the HBM budget   */
#define MPRK_ECUDA (-4)      /* a CUDA call failed (message has details)   */
#define MPRK_ENONFINITE (-5) /* the state holds NaN or Inf                 */
#define MPRK_ECFL (-6)       /* a Courant number exceeded the limit        */
#define MPRK_ETIMEOUT (-7)   /* a bounded device wait gave up              */
#define MPRK_EBUSY (-8)      /* resource busy (e.g. server queue full)     */
#define MPRK_ENOTFOUND (-9)  /* unknown ticket                             */

/* ---- enumerations ------------------------------------------------------ */
#define MPRK_FP64 0     /* every operation in double precision                 */
#define MPRK_FP32FLUX 1 /* fluxes and RHS in float; stage values, the buffer
                           accumulation and all stage combinations in double  */

#define MPRK_SCHEME_MPRK2 0  /* Eq. MRK2 with the Table 1 tableaus (s = 2)     */
#define MPRK_SCHEME_SR_RK2 1 /* single rate: m RK2 steps of dt/m everywhere    */

#define MPRK_WALL_NOSLIP 0 /* outer z walls: no-slip, adiabatic               */
#define MPRK_WALL_SLIP 1   /* outer z walls: free slip, adiabatic             */

#define MPRK_X_PERIODIC 0 /* x is periodic                       */
#define MPRK_X_WALLS 1    /* walls at both ends of x              */

/* Base Runge-Kutta method of the MPRK framework. Sec. 3 builds the coupled
 * method from any base; the coupling keeps it second order at most, so the
 * higher-order bases serve accuracy experiments. RK3 and RK4 run in FP64 on
 * the 2-D model: through mprk_create/mprk_step, mprk_step_batch and the
 * server (not mprk_step_static). */
#define MPRK_BASE_RK2 0 /* Heun's method: the Table 1 tableaus           */
#define MPRK_BASE_RK3 1 /* the three-stage third-order SSP method        */
#define MPRK_BASE_RK4 2 /* the classical four-stage fourth-order method  */

#define MPRK_HOST 0   /* pointer is host memory   */
#define MPRK_DEVICE 1 /* pointer is device memory */

/* ---- configuration ----------------------------------------------------- */
typedef struct {
  int nx;         /* columns, >= 4                                            */
  int nz_S;       /* rows of the slow band, >= 2                              */
  int nz_B;       /* rows of the buffer band, >= 4 (buffer condition, Sec. 3) */
  int nz_F;       /* rows of the fast band, >= 2                              */
  int m;          /* rate ratio, 1..64: dt_fast = dt / m                      */
  int precision;  /* MPRK_FP64 or MPRK_FP32FLUX                               */
  int scheme;     /* MPRK_SCHEME_MPRK2 or MPRK_SCHEME_SR_RK2                  */
  int wall;       /* MPRK_WALL_NOSLIP or MPRK_WALL_SLIP (adiabatic)           */
  int diag_every; /* monitor the state every this many slow steps (0 = never) */
  int x_walls;    /* MPRK_X_PERIODIC (0) or MPRK_X_WALLS: adiabatic walls of
                     kind `wall` at both x ends, as in Sec. 5.2's thermal
                     convection (walls on all boundaries)                     */
  double dt;      /* slow step; 0 = from the initial state at Courant cfl     */
  double cfl;     /* used when dt == 0; 0 means 0.4                           */
  double dx;      /* cell width                                              */
  double dz1;     /* cell height in fluid 1 (S and B rows)                    */
  double dz2;     /* cell height in fluid 2 (F rows)                          */
  double gamma;   /* ratio of specific heats (both fluids)                    */
  double Pr;      /* Prandtl number (both fluids)                             */
  double mu1;     /* nondimensional viscosity of fluid 1 (App. A)             */
  double mu2;     /* nondimensional viscosity of fluid 2                      */
  double G;       /* gravity magnitude: source (0, 0, -rho G, -rho w G)       */
  int ny;         /* columns in y: 1 for the 2-D model; >= 4 for 3-D (App. B):
                     y periodic, 5 components, FP64, MPRK_X_PERIODIC          */
  int base;       /* MPRK_BASE_RK2 (default), MPRK_BASE_RK3 or MPRK_BASE_RK4:
                     the s-stage base of every region (s = 2, 3, 4); a slow
                     step then has s*m stages                                 */
  double dy;      /* cell depth in y (3-D)                                    */
} mprk_config;

typedef struct mprk_instance mprk_instance;

/* Fill cfg with the paper's constants (Sec. 5.2: gamma 1.4, Pr 0.72,
 * mu1 1/20000, mu2 1/5000, G 0.008140864714), dx = 10/nx, dz1 = dz2 = dx,
 * MPRK2, FP64, no-slip walls, dt = 0 (automatic, cfl 0.4), no monitoring,
 * 2-D (ny = 1, dy = dx). */
int mprk_config_default(mprk_config* cfg, int nx, int nz_S, int nz_B, int nz_F, int m);

/* Create an instance: allocate its device buffers (about 3 to 4 states of
 * nz*nx*32 bytes), copy q0 from q0_location (MPRK_HOST or MPRK_DEVICE), pick
 * dt if cfg->dt == 0, and capture the slow step in a CUDA graph.
 * cuda_stream: a cudaStream_t to run on, or NULL for a new non-blocking
 * stream owned by the instance. Synchronises. Errors: MPRK_EINVAL,
 * MPRK_ENOMEM, MPRK_ECUDA, MPRK_ENONFINITE (q0 not finite or not positive). */
int mprk_create(const mprk_config* cfg, const double* q0, int q0_location, void* cuda_stream,
                mprk_instance** out);

/* Free every resource of the instance (synchronises its stream first). */
int mprk_destroy(mprk_instance* inst);

/* Advance n_slow_steps slow steps (Algorithm 1 per step). Asynchronous on the
 * instance stream; monitoring (if diag_every > 0) sets the status word that
 * mprk_status reads. */
int mprk_step(mprk_instance* inst, int n_slow_steps);

/* Advance `count` instances by n_slow_steps each, one CUDA graph launch per
 * slow step. The graph holds one of two forms (the tuning table below picks
 * it per precision and size bucket):
 *  - one persistent launch that covers every instance's stage tiles and step
 *    completions (FP64, and FP32 flux when tuned so): items run in stage
 *    order; a tile of stage s of an instance waits (bounded, about one
 *    second) for all stage s-1 tiles of that instance;
 *  - per-stage launches (FP32 flux, the default there): one launch per stage
 *    index over every instance that has that stage, then one launch of all
 *    step completions, ordered by the stream.
 * Instances may differ in size, m, buffer width, dt and base method, but
 * must share the device and the precision, and each may appear only once.
 * The batch runs on the first instance's stream, ordered after and before
 * the other instances' streams with events. Each instance's result equals
 * what mprk_step gives it alone: bitwise in FP64 with the Heun base (same
 * tile code, same arithmetic), to rounding (within 1e-12) with the RK3 and
 * RK4 bases, and to float rounding in FP32 flux (the batch kernels compile
 * the float tile apart from the single-instance kernel). Asynchronous. A
 * wait of the persistent form that gives up sets MPRK_ETIMEOUT in the
 * affected instances' status words (mprk_status); their states are then
 * undefined. In-graph monitoring (diag_every) does not run in batched
 * steps. Errors: MPRK_EINVAL, MPRK_ENOMEM, MPRK_ECUDA. */
int mprk_step_batch(mprk_instance* const* insts, int count, int n_slow_steps);

/* ---- launch and tile-shape tuning ---------------------------------------
 * Three choices of the batched launch change no result, only its speed:
 * the stage tiles per work item (1, 2, 4, 8 or 16; G consecutive tiles
 * along x; in FP32 flux 0 stands for the per-stage form, which has no work
 * items), the CTAs per SM (1 to 3; with the per-stage form, the number of
 * instance groups, 1, 2 or 4, whose launches run on streams of their own so
 * that one group's launch tail overlaps another's work), and in FP64 the
 * shape of the stage
 * tile of the 256-thread CTA: 32 x 8 cells with one thread per cell or
 * 32 x 4 with two (the FP32-flux tile is 32 x 16). Single-instance FP64
 * stage launches (mprk_step) choose among six tile shapes: 32 x 8, 32 x 4
 * or 32 x 2 cells, with one or two threads per cell. Every shape evaluates
 * the same arithmetic in the same order (Sec. 2.1, App. B), so results are
 * bitwise the same whatever is chosen.
 * A process-wide table keeps the fastest choices measured:
 *  - batches: per precision and size bucket (floor(log2) of the mean cells
 *    per instance); without an entry, in FP64 2 tiles per item, every CTA
 *    that fits and 32 x 8 tiles, in FP32 flux the per-stage form with two
 *    instance groups;
 *  - single-instance FP64 stage launches: per size bucket (floor(log2) of
 *    the cells of the launch); without an entry, the shortest tile whose
 *    launch fits in one wave of the GPU's SMs, with two threads per cell,
 *    or 32 x 8 with one thread per cell when none fits.
 * mprk_step_batch, the server and the FP64 stage launches (including graphs
 * captured afterwards by mprk_create) read the table. */

/* Time every batch choice on these instances (reps batched slow steps each
 * after one warm-up step), record the fastest in the table and return it
 * in out: {tiles per item (0: the per-stage form), CTAs per SM (instance
 * groups with the per-stage form), ms per slow step, tile rows}.
 * The instances' states and step counts are restored afterwards.
 * Synchronises. Errors: MPRK_EINVAL, MPRK_ENOMEM, MPRK_ECUDA. */
int mprk_batch_tune(mprk_instance* const* insts, int count, int reps, double out[4]);

/* The table's batch choice for a precision and a mean instance size in
 * cells: writes it and returns 1, or writes the defaults (ctas_per_sm 0:
 * every CTA that fits, or two instance groups; group 0 in FP32 flux: the
 * per-stage form) and
 * returns 0. tile_rows: 8 or 4 in FP64 (one or two threads per cell), 16 in
 * FP32 flux. Needs no device. */
int mprk_tune_lookup(int precision, double mean_cells, int* group, int* ctas_per_sm, int* tile_rows);

/* Time the six tile shapes of single-instance FP64 stage launches on these
 * 2-D FP64 instances: for each instance the first stage (every row) and the
 * first stage of the second fast substep (B and F rows), reps launches of
 * each shape after a warm-up launch. Both stages read the state and write
 * only stage scratch, so the states are unchanged. Records, per size bucket
 * of a launch's cells, the shape with the smallest summed time over the
 * launches in that bucket, and writes the number of buckets to *entries.
 * Instances created or graphs captured before the call keep their shapes;
 * mprk_create captures with the table's. Synchronises. Errors: MPRK_EINVAL,
 * MPRK_ECUDA. */
int mprk_tile_tune(mprk_instance* const* insts, int count, int reps, int* entries);

/* The table's tile shape for a single-instance FP64 stage launch of `cells`
 * cells: writes it (tile rows 8, 4 or 2; threads per cell 1 or 2) and
 * returns 1, or returns 0 when the table has none (the default rule
 * applies). Needs no device. */
int mprk_tile_lookup(double cells, int* tile_rows, int* threads_per_cell);

/* Save the table to a JSON file, {"gpu": <device name>, "entries": [...]}, or
 * replace it from one. Loading a table measured on a GPU of another name
 * fails with MPRK_EINVAL when a device is present. mprk_tune_clear empties
 * the table. No device is needed to save or clear. */
int mprk_tune_save(const char* path);
int mprk_tune_load(const char* path);
int mprk_tune_clear(void);

/* Test hook for the bounded waits of mprk_step_batch: one batched slow step
 * of the persistent form (in either precision) in which the tiles of stage
 * `stage` of instance inst_index never report completion, and each wait
 * gives up after wait_cycles clock cycles. The waiting tiles give up, set
 * the timeout bit and drain; nothing hangs. */
int mprk_batch_test_withhold(mprk_instance* const* insts, int count, int inst_index, int stage,
                             long long wait_cycles);

/* Copy the current state q_n to q_out ([4][nz][nx], location MPRK_HOST or
 * MPRK_DEVICE). Synchronises the instance stream. */
int mprk_get_state(mprk_instance* inst, double* q_out, int location);

/* Replace the state (checkpoint restore; the step counter is kept by the
 * caller). Synchronises. */
int mprk_set_state(mprk_instance* inst, const double* q, int location);

/* Run `count` independent solves of one slow step each through host
 * memory: for j = 0 .. count-1, set the state from q_in[j], advance one slow
 * step, and copy the result to q_out[j]. All buffers are host memory in the
 * layout of mprk_get_state ([4][nz][nx] doubles; [5][nz][ny][nx] in 3-D),
 * owned by the caller; q_out[j] may alias q_in[j'] only for j' <= j. The
 * results are bitwise those of mprk_set_state, mprk_step(inst, 1) and
 * mprk_get_state in turn. The host copies run on two copy streams of the
 * instance: q_in[j+1] is uploaded while step j runs, and q_out[j]
 * downloads while step j+1 runs. Page-locked host buffers are needed for the overlap; pageable ones
 * give the same results without it. The first call allocates two
 * state-sized device staging buffers, kept until mprk_destroy. The state
 * left in the instance is the last result. Returns after q_out[count-1] is
 * written; MPRK_EINVAL for a NULL pointer or count < 0. The paper has no
 * counterpart: this is host plumbing around the slow step of Algorithm 1. */
int mprk_step_io(mprk_instance* inst, const double* const* q_in, double* const* q_out, int count);

/* Monitoring quantities of the current state (Sec. 5.1), computed on the
 * device in a fixed order: out[0..3] sums of rho, rho u, rho w, rho E times
 * the cell area over fluid 1, out[4..7] over fluid 2, out[8..10] Courant
 * numbers of S, B and F ((max(|u|,|w|)+a) dt_region / min(dx, dz)),
 * out[11] count of non-finite entries, out[12] minimum density, out[13]
 * minimum pressure, out[14] slow steps taken, out[15] dt. In 3-D: out[0..4]
 * sums of rho, rho u, rho v, rho w, rho E times the cell volume over fluid 1,
 * out[5..9] over fluid 2, out[10..12] the Courant numbers
 * ((max(|u|,|v|,|w|)+a) dt_region / min(dx, dy, dz)), out[13] non-finite
 * entries, out[14] minimum density, out[15] minimum pressure. Synchronises. */
int mprk_diagnostics(mprk_instance* inst, double out[16]);

/* Wait for the instance's queued work. */
int mprk_sync(mprk_instance* inst);

/* Status word of the instance: 0, or MPRK_ENONFINITE / MPRK_ECFL /
 * MPRK_ETIMEOUT if monitoring or a batched launch flagged it. Synchronises. */
int mprk_status(mprk_instance* inst);

/* Read-only facts: dt, the number of cell right-hand-side evaluations per
 * slow step (nx ny (2 nz_S + 2 m (nz_B + nz_F)) for MPRK2, Sec. 4), device bytes
 * held, and the CUDA stream. Any out pointer may be NULL. */
int mprk_info(const mprk_instance* inst, double* dt, long long* cell_stages_per_step,
              long long* device_bytes, void** cuda_stream);

/* Test hook: the semi-discrete right-hand side R(W) (Sec. 2.1, App. B) for
 * rows [k_lo, k_hi) of a full state W, computed by the same kernel and
 * precision as the step. W_dev and R_dev are device buffers [4][nz][nx];
 * rows of R outside [k_lo, k_hi) are left untouched. Asynchronous. */
int mprk_rhs(mprk_instance* inst, const double* W_dev, double* R_dev, int k_lo, int k_hi);

/* Timing hook: run one slow step (it advances the state) as a CUDA graph
 * captured like the one mprk_step replays, with an event record node before
 * the first launch and after every launch, on the instance stream.
 * launch_ms[j] receives the duration of launch j and launch_cells[j] the
 * cell right-hand-side evaluations it made (0 for the step completion); the
 * launches are the s*m stages in order (s = 2 for the Heun base), then the
 * completion. Returns the
 * number of launches (at most cap are written) or a negative error code.
 * Synchronises. */
int mprk_profile_step(mprk_instance* inst, double* launch_ms, long long* launch_cells, int cap);

/* Measurement hook: the FP64 fused multiply-add throughput of the current
 * device, the denominator of the FP64 path's arithmetic roofline (the RHS
 * of Sec. 2.1 and App. B is FP64-arithmetic-bound in the FP64 mode).
 * Register-only kernels run independent FMA chains per thread (16 chains
 * of `iters` steps, or 8 of 2 iters; multiplier and addend in registers or
 * literals; 1 <= iters <= 2^30) on one full wave of 256-thread CTAs (as
 * many as fit on each SM), and the fastest of the four is reported. Each
 * CTA times its loop in SM clocks and on the global nanosecond timer. Outputs: gflops (2 flop per FMA, every FMA over
 * the span from the first CTA's start to the last CTA's end),
 * dfma_per_clk_per_sm (that rate per SM clock), sm_mhz (the median over the
 * CTAs of their clocks per nanosecond), sms (the SM count) and max_mhz (the
 * device's peak SM clock, cudaDevAttrClockRate). Allocates and frees three
 * small device buffers; synchronises. Errors: MPRK_EINVAL, MPRK_ECUDA. */
int mprk_probe_fp64(long long iters, double* gflops, double* dfma_per_clk_per_sm, double* sm_mhz, int* sms,
                    double* max_mhz);

/* Test hook for the FP32-flux mode's conversions, which use integer bit
 * operations because this GPU converts between float and double at the FP64
 * rate. For n device doubles in_dev[j] it writes the bit-operation
 * round-to-nearest narrowing and the hardware cast (float), and the
 * bit-operation and hardware widening of (float)in_dev[j] (double). All
 * buffers are device memory of n entries. Runs on the default stream and
 * synchronises. */
int mprk_selftest_convert(const double* in_dev, int n, float* narrow_dev, float* narrow_hw_dev,
                          double* widen_dev, double* widen_hw_dev);

/* Test hook for the FP64 tiles' 1/x, 1/sqrt(x) and sqrt(x): the hardware's
 * approximate reciprocal and reciprocal square root refined by one
 * third-order Householder step, within about one unit in the last place of
 * the exact values (not correctly rounded). For n device doubles in_dev[j]
 * it writes those three results to recip_dev, rsqrt_dev and sqrt_dev (device
 * buffers of n doubles each). Runs on the default stream and synchronises.
 * Errors: MPRK_EINVAL (null buffer, n < 0), MPRK_ECUDA. */
int mprk_selftest_recip(const double* in_dev, int n, double* recip_dev, double* rsqrt_dev, double* sqrt_dev);

/* ---- allocation-free stepping ------------------------------------------ */
/* Largest scratch mprk_step_static may use: 32 MiB. In FP64 a grid needs
 * 8 bytes x 4 components x (2 nx nz + nx (nz_S + nz_B)), each part rounded
 * up to 256 bytes; that is about 350,000 cells, e.g. 512 x 512. */
#define MPRK_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* Advance a state the caller already holds on the device by n_slow_steps
 * slow steps, in place, without allocating any memory. The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc. Examples
 * are code inside another framework's memory pool or allocator, processes
 * that reserve all device memory up front, and real-time loops where an
 * allocation could block or fail mid-run.
 *
 * q_dev: device buffer [4][nz][nx] of double (the layout above), read and
 * overwritten; the caller owns it. cfg: as for mprk_create, but dt must be
 * given (> 0); diag_every is ignored. cuda_stream: the cudaStream_t to run
 * on (NULL = the default stream). Asynchronous: the result is in q_dev once
 * the stream reaches this work. In FP64 it matches mprk_step on the same
 * input to rounding (the parity bound 1e-12 per component; in practice
 * bitwise). In the FP32-flux mode it agrees with mprk_step within that
 * mode's 1e-5: each call rebuilds the mode's per-row reference state and
 * float shadow from the q_dev it is given, while an instance keeps the
 * reference of its initial state. The FP32-flux mode also needs nx to be a
 * multiple of 32 and q_dev to be 256-byte aligned (every row of the
 * unpadded state on a 256-byte boundary, the layouts its tensor copies and
 * 16-byte accesses were tested on); other layouts get MPRK_EINVAL.
 *
 * Scratch comes from one fixed array of MPRK_STATIC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits. A configuration
 * needing more is rejected with MPRK_EINVAL and a message giving both sizes.
 * The function never calls cudaMalloc, cudaFree or any allocating routine.
 * Its first call on a device (with that device current) looks up the
 * array's device address and sets the kernels' shared-memory limits; make
 * that first call before any stream capture on the device. The address is
 * kept per device and CUDA context, so a call after cudaDeviceReset (a new
 * context) looks it up again, and is then also a first call. All calls on a
 * device share the array, which keeps the last call's contents, so calls
 * whose work overlaps on the GPU race and give undefined results: serialise
 * them (one stream, or events). No scratch entry is read before the call
 * writes it, so nothing is cleared between calls. Errors: MPRK_EINVAL,
 * MPRK_ECUDA; the message is in mprk_last_error(). */
int mprk_step_static(const mprk_config* cfg, double* q_dev, int n_slow_steps, void* cuda_stream);

/* ---- serving ----------------------------------------------------------- */
typedef struct mprk_server mprk_server;

typedef struct {
  long long hbm_budget_bytes; /* device bytes the resident instances may hold */
  int max_slots;              /* most instances resident at once              */
  int device;                 /* CUDA device ordinal                         */
  int max_queue;              /* queued requests beyond which submit is EBUSY */
  int solo_cells;             /* instances of at least this many cells step by
                                 their own stage launches on side streams, not
                                 in the batched launch: 0 = the default
                                 (MPRK_SOLO_CELLS_DEFAULT for FP64 requests;
                                 FP32-flux requests all batched), -1 = never */
} mprk_server_config;

/* 2^18 cells, e.g. 512 x 512: from there on an instance's stage launches
 * cover the GPU's SMs about once or more, and its own kernels beat the
 * persistent batch kernel. The per-stage form of FP32-flux batches runs
 * such instances within the batch about as fast, with lower latency for
 * the mix (measured), so the default applies to FP64 requests only. */
#define MPRK_SOLO_CELLS_DEFAULT 262144

#define MPRK_REQ_PENDING 1 /* queued, not admitted          */
#define MPRK_REQ_RUNNING 2 /* resident on the device         */
#define MPRK_REQ_DONE 3    /* finished; result ready to read */

typedef struct {
  double t_submit;        /* seconds on the server's clock (starts at create) */
  double t_admit;
  double t_finish;
  long long cell_stages;  /* cell right-hand-side evaluations done            */
  long long device_bytes; /* bytes the request held while resident           */
  int steps_done;
  int error;              /* 0 or an MPRK_E* code for this request           */
} mprk_stats;

/* Start a server thread on a device. It admits queued requests in arrival
 * order while a slot is free and the HBM ledger has room, advances all
 * resident instances together by one slow step at a time (the batched step
 * of mprk_step_batch per precision, in the form the tuning table picks, for
 * the instances below cfg->solo_cells cells; the larger ones by the same stage kernels as
 * mprk_step, on side streams that run beside each other), and retires each
 * request when it reaches its step count. Either way a request's result is
 * that of the same solve alone: bitwise in FP64, within float rounding in
 * FP32 flux (bitwise for the instances stepped alone). Requests join and
 * leave between slow steps while the others keep running (continuous
 * batching). Uploads and downloads run on a copy stream that overlaps the
 * compute stream, and instance memory is stream-ordered (cudaMallocAsync and
 * cudaFreeAsync). Errors: MPRK_EINVAL, MPRK_ECUDA. */
int mprk_server_create(const mprk_server_config* cfg, mprk_server** out);

/* Queue a solve of n_slow_steps from q0_host ([4][nz][nx], copied before
 * return); cfg->dt == 0 picks dt at admission as mprk_create does.
 * Non-blocking. Returns MPRK_EBUDGET if
 * the instance can never fit the budget, MPRK_EBUSY if the queue is full,
 * MPRK_EINVAL for a bad configuration. A non-finite or non-positive q0 is
 * reported later as that request's MPRK_ENONFINITE. */
int mprk_submit(mprk_server* srv, const mprk_config* cfg, const double* q0_host, int n_slow_steps,
                uint64_t* ticket);

/* Non-blocking status of a ticket: *status is MPRK_REQ_PENDING, _RUNNING or
 * _DONE. When DONE and q_out_host is non-null, the final state is copied
 * there ([4][nz][nx]) and the ticket is released. stats may be NULL. Returns
 * the request's error code (0 if none) or MPRK_ENOTFOUND. */
int mprk_poll(mprk_server* srv, uint64_t ticket, int* status, double* q_out_host,
              mprk_stats* stats);

/* Server-wide counters: out[0] requests done, out[1] cell stages done,
 * out[2] batched slow steps launched, out[3] resident now, out[4] queued now,
 * out[5] ledger bytes now, out[6] seconds since start, out[7] failed requests. */
int mprk_server_stats(mprk_server* srv, double out[8]);

/* Where the server thread's time goes, accumulated since the server started:
 * out[0] loop iterations that launched a batched step, out[1] seconds
 * admitting requests (instance creation: allocation, upload, reference
 * set-up, initial check), out[2] seconds enqueueing the batched steps
 * (including work-list rebuilds when the resident set changed), out[3]
 * seconds retiring finished requests, out[4] seconds waiting for the step
 * two iterations back (the in-flight limit), out[5] GPU seconds of the
 * batched steps (CUDA events around each iteration's launches), out[6]
 * seconds from the first batched step to the last one's end, out[7]
 * requests admitted. The paper has no counterpart; this is instrumentation
 * of the request loop. */
int mprk_server_profile(mprk_server* srv, double out[8]);

/* Stop the server thread (queued and resident requests are dropped) and free
 * its resources. */
int mprk_server_destroy(mprk_server* srv);

/* ---- errors ------------------------------------------------------------ */
/* Message for the last failing call on this thread ("" if none). */
const char* mprk_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
