/*
 * mprk_oracle.h — plain FP64 CPU oracle for one slow step of the multirate
 * partitioned Runge–Kutta method MPRK2 (Kang, Dener, Hamilton, Zhang,
 * Constantinescu, Jacob: "Multirate Partitioned Runge–Kutta Methods for
 * Coupled Navier–Stokes Equations", arXiv 2202.11890).
 *
 * TEST INFRASTRUCTURE. This oracle exists only to check the CUDA library.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it. It shares no code, header, table or helper with the CUDA path.
 *
 * Parity status: every function below is pinned by a CPU test against a
 * fact the paper or the mathematics fixes (Table 1, closed forms, textbook
 * fluxes, conservation, a 50-digit hand expansion, convergence order).
 *
 * Layout of every state array: structure of arrays [4][nz][nx], contiguous,
 * components (rho, rho*u, rho*w, rho*E), rows bottom to top: the slow band S
 * (rows 0..nS-1), the buffer band B (nS..nS+nB-1), the fast band F (the rest).
 * S and B hold fluid 1 (ocean), F holds fluid 2 (atmosphere); the interface
 * Gamma lies between the top B row and the bottom F row. x is periodic.
 */
#ifndef MPRK_ORACLE_H
#define MPRK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_REGION_S = 0, OR_REGION_B = 1, OR_REGION_F = 2 };
enum { OR_WALL_NOSLIP = 0, OR_WALL_SLIP = 1 };
enum { OR_RHS_NS = 0, OR_RHS_LINEAR = 1 };

typedef struct {
  int nx, nS, nB, nF;  /* columns; rows of the S, B and F bands                */
  int m;               /* rate ratio: slow step = m fast steps (Sec. 3)          */
  int wall;            /* outer walls: OR_WALL_NOSLIP or OR_WALL_SLIP (adiabatic) */
  int rhs_mode;        /* OR_RHS_NS, or OR_RHS_LINEAR (R = lin_lambda*q, tests)  */
  int xwall;           /* 0: x periodic; 1: walls of the same kind at both x ends
                        * (Sec. 5.2, walls on all boundaries)                    */
  double dt;           /* slow step Delta t                                     */
  double dx, dz1, dz2; /* cell sizes: x, fluid-1 rows, fluid-2 rows             */
  double gamma, Pr;    /* ratio of specific heats, Prandtl number               */
  double mu1, mu2;     /* nondimensional viscosities mu~ of fluid 1 and 2        */
  double G;            /* gravity magnitude; source (0,0,-rho G,-rho w G)        */
  double lin_lambda;   /* only for OR_RHS_LINEAR                                */
} or_problem;

/* Butcher tableau of region (S, B or F) of MPRK2 with base RK2 (s = 2) and
 * rate ratio m; a is (2m)x(2m) row-major, b and c have 2m entries. */
int or_tableau(int m, int region, double* a, double* b, double* c);

/* Semi-discrete right-hand side R(W) of the finite-volume scheme (Sec. 2.1,
 * App. B) for rows [k_lo, k_hi) of the composite state W; other rows of R are
 * left untouched. */
int or_rhs(const or_problem* P, const double* W, double* R, int k_lo, int k_hi);

/* One MPRK2 slow step (Eq. MRK2, Algorithm 1) in place on q. If rhs_cells is
 * non-null it receives the number of cell right-hand-side evaluations. */
int or_mprk_step(const or_problem* P, double* q, long long* rhs_cells);

/* The same step, keeping every stage: Q and R are [2m][4][nz][nx]. Rows of R
 * that a stage does not evaluate are set to zero. */
int or_mprk_step_trace(const or_problem* P, const double* q, double* Q, double* R,
                       double* q_next);

/* MPRK with a general s-stage base method (A s x s row-major, b, c; the
 * Sec. 3 remark): the region tableaus built from the base as Table 1 builds
 * them from RK2 (or_tableau's entries for Heun's base), one slow step, and
 * the base method alone over the whole grid. */
int or_tableau_base(int m, int region, int s, const double* A, const double* b, const double* c, double* a_out,
                    double* b_out, double* c_out);
int or_mprk_step_base(const or_problem* P, int s, const double* A, const double* b, const double* c, double* q);
int or_rk_step_base(const or_problem* P, int s, const double* A, const double* b, double* q, double h);

/* Single-rate base RK2 (Heun, Table 1 "Base RK2") over the whole grid, step h. */
int or_rk2_step(const or_problem* P, double* q, double h);

/* Classical fourth-order Runge–Kutta over the whole grid, step h (reference
 * solutions for the convergence tests only). */
int or_rk4_step(const or_problem* P, double* q, double h);

/* Monitoring quantities (Sec. 5.1): out[0..3] = sums of rho, rho u, rho w,
 * rho E times |K| over fluid 1; out[4..7] over fluid 2; out[8..10] = Courant
 * numbers of S, B, F; out[11] = count of non-finite entries; out[12] = minimum
 * density; out[13] = minimum pressure; out[14..15] = 0. */
int or_diagnostics(const or_problem* P, const double* q, double out[16]);

/* Slow step for a Courant number cfl: cfl*min(dx,dz1,dz2)/max(|u|,|w|)+a. */
double or_stable_dt(const or_problem* P, const double* q, double cfl);

/* Pieces exposed for the pins. d = 0 for an x face, 1 for a z face. */
void or_euler_flux(const double q[4], int d, double gamma, double F[4]);
void or_lf_flux(const double ql[4], const double qr[4], int d, double gamma, double F[4]);
/* Interface wall states of column i (App. B): out = {sigma_xz, Pi_z, u_w1,
 * T_w1, u_w2, T_w2}. */
int or_interface_state(const or_problem* P, const double* W, int i, double out[6]);

/* Cell right-hand-side evaluations made by or_rhs so far (a counter). */
long long or_rhs_cell_count(void);

/* OpenMP threads used by or_rhs (1 = serial). Results do not depend on it. */
void or_set_threads(int n);
int or_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
