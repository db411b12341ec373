/*
 * mprk_oracle3d.h — the oracle in three dimensions: App. B of Kang, Dener,
 * Hamilton, Zhang, Constantinescu, Jacob (arXiv 2202.11890), Eq.
 * ns-fv-cartesian-3d in full, with the MPRK2 slow step of Algorithm 1.
 *
 * TEST INFRASTRUCTURE, like mprk_oracle.h: only the tests, the smoke check
 * and the benchmark's CPU legs load it; it shares nothing with the CUDA path.
 *
 * Layout of every state array: [5][nz][ny][nx], contiguous, components
 * (rho, rho u, rho v, rho w, rho E); rows bottom to top as in 2-D (S, B, F
 * bands; Gamma between the top B row and the bottom F row); x and y periodic.
 */
#ifndef MPRK_ORACLE3D_H
#define MPRK_ORACLE3D_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nS, nB, nF; /* columns in x and y; rows of the S, B and F bands */
  int m;                  /* rate ratio                                        */
  int wall;               /* outer z walls: 0 no-slip, 1 slip (adiabatic)      */
  int pad_;
  double dt;              /* slow step                                         */
  double dx, dy, dz1, dz2;
  double gamma, Pr, mu1, mu2, G;
} or3_problem;

/* R(W) of Eq. ns-fv-cartesian-3d for rows [k_lo, k_hi); other rows of R
 * are left untouched. */
int or3_rhs(const or3_problem* P, const double* W, double* R, int k_lo, int k_hi);

/* One MPRK2 slow step (Algorithm 1, full stage arrays) in place on q. */
int or3_mprk_step(const or3_problem* P, double* q);

/* Single-rate Heun (base RK2) and classical RK4 over the whole grid. */
int or3_rk2_step(const or3_problem* P, double* q, double h);
int or3_rk4_step(const or3_problem* P, double* q, double h);

/* out[0..4] = sums of (rho, rho u, rho v, rho w, rho E) times |K| over
 * fluid 1, out[5..9] over fluid 2, out[10..12] = Courant numbers of S, B, F
 * (max(|u|,|v|,|w|) + a over the region times its step over min(dx, dy,
 * dz)), out[13] = non-finite entries, out[14] = minimum density, out[15] =
 * minimum pressure. */
int or3_diagnostics(const or3_problem* P, const double* q, double out[16]);

/* dt for Courant number cfl in every region (fast band at step dt/m). */
double or3_stable_dt(const or3_problem* P, const double* q, double cfl);

/* Interface state of column (i, j): out = {sigma_xz, sigma_yz, Pi_z, u_w1,
 * v_w1, T_w1, u_w2, v_w2, T_w2} (App. B, Eq. bulk-flux and the wall states). */
int or3_interface_state(const or3_problem* P, const double* W, int j, int i, double out[9]);

/* Lax–Friedrichs flux of Sec. 2.1 in direction d (0 x, 1 y, 2 z). */
void or3_lf_flux(const double ql[5], const double qr[5], int d, double gamma, double F[5]);

#ifdef __cplusplus
}
#endif
#endif
