/*
 * mprk_oracle.c — plain FP64 CPU oracle for one MPRK2 slow step.
 *
 * TEST INFRASTRUCTURE ONLY: it checks the CUDA library and is never part of
 * the product path. It shares no code with the CUDA sources. Build it with
 * -O2 -ffp-contract=off so that every operation is rounded as written.
 *
 * Paper: Kang, Dener, Hamilton, Zhang, Constantinescu, Jacob, "Multirate
 * Partitioned Runge–Kutta Methods for Coupled Navier–Stokes Equations"
 * (arXiv 2202.11890). Section, equation, table and algorithm names below are
 * the paper's.
 *
 * The 2-D x–z scheme is App. B with the y direction dropped:
 *   dq/dt = -(F*_{i+1/2} - F*_{i-1/2})/dx - (H*_{k+1/2} - H*_{k-1/2})/dz + s,
 * F* = F^{I*} - F^{V*}, with the Lax–Friedrichs inviscid flux of Sec. 2.1,
 * linear reconstruction of conserved variables from central-difference cell
 * gradients (App. B), and the viscous flux from common face values (App. B).
 *
 * Readings where the paper is silent (each one is a choice of this oracle):
 *  - beyond a wall or the interface the conserved-variable slope uses a mirror
 *    ghost (rho, rho u, rho E even; rho w odd);
 *  - u, w, T slopes there use a ghost equal to 2*(wall state) - (interior);
 *    outer walls are adiabatic (T ghost = T), no-slip (u_w = w_w = 0) or slip
 *    (u ghost = u, w_w = 0); at the interface the wall state is (u_w, 0, T_w)
 *    of App. B, each fluid using its own formula;
 *  - the inviscid flux through a wall or the interface is the Lax–Friedrichs
 *    flux between the reconstructed boundary state and its mirror;
 *  - the viscous flux through an outer wall is the common-value recipe of
 *    App. B applied between the cell and its ghost;
 *  - x walls (xwall = 1; Sec. 5.2 puts adiabatic no-slip walls on all
 *    boundaries) follow the z-wall rules with x as the normal: the mirror
 *    ghost flips rho u, and the (u, w, T) ghost flips u, flips w for no-slip
 *    and keeps it for slip;
 *  - the viscous flux through the interface is (0, sigma_xz, 0,
 *    u_w*sigma_xz - Pi_z) from the bulk formulas of App. B (w = 0,
 *    sigma_zz = 0);
 *  - the heat flux is Pi = -kappa grad T (Sec. 2, the physical sign);
 *  - gravity: source (0, 0, -rho G, -rho w G) with G > 0 (Sec. 2, Eq.
 *    cns-gov with g pointing down).
 */
#include "mprk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;
/* cell right-hand-side evaluations made by or_rhs since the library loaded */
static long long g_rhs_cells = 0;

void or_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int or_get_threads(void) { return g_threads; }
long long or_rhs_cell_count(void) { return g_rhs_cells; }

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static int nz_of(const or_problem* P) { return P->nS + P->nB + P->nF; }
/* rows of fluid 1 (the ocean: S and B bands) */
static int n1_of(const or_problem* P) { return P->nS + P->nB; }

static size_t at(const or_problem* P, int c, int k, int i) {
  return ((size_t)c * (size_t)nz_of(P) + (size_t)k) * (size_t)P->nx + (size_t)i;
}

static int fluid_of(const or_problem* P, int k) { return k < n1_of(P) ? 1 : 2; }
static double dz_of(const or_problem* P, int k) { return fluid_of(P, k) == 1 ? P->dz1 : P->dz2; }
static double mu_of_fluid(const or_problem* P, int f) { return f == 1 ? P->mu1 : P->mu2; }
/* kappa~ = c~_p mu~ / Pr with c~_p = 1/(gamma-1) (App. A) */
static double kappa_of_fluid(const or_problem* P, int f) {
  double cp = 1.0 / (P->gamma - 1.0);
  return cp * mu_of_fluid(P, f) / P->Pr;
}
static int wrap(const or_problem* P, int i) { return ((i % P->nx) + P->nx) % P->nx; }

static void load(const or_problem* P, const double* W, int k, int i, double q[4]) {
  for (int c = 0; c < 4; c++) q[c] = W[at(P, c, k, i)];
}

/* ------------------------------------------------------------------------ */
/* Thermodynamics (Sec. 2 and App. A): p = (gamma-1)(rho E - rho|u|^2/2),     */
/* T = gamma p / rho, a = sqrt(gamma p / rho), H = (rho E + p)/rho            */
/* ------------------------------------------------------------------------ */

typedef struct { double rho, u, w, p, T, a, H; } prim;

static prim to_prim(const double q[4], double gamma) {
  prim s;
  s.rho = q[0];
  s.u = q[1] / q[0];
  s.w = q[2] / q[0];
  s.p = (gamma - 1.0) * (q[3] - 0.5 * q[0] * (s.u * s.u + s.w * s.w));
  s.T = gamma * s.p / q[0];
  s.a = sqrt(gamma * s.p / q[0]);
  s.H = (q[3] + s.p) / q[0];
  return s;
}

/* Inviscid flux of the state q in direction d (0: x, 1: z): App. B, the F^I
 * and H^I columns restricted to (rho, rho u, rho w, rho E). */
void or_euler_flux(const double q[4], int d, double gamma, double F[4]) {
  prim s = to_prim(q, gamma);
  double un = d == 0 ? s.u : s.w;
  F[0] = q[0] * un;
  F[1] = q[1] * un + (d == 0 ? s.p : 0.0);
  F[2] = q[2] * un + (d == 1 ? s.p : 0.0);
  F[3] = q[0] * un * s.H;
}

/* Lax–Friedrichs numerical flux (Sec. 2.1): 1/2 (F(ql)+F(qr)).n +
 * lambda/2 (ql - qr), lambda = max of |u.n|+a over ql, qr and their Roe
 * average (Roe averages: sqrt(rho)-weighted u, w, H; a~^2 = (gamma-1)(H~ -
 * |u~|^2/2)). */
void or_lf_flux(const double ql[4], const double qr[4], int d, double gamma, double F[4]) {
  double Fl[4], Fr[4];
  or_euler_flux(ql, d, gamma, Fl);
  or_euler_flux(qr, d, gamma, Fr);
  prim L = to_prim(ql, gamma), R = to_prim(qr, gamma);
  double sl = sqrt(L.rho), sr = sqrt(R.rho);
  double ur = (sl * L.u + sr * R.u) / (sl + sr);
  double wr = (sl * L.w + sr * R.w) / (sl + sr);
  double Hr = (sl * L.H + sr * R.H) / (sl + sr);
  double ar = sqrt((gamma - 1.0) * (Hr - 0.5 * (ur * ur + wr * wr)));
  double unl = d == 0 ? L.u : L.w;
  double unr = d == 0 ? R.u : R.w;
  double unroe = d == 0 ? ur : wr;
  double lam = fmax(fabs(unl) + L.a, fmax(fabs(unr) + R.a, fabs(unroe) + ar));
  for (int c = 0; c < 4; c++) F[c] = 0.5 * (Fl[c] + Fr[c]) + 0.5 * lam * (ql[c] - qr[c]);
}

/* ------------------------------------------------------------------------ */
/* Interface wall states (App. B, Eq. bulk-flux and the wall states after it) */
/* ------------------------------------------------------------------------ */

int or_interface_state(const or_problem* P, const double* W, int i, double out[6]) {
  int k1 = n1_of(P) - 1, k2 = n1_of(P);
  double q1[4], q2[4];
  load(P, W, k1, i, q1);
  load(P, W, k2, i, q2);
  prim c1 = to_prim(q1, P->gamma), c2 = to_prim(q2, P->gamma);
  double mu1 = P->mu1, mu2 = P->mu2;
  double ka1 = kappa_of_fluid(P, 1), ka2 = kappa_of_fluid(P, 2);
  double dz1 = P->dz1, dz2 = P->dz2;
  double bu = 2.0 * mu1 * mu2 / (dz2 * mu1 + dz1 * mu2);
  double bT = 2.0 * ka1 * ka2 / (dz2 * ka1 + dz1 * ka2);
  double sxz = bu * (c2.u - c1.u);
  double Piz = -bT * (c2.T - c1.T);
  out[0] = sxz;
  out[1] = Piz;
  out[2] = c1.u + sxz * dz1 / (2.0 * mu1);
  out[3] = c1.T - Piz * dz1 / (2.0 * ka1);
  out[4] = c2.u - sxz * dz2 / (2.0 * mu2);
  out[5] = c2.T + Piz * dz2 / (2.0 * ka2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Neighbours with ghost rules                                                */
/* ------------------------------------------------------------------------ */

/* Is row k+s outside the fluid of row k (beyond an outer wall or Gamma)? */
static int beyond(const or_problem* P, int k, int s) {
  int kk = k + s;
  if (kk < 0 || kk >= nz_of(P)) return 1;
  return fluid_of(P, kk) != fluid_of(P, k);
}
static int beyond_gamma(const or_problem* P, int k, int s) {
  int kk = k + s;
  return kk >= 0 && kk < nz_of(P) && fluid_of(P, kk) != fluid_of(P, k);
}

/* conserved neighbour of (k,i) in z at offset s, mirror ghost beyond a boundary */
static void nb_cons_z(const or_problem* P, const double* W, int k, int i, int s, double q[4]) {
  if (!beyond(P, k, s)) {
    load(P, W, k + s, i, q);
  } else {
    load(P, W, k, i, q);
    q[2] = -q[2];
  }
}

/* (u, w, T) of the z-neighbour of (k,i) at offset s; beyond a boundary the
 * ghost is 2*(wall state) - (interior value). */
static void nb_uwT_z(const or_problem* P, const double* W, int k, int i, int s, double v[3]) {
  double q[4];
  if (!beyond(P, k, s)) {
    load(P, W, k + s, i, q);
    prim c = to_prim(q, P->gamma);
    v[0] = c.u; v[1] = c.w; v[2] = c.T;
    return;
  }
  load(P, W, k, i, q);
  prim c = to_prim(q, P->gamma);
  if (beyond_gamma(P, k, s)) {
    double st[6];
    or_interface_state(P, W, i, st);
    double uw = fluid_of(P, k) == 1 ? st[2] : st[4];
    double Tw = fluid_of(P, k) == 1 ? st[3] : st[5];
    v[0] = 2.0 * uw - c.u;
    v[1] = -c.w;
    v[2] = 2.0 * Tw - c.T;
  } else if (P->wall == OR_WALL_SLIP) {
    v[0] = c.u;
    v[1] = -c.w;
    v[2] = c.T;
  } else {
    v[0] = -c.u;
    v[1] = -c.w;
    v[2] = c.T;
  }
}

/* Is column i+s beyond an x wall? */
static int beyond_x(const or_problem* P, int i, int s) {
  return P->xwall && (i + s < 0 || i + s >= P->nx);
}

/* conserved neighbour of (k,i) in x at offset s: periodic, or the mirror
 * ghost (rho u flipped) beyond an x wall */
static void nb_cons_x(const or_problem* P, const double* W, int k, int i, int s, double q[4]) {
  if (!beyond_x(P, i, s)) {
    load(P, W, k, wrap(P, i + s), q);
  } else {
    load(P, W, k, i, q);
    q[1] = -q[1];
  }
}

/* Cell gradients by central differences (App. B, LS gradient on a uniform grid) */
static void grad_x_cons(const or_problem* P, const double* W, int k, int i, double g[4]) {
  double qe[4], qw[4];
  nb_cons_x(P, W, k, i, +1, qe);
  nb_cons_x(P, W, k, i, -1, qw);
  for (int c = 0; c < 4; c++) g[c] = (qe[c] - qw[c]) / (2.0 * P->dx);
}
static void grad_z_cons(const or_problem* P, const double* W, int k, int i, double g[4]) {
  double qn[4], qs[4];
  nb_cons_z(P, W, k, i, +1, qn);
  nb_cons_z(P, W, k, i, -1, qs);
  for (int c = 0; c < 4; c++) g[c] = (qn[c] - qs[c]) / (2.0 * dz_of(P, k));
}
static void uwT_at(const or_problem* P, const double* W, int k, int i, double v[3]) {
  double q[4];
  load(P, W, k, i, q);
  prim c = to_prim(q, P->gamma);
  v[0] = c.u; v[1] = c.w; v[2] = c.T;
}
/* (u, w, T) of the x-neighbour of (k,i) at offset s; beyond an x wall the
 * ghost is 2*(wall state) - (interior value): u flips (normal), w flips for
 * no-slip and stays for slip, T stays (adiabatic) */
static void nb_uwT_x(const or_problem* P, const double* W, int k, int i, int s, double v[3]) {
  if (!beyond_x(P, i, s)) {
    uwT_at(P, W, k, wrap(P, i + s), v);
    return;
  }
  uwT_at(P, W, k, i, v);
  v[0] = -v[0];
  if (P->wall != OR_WALL_SLIP) v[1] = -v[1];
}
static void grad_x_uwT(const or_problem* P, const double* W, int k, int i, double g[3]) {
  double ve[3], vw[3];
  nb_uwT_x(P, W, k, i, +1, ve);
  nb_uwT_x(P, W, k, i, -1, vw);
  for (int c = 0; c < 3; c++) g[c] = (ve[c] - vw[c]) / (2.0 * P->dx);
}
static void grad_z_uwT(const or_problem* P, const double* W, int k, int i, double g[3]) {
  double vn[3], vs[3];
  nb_uwT_z(P, W, k, i, +1, vn);
  nb_uwT_z(P, W, k, i, -1, vs);
  for (int c = 0; c < 3; c++) g[c] = (vn[c] - vs[c]) / (2.0 * dz_of(P, k));
}

/* ------------------------------------------------------------------------ */
/* Viscous flux from common face values (App. B)                              */
/* ------------------------------------------------------------------------ */

/* one side of a face: cell values of u, w, T and the tangential derivatives of
 * u and w at the cell centre */
typedef struct { double u, w, T, dut, dwt; } vside;

static void viscous_flux(const vside* L, const vside* R, int d, double dn, double mu, double kap,
                         double FV[4]) {
  double uh = 0.5 * (L->u + R->u);
  double wh = 0.5 * (L->w + R->w);
  double dun = (R->u - L->u) / dn;
  double dwn = (R->w - L->w) / dn;
  double dTn = (R->T - L->T) / dn;
  double dut = 0.5 * (L->dut + R->dut);
  double dwt = 0.5 * (L->dwt + R->dwt);
  if (d == 0) { /* x face: normal x, tangential z */
    double ux = dun, wx = dwn, Tx = dTn, uz = dut, wz = dwt;
    double sxx = mu * (2.0 * ux - (2.0 / 3.0) * (ux + wz));
    double sxz = mu * (uz + wx);
    FV[0] = 0.0;
    FV[1] = sxx;
    FV[2] = sxz;
    FV[3] = uh * sxx + wh * sxz + kap * Tx; /* u.sigma_x - Pi_x, Pi = -kappa grad T */
  } else { /* z face: normal z, tangential x */
    double uz = dun, wz = dwn, Tz = dTn, ux = dut, wx = dwt;
    double szz = mu * (2.0 * wz - (2.0 / 3.0) * (ux + wz));
    double sxz = mu * (uz + wx);
    FV[0] = 0.0;
    FV[1] = sxz;
    FV[2] = szz;
    FV[3] = uh * sxz + wh * szz + kap * Tz;
  }
}

/* ------------------------------------------------------------------------ */
/* Face fluxes F* = F^{I*} - F^{V*}                                           */
/* ------------------------------------------------------------------------ */

/* x face between (k,i) and (k,i+1) (periodic wrap when x is periodic) */
static void xface(const or_problem* P, const double* W, int k, int i, double F[4]) {
  int ip = wrap(P, i + 1);
  double qL[4], qR[4], gL[4], gR[4], ql[4], qr[4], FI[4], FV[4];
  load(P, W, k, i, qL);
  load(P, W, k, ip, qR);
  grad_x_cons(P, W, k, i, gL);
  grad_x_cons(P, W, k, ip, gR);
  for (int c = 0; c < 4; c++) {
    ql[c] = qL[c] + gL[c] * (P->dx / 2.0);
    qr[c] = qR[c] - gR[c] * (P->dx / 2.0);
  }
  or_lf_flux(ql, qr, 0, P->gamma, FI);
  double vL[3], vR[3], tL[3], tR[3];
  uwT_at(P, W, k, i, vL);
  uwT_at(P, W, k, ip, vR);
  grad_z_uwT(P, W, k, i, tL);
  grad_z_uwT(P, W, k, ip, tR);
  vside L = {vL[0], vL[1], vL[2], tL[0], tL[1]};
  vside R = {vR[0], vR[1], vR[2], tR[0], tR[1]};
  int f = fluid_of(P, k);
  viscous_flux(&L, &R, 0, P->dx, mu_of_fluid(P, f), kappa_of_fluid(P, f), FV);
  for (int c = 0; c < 4; c++) F[c] = FI[c] - FV[c];
}

/* z face between (k,i) and (k+1,i), both rows in the same fluid */
static void zface_interior(const or_problem* P, const double* W, int k, int i, double F[4]) {
  double dz = dz_of(P, k);
  double qL[4], qR[4], gL[4], gR[4], ql[4], qr[4], FI[4], FV[4];
  load(P, W, k, i, qL);
  load(P, W, k + 1, i, qR);
  grad_z_cons(P, W, k, i, gL);
  grad_z_cons(P, W, k + 1, i, gR);
  for (int c = 0; c < 4; c++) {
    ql[c] = qL[c] + gL[c] * (dz / 2.0);
    qr[c] = qR[c] - gR[c] * (dz / 2.0);
  }
  or_lf_flux(ql, qr, 1, P->gamma, FI);
  double vL[3], vR[3], tL[3], tR[3];
  uwT_at(P, W, k, i, vL);
  uwT_at(P, W, k + 1, i, vR);
  grad_x_uwT(P, W, k, i, tL);
  grad_x_uwT(P, W, k + 1, i, tR);
  vside L = {vL[0], vL[1], vL[2], tL[0], tL[1]};
  vside R = {vR[0], vR[1], vR[2], tR[0], tR[1]};
  int f = fluid_of(P, k);
  viscous_flux(&L, &R, 1, dz, mu_of_fluid(P, f), kappa_of_fluid(P, f), FV);
  for (int c = 0; c < 4; c++) F[c] = FI[c] - FV[c];
}

static void mirror(const double q[4], double g[4]) {
  g[0] = q[0]; g[1] = q[1]; g[2] = -q[2]; g[3] = q[3];
}

/* x wall on the left of column 0 (s = -1) or on the right of column nx-1
 * (s = +1): the z-wall construction with x as the normal direction. */
static void xface_wall(const or_problem* P, const double* W, int k, int i, int s, double F[4]) {
  double q[4], g[4], qb[4], qg[4], FI[4], FV[4];
  load(P, W, k, i, q);
  grad_x_cons(P, W, k, i, g);
  for (int c = 0; c < 4; c++) qb[c] = q[c] + (double)s * g[c] * (P->dx / 2.0);
  for (int c = 0; c < 4; c++) qg[c] = qb[c];
  qg[1] = -qb[1];
  if (s < 0) or_lf_flux(qg, qb, 0, P->gamma, FI);
  else or_lf_flux(qb, qg, 0, P->gamma, FI);
  /* viscous: the cell and its ghost (2*wall - interior; adiabatic) */
  double v[3], t[3];
  uwT_at(P, W, k, i, v);
  grad_z_uwT(P, W, k, i, t);
  vside C = {v[0], v[1], v[2], t[0], t[1]};
  vside Gh;
  Gh.u = -v[0]; Gh.dut = -t[0];
  if (P->wall == OR_WALL_SLIP) {
    Gh.w = v[1]; Gh.dwt = t[1];
  } else {
    Gh.w = -v[1]; Gh.dwt = -t[1];
  }
  Gh.T = v[2];
  int f = fluid_of(P, k);
  if (s < 0) viscous_flux(&Gh, &C, 0, P->dx, mu_of_fluid(P, f), kappa_of_fluid(P, f), FV);
  else viscous_flux(&C, &Gh, 0, P->dx, mu_of_fluid(P, f), kappa_of_fluid(P, f), FV);
  for (int c = 0; c < 4; c++) F[c] = FI[c] - FV[c];
}

/* Outer wall below row 0 (s = -1) or above the top row (s = +1). */
static void zface_wall(const or_problem* P, const double* W, int k, int i, int s, double F[4]) {
  double dz = dz_of(P, k);
  double q[4], g[4], qb[4], qg[4], FI[4], FV[4];
  load(P, W, k, i, q);
  grad_z_cons(P, W, k, i, g);
  for (int c = 0; c < 4; c++) qb[c] = q[c] + (double)s * g[c] * (dz / 2.0);
  mirror(qb, qg);
  if (s < 0) or_lf_flux(qg, qb, 1, P->gamma, FI);
  else or_lf_flux(qb, qg, 1, P->gamma, FI);
  /* viscous: the cell and its ghost (2*wall - interior; adiabatic) */
  double v[3], t[3];
  uwT_at(P, W, k, i, v);
  grad_x_uwT(P, W, k, i, t);
  vside C = {v[0], v[1], v[2], t[0], t[1]};
  vside Gh;
  if (P->wall == OR_WALL_SLIP) {
    Gh.u = v[0]; Gh.dut = t[0];
  } else {
    Gh.u = -v[0]; Gh.dut = -t[0];
  }
  Gh.w = -v[1]; Gh.dwt = -t[1];
  Gh.T = v[2];
  int f = fluid_of(P, k);
  if (s < 0) viscous_flux(&Gh, &C, 1, dz, mu_of_fluid(P, f), kappa_of_fluid(P, f), FV);
  else viscous_flux(&C, &Gh, 1, dz, mu_of_fluid(P, f), kappa_of_fluid(P, f), FV);
  for (int c = 0; c < 4; c++) F[c] = FI[c] - FV[c];
}

/* The interface Gamma as seen by fluid 1's top row (f = 1) or by fluid 2's
 * bottom row (f = 2). Inviscid: rigid lid (w^ = 0), a wall from each side;
 * viscous: the bulk fluxes of App. B. */
static void zface_gamma(const or_problem* P, const double* W, int i, int f, double F[4]) {
  int k = f == 1 ? n1_of(P) - 1 : n1_of(P);
  int s = f == 1 ? +1 : -1;
  double dz = dz_of(P, k);
  double q[4], g[4], qb[4], qg[4], FI[4];
  load(P, W, k, i, q);
  grad_z_cons(P, W, k, i, g);
  for (int c = 0; c < 4; c++) qb[c] = q[c] + (double)s * g[c] * (dz / 2.0);
  mirror(qb, qg);
  if (f == 1) or_lf_flux(qb, qg, 1, P->gamma, FI);
  else or_lf_flux(qg, qb, 1, P->gamma, FI);
  double st[6];
  or_interface_state(P, W, i, st);
  double sxz = st[0], Piz = st[1];
  double uw = f == 1 ? st[2] : st[4];
  double FV[4] = {0.0, sxz, 0.0, uw * sxz - Piz};
  for (int c = 0; c < 4; c++) F[c] = FI[c] - FV[c];
}

/* flux through the lower (s=-1) or upper (s=+1) z face of row k */
static void zflux_of_cell(const or_problem* P, const double* W, int k, int i, int s, double F[4]) {
  int nz = nz_of(P), n1 = n1_of(P);
  if (s < 0) {
    if (k == 0) zface_wall(P, W, k, i, -1, F);
    else if (k == n1) zface_gamma(P, W, i, 2, F);
    else zface_interior(P, W, k - 1, i, F);
  } else {
    if (k == nz - 1) zface_wall(P, W, k, i, +1, F);
    else if (k == n1 - 1) zface_gamma(P, W, i, 1, F);
    else zface_interior(P, W, k, i, F);
  }
}

/* ------------------------------------------------------------------------ */
/* Right-hand side (Sec. 2.1 Eq. cns-fv; App. B Eq. ns-fv-cartesian-3d in 2-D) */
/* ------------------------------------------------------------------------ */

static void rhs_cell(const or_problem* P, const double* W, int k, int i, double r[4]) {
  if (P->rhs_mode == OR_RHS_LINEAR) {
    for (int c = 0; c < 4; c++) r[c] = P->lin_lambda * W[at(P, c, k, i)];
    return;
  }
  double Fe[4], Fw[4], Hn[4], Hs[4], q[4];
  if (P->xwall && i == P->nx - 1) xface_wall(P, W, k, i, +1, Fe);
  else xface(P, W, k, i, Fe);
  if (P->xwall && i == 0) xface_wall(P, W, k, i, -1, Fw);
  else xface(P, W, k, wrap(P, i - 1), Fw);
  zflux_of_cell(P, W, k, i, +1, Hn);
  zflux_of_cell(P, W, k, i, -1, Hs);
  load(P, W, k, i, q);
  double dz = dz_of(P, k);
  double src[4] = {0.0, 0.0, -q[0] * P->G, -q[2] * P->G};
  for (int c = 0; c < 4; c++) r[c] = -(Fe[c] - Fw[c]) / P->dx - (Hn[c] - Hs[c]) / dz + src[c];
}

static int check_problem(const or_problem* P) {
  if (!P || P->nx < 4 || P->nS < 1 || P->nB < 1 || P->nF < 2 || P->m < 1) return -1;
  if (!(P->dx > 0) || !(P->dz1 > 0) || !(P->dz2 > 0)) return -1;
  return 0;
}

int or_rhs(const or_problem* P, const double* W, double* R, int k_lo, int k_hi) {
  if (check_problem(P) || k_lo < 0 || k_hi > nz_of(P) || k_lo > k_hi) return -1;
  int nx = P->nx;
  long long ncell = (long long)(k_hi - k_lo) * nx;
  g_rhs_cells += ncell;
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (long long e = 0; e < ncell; e++) {
    int k = k_lo + (int)(e / nx), i = (int)(e % nx);
    double r[4];
    rhs_cell(P, W, k, i, r);
    for (int c = 0; c < 4; c++) R[at(P, c, k, i)] = r[c];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Butcher tableaus (Table 1 for m = 2, generalised to any m)                 */
/* ------------------------------------------------------------------------ */
/*
 * Stages are numbered i = 1..2m; stage i = 2k+1 or 2k+2 belongs to fast
 * substep k = 0..m-1.
 *  F: m Heun substeps of dt/m (Sec. 3: the fast region takes m steps of the
 *     base RK2): c_{2k+1} = k/m, c_{2k+2} = (k+1)/m; a_{i,j} = 1/(2m) for all
 *     j <= 2k, a_{2k+2,2k+1} = 1/m; b_j = 1/(2m).
 *  B: the base RK2 restarted at every substep from q_n, its weights spread
 *     uniformly: a_{2k+2,2k+1} = 1; c = (0,1,0,1,...); b_j = 1/(2m).
 *  S: the base RK2 once; stages past s = 2 repeat stage mod(i-1,2)+1
 *     (Algorithm 1): a_{2k+2,1} = 1; c = (0,1,0,1,...); b = (1/2,1/2,0,...).
 * For m = 2 these are Table 1 entry by entry; for m = 1 all three are RK2.
 */
int or_tableau(int m, int region, double* a, double* b, double* c) {
  if (m < 1 || region < 0 || region > 2) return -1;
  int ms = 2 * m;
  for (int e = 0; e < ms * ms; e++) a[e] = 0.0;
  for (int k = 0; k < m; k++) {
    int i1 = 2 * k, i2 = 2 * k + 1; /* 0-based rows of stages 2k+1, 2k+2 */
    if (region == OR_REGION_F) {
      for (int j = 0; j < 2 * k; j++) {
        a[i1 * ms + j] = 1.0 / (2.0 * m);
        a[i2 * ms + j] = 1.0 / (2.0 * m);
      }
      a[i2 * ms + i1] = 1.0 / m;
      c[i1] = (double)k / m;
      c[i2] = (double)(k + 1) / m;
    } else if (region == OR_REGION_B) {
      a[i2 * ms + i1] = 1.0;
      c[i1] = 0.0;
      c[i2] = 1.0;
    } else {
      a[i2 * ms + 0] = 1.0;
      c[i1] = 0.0;
      c[i2] = 1.0;
    }
  }
  for (int j = 0; j < ms; j++) {
    if (region == OR_REGION_S) b[j] = j < 2 ? 0.5 : 0.0;
    else b[j] = 1.0 / (2.0 * m);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* MPRK2 slow step: Algorithm 1 with full stage arrays (Eq. MRK2)             */
/* ------------------------------------------------------------------------ */

/* Q_i = q + dt * sum_{j<i} a_ij R_j over rows [k_lo,k_hi), j ascending,
 * zero coefficients skipped (Eq. MRK2-qi) */
static void stage_value(const or_problem* P, const double* q, const double* Rall, double* Qi,
                        const double* a, int ms, int i, int k_lo, int k_hi) {
  size_t N = (size_t)4 * nz_of(P) * P->nx;
  for (int c = 0; c < 4; c++)
    for (int k = k_lo; k < k_hi; k++)
      for (int x = 0; x < P->nx; x++) {
        size_t e = at(P, c, k, x);
        double sum = 0.0;
        for (int j = 0; j < i; j++) {
          double aij = a[i * ms + j];
          if (aij != 0.0) sum += aij * Rall[(size_t)j * N + e];
        }
        Qi[e] = q[e] + P->dt * sum;
      }
}

/* q_{n+1} = q_n + dt * sum_i b_i R_i over rows [k_lo,k_hi) (Eq. MRK2-qn) */
static void completion(const or_problem* P, const double* q, const double* Rall, double* qn,
                       const double* b, int ms, int k_lo, int k_hi) {
  size_t N = (size_t)4 * nz_of(P) * P->nx;
  for (int c = 0; c < 4; c++)
    for (int k = k_lo; k < k_hi; k++)
      for (int x = 0; x < P->nx; x++) {
        size_t e = at(P, c, k, x);
        double sum = 0.0;
        for (int i = 0; i < ms; i++)
          if (b[i] != 0.0) sum += b[i] * Rall[(size_t)i * N + e];
        qn[e] = q[e] + P->dt * sum;
      }
}

static void copy_rows(const or_problem* P, const double* src, double* dst, int k_lo, int k_hi) {
  for (int c = 0; c < 4; c++)
    for (int k = k_lo; k < k_hi; k++)
      memcpy(&dst[at(P, c, k, 0)], &src[at(P, c, k, 0)], sizeof(double) * (size_t)P->nx);
}

int or_mprk_step_trace(const or_problem* P, const double* q, double* Q, double* R, double* q_next) {
  if (check_problem(P)) return -1;
  const int s = 2, m = P->m, ms = s * m;
  const int nS = P->nS, n1 = n1_of(P), nz = nz_of(P);
  const size_t N = (size_t)4 * nz * P->nx;
  double* aS = malloc(sizeof(double) * ms * ms * 3);
  double* bS = malloc(sizeof(double) * ms * 3);
  double* cc = malloc(sizeof(double) * ms);
  if (!aS || !bS || !cc) { free(aS); free(bS); free(cc); return -2; }
  double *aB = aS + ms * ms, *aF = aS + 2 * ms * ms;
  double *bB = bS + ms, *bF = bS + 2 * ms;
  or_tableau(m, OR_REGION_S, aS, bS, cc);
  or_tableau(m, OR_REGION_B, aB, bB, cc);
  or_tableau(m, OR_REGION_F, aF, bF, cc);
  memset(R, 0, sizeof(double) * N * ms);

  for (int i = 0; i < ms; i++) { /* stage i+1 of Algorithm 1 */
    double* Qi = Q + (size_t)i * N;
    double* Ri = R + (size_t)i * N;
    /* buffer stage value */
    stage_value(P, q, R, Qi, aB, ms, i, nS, n1);
    /* slow stage value, or a copy of stage mod(i-1,s)+1 */
    if (i < s) stage_value(P, q, R, Qi, aS, ms, i, 0, nS);
    else copy_rows(P, Q + (size_t)(i % s) * N, Qi, 0, nS);
    /* fast stage value */
    stage_value(P, q, R, Qi, aF, ms, i, n1, nz);
    /* right-hand sides on the composite stage state */
    or_rhs(P, Qi, Ri, nS, n1);
    if (i < s) or_rhs(P, Qi, Ri, 0, nS);
    or_rhs(P, Qi, Ri, n1, nz);
  }
  /* step completion */
  completion(P, q, R, q_next, bS, ms, 0, nS);
  completion(P, q, R, q_next, bB, ms, nS, n1);
  completion(P, q, R, q_next, bF, ms, n1, nz);
  free(aS); free(bS); free(cc);
  return 0;
}

int or_mprk_step(const or_problem* P, double* q, long long* rhs_cells) {
  if (check_problem(P)) return -1;
  const int ms = 2 * P->m;
  const size_t N = (size_t)4 * nz_of(P) * P->nx;
  double* Q = malloc(sizeof(double) * N * ms);
  double* R = malloc(sizeof(double) * N * ms);
  double* qn = malloc(sizeof(double) * N);
  if (!Q || !R || !qn) { free(Q); free(R); free(qn); return -2; }
  long long before = g_rhs_cells;
  int rc = or_mprk_step_trace(P, q, Q, R, qn);
  if (rc == 0) memcpy(q, qn, sizeof(double) * N);
  free(Q); free(R); free(qn);
  /* cell right-hand-side evaluations this step actually made */
  if (rhs_cells) *rhs_cells = g_rhs_cells - before;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* MPRK with a general base method (Sec. 3 remark: the base of the MPRK2     */
/* framework can be any Runge–Kutta method; the coupled method stays second  */
/* order at most)                                                             */
/* ------------------------------------------------------------------------ */

/* The three region tableaus for an s-stage base method (A s x s row-major,
 * b, c) and rate ratio m, built the way Table 1 builds them from RK2; stage
 * i = k s + p is stage p of fast substep k:
 *  F: m base steps of dt/m: a_{i, k's+q} = b_q/m for k' < k,
 *     a_{i, ks+q} = A_pq/m, c_i = (k + c_p)/m, b_i = b_p/m;
 *  B: the base restarted from q_n every substep: a_{i, ks+q} = A_pq,
 *     c_i = c_p, b_i = b_p/m;
 *  S: the base once; stages past s repeat stage p of the first substep:
 *     a_{i, q} = A_pq, c_i = c_p, b = (b, 0, ..., 0).
 * With Heun's base these are or_tableau's entries exactly. */
int or_tableau_base(int m, int region, int s, const double* A, const double* bb, const double* cc, double* a,
                    double* b, double* c) {
  if (m < 1 || s < 1 || region < 0 || region > 2) return -1;
  const int ms = m * s;
  for (int e = 0; e < ms * ms; e++) a[e] = 0.0;
  for (int k = 0; k < m; k++)
    for (int p = 0; p < s; p++) {
      const int i = k * s + p;
      if (region == OR_REGION_F) {
        for (int kk = 0; kk < k; kk++)
          for (int q = 0; q < s; q++) a[i * ms + kk * s + q] = bb[q] / m;
        for (int q = 0; q < p; q++) a[i * ms + k * s + q] = A[p * s + q] / m;
        c[i] = (k + cc[p]) / m;
        b[i] = bb[p] / m;
      } else if (region == OR_REGION_B) {
        for (int q = 0; q < p; q++) a[i * ms + k * s + q] = A[p * s + q];
        c[i] = cc[p];
        b[i] = bb[p] / m;
      } else {
        for (int q = 0; q < p; q++) a[i * ms + q] = A[p * s + q];
        c[i] = cc[p];
        b[i] = k == 0 ? bb[p] : 0.0;
      }
    }
  return 0;
}

/* One slow step of MPRK with the s-stage base (A, b, c): Algorithm 1 with s
 * in place of 2 (S stages past s copy stage mod(i-1, s)+1 of the first
 * substep and skip their RHS). */
int or_mprk_step_base(const or_problem* P, int s, const double* A, const double* bb, const double* cc, double* q) {
  if (check_problem(P) || s < 1 || s > 8) return -1;
  const int m = P->m, ms = s * m;
  const int nS = P->nS, n1 = n1_of(P), nz = nz_of(P);
  const size_t N = (size_t)4 * nz * P->nx;
  double* Q = malloc(sizeof(double) * N * ms);
  double* R = calloc(N * ms, sizeof(double));
  double* qn = malloc(sizeof(double) * N);
  double* tab = malloc(sizeof(double) * (3 * ms * ms + 4 * ms));
  if (!Q || !R || !qn || !tab) { free(Q); free(R); free(qn); free(tab); return -2; }
  double *aS = tab, *aB = tab + ms * ms, *aF = tab + 2 * ms * ms;
  double *bS = tab + 3 * ms * ms, *bB = bS + ms, *bF = bS + 2 * ms, *cx = bS + 3 * ms;
  or_tableau_base(m, OR_REGION_S, s, A, bb, cc, aS, bS, cx);
  or_tableau_base(m, OR_REGION_B, s, A, bb, cc, aB, bB, cx);
  or_tableau_base(m, OR_REGION_F, s, A, bb, cc, aF, bF, cx);
  for (int i = 0; i < ms; i++) {
    double* Qi = Q + (size_t)i * N;
    double* Ri = R + (size_t)i * N;
    stage_value(P, q, R, Qi, aB, ms, i, nS, n1);
    if (i < s) stage_value(P, q, R, Qi, aS, ms, i, 0, nS);
    else copy_rows(P, Q + (size_t)(i % s) * N, Qi, 0, nS);
    stage_value(P, q, R, Qi, aF, ms, i, n1, nz);
    or_rhs(P, Qi, Ri, nS, n1);
    if (i < s) or_rhs(P, Qi, Ri, 0, nS);
    or_rhs(P, Qi, Ri, n1, nz);
  }
  completion(P, q, R, qn, bS, ms, 0, nS);
  completion(P, q, R, qn, bB, ms, nS, n1);
  completion(P, q, R, qn, bF, ms, n1, nz);
  memcpy(q, qn, sizeof(double) * N);
  free(Q); free(R); free(qn); free(tab);
  return 0;
}

/* The s-stage base method alone over the whole grid, step h:
 * K_i = R(q + h sum_{j<i} A_ij K_j), q <- q + h sum_i b_i K_i. */
int or_rk_step_base(const or_problem* P, int s, const double* A, const double* bb, double* q, double h) {
  if (check_problem(P) || s < 1 || s > 8) return -1;
  const int nz = nz_of(P);
  const size_t N = (size_t)4 * nz * P->nx;
  double* K = malloc(sizeof(double) * N * (s + 1));
  if (!K) return -2;
  double* y = K + (size_t)s * N;
  for (int i = 0; i < s; i++) {
    for (size_t e = 0; e < N; e++) {
      double sum = 0.0;
      for (int j = 0; j < i; j++)
        if (A[i * s + j] != 0.0) sum += A[i * s + j] * K[(size_t)j * N + e];
      y[e] = q[e] + h * sum;
    }
    or_rhs(P, y, K + (size_t)i * N, 0, nz);
  }
  for (size_t e = 0; e < N; e++) {
    double sum = 0.0;
    for (int i = 0; i < s; i++)
      if (bb[i] != 0.0) sum += bb[i] * K[(size_t)i * N + e];
    q[e] = q[e] + h * sum;
  }
  free(K);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Single-rate integrators over the whole grid                                */
/* ------------------------------------------------------------------------ */

/* Heun's method, the base RK2 of Table 1: q1 = q + h R(q);
 * q <- q + h/2 (R(q) + R(q1)) */
int or_rk2_step(const or_problem* P, double* q, double h) {
  if (check_problem(P)) return -1;
  const int nz = nz_of(P);
  const size_t N = (size_t)4 * nz * P->nx;
  double* R1 = malloc(sizeof(double) * N);
  double* R2 = malloc(sizeof(double) * N);
  double* q1 = malloc(sizeof(double) * N);
  if (!R1 || !R2 || !q1) { free(R1); free(R2); free(q1); return -2; }
  or_rhs(P, q, R1, 0, nz);
  for (size_t e = 0; e < N; e++) q1[e] = q[e] + h * R1[e];
  or_rhs(P, q1, R2, 0, nz);
  for (size_t e = 0; e < N; e++) q[e] = q[e] + (h / 2.0) * (R1[e] + R2[e]);
  free(R1); free(R2); free(q1);
  return 0;
}

/* classical RK4 */
int or_rk4_step(const or_problem* P, double* q, double h) {
  if (check_problem(P)) return -1;
  const int nz = nz_of(P);
  const size_t N = (size_t)4 * nz * P->nx;
  double* k1 = malloc(sizeof(double) * N * 5);
  if (!k1) return -2;
  double *k2 = k1 + N, *k3 = k1 + 2 * N, *k4 = k1 + 3 * N, *y = k1 + 4 * N;
  or_rhs(P, q, k1, 0, nz);
  for (size_t e = 0; e < N; e++) y[e] = q[e] + (h / 2.0) * k1[e];
  or_rhs(P, y, k2, 0, nz);
  for (size_t e = 0; e < N; e++) y[e] = q[e] + (h / 2.0) * k2[e];
  or_rhs(P, y, k3, 0, nz);
  for (size_t e = 0; e < N; e++) y[e] = q[e] + h * k3[e];
  or_rhs(P, y, k4, 0, nz);
  for (size_t e = 0; e < N; e++)
    q[e] = q[e] + (h / 6.0) * (k1[e] + 2.0 * k2[e] + 2.0 * k3[e] + k4[e]);
  free(k1);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (Sec. 5.1 total mass and energy) and the Courant numbers       */
/* ------------------------------------------------------------------------ */

static double wave_speed(const double q[4], double gamma) {
  prim c = to_prim(q, gamma);
  return fmax(fabs(c.u), fabs(c.w)) + c.a;
}

int or_diagnostics(const or_problem* P, const double* q, double out[16]) {
  if (check_problem(P)) return -1;
  const int nz = nz_of(P), nS = P->nS, n1 = n1_of(P);
  for (int e = 0; e < 16; e++) out[e] = 0.0;
  double cmax[3] = {0.0, 0.0, 0.0};
  double nonfinite = 0.0, rmin = INFINITY, pmin = INFINITY;
  for (int k = 0; k < nz; k++) {
    int f = fluid_of(P, k);
    int region = k < nS ? 0 : (k < n1 ? 1 : 2);
    double vol = P->dx * dz_of(P, k);
    for (int i = 0; i < P->nx; i++) {
      double v[4];
      load(P, q, k, i, v);
      for (int c = 0; c < 4; c++) {
        if (!isfinite(v[c])) nonfinite += 1.0;
        out[(f - 1) * 4 + c] += v[c] * vol;
      }
      prim pr = to_prim(v, P->gamma);
      double ws = wave_speed(v, P->gamma);
      if (ws > cmax[region]) cmax[region] = ws;
      if (v[0] < rmin) rmin = v[0];
      if (pr.p < pmin) pmin = pr.p;
    }
  }
  out[8] = P->dt * cmax[0] / fmin(P->dx, P->dz1);
  out[9] = P->dt * cmax[1] / fmin(P->dx, P->dz1);
  out[10] = (P->dt / P->m) * cmax[2] / fmin(P->dx, P->dz2);
  out[11] = nonfinite;
  out[12] = rmin;
  out[13] = pmin;
  return 0;
}

/* dt = min(cfl*min(dx,dz1)/c_max over fluid 1, m*cfl*min(dx,dz2)/c_max over
 * fluid 2): the slow step for which every region runs at Courant number cfl
 * or less. */
double or_stable_dt(const or_problem* P, const double* q, double cfl) {
  if (check_problem(P)) return -1.0;
  const int nz = nz_of(P), n1 = n1_of(P);
  double c1 = 0.0, c2 = 0.0;
  for (int k = 0; k < nz; k++)
    for (int i = 0; i < P->nx; i++) {
      double v[4];
      load(P, q, k, i, v);
      double ws = wave_speed(v, P->gamma);
      if (k < n1) { if (ws > c1) c1 = ws; }
      else { if (ws > c2) c2 = ws; }
    }
  double d1 = cfl * fmin(P->dx, P->dz1) / c1;
  double d2 = P->m * cfl * fmin(P->dx, P->dz2) / c2;
  return fmin(d1, d2);
}
