/*
 * mprk_oracle3d.c — plain FP64 CPU oracle of the 3-D scheme (App. B,
 * Eq. ns-fv-cartesian-3d) and its MPRK2 slow step (Eq. MRK2, Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY: it checks the CUDA library and is never part of
 * the product path. It shares no code with the CUDA sources. Build it with
 * -O2 -ffp-contract=off so that every operation is rounded as written.
 *
 * The scheme is the 2-D oracle's with y added, as App. B writes it:
 *   dq/dt = -(F*_{i+1/2} - F*_{i-1/2})/dx - (G*_{j+1/2} - G*_{j-1/2})/dy
 *           - (H*_{k+1/2} - H*_{k-1/2})/dz + s,
 * Lax–Friedrichs inviscid fluxes of linearly reconstructed conserved
 * variables (central-difference cell gradients), viscous fluxes from common
 * face values (mean velocity; two-point normal derivatives; tangential
 * derivatives averaged from the two cells), sigma = mu (grad u + grad u^T
 * - 2/3 div u I), Pi = -kappa grad T.
 *
 * Readings, as in the 2-D oracle:
 *  - x and y are periodic;
 *  - beyond a z wall or Gamma the conserved slope uses a mirror ghost (rho w
 *    flipped); u, v, w, T use 2*(wall state) - interior: no-slip walls
 *    u_w = v_w = w_w = 0, slip walls keep u and v, adiabatic (T kept);
 *    Gamma's wall state is (u_w, v_w, 0, T_w) of each fluid's own formula;
 *  - the inviscid flux through a wall or Gamma is Lax–Friedrichs between the
 *    reconstructed boundary state and its mirror;
 *  - the viscous flux through an outer wall is the common-value recipe
 *    between the cell and its ghost; through Gamma it is
 *    (0, sigma^_xz, sigma^_yz, 0, u_w sigma^_xz + v_w sigma^_yz - Pi^_z);
 *  - gravity: source (0, 0, 0, -rho G, -rho w G), G > 0.
 */
#include "mprk_oracle3d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "mprk_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static int nz3(const or3_problem* P) { return P->nS + P->nB + P->nF; }
static int n13(const or3_problem* P) { return P->nS + P->nB; }
static int fluid3(const or3_problem* P, int k) { return k < n13(P) ? 1 : 2; }
static double dz3(const or3_problem* P, int k) { return fluid3(P, k) == 1 ? P->dz1 : P->dz2; }
static double mu3(const or3_problem* P, int f) { return f == 1 ? P->mu1 : P->mu2; }
/* kappa~ = c~_p mu~ / Pr with c~_p = 1/(gamma-1) (App. A) */
static double kap3(const or3_problem* P, int f) { return mu3(P, f) / ((P->gamma - 1.0) * P->Pr); }
static double delta3(const or3_problem* P, int d, int k) {
  return d == 0 ? P->dx : (d == 1 ? P->dy : dz3(P, k));
}

static size_t at3(const or3_problem* P, int c, int k, int j, int i) {
  return (((size_t)c * nz3(P) + (size_t)k) * (size_t)P->ny + (size_t)j) * (size_t)P->nx + (size_t)i;
}
static int wx(const or3_problem* P, int i) { return ((i % P->nx) + P->nx) % P->nx; }
static int wy(const or3_problem* P, int j) { return ((j % P->ny) + P->ny) % P->ny; }

static void load3(const or3_problem* P, const double* W, int k, int j, int i, double q[5]) {
  for (int c = 0; c < 5; c++) q[c] = W[at3(P, c, k, j, i)];
}

/* ------------------------------------------------------------------------ */
/* Thermodynamics and the inviscid flux                                       */
/* ------------------------------------------------------------------------ */

typedef struct { double rho, u, v, w, p, T, a, H; } prim3;

static prim3 prim_of(const double q[5], double gamma) {
  prim3 s;
  s.rho = q[0];
  s.u = q[1] / q[0];
  s.v = q[2] / q[0];
  s.w = q[3] / q[0];
  s.p = (gamma - 1.0) * (q[4] - 0.5 * q[0] * (s.u * s.u + s.v * s.v + s.w * s.w));
  s.T = gamma * s.p / q[0];
  s.a = sqrt(gamma * s.p / q[0]);
  s.H = (q[4] + s.p) / q[0];
  return s;
}

static double normal_velocity(const prim3* s, int d) { return d == 0 ? s->u : (d == 1 ? s->v : s->w); }

/* F^I, G^I or H^I of App. B for d = 0, 1, 2 */
static void euler3(const double q[5], int d, double gamma, double F[5]) {
  prim3 s = prim_of(q, gamma);
  double un = normal_velocity(&s, d);
  F[0] = q[0] * un;
  for (int a = 0; a < 3; a++) F[1 + a] = q[1 + a] * un + (a == d ? s.p : 0.0);
  F[4] = q[0] * un * s.H;
}

void or3_lf_flux(const double ql[5], const double qr[5], int d, double gamma, double F[5]) {
  double Fl[5], Fr[5];
  euler3(ql, d, gamma, Fl);
  euler3(qr, d, gamma, Fr);
  prim3 L = prim_of(ql, gamma), R = prim_of(qr, gamma);
  double sl = sqrt(L.rho), sr = sqrt(R.rho);
  double ur = (sl * L.u + sr * R.u) / (sl + sr);
  double vr = (sl * L.v + sr * R.v) / (sl + sr);
  double wr = (sl * L.w + sr * R.w) / (sl + sr);
  double Hr = (sl * L.H + sr * R.H) / (sl + sr);
  double ar = sqrt((gamma - 1.0) * (Hr - 0.5 * (ur * ur + vr * vr + wr * wr)));
  double unroe = d == 0 ? ur : (d == 1 ? vr : wr);
  double lam = fmax(fabs(normal_velocity(&L, d)) + L.a, fmax(fabs(normal_velocity(&R, d)) + R.a, fabs(unroe) + ar));
  for (int c = 0; c < 5; c++) F[c] = 0.5 * (Fl[c] + Fr[c]) + 0.5 * lam * (ql[c] - qr[c]);
}

/* ------------------------------------------------------------------------ */
/* Interface state (App. B, Eq. bulk-flux and the wall states after it)       */
/* ------------------------------------------------------------------------ */

int or3_interface_state(const or3_problem* P, const double* W, int j, int i, double out[9]) {
  double q1[5], q2[5];
  load3(P, W, n13(P) - 1, j, i, q1);
  load3(P, W, n13(P), j, i, q2);
  prim3 c1 = prim_of(q1, P->gamma), c2 = prim_of(q2, P->gamma);
  double mu1 = P->mu1, mu2 = P->mu2, ka1 = kap3(P, 1), ka2 = kap3(P, 2);
  double dz1 = P->dz1, dz2 = P->dz2;
  double bu = 2.0 * mu1 * mu2 / (dz2 * mu1 + dz1 * mu2); /* = b_v */
  double bT = 2.0 * ka1 * ka2 / (dz2 * ka1 + dz1 * ka2);
  double sxz = bu * (c2.u - c1.u);
  double syz = bu * (c2.v - c1.v);
  double Piz = -bT * (c2.T - c1.T);
  out[0] = sxz;
  out[1] = syz;
  out[2] = Piz;
  out[3] = c1.u + sxz * dz1 / (2.0 * mu1);
  out[4] = c1.v + syz * dz1 / (2.0 * mu1);
  out[5] = c1.T - Piz * dz1 / (2.0 * ka1);
  out[6] = c2.u - sxz * dz2 / (2.0 * mu2);
  out[7] = c2.v - syz * dz2 / (2.0 * mu2);
  out[8] = c2.T + Piz * dz2 / (2.0 * ka2);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Neighbours and cell gradients                                              */
/* ------------------------------------------------------------------------ */

/* Is row k+s outside the fluid of row k (beyond a wall or Gamma)? */
static int beyond3(const or3_problem* P, int k, int s) {
  int kk = k + s;
  if (kk < 0 || kk >= nz3(P)) return 1;
  return fluid3(P, kk) != fluid3(P, k);
}
static int beyond_gamma3(const or3_problem* P, int k, int s) {
  int kk = k + s;
  return kk >= 0 && kk < nz3(P) && fluid3(P, kk) != fluid3(P, k);
}

/* conserved neighbour of (k,j,i) at offset s in direction d; mirror ghost
 * (rho w flipped) beyond a z wall or Gamma */
static void nb_cons3(const or3_problem* P, const double* W, int k, int j, int i, int d, int s, double q[5]) {
  if (d == 0) {
    load3(P, W, k, j, wx(P, i + s), q);
  } else if (d == 1) {
    load3(P, W, k, wy(P, j + s), i, q);
  } else if (!beyond3(P, k, s)) {
    load3(P, W, k + s, j, i, q);
  } else {
    load3(P, W, k, j, i, q);
    q[3] = -q[3];
  }
}

static void uvwT_at(const or3_problem* P, const double* W, int k, int j, int i, double v[4]) {
  double q[5];
  load3(P, W, k, j, i, q);
  prim3 c = prim_of(q, P->gamma);
  v[0] = c.u; v[1] = c.v; v[2] = c.w; v[3] = c.T;
}

/* (u, v, w, T) of the neighbour at offset s in direction d; beyond a z wall
 * or Gamma the ghost is 2*(wall state) - (interior value) */
static void nb_uvwT3(const or3_problem* P, const double* W, int k, int j, int i, int d, int s, double v[4]) {
  if (d == 0) { uvwT_at(P, W, k, j, wx(P, i + s), v); return; }
  if (d == 1) { uvwT_at(P, W, k, wy(P, j + s), i, v); return; }
  if (!beyond3(P, k, s)) { uvwT_at(P, W, k + s, j, i, v); return; }
  double c[4];
  uvwT_at(P, W, k, j, i, c);
  if (beyond_gamma3(P, k, s)) {
    double st[9];
    or3_interface_state(P, W, j, i, st);
    int f1 = fluid3(P, k) == 1;
    double uw = f1 ? st[3] : st[6], vw = f1 ? st[4] : st[7], Tw = f1 ? st[5] : st[8];
    v[0] = 2.0 * uw - c[0];
    v[1] = 2.0 * vw - c[1];
    v[2] = -c[2];
    v[3] = 2.0 * Tw - c[3];
  } else if (P->wall == 1) { /* slip */
    v[0] = c[0]; v[1] = c[1]; v[2] = -c[2]; v[3] = c[3];
  } else { /* no-slip */
    v[0] = -c[0]; v[1] = -c[1]; v[2] = -c[2]; v[3] = c[3];
  }
}

/* central-difference cell gradients (App. B footnote, read as central) */
static void grad_cons3(const or3_problem* P, const double* W, int k, int j, int i, int d, double g[5]) {
  double qp[5], qm[5];
  nb_cons3(P, W, k, j, i, d, +1, qp);
  nb_cons3(P, W, k, j, i, d, -1, qm);
  double h = delta3(P, d, k);
  for (int c = 0; c < 5; c++) g[c] = (qp[c] - qm[c]) / (2.0 * h);
}
static void grad_uvwT3(const or3_problem* P, const double* W, int k, int j, int i, int d, double g[4]) {
  double vp[4], vm[4];
  nb_uvwT3(P, W, k, j, i, d, +1, vp);
  nb_uvwT3(P, W, k, j, i, d, -1, vm);
  double h = delta3(P, d, k);
  for (int c = 0; c < 4; c++) g[c] = (vp[c] - vm[c]) / (2.0 * h);
}

/* ------------------------------------------------------------------------ */
/* Viscous flux from common face values                                        */
/* ------------------------------------------------------------------------ */

/* one side of a face: (u, v, w, T) and, for the two tangential directions
 * b, the cell gradients du_a/dx_b (gt[b][a], a = u, v, w) */
typedef struct { double v[4]; double gt[3][3]; } vside3;

static void side_of(const or3_problem* P, const double* W, int k, int j, int i, int d, vside3* s) {
  uvwT_at(P, W, k, j, i, s->v);
  for (int b = 0; b < 3; b++) {
    if (b == d) { s->gt[b][0] = s->gt[b][1] = s->gt[b][2] = 0.0; continue; }
    double g[4];
    grad_uvwT3(P, W, k, j, i, b, g);
    for (int a = 0; a < 3; a++) s->gt[b][a] = g[a];
  }
}

/* F^V, G^V or H^V (d = 0, 1, 2) of App. B at a face of width dn */
static void viscous3(const vside3* L, const vside3* R, int d, double dn, double mu, double kap, double FV[5]) {
  double uh[3], G[3][3]; /* G[a][b] = d u_a / d x_b at the face */
  for (int a = 0; a < 3; a++) {
    uh[a] = 0.5 * (L->v[a] + R->v[a]);
    for (int b = 0; b < 3; b++)
      G[a][b] = (b == d) ? (R->v[a] - L->v[a]) / dn : 0.5 * (L->gt[b][a] + R->gt[b][a]);
  }
  double div = G[0][0] + G[1][1] + G[2][2];
  double sig[3]; /* sigma_{d a} */
  for (int a = 0; a < 3; a++)
    sig[a] = mu * (G[a][d] + G[d][a]) - (a == d ? (2.0 / 3.0) * mu * div : 0.0);
  double dTn = (R->v[3] - L->v[3]) / dn;
  FV[0] = 0.0;
  for (int a = 0; a < 3; a++) FV[1 + a] = sig[a];
  FV[4] = uh[0] * sig[0] + uh[1] * sig[1] + uh[2] * sig[2] + kap * dTn; /* u.sigma_d - Pi_d */
}

/* ------------------------------------------------------------------------ */
/* Face fluxes                                                               */
/* ------------------------------------------------------------------------ */

/* face between (k,j,i) and its neighbour at +1 in direction d (periodic in
 * x and y; in z both rows lie in the same fluid) */
static void face3(const or3_problem* P, const double* W, int k, int j, int i, int d, double F[5]) {
  int k2 = k + (d == 2), j2 = d == 1 ? wy(P, j + 1) : j, i2 = d == 0 ? wx(P, i + 1) : i;
  double h = delta3(P, d, k);
  double qL[5], qR[5], gL[5], gR[5], ql[5], qr[5], FI[5], FV[5];
  load3(P, W, k, j, i, qL);
  load3(P, W, k2, j2, i2, qR);
  grad_cons3(P, W, k, j, i, d, gL);
  grad_cons3(P, W, k2, j2, i2, d, gR);
  for (int c = 0; c < 5; c++) {
    ql[c] = qL[c] + gL[c] * (h / 2.0);
    qr[c] = qR[c] - gR[c] * (h / 2.0);
  }
  or3_lf_flux(ql, qr, d, P->gamma, FI);
  vside3 sL, sR;
  side_of(P, W, k, j, i, d, &sL);
  side_of(P, W, k2, j2, i2, d, &sR);
  int f = fluid3(P, k);
  viscous3(&sL, &sR, d, h, mu3(P, f), kap3(P, f), FV);
  for (int c = 0; c < 5; c++) F[c] = FI[c] - FV[c];
}

static void mirror3(const double q[5], double g[5]) {
  for (int c = 0; c < 5; c++) g[c] = q[c];
  g[3] = -q[3];
}

/* outer wall below row 0 (s = -1) or above the top row (s = +1) */
static void zwall3(const or3_problem* P, const double* W, int k, int j, int i, int s, double F[5]) {
  double dz = dz3(P, k);
  double q[5], g[5], qb[5], qg[5], FI[5], FV[5];
  load3(P, W, k, j, i, q);
  grad_cons3(P, W, k, j, i, 2, g);
  for (int c = 0; c < 5; c++) qb[c] = q[c] + (double)s * g[c] * (dz / 2.0);
  mirror3(qb, qg);
  if (s < 0) or3_lf_flux(qg, qb, 2, P->gamma, FI);
  else or3_lf_flux(qb, qg, 2, P->gamma, FI);
  /* viscous: the cell and its ghost 2*wall - interior (adiabatic) */
  vside3 C, Gh;
  side_of(P, W, k, j, i, 2, &C);
  Gh = C;
  int slip = P->wall == 1;
  for (int a = 0; a < 3; a++) {
    double sg = (a == 2 || !slip) ? -1.0 : 1.0; /* w always flips; u, v flip at no-slip walls */
    Gh.v[a] = sg * C.v[a];
    for (int b = 0; b < 2; b++) Gh.gt[b][a] = sg * C.gt[b][a];
  }
  int f = fluid3(P, k);
  if (s < 0) viscous3(&Gh, &C, 2, dz, mu3(P, f), kap3(P, f), FV);
  else viscous3(&C, &Gh, 2, dz, mu3(P, f), kap3(P, f), FV);
  for (int c = 0; c < 5; c++) F[c] = FI[c] - FV[c];
}

/* Gamma seen by fluid 1's top row (f = 1) or fluid 2's bottom row (f = 2):
 * a rigid lid (inviscid) and the bulk fluxes of App. B (viscous) */
static void zgamma3(const or3_problem* P, const double* W, int j, int i, int f, double F[5]) {
  int k = f == 1 ? n13(P) - 1 : n13(P);
  int s = f == 1 ? +1 : -1;
  double dz = dz3(P, k);
  double q[5], g[5], qb[5], qg[5], FI[5];
  load3(P, W, k, j, i, q);
  grad_cons3(P, W, k, j, i, 2, g);
  for (int c = 0; c < 5; c++) qb[c] = q[c] + (double)s * g[c] * (dz / 2.0);
  mirror3(qb, qg);
  if (f == 1) or3_lf_flux(qb, qg, 2, P->gamma, FI);
  else or3_lf_flux(qg, qb, 2, P->gamma, FI);
  double st[9];
  or3_interface_state(P, W, j, i, st);
  double sxz = st[0], syz = st[1], Piz = st[2];
  double uw = f == 1 ? st[3] : st[6], vw = f == 1 ? st[4] : st[7];
  double FV[5] = {0.0, sxz, syz, 0.0, uw * sxz + vw * syz - Piz};
  for (int c = 0; c < 5; c++) F[c] = FI[c] - FV[c];
}

/* flux through the lower (s = -1) or upper (s = +1) z face of row k */
static void zflux3(const or3_problem* P, const double* W, int k, int j, int i, int s, double F[5]) {
  int nz = nz3(P), n1 = n13(P);
  if (s < 0) {
    if (k == 0) zwall3(P, W, k, j, i, -1, F);
    else if (k == n1) zgamma3(P, W, j, i, 2, F);
    else face3(P, W, k - 1, j, i, 2, F);
  } else {
    if (k == nz - 1) zwall3(P, W, k, j, i, +1, F);
    else if (k == n1 - 1) zgamma3(P, W, j, i, 1, F);
    else face3(P, W, k, j, i, 2, F);
  }
}

/* ------------------------------------------------------------------------ */
/* Right-hand side (Eq. ns-fv-cartesian-3d)                                   */
/* ------------------------------------------------------------------------ */

static void rhs_cell3(const or3_problem* P, const double* W, int k, int j, int i, double r[5]) {
  double Fe[5], Fw[5], Gn[5], Gs[5], Hu[5], Hd[5], q[5];
  face3(P, W, k, j, i, 0, Fe);
  face3(P, W, k, j, wx(P, i - 1), 0, Fw);
  face3(P, W, k, j, i, 1, Gn);
  face3(P, W, k, wy(P, j - 1), i, 1, Gs);
  zflux3(P, W, k, j, i, +1, Hu);
  zflux3(P, W, k, j, i, -1, Hd);
  load3(P, W, k, j, i, q);
  double dz = dz3(P, k);
  double src[5] = {0.0, 0.0, 0.0, -q[0] * P->G, -q[3] * P->G};
  for (int c = 0; c < 5; c++)
    r[c] = -(Fe[c] - Fw[c]) / P->dx - (Gn[c] - Gs[c]) / P->dy - (Hu[c] - Hd[c]) / dz + src[c];
}

static int check3(const or3_problem* P) {
  if (!P || P->nx < 3 || P->ny < 3 || P->nS < 1 || P->nB < 1 || P->nF < 2 || P->m < 1) return -1;
  if (!(P->dx > 0) || !(P->dy > 0) || !(P->dz1 > 0) || !(P->dz2 > 0)) return -1;
  return 0;
}

int or3_rhs(const or3_problem* P, const double* W, double* R, int k_lo, int k_hi) {
  if (check3(P) || k_lo < 0 || k_hi > nz3(P) || k_lo > k_hi) return -1;
  const int nx = P->nx, ny = P->ny;
  const long long ncell = (long long)(k_hi - k_lo) * ny * nx;
#pragma omp parallel for schedule(static) num_threads(or_get_threads())
  for (long long e = 0; e < ncell; e++) {
    int i = (int)(e % nx);
    int j = (int)((e / nx) % ny);
    int k = k_lo + (int)(e / ((long long)nx * ny));
    double r[5];
    rhs_cell3(P, W, k, j, i, r);
    for (int c = 0; c < 5; c++) R[at3(P, c, k, j, i)] = r[c];
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* MPRK2 slow step: Algorithm 1 with full stage arrays (Eq. MRK2)             */
/* ------------------------------------------------------------------------ */

/* Q_i = q + dt sum_{j<i} a_ij R_j over rows [k_lo,k_hi), j ascending,
 * zero coefficients skipped */
static void stage_value3(const or3_problem* P, const double* q, const double* Rall, double* Qi, const double* a,
                         int ms, int i, int k_lo, int k_hi) {
  const size_t N = (size_t)5 * nz3(P) * P->ny * P->nx, row = (size_t)P->ny * P->nx;
  for (int c = 0; c < 5; c++)
    for (int k = k_lo; k < k_hi; k++)
      for (size_t x = 0; x < row; x++) {
        size_t e = at3(P, c, k, 0, 0) + x;
        double sum = 0.0;
        for (int jj = 0; jj < i; jj++) {
          double aij = a[i * ms + jj];
          if (aij != 0.0) sum += aij * Rall[(size_t)jj * N + e];
        }
        Qi[e] = q[e] + P->dt * sum;
      }
}

static void completion3(const or3_problem* P, const double* q, const double* Rall, double* qn, const double* b,
                        int ms, int k_lo, int k_hi) {
  const size_t N = (size_t)5 * nz3(P) * P->ny * P->nx, row = (size_t)P->ny * P->nx;
  for (int c = 0; c < 5; c++)
    for (int k = k_lo; k < k_hi; k++)
      for (size_t x = 0; x < row; x++) {
        size_t e = at3(P, c, k, 0, 0) + x;
        double sum = 0.0;
        for (int i = 0; i < ms; i++)
          if (b[i] != 0.0) sum += b[i] * Rall[(size_t)i * N + e];
        qn[e] = q[e] + P->dt * sum;
      }
}

static void copy_rows3(const or3_problem* P, const double* src, double* dst, int k_lo, int k_hi) {
  const size_t row = (size_t)P->ny * P->nx;
  for (int c = 0; c < 5; c++)
    for (int k = k_lo; k < k_hi; k++) memcpy(&dst[at3(P, c, k, 0, 0)], &src[at3(P, c, k, 0, 0)], sizeof(double) * row);
}

int or3_mprk_step(const or3_problem* P, double* q) {
  if (check3(P)) return -1;
  const int s = 2, m = P->m, ms = s * m;
  const int nS = P->nS, n1 = n13(P), nz = nz3(P);
  const size_t N = (size_t)5 * nz * P->ny * P->nx;
  double* Q = malloc(sizeof(double) * N * ms);
  double* R = calloc(N * ms, sizeof(double));
  double* qn = malloc(sizeof(double) * N);
  double* tab = malloc(sizeof(double) * (3 * ms * ms + 3 * ms + ms));
  if (!Q || !R || !qn || !tab) { free(Q); free(R); free(qn); free(tab); return -2; }
  double *aS = tab, *aB = tab + ms * ms, *aF = tab + 2 * ms * ms;
  double *bS = tab + 3 * ms * ms, *bB = bS + ms, *bF = bS + 2 * ms, *cc = bS + 3 * ms;
  or_tableau(m, OR_REGION_S, aS, bS, cc);
  or_tableau(m, OR_REGION_B, aB, bB, cc);
  or_tableau(m, OR_REGION_F, aF, bF, cc);
  for (int i = 0; i < ms; i++) { /* stage i+1 of Algorithm 1 */
    double* Qi = Q + (size_t)i * N;
    double* Ri = R + (size_t)i * N;
    stage_value3(P, q, R, Qi, aB, ms, i, nS, n1);
    if (i < s) stage_value3(P, q, R, Qi, aS, ms, i, 0, nS);
    else copy_rows3(P, Q + (size_t)(i % s) * N, Qi, 0, nS);
    stage_value3(P, q, R, Qi, aF, ms, i, n1, nz);
    or3_rhs(P, Qi, Ri, nS, n1);
    if (i < s) or3_rhs(P, Qi, Ri, 0, nS);
    or3_rhs(P, Qi, Ri, n1, nz);
  }
  completion3(P, q, R, qn, bS, ms, 0, nS);
  completion3(P, q, R, qn, bB, ms, nS, n1);
  completion3(P, q, R, qn, bF, ms, n1, nz);
  memcpy(q, qn, sizeof(double) * N);
  free(Q); free(R); free(qn); free(tab);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Single-rate integrators                                                    */
/* ------------------------------------------------------------------------ */

int or3_rk2_step(const or3_problem* P, double* q, double h) {
  if (check3(P)) return -1;
  const int nz = nz3(P);
  const size_t N = (size_t)5 * nz * P->ny * P->nx;
  double* R1 = malloc(sizeof(double) * N * 3);
  if (!R1) return -2;
  double *R2 = R1 + N, *q1 = R1 + 2 * N;
  or3_rhs(P, q, R1, 0, nz);
  for (size_t e = 0; e < N; e++) q1[e] = q[e] + h * R1[e];
  or3_rhs(P, q1, R2, 0, nz);
  for (size_t e = 0; e < N; e++) q[e] = q[e] + (h / 2.0) * (R1[e] + R2[e]);
  free(R1);
  return 0;
}

int or3_rk4_step(const or3_problem* P, double* q, double h) {
  if (check3(P)) return -1;
  const int nz = nz3(P);
  const size_t N = (size_t)5 * nz * P->ny * P->nx;
  double* k1 = malloc(sizeof(double) * N * 5);
  if (!k1) return -2;
  double *k2 = k1 + N, *k3 = k1 + 2 * N, *k4 = k1 + 3 * N, *y = k1 + 4 * N;
  or3_rhs(P, q, k1, 0, nz);
  for (size_t e = 0; e < N; e++) y[e] = q[e] + (h / 2.0) * k1[e];
  or3_rhs(P, y, k2, 0, nz);
  for (size_t e = 0; e < N; e++) y[e] = q[e] + (h / 2.0) * k2[e];
  or3_rhs(P, y, k3, 0, nz);
  for (size_t e = 0; e < N; e++) y[e] = q[e] + h * k3[e];
  or3_rhs(P, y, k4, 0, nz);
  for (size_t e = 0; e < N; e++) q[e] = q[e] + (h / 6.0) * (k1[e] + 2.0 * k2[e] + 2.0 * k3[e] + k4[e]);
  free(k1);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics and the Courant step                                           */
/* ------------------------------------------------------------------------ */

static double wave3(const double q[5], double gamma) {
  prim3 c = prim_of(q, gamma);
  return fmax(fabs(c.u), fmax(fabs(c.v), fabs(c.w))) + c.a;
}

int or3_diagnostics(const or3_problem* P, const double* q, double out[16]) {
  if (check3(P)) return -1;
  const int nz = nz3(P), nS = P->nS, n1 = n13(P);
  for (int e = 0; e < 16; e++) out[e] = 0.0;
  double cmax[3] = {0.0, 0.0, 0.0}, nonfinite = 0.0, rmin = INFINITY, pmin = INFINITY;
  for (int k = 0; k < nz; k++) {
    int f = fluid3(P, k);
    int region = k < nS ? 0 : (k < n1 ? 1 : 2);
    double vol = P->dx * P->dy * dz3(P, k);
    for (int j = 0; j < P->ny; j++)
      for (int i = 0; i < P->nx; i++) {
        double v[5];
        load3(P, q, k, j, i, v);
        for (int c = 0; c < 5; c++) {
          if (!isfinite(v[c])) nonfinite += 1.0;
          out[(f - 1) * 5 + c] += v[c] * vol;
        }
        prim3 pr = prim_of(v, P->gamma);
        double ws = wave3(v, P->gamma);
        if (ws > cmax[region]) cmax[region] = ws;
        if (v[0] < rmin) rmin = v[0];
        if (pr.p < pmin) pmin = pr.p;
      }
  }
  double h1 = fmin(fmin(P->dx, P->dy), P->dz1), h2 = fmin(fmin(P->dx, P->dy), P->dz2);
  out[10] = P->dt * cmax[0] / h1;
  out[11] = P->dt * cmax[1] / h1;
  out[12] = (P->dt / P->m) * cmax[2] / h2;
  out[13] = nonfinite;
  out[14] = rmin;
  out[15] = pmin;
  return 0;
}

double or3_stable_dt(const or3_problem* P, const double* q, double cfl) {
  if (check3(P)) return -1.0;
  const int nz = nz3(P), n1 = n13(P);
  double c1 = 0.0, c2 = 0.0;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < P->ny; j++)
      for (int i = 0; i < P->nx; i++) {
        double v[5];
        load3(P, q, k, j, i, v);
        double ws = wave3(v, P->gamma);
        if (k < n1) { if (ws > c1) c1 = ws; }
        else { if (ws > c2) c2 = ws; }
      }
  double h1 = fmin(fmin(P->dx, P->dy), P->dz1), h2 = fmin(fmin(P->dx, P->dy), P->dz2);
  return fmin(cfl * h1 / c1, P->m * cfl * h2 / c2);
}
