// stage_tile3d.cuh — the 3-D stage (App. B, Eq. ns-fv-cartesian-3d in full),
// FP64: five conserved variables (rho, rho u, rho v, rho w, rho E), x and y
// periodic, the S/B/F row bands and Gamma in z as in 2-D. Layout of every
// state-sized array: [5][nz][ny][pitch].
//
// A stage is two launches over the active rows:
//  * yface3: one CTA per TX x TZ tile of an x–z plane j computes the y-face
//    fluxes G* between planes j and j+1 of its cells and stores G*/dy (face
//    j+1/2 at index j) in a state-sized buffer;
//  * stage3: one CTA per TX x TZ tile of plane j computes its x and z faces
//    as the 2-D tile does, takes the y divergence from the stored y faces,
//    adds the source and applies the stage combination.
// Every face is computed once. Viscous fluxes use the common face values
// of App. B: mean velocity, two-point normal derivatives, tangential
// derivatives averaged from the two cells' central differences, sigma =
// mu (grad u + grad u^T - 2/3 div u I), heat flux -kappa grad T.
// Central differences are stored unscaled; their factors (1/4 for the
// reconstruction, 1/(2 d) for a derivative), the viscosity and the
// divergence's 1/dx, 1/dy, 1/dz are folded into per-face constants, so each
// face flux comes out multiplied by 1/d of its normal direction.
#pragma once

#include "fp64_recip.cuh"
#include "mprk_internal.h"

namespace mprk {

constexpr int NC3 = 5;

// Face constants of one face direction in one fluid: sc = 1/d_n is the
// divergence factor, d_n, d_t1, d_t2 the spacings normal to the face and
// along its two tangents.
enum {
  F3_HS,  // sc / 2
  F3_A,   // (4/3) mu sc / d_n
  F3_B1,  // mu sc / (6 d_t1)
  F3_B2,  // mu sc / (6 d_t2)
  F3_C,   // mu sc / d_n
  F3_D1,  // mu sc / (4 d_t1)
  F3_D2,  // mu sc / (4 d_t2)
  F3_K,   // kappa sc / d_n
  F3_SC,  // sc
  F3_N
};

// The constants of a face with normal spacing inv_dn (= sc) and tangential
// spacings inv_dt1, inv_dt2 (reciprocals) into fc[F3_N].
__device__ __forceinline__ void face_consts3(double inv_dn, double inv_dt1, double inv_dt2, double mu, double kap,
                                             double* fc) {
  const double sc = inv_dn;
  fc[F3_HS] = 0.5 * sc;
  fc[F3_A] = 4.0 / 3.0 * mu * inv_dn * sc;
  fc[F3_B1] = mu * inv_dt1 * sc / 6.0;
  fc[F3_B2] = mu * inv_dt2 * sc / 6.0;
  fc[F3_C] = mu * inv_dn * sc;
  fc[F3_D1] = 0.25 * mu * inv_dt1 * sc;
  fc[F3_D2] = 0.25 * mu * inv_dt2 * sc;
  fc[F3_K] = kap * inv_dn * sc;
  fc[F3_SC] = sc;
}

// Lax–Friedrichs flux (Sec. 2.1) in a face frame, times sc = 2 hs: a state
// is (rho, m_n, m_t1, m_t2, rho E); lambda is the largest |u_n| + a over the
// left, right and Roe-averaged states. The Roe weights times the enthalpy
// (rho E + p)/rho are formed as (rho E + p)/sqrt(rho).
__device__ __forceinline__ void lf_face5(const double l[5], const double r[5], double gamma, double gm1, double hs,
                                         double out[5]) {
  const double rsL = rsqrt_f64(l[0]), rsR = rsqrt_f64(r[0]);
  const double invL = rsL * rsL, invR = rsR * rsR;
  const double sL = l[0] * rsL, sR = r[0] * rsR;  // sqrt(rho)
  const double unL = l[1] * invL, t1L = l[2] * invL, t2L = l[3] * invL;
  const double unR = r[1] * invR, t1R = r[2] * invR, t2R = r[3] * invR;
  const double pL = gm1 * (l[4] - 0.5 * (l[1] * unL + l[2] * t1L + l[3] * t2L));
  const double pR = gm1 * (r[4] - 0.5 * (r[1] * unR + r[2] * t1R + r[3] * t2R));
  const double XL = gamma * pL * invL, XR = gamma * pR * invR;
  const double cL = XL * rsqrt_f64(XL), cR = XR * rsqrt_f64(XR);
  const double eL = l[4] + pL, eR = r[4] + pR;
  const double den = recip_f64(sL + sR);
  const double un = (sL * unL + sR * unR) * den;
  const double t1 = (sL * t1L + sR * t1R) * den;
  const double t2 = (sL * t2L + sR * t2R) * den;
  const double H = (eL * rsL + eR * rsR) * den;
  const double X = gm1 * (H - 0.5 * (un * un + t1 * t1 + t2 * t2));
  const double c = X * rsqrt_f64(X);
  const double lam = max_speed(max_speed(fabs(unL) + cL, fabs(unR) + cR), fabs(un) + c);
  const double hl = hs * lam;
  out[0] = hs * (l[1] + r[1]) + hl * (l[0] - r[0]);
  out[1] = hs * ((l[1] * unL + pL) + (r[1] * unR + pR)) + hl * (l[1] - r[1]);
  out[2] = hs * (l[2] * unL + r[2] * unR) + hl * (l[2] - r[2]);
  out[3] = hs * (l[3] * unL + r[3] * unR) + hl * (l[3] - r[3]);
  out[4] = hs * (unL * eL + unR * eR) + hl * (l[4] - r[4]);
}

// One side of a face in its frame: velocity (u_n, u_t1, u_t2), T, and the
// cell's central differences (unscaled) of the velocity along t1 (d1) and
// t2 (d2).
struct VSide {
  double u[3], T, d1[3], d2[3];
};

// Viscous flux in the face frame, times sc: (0, sigma_nn, sigma_nt1,
// sigma_nt2, u^.sigma_n + kappa dT/dn). With G[a][b] = d u_a / d x_b
// (b = normal, t1, t2): sigma_nn = mu (4/3 G00 - 2/3 (G11 + G22)),
// sigma_nt = mu (G_t0 + G_0t); the derivative factors sit in fc.
__device__ __forceinline__ void visc_face5(const VSide& L, const VSide& R, const double* fc, double out[5]) {
  const double snn = fc[F3_A] * (R.u[0] - L.u[0]) - fc[F3_B1] * (L.d1[1] + R.d1[1]) -
                     fc[F3_B2] * (L.d2[2] + R.d2[2]);
  const double snt1 = fc[F3_C] * (R.u[1] - L.u[1]) + fc[F3_D1] * (L.d1[0] + R.d1[0]);
  const double snt2 = fc[F3_C] * (R.u[2] - L.u[2]) + fc[F3_D2] * (L.d2[0] + R.d2[0]);
  out[0] = 0.0;
  out[1] = snn;
  out[2] = snt1;
  out[3] = snt2;
  out[4] = 0.5 * ((L.u[0] + R.u[0]) * snn + (L.u[1] + R.u[1]) * snt1 + (L.u[2] + R.u[2]) * snt2) +
           fc[F3_K] * (R.T - L.T);
}

// ---- shared helpers --------------------------------------------------------

struct Geo3 {
  int nx, ny, nz, n1, pitch;
  size_t plane;  // elements of one component
  __device__ __forceinline__ size_t at(int c, int k, int j, int i) const {
    return ((size_t)c * nz + k) * ny * (size_t)pitch + (size_t)j * pitch + i;
  }
};
__device__ __forceinline__ Geo3 geo3(const Geom& g) {
  Geo3 s;
  s.nx = g.nx;
  s.ny = g.ny;
  s.nz = g.nz;
  s.n1 = g.n1;
  s.pitch = g.pitch;
  s.plane = (size_t)g.nz * g.ny * g.pitch;
  return s;
}
__device__ __forceinline__ int wrap3(int i, int n) {
  if (i < 0) i += n;
  if (i >= n) i -= n;
  if (i < 0 || i >= n) i = ((i % n) + n) % n;  // only for grids narrower than the tile halo
  return i;
}

// The stage value (q_n, or q_n + h R_a on the second stage of a substep) of
// component c at (k, j, i); the full state given by rhs_in for the test hook.
__device__ __forceinline__ double stage_val3(const StageArgs& a, const Geo3& G, int c, int k, int j, int i) {
  const size_t o = G.at(c, k, j, i);
  if (a.rhs_only) return a.rhs_in[o];
  const Geom& g = a.g;
  const double* base = k < g.n1_r ? a.b.qA : a.qF;
  if (!a.rhs_only && (a.stage & 1)) {
    const double h = k < g.n1_r ? g.dt : g.hF;
    return base[o] + h * reinterpret_cast<const double*>(a.b.Ra)[o];
  }
  return base[o];
}

// (u, v, w, T) from a conserved state; gg = gamma (gamma - 1), T = gamma p / rho
__device__ __forceinline__ void prim5(const double q[5], double gg, double v[4]) {
  const double inv = recip_f64(q[0]);
  v[0] = q[1] * inv;
  v[1] = q[2] * inv;
  v[2] = q[3] * inv;
  v[3] = gg * (q[4] - 0.5 * (q[1] * v[0] + q[2] * v[1] + q[3] * v[2])) * inv;
}

// Interface state of column (i, j) (App. B, Eq. bulk-flux and the wall
// states after it): {sigma_xz, sigma_yz, Pi_z, u_w1, v_w1, T_w1, u_w2, v_w2,
// T_w2}, each fluid using its own formula.
__device__ __forceinline__ void interface3(const StageArgs& a, const Geo3& G, int j, int i, double out[9]) {
  const Geom& g = a.g;
  double v1[4], v2[4], q[5];
#pragma unroll
  for (int c = 0; c < 5; c++) q[c] = stage_val3(a, G, c, G.n1 - 1, j, i);
  prim5(q, g.gamma * g.gm1, v1);
#pragma unroll
  for (int c = 0; c < 5; c++) q[c] = stage_val3(a, G, c, G.n1, j, i);
  prim5(q, g.gamma * g.gm1, v2);
  const double sxz = g.bu * (v2[0] - v1[0]);
  const double syz = g.bu * (v2[1] - v1[1]);  // b_v = b_u
  const double Pi = -g.bT * (v2[3] - v1[3]);
  out[0] = sxz;
  out[1] = syz;
  out[2] = Pi;
  out[3] = v1[0] + sxz * g.cu1;
  out[4] = v1[1] + syz * g.cu1;
  out[5] = v1[3] - Pi * g.cT1;
  out[6] = v2[0] - sxz * g.cu2;
  out[7] = v2[1] - syz * g.cu2;
  out[8] = v2[3] + Pi * g.cT2;
}

// Central z difference (unscaled) of (u, v, w) at row k from the cell (c)
// and its neighbours above (up) and below (dn), with the ghost
// 2*(wall state) - interior beyond a wall or Gamma; gam holds the column's
// interface state.
__device__ __forceinline__ void dz_uvw(const Geom& g, int k, const double* c, const double* up, const double* dn,
                                       const double* gam, double out[3]) {
  double U[3], D[3];
  const int nz = g.nz, n1 = g.n1;
  const double st = g.wall ? 1.0 : -1.0;  // tangential ghost sign at a slip / no-slip wall
  if (k + 1 == nz) {
    U[0] = st * c[0]; U[1] = st * c[1]; U[2] = -c[2];
  } else if (k + 1 == n1) {  // fluid 1's top row: Gamma above
    U[0] = 2.0 * gam[3] - c[0]; U[1] = 2.0 * gam[4] - c[1]; U[2] = -c[2];
  } else {
    U[0] = up[0]; U[1] = up[1]; U[2] = up[2];
  }
  if (k == 0) {
    D[0] = st * c[0]; D[1] = st * c[1]; D[2] = -c[2];
  } else if (k == n1) {  // fluid 2's bottom row: Gamma below
    D[0] = 2.0 * gam[6] - c[0]; D[1] = 2.0 * gam[7] - c[1]; D[2] = -c[2];
  } else {
    D[0] = dn[0]; D[1] = dn[1]; D[2] = dn[2];
  }
#pragma unroll
  for (int a = 0; a < 3; a++) out[a] = U[a] - D[a];
}

// ---- y faces ------------------------------------------------------------------

struct YfaceSmem {
  double q0[5][TZ + 2][TX + 2];  // plane j, rows k0-1.., cols i0-1..
  double q1[5][TZ + 2][TX + 2];  // plane j+1
  double qm[5][TZ][TX];          // plane j-1, tile cells
  double qp[5][TZ][TX];          // plane j+2, tile cells
  double v0[4][TZ + 2][TX + 2];  // u, v, w, T of plane j on the ring
  double v1[4][TZ + 2][TX + 2];
  double gam0[9][TX];            // interface state of the tile columns, planes j and j+1
  double gam1[9][TX];
  double fc[2][F3_N];            // y-face constants per fluid
  double gg;                     // gamma (gamma - 1)
};

// The y faces between planes j and j+1 of the TX x TZ tile from row k0,
// column i0, times 1/dy, written to a.gy at index j.
__device__ __forceinline__ void yface_tile(const StageArgs& a, int k0, int i0, int j, YfaceSmem& S) {
  const Geom& g = a.g;
  const Geo3 G = geo3(g);
  const int tid = threadIdx.x;
  const int nz = g.nz, nx = g.nx, ny = g.ny, n1 = g.n1;
  const int row_hi = a.rhs_only ? a.rhs_hi : nz;
  const int jm = wrap3(j - 1, ny), j1 = wrap3(j + 1, ny), jp = wrap3(j + 2, ny);

  if (tid < 2) {
    // y faces: t1 = x, t2 = z
    face_consts3(g.inv_dy, g.inv_dx, tid ? g.inv_dz2 : g.inv_dz1, tid ? g.mu2 : g.mu1, tid ? g.kap2 : g.kap1,
                 S.fc[tid]);
    if (tid == 0) S.gg = g.gamma * g.gm1;
  }
  for (int e = tid; e < 5 * (TZ + 2) * (TX + 2); e += NTHREADS) {
    const int c = e / ((TZ + 2) * (TX + 2)), rem = e - c * (TZ + 2) * (TX + 2);
    const int rr = rem / (TX + 2), cc = rem - rr * (TX + 2);
    const int k = k0 - 1 + rr, i = wrap3(i0 - 1 + cc, nx);
    double x0 = 0.0, x1 = 0.0;
    if (k >= 0 && k < nz) {
      x0 = stage_val3(a, G, c, k, j, i);
      x1 = stage_val3(a, G, c, k, j1, i);
    }
    S.q0[c][rr][cc] = x0;
    S.q1[c][rr][cc] = x1;
  }
  for (int e = tid; e < 5 * TZ * TX; e += NTHREADS) {
    const int c = e / (TZ * TX), rem = e - c * TZ * TX;
    const int rr = rem / TX, cc = rem - rr * TX;
    const int k = k0 + rr, i = wrap3(i0 + cc, nx);
    double xm = 0.0, xp = 0.0;
    if (k < nz) {
      xm = stage_val3(a, G, c, k, jm, i);
      xp = stage_val3(a, G, c, k, jp, i);
    }
    S.qm[c][rr][cc] = xm;
    S.qp[c][rr][cc] = xp;
  }
  const bool has_gamma = (n1 >= k0 && n1 <= k0 + TZ);
  if (has_gamma && tid < 2 * TX) {
    const int side = tid / TX, cc = tid - side * TX;
    double st[9];
    interface3(a, G, side ? j1 : j, wrap3(i0 + cc, nx), st);
#pragma unroll
    for (int s = 0; s < 9; s++) (side ? S.gam1 : S.gam0)[s][cc] = st[s];
  }
  __syncthreads();
  for (int e = tid; e < 2 * (TZ + 2) * (TX + 2); e += NTHREADS) {
    const int side = e / ((TZ + 2) * (TX + 2)), rem = e - side * (TZ + 2) * (TX + 2);
    const int rr = rem / (TX + 2), cc = rem - rr * (TX + 2);
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    double q[5], v[4];
#pragma unroll
    for (int c = 0; c < 5; c++) q[c] = side ? S.q1[c][rr][cc] : S.q0[c][rr][cc];
    prim5(q, S.gg, v);
#pragma unroll
    for (int c = 0; c < 4; c++) (side ? S.v1 : S.v0)[c][rr][cc] = v[c];
  }
  __syncthreads();

  const int rr = tid / TX, cc = tid - rr * TX;
  const int k = k0 + rr, i = i0 + cc;
  if (k >= row_hi || i >= nx) return;
  // reconstructed states: d/dy central differences of q at j and j+1
  double L[5], R[5];
#pragma unroll
  for (int c = 0; c < 5; c++) {
    const double a0 = S.q0[c][rr + 1][cc + 1], a1 = S.q1[c][rr + 1][cc + 1];
    L[c] = a0 + 0.25 * (a1 - S.qm[c][rr][cc]);
    R[c] = a1 - 0.25 * (S.qp[c][rr][cc] - a0);
  }
  // face frame: normal rho v, tangential rho u, rho w
  const double lf[5] = {L[0], L[2], L[1], L[3], L[4]}, rf[5] = {R[0], R[2], R[1], R[3], R[4]};
  const double* fc = S.fc[k >= n1];
  double FI[5], FV[5];
  lf_face5(lf, rf, g.gamma, g.gm1, fc[F3_HS], FI);
  VSide s[2];
#pragma unroll
  for (int side = 0; side < 2; side++) {
    double (*V)[TZ + 2][TX + 2] = side ? S.v1 : S.v0;
    const double(*gam)[TX] = side ? S.gam1 : S.gam0;
    // frame order (v, u, w)
    s[side].u[0] = V[1][rr + 1][cc + 1];
    s[side].u[1] = V[0][rr + 1][cc + 1];
    s[side].u[2] = V[2][rr + 1][cc + 1];
    s[side].T = V[3][rr + 1][cc + 1];
    // x (t1) differences of (v, u, w)
    s[side].d1[0] = V[1][rr + 1][cc + 2] - V[1][rr + 1][cc];
    s[side].d1[1] = V[0][rr + 1][cc + 2] - V[0][rr + 1][cc];
    s[side].d1[2] = V[2][rr + 1][cc + 2] - V[2][rr + 1][cc];
    // z (t2) differences of (v, u, w), ghosts beyond a wall or Gamma
    const double cv[3] = {V[0][rr + 1][cc + 1], V[1][rr + 1][cc + 1], V[2][rr + 1][cc + 1]};
    const double uv[3] = {V[0][rr + 2][cc + 1], V[1][rr + 2][cc + 1], V[2][rr + 2][cc + 1]};
    const double dv[3] = {V[0][rr][cc + 1], V[1][rr][cc + 1], V[2][rr][cc + 1]};
    double gz[9];
#pragma unroll
    for (int q = 0; q < 9; q++) gz[q] = has_gamma ? gam[q][cc] : 0.0;
    double dz[3];
    dz_uvw(g, k, cv, uv, dv, gz, dz);
    s[side].d2[0] = dz[1];
    s[side].d2[1] = dz[0];
    s[side].d2[2] = dz[2];
  }
  visc_face5(s[0], s[1], fc, FV);
  const double F[5] = {FI[0] - FV[0], FI[2] - FV[2], FI[1] - FV[1], FI[3] - FV[3], FI[4] - FV[4]};
#pragma unroll
  for (int c = 0; c < 5; c++) a.gy[G.at(c, k, j, i)] = F[c];
}

// ---- x and z faces, divergence and stage combination ----------------------

struct Tile3Smem {
  double q[5][TZ + 4][TX + 4];   // plane j, rows k0-2.., cols i0-2..
  double v[4][TZ + 2][TX + 2];   // u, v, w, T on the ring
  double vy[3][TZ + 2][TX + 2];  // central y differences of u, v, w on the ring
  double hx[5][TZ][TX + 2];      // central x differences of q, tile rows, cols i0-1..
  double hz[5][TZ + 2][TX];      // central z differences of q, rows k0-1.., tile cols
  double tz[3][TZ][TX + 2];      // central z differences of u, v, w at x-face cells
  double tx[3][TZ + 2][TX];      // central x differences of u, v, w at z-face cells
  double fx[5][TZ][TX + 1];      // x face fluxes / dx, face f between cols f-1, f
  double fz[5][TZ + 1][TX];      // z face fluxes / dz seen from above
  double fg[5][TX];              // interface flux seen from fluid 1
  double gam[9][TX + 2];         // interface state per ring column
  double fc[2][2][F3_N];         // face constants per direction (x, z) and fluid
  double gg;                     // gamma (gamma - 1)
};

__device__ __forceinline__ void stage_tile3(const StageArgs& a, int k0, int i0, int j, Tile3Smem& S) {
  const Geom& g = a.g;
  const Geo3 G = geo3(g);
  const int tid = threadIdx.x;
  const int nz = g.nz, nx = g.nx, ny = g.ny, n1 = g.n1;
  const int row_hi = a.rhs_only ? a.rhs_hi : nz;
  const double gamma = g.gamma, gm1 = g.gm1;
  const int jm = wrap3(j - 1, ny), jp = wrap3(j + 1, ny);

  // ---- 1. stage state with a two-cell halo; y differences of the velocity
  // on the ring from planes j-1 and j+1; the interface state
  if (tid < 4) {
    // x faces: t1 = y, t2 = z; z faces: t1 = x, t2 = y
    const int dir = tid >> 1, fl = tid & 1;
    const double inv_dz = fl ? g.inv_dz2 : g.inv_dz1;
    const double mu = fl ? g.mu2 : g.mu1, kap = fl ? g.kap2 : g.kap1;
    if (dir == 0) face_consts3(g.inv_dx, g.inv_dy, inv_dz, mu, kap, S.fc[0][fl]);
    else face_consts3(inv_dz, g.inv_dx, g.inv_dy, mu, kap, S.fc[1][fl]);
    if (tid == 0) S.gg = g.gamma * g.gm1;
  }
  for (int e = tid; e < 5 * (TZ + 4) * (TX + 4); e += NTHREADS) {
    const int c = e / ((TZ + 4) * (TX + 4)), rem = e - c * (TZ + 4) * (TX + 4);
    const int rr = rem / (TX + 4), cc = rem - rr * (TX + 4);
    const int k = k0 - 2 + rr;
    S.q[c][rr][cc] = (k >= 0 && k < nz) ? stage_val3(a, G, c, k, j, wrap3(i0 - 2 + cc, nx)) : 0.0;
  }
  for (int e = tid; e < (TZ + 2) * (TX + 2); e += NTHREADS) {
    const int rr = e / (TX + 2), cc = e - rr * (TX + 2);
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    const int i = wrap3(i0 - 1 + cc, nx);
    double up[3], dn[3];
    {
      const double inv = recip_f64(stage_val3(a, G, 0, k, jp, i));
      up[0] = stage_val3(a, G, 1, k, jp, i) * inv;
      up[1] = stage_val3(a, G, 2, k, jp, i) * inv;
      up[2] = stage_val3(a, G, 3, k, jp, i) * inv;
    }
    {
      const double inv = recip_f64(stage_val3(a, G, 0, k, jm, i));
      dn[0] = stage_val3(a, G, 1, k, jm, i) * inv;
      dn[1] = stage_val3(a, G, 2, k, jm, i) * inv;
      dn[2] = stage_val3(a, G, 3, k, jm, i) * inv;
    }
#pragma unroll
    for (int q = 0; q < 3; q++) S.vy[q][rr][cc] = up[q] - dn[q];
  }
  const bool has_gamma = (n1 >= k0 && n1 <= k0 + TZ);
  if (has_gamma && tid < TX + 2) {
    double st[9];
    interface3(a, G, j, wrap3(i0 - 1 + tid, nx), st);
#pragma unroll
    for (int s = 0; s < 9; s++) S.gam[s][tid] = st[s];
  }
  __syncthreads();

  // ---- 2. u, v, w, T on the ring --------------------------------------------
  for (int e = tid; e < (TZ + 2) * (TX + 2); e += NTHREADS) {
    const int rr = e / (TX + 2), cc = e - rr * (TX + 2);
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    double q[5], v[4];
#pragma unroll
    for (int c = 0; c < 5; c++) q[c] = S.q[c][rr + 1][cc + 1];
    prim5(q, S.gg, v);
#pragma unroll
    for (int c = 0; c < 4; c++) S.v[c][rr][cc] = v[c];
  }
  __syncthreads();

  // ---- 3. slopes and tangential differences --------------------------------
  for (int e = tid; e < TZ * (TX + 2); e += NTHREADS) {
    const int rr = e / (TX + 2), cc = e - rr * (TX + 2);
    const int k = k0 + rr;
    if (k >= row_hi) continue;
#pragma unroll
    for (int c = 0; c < 5; c++) S.hx[c][rr][cc] = S.q[c][rr + 2][cc + 2] - S.q[c][rr + 2][cc];
    const double cv[3] = {S.v[0][rr + 1][cc], S.v[1][rr + 1][cc], S.v[2][rr + 1][cc]};
    const double uv[3] = {S.v[0][rr + 2][cc], S.v[1][rr + 2][cc], S.v[2][rr + 2][cc]};
    const double dv[3] = {S.v[0][rr][cc], S.v[1][rr][cc], S.v[2][rr][cc]};
    double gz[9];
#pragma unroll
    for (int q = 0; q < 9; q++) gz[q] = has_gamma ? S.gam[q][cc] : 0.0;
    double dz[3];
    dz_uvw(g, k, cv, uv, dv, gz, dz);
#pragma unroll
    for (int q = 0; q < 3; q++) S.tz[q][rr][cc] = dz[q];
  }
  for (int e = tid; e < (TZ + 2) * TX; e += NTHREADS) {
    const int rr = e / TX, cc = e - rr * TX;
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    const bool up_in = (k + 1 < nz) && ((k + 1 < n1) == (k < n1));
    const bool dn_in = (k - 1 >= 0) && ((k - 1 < n1) == (k < n1));
#pragma unroll
    for (int c = 0; c < 5; c++) {
      const double own = S.q[c][rr + 1][cc + 2];
      const double mir = (c == 3) ? -own : own;  // mirror ghost: rho w odd
      const double up = up_in ? S.q[c][rr + 2][cc + 2] : mir;
      const double dn = dn_in ? S.q[c][rr][cc + 2] : mir;
      S.hz[c][rr][cc] = up - dn;
    }
#pragma unroll
    for (int q = 0; q < 3; q++) S.tx[q][rr][cc] = S.v[q][rr][cc + 2] - S.v[q][rr][cc];
  }
  __syncthreads();

  // ---- 4. face fluxes -----------------------------------------------------
  constexpr int NZF = (TZ + 1) * TX, NXF = TZ * (TX + 1);
  const double st = g.wall ? 1.0 : -1.0;
  for (int e = tid; e < NZF + NXF; e += NTHREADS) {
    if (e < NZF) {
      const int f = e / TX, cc = e - f * TX;
      const int ku = k0 + f, kd = ku - 1;
      if (kd >= row_hi) continue;
      // z-frame side of ring row rh (q row rh + 1): (u_n, u_t1, u_t2) = (w, u, v)
      auto zside = [&](int rh, VSide& s) {
        s.u[0] = S.v[2][rh][cc + 1];
        s.u[1] = S.v[0][rh][cc + 1];
        s.u[2] = S.v[1][rh][cc + 1];
        s.T = S.v[3][rh][cc + 1];
        s.d1[0] = S.tx[2][rh][cc];
        s.d1[1] = S.tx[0][rh][cc];
        s.d1[2] = S.tx[1][rh][cc];
        s.d2[0] = S.vy[2][rh][cc + 1];
        s.d2[1] = S.vy[0][rh][cc + 1];
        s.d2[2] = S.vy[1][rh][cc + 1];
      };
      // reconstructed state of ring row rh in the z frame,
      // q + sq * (central difference), sq = +-1/4
      auto zstate = [&](int rh, double sq, double o[5]) {
        const double x[5] = {S.q[0][rh + 1][cc + 2] + sq * S.hz[0][rh][cc],
                             S.q[1][rh + 1][cc + 2] + sq * S.hz[1][rh][cc],
                             S.q[2][rh + 1][cc + 2] + sq * S.hz[2][rh][cc],
                             S.q[3][rh + 1][cc + 2] + sq * S.hz[3][rh][cc],
                             S.q[4][rh + 1][cc + 2] + sq * S.hz[4][rh][cc]};
        o[0] = x[0];
        o[1] = x[3];
        o[2] = x[1];
        o[3] = x[2];
        o[4] = x[4];
      };
      double FI[5], FV[5], Ff[5];
      if (ku == 0 || ku == nz) {
        // outer wall: the boundary state against its mirror; the cell
        // against its ghost 2*wall - interior (adiabatic)
        const bool below = (ku == 0);
        const int rh = below ? f + 1 : f;
        const int k = below ? ku : kd;
        const double* fc = S.fc[1][k >= n1];
        double b[5], m[5];
        zstate(rh, below ? -0.25 : 0.25, b);
#pragma unroll
        for (int c = 0; c < 5; c++) m[c] = b[c];
        m[1] = -b[1];
        if (below) lf_face5(m, b, gamma, gm1, fc[F3_HS], FI);
        else lf_face5(b, m, gamma, gm1, fc[F3_HS], FI);
        VSide C, Gh;
        zside(rh, C);
        Gh = C;
        Gh.u[0] = -C.u[0];
        Gh.d1[0] = -C.d1[0];
        Gh.d2[0] = -C.d2[0];
#pragma unroll
        for (int q = 1; q < 3; q++) {
          Gh.u[q] = st * C.u[q];
          Gh.d1[q] = st * C.d1[q];
          Gh.d2[q] = st * C.d2[q];
        }
        if (below) visc_face5(Gh, C, fc, FV);
        else visc_face5(C, Gh, fc, FV);
#pragma unroll
        for (int c = 0; c < 5; c++) Ff[c] = FI[c] - FV[c];
        // frame (rho, w, u, v, E) -> (rho, u, v, w, E)
        S.fz[0][f][cc] = Ff[0];
        S.fz[1][f][cc] = Ff[2];
        S.fz[2][f][cc] = Ff[3];
        S.fz[3][f][cc] = Ff[1];
        S.fz[4][f][cc] = Ff[4];
      } else if (ku == n1) {
        // Gamma: a rigid lid from each side (inviscid) and the bulk fluxes
        // (viscous) with each side's wall state
        const double sxz = S.gam[0][cc + 1], syz = S.gam[1][cc + 1], Pi = S.gam[2][cc + 1];
        const double *fc2 = S.fc[1][1], *fc1 = S.fc[1][0];
        double b[5], m[5];
        zstate(f + 1, -0.25, b);  // fluid 2, above
#pragma unroll
        for (int c = 0; c < 5; c++) m[c] = b[c];
        m[1] = -b[1];
        lf_face5(m, b, gamma, gm1, fc2[F3_HS], FI);
        S.fz[0][f][cc] = FI[0];
        S.fz[1][f][cc] = FI[2] - sxz * fc2[F3_SC];
        S.fz[2][f][cc] = FI[3] - syz * fc2[F3_SC];
        S.fz[3][f][cc] = FI[1];
        S.fz[4][f][cc] = FI[4] - (S.gam[6][cc + 1] * sxz + S.gam[7][cc + 1] * syz - Pi) * fc2[F3_SC];
        zstate(f, 0.25, b);  // fluid 1, below
#pragma unroll
        for (int c = 0; c < 5; c++) m[c] = b[c];
        m[1] = -b[1];
        lf_face5(b, m, gamma, gm1, fc1[F3_HS], FI);
        S.fg[0][cc] = FI[0];
        S.fg[1][cc] = FI[2] - sxz * fc1[F3_SC];
        S.fg[2][cc] = FI[3] - syz * fc1[F3_SC];
        S.fg[3][cc] = FI[1];
        S.fg[4][cc] = FI[4] - (S.gam[3][cc + 1] * sxz + S.gam[4][cc + 1] * syz - Pi) * fc1[F3_SC];
      } else {
        const double* fc = S.fc[1][kd >= n1];
        double l[5], r[5];
        zstate(f, 0.25, l);
        zstate(f + 1, -0.25, r);
        lf_face5(l, r, gamma, gm1, fc[F3_HS], FI);
        VSide sL, sR;
        zside(f, sL);
        zside(f + 1, sR);
        visc_face5(sL, sR, fc, FV);
        S.fz[0][f][cc] = FI[0] - FV[0];
        S.fz[1][f][cc] = FI[2] - FV[2];
        S.fz[2][f][cc] = FI[3] - FV[3];
        S.fz[3][f][cc] = FI[1] - FV[1];
        S.fz[4][f][cc] = FI[4] - FV[4];
      }
    } else {
      const int x = e - NZF;
      const int rr = x / (TX + 1), f = x - rr * (TX + 1);
      const int k = k0 + rr;
      if (k >= row_hi) continue;
      // face between ring cols f (L) and f+1 (R); frame = Cartesian (n = x)
      double l[5], r[5], FI[5], FV[5];
#pragma unroll
      for (int c = 0; c < 5; c++) {
        l[c] = S.q[c][rr + 2][f + 1] + 0.25 * S.hx[c][rr][f];
        r[c] = S.q[c][rr + 2][f + 2] - 0.25 * S.hx[c][rr][f + 1];
      }
      const double* fc = S.fc[0][k >= n1];
      lf_face5(l, r, gamma, gm1, fc[F3_HS], FI);
      VSide s[2];
#pragma unroll
      for (int side = 0; side < 2; side++) {
        const int col = f + side;
#pragma unroll
        for (int q = 0; q < 3; q++) {
          s[side].u[q] = S.v[q][rr + 1][col];
          s[side].d1[q] = S.vy[q][rr + 1][col];
          s[side].d2[q] = S.tz[q][rr][col];
        }
        s[side].T = S.v[3][rr + 1][col];
      }
      visc_face5(s[0], s[1], fc, FV);
#pragma unroll
      for (int c = 0; c < 5; c++) S.fx[c][rr][f] = FI[c] - FV[c];
    }
  }
  __syncthreads();

  // ---- 5. R = -div F* + s and the stage combination -------------------------
  const int rr = tid / TX, cc = tid - rr * TX;
  const int k = k0 + rr, i = i0 + cc;
  if (k >= row_hi || i >= nx) return;
  const bool under_gamma = (k == n1 - 1);
  double R[5];
#pragma unroll
  for (int c = 0; c < 5; c++) {
    // every face flux carries the 1/d of its direction already
    const double up = under_gamma ? S.fg[c][cc] : S.fz[c][rr + 1][cc];
    R[c] = (S.fx[c][rr][cc] - S.fx[c][rr][cc + 1]) + (S.fz[c][rr][cc] - up) +
           (a.gy[G.at(c, k, jm, i)] - a.gy[G.at(c, k, j, i)]);
  }
  R[3] -= S.q[0][rr + 2][cc + 2] * g.G;
  R[4] -= S.q[3][rr + 2][cc + 2] * g.G;

  const size_t row = (size_t)(k * ny + j) * g.pitch + i;  // offset within a component
  const size_t plane = G.plane;
  if (a.rhs_only) {
#pragma unroll
    for (int c = 0; c < 5; c++) a.rhs_out[(size_t)c * plane + row] = R[c];
    return;
  }
  double* Ra = reinterpret_cast<double*>(a.b.Ra);
  const int sg = a.stage;
  if (k >= g.n1_r) {
    // fast region: m Heun substeps of dt/m
#pragma unroll
    for (int c = 0; c < 5; c++) {
      const size_t o = (size_t)c * plane + row;
      if (!(sg & 1)) Ra[o] = R[c];
      else a.qF_next[o] = a.qF[o] + g.h2 * (Ra[o] + R[c]);
    }
  } else if (k >= g.nS_r) {
    // buffer: RK2 restarted from q_n each substep, weights 1/(2m)
    const size_t pb = (size_t)(g.n1_r - g.nS_r) * ny * g.pitch;
    const size_t ob = (size_t)((k - g.nS_r) * ny + j) * g.pitch + i;
    const bool last = (sg == 2 * g.m - 1);
#pragma unroll
    for (int c = 0; c < 5; c++) {
      const size_t o = (size_t)c * plane + row;
      double* acc = a.b.accB + (size_t)c * pb + ob;
      if (!(sg & 1)) Ra[o] = R[c];
      if (sg == 0) *acc = R[c];
      else if (last) *acc = a.b.qA[o] + g.h2 * (*acc + R[c]);
      else *acc = *acc + R[c];
    }
  } else {
    // slow region: stages 1 and 2 only (Algorithm 1)
    const size_t ps = (size_t)g.nS_r * ny * g.pitch;
#pragma unroll
    for (int c = 0; c < 5; c++) {
      const size_t o = (size_t)c * plane + row;
      if (sg == 0) Ra[o] = R[c];
      else a.b.accS[(size_t)c * ps + row] = a.b.qA[o] + g.hdt * (Ra[o] + R[c]);
    }
  }
}

}  // namespace mprk
