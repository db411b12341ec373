// stage_tile.cuh — the fused right-hand-side + stage-combination tile of one
// MPRK2 stage (device code; included by the kernel translation units).
//
// One CTA of TX x TZR threads owns a TX x TZR tile of cells (TZR = TZ rows,
// or TZ/2 or TZ/4 for launches of few tiles). It
//   1. stages the stage state of the tile plus a two-cell halo in shared
//      memory (x periodic; stage values q + h R_a rebuilt on the fly),
//   2. computes u, w, T on the tile plus a one-cell ring, and the interface
//      state (bulk fluxes and wall states of App. B) when the tile touches it,
//   3. computes the cell slopes: central differences of the conserved
//      variables (reconstruction) and of u, w (tangential viscous gradients),
//      with mirror or wall-state ghosts beyond walls and the interface; the
//      differences are stored unscaled and their factors (1/4 for the
//      reconstruction, 1/(2 d) for a derivative) taken up where they are used,
//   4. computes every x and z face flux of the tile once (Lax–Friedrichs
//      inviscid flux of Sec. 2.1 minus the common-value viscous flux of
//      App. B), in one direction-generic routine written in the face frame;
//      each flux comes out multiplied by the 1/dx or 1/dz of the divergence,
//   5. forms R = -div F* + s per cell and applies the partition's stage
//      combination (Eq. MRK2 in low-storage form) in double precision.
//
// Real is the arithmetic type of steps 1-5 up to R (double, or float in the
// FP32-flux mode); Store is the type of the saved stage-one right-hand side.
#pragma once

#include "fp64_recip.cuh"
#include "mprk_internal.h"

namespace mprk {

// Face constants of one face direction in one fluid (scaled by the divergence
// factor sc = 1/dx at x faces, 1/dz of the fluid at z faces; d_n and d_t are
// the spacings normal and tangential to the face).
enum {
  FC_HS,  // sc / 2: the averages of the Lax–Friedrichs flux
  FC_A,   // (4/3) mu sc / d_n: sigma_nn from the normal difference of u_n
  FC_B,   // mu sc / (6 d_t): sigma_nn from the two cells' tangential differences of u_t
  FC_C,   // mu sc / d_n: sigma_nt from the normal difference of u_t
  FC_D,   // mu sc / (4 d_t): sigma_nt from the two cells' tangential differences of u_n
  FC_K,   // kappa gamma (gamma - 1) sc / d_n: heat flux from the normal difference of e = T / (gamma (gamma - 1))
  FC_SC,  // sc
  FC_N
};

template <typename Real, int TZR = TZ>
struct TileSmem {
  Real q[4][TZR + 4][TX + 4];   // stage state, rows k0-2.., cols i0-2..
  Real v[3][TZR + 2][TX + 2];   // u, w, e = T / (gamma (gamma - 1)), rows k0-1.., cols i0-1..
  Real hx[4][TZR][TX + 2];      // central x differences of q, cols i0-1..
  Real hz[4][TZR + 2][TX];      // central z differences of q, rows k0-1..
  Real tz[2][TZR][TX + 2];      // central z differences of u, w (tangential at x faces)
  Real tx[2][TZR + 2][TX];      // central x differences of u, w (tangential at z faces)
  Real fx[4][TZR][TX + 1];      // x face fluxes / dx, face f between cols f-1, f
  Real fz[4][TZR + 1][TX];      // z face fluxes / dz seen from above
  Real fg[4][TX];              // interface flux / dz1 seen from fluid 1 (below)
  double gam[4][TX + 2];       // sigma_xz, Pi_z, u_w, T_w per column i0-1..
  Real fc[2][2][FC_N];         // face constants per direction (x, z) and fluid (1, 2)
};

template <typename Real>
__device__ __forceinline__ Real rsq(Real x);
template <>
__device__ __forceinline__ double rsq<double>(double x) { return rsqrt_f64(x); }
template <>
__device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }

template <typename Real>
__device__ __forceinline__ Real sqr(Real x);
template <>
__device__ __forceinline__ double sqr<double>(double x) { return sqrt_f64(x); }
template <>
__device__ __forceinline__ float sqr<float>(float x) { return x * rsqrtf(x); }

template <typename Real>
__device__ __forceinline__ Real rcp(Real x);
template <>
__device__ __forceinline__ double rcp<double>(double x) { return recip_f64(x); }
template <>
__device__ __forceinline__ float rcp<float>(float x) { return 1.0f / x; }

// Lax–Friedrichs flux in the face frame. A state is (rho, m_n, m_t, rho E):
// m_n is the momentum along the face normal, m_t along the face. Output is
// sc (F_rho, F_mn, F_mt, F_E) - sub, where hs = sc/2 and each component is
// hs (f(q_L) + f(q_R) + lambda (q_L - q_R)) - sub: sub carries the viscous
// or interface part of the face flux, taken off in the last fused
// multiply-add. lambda is the largest |u_n| + a over the left, right and
// Roe-averaged states (Sec. 2.1); the Roe weights sqrt(rho)/(sqrt(rho_L) +
// sqrt(rho_R)) times the enthalpy H = (rho E + p)/rho are formed as
// (rho E + p)/sqrt(rho).
template <typename Real>
__device__ __forceinline__ void lf_face(Real lr, Real lmn, Real lmt, Real lE, Real rr, Real rmn,
                                        Real rmt, Real rE, Real gamma, Real gm1, Real hs, const Real sub[4],
                                        Real out[4]) {
  const Real half = Real(0.5);
  const Real rsL = rsq(lr), rsR = rsq(rr);
  const Real invL = rsL * rsL, invR = rsR * rsR;
  const Real sL = lr * rsL, sR = rr * rsR;  // sqrt(rho)
  const Real unL = lmn * invL, utL = lmt * invL;
  const Real unR = rmn * invR, utR = rmt * invR;
  const Real pL = gm1 * (lE - half * (lmn * unL + lmt * utL));
  const Real pR = gm1 * (rE - half * (rmn * unR + rmt * utR));
  const Real cL = sqr(gamma * pL * invL), cR = sqr(gamma * pR * invR);
  const Real eL = lE + pL, eR = rE + pR;
  const Real den = rcp(sL + sR);
  const Real un = (sL * unL + sR * unR) * den;
  const Real ut = (sL * utL + sR * utR) * den;
  const Real H = (eL * rsL + eR * rsR) * den;
  const Real c = sqr(gm1 * (H - half * (un * un + ut * ut)));
  const Real lam = max_speed(max_speed(fabs(unL) + cL, fabs(unR) + cR), fabs(un) + c);
  out[0] = hs * fma(lam, lr - rr, lmn + rmn) - sub[0];
  out[1] = fma(hs, fma(lam, lmn - rmn, (lmn * unL + pL) + (rmn * unR + pR)), -sub[1]);
  out[2] = fma(hs, fma(lam, lmt - rmt, lmt * unL + rmt * unR), -sub[2]);
  out[3] = fma(hs, fma(lam, lE - rE, unL * eL + unR * eR), -sub[3]);
}

// Viscous flux in the face frame from the common values of App. B: face
// velocity = mean of the two cells, normal derivatives = two-point
// differences, tangential derivatives = mean of the two cells' central
// differences. Output (0, sigma_nn, sigma_nt, u.sigma_n + kappa dT/dn).
template <typename Real>
__device__ __forceinline__ void visc_face(Real unL, Real utL, Real TL, Real gnL, Real gtL,
                                          Real unR, Real utR, Real TR, Real gnR, Real gtR,
                                          Real inv_dn, Real mu, Real kap, Real out[4]) {
  const Real half = Real(0.5);
  const Real un = half * (unL + unR), ut = half * (utL + utR);
  const Real dn_un = (unR - unL) * inv_dn;
  const Real dn_ut = (utR - utL) * inv_dn;
  const Real dn_T = (TR - TL) * inv_dn;
  const Real dt_un = half * (gnL + gnR);  // tangential derivative of u_n
  const Real dt_ut = half * (gtL + gtR);  // tangential derivative of u_t
  const Real snn = mu * (Real(2) * dn_un - Real(2.0 / 3.0) * (dn_un + dt_ut));
  const Real snt = mu * (dn_ut + dt_un);
  out[0] = Real(0);
  out[1] = snn;
  out[2] = snt;
  out[3] = un * snn + ut * snt + kap * dn_T;
}

// visc_face with the spacings, viscosity and divergence factor folded into
// the face constants fc (FC_*): the tangential inputs gn, gt are the cells'
// unscaled central differences of u_n, u_t along the face, and TL, TR the
// cells' temperatures in the units of fc[FC_K] (the tile passes e = T /
// (gamma (gamma - 1)) and folds that factor into FC_K). Output
// sc (0, sigma_nn, sigma_nt, u.sigma_n + kappa dT/dn); the same sums as
// visc_face, regrouped.
template <typename Real>
__device__ __forceinline__ void visc_face_fc(Real unL, Real utL, Real TL, Real gnL, Real gtL, Real unR,
                                             Real utR, Real TR, Real gnR, Real gtR, const Real* fc,
                                             Real out[4]) {
  const Real snn = fc[FC_A] * (unR - unL) - fc[FC_B] * (gtL + gtR);
  const Real snt = fc[FC_C] * (utR - utL) + fc[FC_D] * (gnL + gnR);
  out[0] = Real(0);
  out[1] = snn;
  out[2] = snt;
  out[3] = Real(0.5) * ((unL + unR) * snn + (utL + utR) * snt) + fc[FC_K] * (TR - TL);
}

__device__ __forceinline__ int wrap_col(int i, int nx) {
  if (i < 0) i += nx;
  if (i >= nx) i %= nx;
  return i;
}

// The cell that halo column i stands for: its periodic image, or with x
// walls its mirror image across the nearer wall. In that case *ghost is set
// and the caller builds the wall ghosts: rho u flips (mirror state), u flips
// and, at a no-slip wall, w flips ((u, w, T) ghost = 2 wall state - cell).
// Far ghosts of a tile wider than the grid feed no cell of the grid and are
// clamped into it.
__device__ __forceinline__ int halo_col(int i, int nx, int xwall, bool* ghost) {
  *ghost = false;
  if (!xwall) return wrap_col(i, nx);
  if (i < 0) {
    *ghost = true;
    i = -1 - i;
  } else if (i >= nx) {
    *ghost = true;
    i = 2 * nx - 1 - i;
  }
  return i < 0 ? 0 : (i >= nx ? nx - 1 : i);
}
// Is halo column i an x-wall ghost?
__device__ __forceinline__ bool x_ghost(int i, int nx, int xwall) { return xwall && (i < 0 || i >= nx); }

// The tile body. tile = linear tile index within the launch's row range.
// Not inlined: the single-instance kernel and the persistent batch kernel
// then run the very same compiled body, so an instance's results are bitwise
// the same alone and in a batch.
// The stage value of a general s-stage base (GEN): base + h sum_{q<p}
// A_pq R_q over the R_a slots of the current substep (slot q at
// Ra + q * slot); p = 0 gives the base value. Every product-sum is an
// explicit fused multiply-add, so no launch shape or kernel that compiles
// this code can round it differently.
__device__ __forceinline__ double gen_stage_value(const Geom& g, const double* base, const double* Ra, size_t slot,
                                                  size_t off, int p, double h) {
  if (p == 0) return base[off];
  double sum = 0.0;
  for (int q = 0; q < p; q++)
    if (g.bA[p][q] != 0.0) sum = __fma_rn(g.bA[p][q], Ra[(size_t)q * slot + off], sum);
  return __fma_rn(h, sum, base[off]);
}

// sum_q b_q R_q over the first s - 1 R_a slots and the current R (slot
// s - 1), as explicit fused multiply-adds in ascending q.
__device__ __forceinline__ double gen_weighted_sum(const Geom& g, const double* Rs, size_t slot, size_t o, double r) {
  double sum = 0.0;
  for (int q = 0; q < g.s - 1; q++) sum = __fma_rn(g.bb[q], Rs[(size_t)q * slot + o], sum);
  return __fma_rn(g.bb[g.s - 1], r, sum);
}

// GEN selects the general s-stage base method (Sec. 3 remark) in place of
// Heun's low-storage path: s R_a slots, the stage values of the region
// tableaus built from the base, and its weights b in the combinations.
// NT: threads of the CTA. TX x TZR gives one thread per cell; launches with
// fewer tiles than the GPU has SMs take twice that, so that each SM holds
// more warps of the few tiles there are: every phase but the last spreads
// its work over all threads, and the last (one cell per thread) uses the
// first TX x TZR. TZR: tile rows.
template <typename Real, typename Store, bool GEN = false, int NT = NTHREADS, int TZR = TZ>
__device__ __noinline__ void stage_tile(const StageArgs& __restrict__ a, int tile,
                                       TileSmem<Real, TZR>& __restrict__ S) {
  // __restrict__: the argument block and shared memory never alias, so its
  // fields need not be reloaded after shared-memory stores
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int tzi = tile / a.tiles_x;
  const int txi = tile - tzi * a.tiles_x;
  const int k0 = a.row0 + tzi * TZR;
  const int i0 = txi * TX;
  const int nz = g.nz, nx = g.nx, n1 = g.n1;
  const int row_hi = a.rhs_only ? a.rhs_hi : nz;
  const size_t plane = (size_t)nz * g.pitch;
  const bool odd_stage = !a.rhs_only && (a.stage & 1);  // stages 2, 4, ... (1-based)
  const Store* Ra = reinterpret_cast<const Store*>(a.b.Ra);
  const double hF = g.hF;

  // ---- 1. stage state of the tile and its halo --------------------------
  if (tid < 4) {
    // face constants of direction tid >> 1 (x, z) in fluid tid & 1
    const int dir = tid >> 1, fl = tid & 1;
    const double inv_dz = fl ? g.inv_dz2 : g.inv_dz1;
    const double mu = fl ? g.mu2 : g.mu1, kap = fl ? g.kap2 : g.kap1;
    const double inv_dn = dir ? inv_dz : g.inv_dx, inv_dt = dir ? g.inv_dx : inv_dz;
    const double sc = inv_dn;  // the divergence factor is the normal one
    Real* fc = S.fc[dir][fl];
    fc[FC_HS] = (Real)(0.5 * sc);
    fc[FC_A] = (Real)(4.0 / 3.0 * mu * inv_dn * sc);
    fc[FC_B] = (Real)(mu * inv_dt * sc / 6.0);
    fc[FC_C] = (Real)(mu * inv_dn * sc);
    fc[FC_D] = (Real)(0.25 * mu * inv_dt * sc);
    fc[FC_K] = (Real)(kap * inv_dn * sc * (g.gamma * g.gm1));  // times the factor T / e of S.v[2]
    fc[FC_SC] = (Real)sc;
  }
  for (int e = tid; e < 4 * (TZR + 4) * (TX + 4); e += NT) {
    const int c = e / ((TZR + 4) * (TX + 4));
    const int rem = e - c * ((TZR + 4) * (TX + 4));
    const int rr = rem / (TX + 4), cc = rem - rr * (TX + 4);
    const int k = k0 - 2 + rr;
    Real val = Real(0);
    if (k >= 0 && k < nz) {
      bool gh;
      const int i = halo_col(i0 - 2 + cc, nx, g.xwall, &gh);
      const size_t off = (size_t)c * plane + (size_t)k * g.pitch + i;
      if (a.rhs_only) {
        val = (Real)a.rhs_in[off];
      } else {
        const double* base = k < g.n1_r ? a.b.qA : a.qF;
        if (GEN) {
          val = (Real)gen_stage_value(g, base, reinterpret_cast<const double*>(Ra), 4 * plane, off,
                                      a.stage % g.s, k < g.n1_r ? g.dt : hF);
        } else if (odd_stage) {
          const Real h = (Real)(k < g.n1_r ? g.dt : hF);
          val = (Real)base[off] + h * (Real)Ra[off];
        } else {
          val = (Real)base[off];
        }
      }
      if (gh && c == 1) val = -val;  // mirror state beyond an x wall
    }
    S.q[c][rr][cc] = val;
  }
  const bool has_gamma = (n1 >= k0 && n1 <= k0 + TZR);
  __syncthreads();

  // ---- 2. u, w, T on the one-cell ring; interface state -----------------
  const Real gamma = (Real)g.gamma, gm1 = (Real)g.gm1;
  for (int e = tid; e < (TZR + 2) * (TX + 2); e += NT) {
    const int rr = e / (TX + 2), cc = e - rr * (TX + 2);
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    const Real r = S.q[0][rr + 1][cc + 1], mu_ = S.q[1][rr + 1][cc + 1];
    const Real mw = S.q[2][rr + 1][cc + 1], E = S.q[3][rr + 1][cc + 1];
    const Real inv = rcp(r);
    const Real u = mu_ * inv, w = mw * inv;
    S.v[0][rr][cc] = u;
    // the mirror state's u is already flipped; a no-slip wall flips w too
    S.v[1][rr][cc] = (x_ghost(i0 - 1 + cc, nx, g.xwall) && g.wall == 0) ? -w : w;
    // internal energy per mass e = T / (gamma (gamma - 1)) with T = gamma p / rho;
    // the heat-flux constant carries the factor
    S.v[2][rr][cc] = (E - Real(0.5) * (mu_ * u + mw * w)) * inv;
  }
  if (has_gamma && tid < TX + 2) {
    // Interface state of column i0-1+tid in double precision from the two
    // cells touching Gamma (App. B, Eq. bulk-flux and the wall states).
    bool gh;
    const int i = halo_col(i0 - 1 + tid, nx, g.xwall, &gh);
    double u[2], T[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const int k = n1 - 1 + s;
      double qq[4];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const size_t off = (size_t)c * plane + (size_t)k * g.pitch + i;
        if (a.rhs_only) {
          qq[c] = a.rhs_in[off];
        } else {
          const double* base = k < g.n1_r ? a.b.qA : a.qF;
          if (GEN) {
            qq[c] = gen_stage_value(g, base, reinterpret_cast<const double*>(Ra), 4 * plane, off, a.stage % g.s,
                                    k < g.n1_r ? g.dt : hF);
          } else if (odd_stage) {
            qq[c] = base[off] + (k < g.n1_r ? g.dt : hF) * (double)Ra[off];
          } else {
            qq[c] = base[off];
          }
        }
      }
      if (gh) qq[1] = -qq[1];  // mirror state beyond an x wall
      const double inv = 1.0 / qq[0];
      u[s] = qq[1] * inv;
      const double w = qq[2] * inv;
      const double p = g.gm1 * (qq[3] - 0.5 * (qq[1] * u[s] + qq[2] * w));
      T[s] = g.gamma * p * inv;
    }
    const double sig = g.bu * (u[1] - u[0]);
    const double Pi = -g.bT * (T[1] - T[0]);
    S.gam[0][tid] = sig;
    S.gam[1][tid] = Pi;
    S.gam[2][tid] = u[0] + sig * g.cu1;
    S.gam[3][tid] = T[0] - Pi * g.cT1;
  }
  __syncthreads();

  // ---- 3. slopes ---------------------------------------------------------
  // (a) central x differences of q on tile rows, cols i0-1 .. i0+TX
  for (int e = tid; e < TZR * (TX + 2); e += NT) {
    const int rr = e / (TX + 2), cc = e - rr * (TX + 2);
    if (k0 + rr >= row_hi) continue;
#pragma unroll
    for (int c = 0; c < 4; c++) S.hx[c][rr][cc] = S.q[c][rr + 2][cc + 2] - S.q[c][rr + 2][cc];
    // z differences of u, w at the same cells (tangential at x faces)
    const int k = k0 + rr;
    const Real u = S.v[0][rr + 1][cc], w = S.v[1][rr + 1][cc];
    Real uu, wu, ud, wd;  // values above and below, or their ghosts
    const bool top_wall = (k + 1 == nz), bot_wall = (k == 0);
    const bool top_gam = (k + 1 == n1), bot_gam = (k == n1);
    if (top_wall) { uu = g.wall ? u : -u; wu = -w; }
    else if (top_gam) { uu = Real(2) * (Real)S.gam[2][cc] - u; wu = -w; }
    else { uu = S.v[0][rr + 2][cc]; wu = S.v[1][rr + 2][cc]; }
    if (bot_wall) { ud = g.wall ? u : -u; wd = -w; }
    else if (bot_gam) { ud = Real(2) * (Real)S.gam[2][cc] - u; wd = -w; }
    else { ud = S.v[0][rr][cc]; wd = S.v[1][rr][cc]; }
    S.tz[0][rr][cc] = uu - ud;
    S.tz[1][rr][cc] = wu - wd;
  }
  // (b) central z differences of q on ring rows k0-1 .. k0+TZR, tile cols
  for (int e = tid; e < (TZR + 2) * TX; e += NT) {
    const int rr = e / TX, cc = e - rr * TX;
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    const bool up_in = (k + 1 < nz) && ((k + 1 < n1) == (k < n1));
    const bool dn_in = (k - 1 >= 0) && ((k - 1 < n1) == (k < n1));
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const Real own = S.q[c][rr + 1][cc + 2];
      const Real mir = (c == 2) ? -own : own;  // mirror ghost: rho w odd
      const Real up = up_in ? S.q[c][rr + 2][cc + 2] : mir;
      const Real dn = dn_in ? S.q[c][rr][cc + 2] : mir;
      S.hz[c][rr][cc] = up - dn;
    }
    S.tx[0][rr][cc] = S.v[0][rr][cc + 2] - S.v[0][rr][cc];
    S.tx[1][rr][cc] = S.v[1][rr][cc + 2] - S.v[1][rr][cc];
  }
  __syncthreads();

  // ---- 4. face fluxes ----------------------------------------------------
  // z faces first: (TZR+1) rows of TX faces, one warp per face row; then x
  // faces. Every warp sees one face kind.
  const Real quarter = Real(0.25);
  constexpr int NZF = (TZR + 1) * TX, NXF = TZR * (TX + 1);
  for (int e = tid; e < NZF + NXF; e += NT) {
    Real F[4];
    if (e < NZF) {
      const int f = e / TX, cc = e - f * TX;
      const int ku = k0 + f;  // row above the face
      const int kd = ku - 1;  // row below the face
      // needed by a cell of the tile: the cell below (f >= 1) or above (f == 0)
      if (kd >= row_hi) continue;
      // reconstructed state of the cell at tile row rq (halo rows) / ring row
      // rh in the face frame (normal = z): q + sq * (central z difference),
      // sq = +-1/4
      auto load_side = [&](int rq, int rh, Real& r, Real& mn, Real& mt, Real& E, Real sq) {
        r = S.q[0][rq][cc + 2] + sq * S.hz[0][rh][cc];
        mt = S.q[1][rq][cc + 2] + sq * S.hz[1][rh][cc];
        mn = S.q[2][rq][cc + 2] + sq * S.hz[2][rh][cc];
        E = S.q[3][rq][cc + 2] + sq * S.hz[3][rh][cc];
      };
      if (ku == 0 || ku == nz) {
        // outer wall: the boundary cell against its mirror (inviscid) and its
        // ghost 2*wall - interior (viscous); no-slip or slip, adiabatic
        const bool below = (ku == 0);  // wall under row 0
        const int rq = below ? f + 2 : f + 1;
        const int rh = below ? f + 1 : f;
        const int rv = below ? f + 1 : f;
        const int k = below ? ku : kd;
        const Real* fc = S.fc[1][k >= n1];
        Real r, mn, mt, E;
        load_side(rq, rh, r, mn, mt, E, below ? -quarter : quarter);
        Real F[4], FV[4];
        const Real un = S.v[1][rv][cc + 1], ut = S.v[0][rv][cc + 1], T = S.v[2][rv][cc + 1];
        const Real gn = S.tx[1][rv][cc], gt = S.tx[0][rv][cc];
        const Real utg = g.wall ? ut : -ut, gtg = g.wall ? gt : -gt;
        if (below) visc_face_fc(-un, utg, T, -gn, gtg, un, ut, T, gn, gt, fc, FV);
        else visc_face_fc(un, ut, T, gn, gt, -un, utg, T, -gn, gtg, fc, FV);
        if (below) lf_face(r, -mn, mt, E, r, mn, mt, E, gamma, gm1, fc[FC_HS], FV, F);
        else lf_face(r, mn, mt, E, r, -mn, mt, E, gamma, gm1, fc[FC_HS], FV, F);
        S.fz[0][f][cc] = F[0];
        S.fz[1][f][cc] = F[2];
        S.fz[2][f][cc] = F[1];
        S.fz[3][f][cc] = F[3];
      } else if (ku == n1) {
        // the interface: a rigid lid seen from each fluid (inviscid), the bulk
        // fluxes of App. B (viscous, shared by both fluids)
        const double sig = S.gam[0][cc + 1], Pi = S.gam[1][cc + 1], uw = S.gam[2][cc + 1];
        const Real Vt = (Real)sig, VE = (Real)(uw * sig - Pi);
        const Real *fc2 = S.fc[1][1], *fc1 = S.fc[1][0];
        Real r, mn, mt, E, F[4];
        load_side(f + 2, f + 1, r, mn, mt, E, -quarter);  // fluid 2, above
        const Real sub2[4] = {Real(0), Real(0), Vt * fc2[FC_SC], VE * fc2[FC_SC]};
        lf_face(r, -mn, mt, E, r, mn, mt, E, gamma, gm1, fc2[FC_HS], sub2, F);
        S.fz[0][f][cc] = F[0];
        S.fz[1][f][cc] = F[2];
        S.fz[2][f][cc] = F[1];
        S.fz[3][f][cc] = F[3];
        load_side(f + 1, f, r, mn, mt, E, quarter);  // fluid 1, below
        const Real sub1[4] = {Real(0), Real(0), Vt * fc1[FC_SC], VE * fc1[FC_SC]};
        lf_face(r, mn, mt, E, r, -mn, mt, E, gamma, gm1, fc1[FC_HS], sub1, F);
        S.fg[0][cc] = F[0];
        S.fg[1][cc] = F[2];
        S.fg[2][cc] = F[1];
        S.fg[3][cc] = F[3];
      } else {
        const Real* fc = S.fc[1][kd >= n1];
        Real lr, lmn, lmt, lE, rr_, rmn, rmt, rE, F[4], FV[4];
        load_side(f + 1, f, lr, lmn, lmt, lE, quarter);
        load_side(f + 2, f + 1, rr_, rmn, rmt, rE, -quarter);
        visc_face_fc(S.v[1][f][cc + 1], S.v[0][f][cc + 1], S.v[2][f][cc + 1], S.tx[1][f][cc], S.tx[0][f][cc],
                     S.v[1][f + 1][cc + 1], S.v[0][f + 1][cc + 1], S.v[2][f + 1][cc + 1], S.tx[1][f + 1][cc],
                     S.tx[0][f + 1][cc], fc, FV);
        lf_face(lr, lmn, lmt, lE, rr_, rmn, rmt, rE, gamma, gm1, fc[FC_HS], FV, F);
        S.fz[0][f][cc] = F[0];
        S.fz[1][f][cc] = F[2];
        S.fz[2][f][cc] = F[1];
        S.fz[3][f][cc] = F[3];
      }
    } else {
      const int x = e - NZF;
      const int rr = x / (TX + 1), f = x - rr * (TX + 1);
      const int k = k0 + rr;
      if (k >= row_hi) continue;
      // face between columns i0+f-1 (L, ring col f) and i0+f (R, ring col f+1)
      // q +- 1/4 (central difference); the products are exact, so each sum
      // rounds once
      const Real lr = S.q[0][rr + 2][f + 1] + quarter * S.hx[0][rr][f];
      const Real lmn = S.q[1][rr + 2][f + 1] + quarter * S.hx[1][rr][f];
      const Real lmt = S.q[2][rr + 2][f + 1] + quarter * S.hx[2][rr][f];
      const Real lE = S.q[3][rr + 2][f + 1] + quarter * S.hx[3][rr][f];
      const Real rr_ = S.q[0][rr + 2][f + 2] - quarter * S.hx[0][rr][f + 1];
      const Real rmn = S.q[1][rr + 2][f + 2] - quarter * S.hx[1][rr][f + 1];
      const Real rmt = S.q[2][rr + 2][f + 2] - quarter * S.hx[2][rr][f + 1];
      const Real rE = S.q[3][rr + 2][f + 2] - quarter * S.hx[3][rr][f + 1];
      const Real* fc = S.fc[0][k >= n1];
      Real F[4], FV[4];
      visc_face_fc(S.v[0][rr + 1][f], S.v[1][rr + 1][f], S.v[2][rr + 1][f], S.tz[0][rr][f], S.tz[1][rr][f],
                   S.v[0][rr + 1][f + 1], S.v[1][rr + 1][f + 1], S.v[2][rr + 1][f + 1], S.tz[0][rr][f + 1],
                   S.tz[1][rr][f + 1], fc, FV);
      lf_face(lr, lmn, lmt, lE, rr_, rmn, rmt, rE, gamma, gm1, fc[FC_HS], FV, F);
      S.fx[0][rr][f] = F[0];
      S.fx[1][rr][f] = F[1];
      S.fx[2][rr][f] = F[2];
      S.fx[3][rr][f] = F[3];
    }
  }
  __syncthreads();

  // ---- 5. R = -div F* + s and the stage combination ----------------------
  {
    const int rr = tid / TX, cc = tid - rr * TX;
    const int k = k0 + rr, i = i0 + cc;
    if (rr >= TZR || k >= row_hi || i >= nx) return;
    const bool under_gamma = (k == n1 - 1);
    Real R[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      // the face fluxes carry 1/dx and 1/dz already
      const Real up = under_gamma ? S.fg[c][cc] : S.fz[c][rr + 1][cc];
      R[c] = (S.fx[c][rr][cc] - S.fx[c][rr][cc + 1]) + (S.fz[c][rr][cc] - up);
    }
    const Real Gr = (Real)g.G;
    R[2] -= S.q[0][rr + 2][cc + 2] * Gr;
    R[3] -= S.q[2][rr + 2][cc + 2] * Gr;

    const size_t row_off = (size_t)k * g.pitch + i;
    if (a.rhs_only) {
#pragma unroll
      for (int c = 0; c < 4; c++) a.rhs_out[(size_t)c * plane + row_off] = (double)R[c];
      return;
    }
    Store* Ra_w = reinterpret_cast<Store*>(a.b.Ra);
    const int st = a.stage;
    const double h2 = g.h2;
    if (GEN) {
      // general s-stage base: R to slot p; F rows finish a substep with the
      // weights b/m, B rows accumulate b_p R over the slow step, S rows finish
      // after the first substep
      double* Rs = reinterpret_cast<double*>(a.b.Ra);
      const size_t slot = 4 * plane;
      const int s = g.s, p = st % s;
      const bool sub_end = (p == s - 1);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const size_t o = (size_t)c * plane + row_off;
        const double r = (double)R[c];
        if (!sub_end) Rs[(size_t)p * slot + o] = r;
        if (k >= g.n1_r) {
          if (sub_end) a.qF_next[o] = __fma_rn(g.hF, gen_weighted_sum(g, Rs, slot, o, r), a.qF[o]);
        } else if (k >= g.nS_r) {
          const size_t pb = (size_t)(g.n1_r - g.nS_r) * g.pitch;
          double* acc = a.b.accB + (size_t)c * pb + (size_t)(k - g.nS_r) * g.pitch + i;
          const double v = (st == 0) ? __dmul_rn(g.bb[p], r) : __fma_rn(g.bb[p], r, *acc);
          *acc = (st == s * g.m - 1) ? __fma_rn(g.hF, v, a.b.qA[o]) : v;
        } else if (sub_end) {
          a.b.accS[(size_t)c * ((size_t)g.nS_r * g.pitch) + row_off] =
              __fma_rn(g.dt, gen_weighted_sum(g, Rs, slot, o, r), a.b.qA[o]);
        }
      }
      return;
    }
    if (k >= g.n1_r) {
      // fast region: m Heun substeps of dt/m
      if (!(st & 1)) {
#pragma unroll
        for (int c = 0; c < 4; c++) Ra_w[(size_t)c * plane + row_off] = (Store)R[c];
      } else {
#pragma unroll
        for (int c = 0; c < 4; c++) {
          const size_t o = (size_t)c * plane + row_off;
          a.qF_next[o] = a.qF[o] + h2 * ((double)Ra[o] + (double)R[c]);
        }
      }
    } else if (k >= g.nS_r) {
      // buffer: RK2 restarted from q_n each substep, weights 1/(2m)
      const size_t pb = (size_t)(g.n1_r - g.nS_r) * g.pitch;
      const size_t ob = (size_t)(k - g.nS_r) * g.pitch + i;
      const bool last = (st == 2 * g.m - 1);
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const size_t o = (size_t)c * plane + row_off;
        double* acc = a.b.accB + (size_t)c * pb + ob;
        if (!(st & 1)) Ra_w[o] = (Store)R[c];
        if (st == 0) {
          *acc = (double)R[c];
        } else if (last) {
          *acc = a.b.qA[o] + h2 * (*acc + (double)R[c]);
        } else {
          *acc = *acc + (double)R[c];
        }
      }
    } else {
      // slow region: evaluated at stages 1 and 2 only (Algorithm 1)
      const size_t ps = (size_t)g.nS_r * g.pitch;
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const size_t o = (size_t)c * plane + row_off;
        if (st == 0) {
          Ra_w[o] = (Store)R[c];
        } else {
          a.b.accS[(size_t)c * ps + row_off] = a.b.qA[o] + g.hdt * ((double)Ra[o] + (double)R[c]);
        }
      }
    }
  }
}

}  // namespace mprk
