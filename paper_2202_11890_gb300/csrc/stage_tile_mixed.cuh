// stage_tile_mixed.cuh — the fused stage tile of the FP32-flux mode.
//
// Fluxes and R are evaluated in float. Stage values, the buffer
// accumulation, the interface bulk fluxes and every stage combination stay
// double. To keep float's rounding away from the large, nearly cancelling
// hydrostatic pressure, the tile works on deviations from a per-row
// reference state q_ref(k) (the row means of the initial state). The kernel
// reads a float shadow d = q - q_ref of the double state. The pressure enters
// the normal-momentum flux only as p - p_ref. The reference pressure's
// divergence and the reference gravity source are folded, in double, into
// one per-row constant added to R(rho w). Everything else (velocities, wave
// speeds, the viscous terms, the energy flux) uses full float states
// q_ref + d.
//
// The GB300 converts between float and double at the FP64 rate (2 per
// clock per SM, measured), so the hot loop converts with integer bit
// operations (IEEE-754 round-to-nearest-even; exact widening). The FP64 pipe
// only sees the accumulation into the double state: one DFMA per component
// per fast substep.
//
// Layout for few instructions per cell: one thread owns one cell of the
// TX x TZ tile and computes the x face on its left and the z face below it;
// a ninth warp computes the faces on the tile's right and top edges.
// Per-cell quantities sit in shared memory as float4 (one 16-byte load
// each). The right x face of a cell comes from the neighbouring lane by a
// warp shuffle.
#pragma once

#include "mprk_internal.h"
#include "stage_tile.cuh"

namespace mprk {

// ---- conversions by bit operations (IEEE-754 binary32 / binary64) --------

// float -> double, exact. Zero, subnormal, Inf and NaN take the hardware path.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)f;
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(e + (1023u - 127u)) << 52) |
                                  ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// double -> float, rounded to nearest, ties to even. Results that would be
// zero, subnormal, out of range, Inf or NaN take the hardware path.
__device__ __forceinline__ float narrow(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int fe = (int)((b >> 52) & 0x7FFu) - 1023 + 127;
  if (fe < 1 || fe > 254) return (float)x;
  const unsigned hi = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned m = (unsigned)((b >> 29) & 0x7FFFFFu);
  const unsigned rem = (unsigned)(b & 0x1FFFFFFFu);
  unsigned f = hi | ((unsigned)fe << 23) | m;
  // a carry out of the mantissa correctly bumps the exponent (to Inf at the top)
  f += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float(f);
}

// Per-row constants (float), index [j * nz + k]:
//   0-3   q_ref (rho, rho u, rho w, rho E)
//   4-7   quarter z difference of q_ref with the mirror rule at walls and Gamma
//   8-11  q_ref(k) - q_ref(k+1)
//   12    kinetic energy of q_ref
//   13    reference pressure divergence and gravity for R(rho w)
//   14    p_ref
constexpr int NROWC = 16;

// Nine warps: warps 0-7 own the TX x TZ cells, warp 8 computes the faces on
// the tile's top edge (one pass) and right edge (one pass), so every warp
// makes two face passes.
constexpr int MIXED_THREADS = NTHREADS + 32;

struct MixedSmem {
  float4 q[TZ + 4][TX + 4];   // deviation d of the stage state (rho, mu, mw, E)
  float4 v[TZ + 2][TX + 2];   // (u, w, T, -) full values on the one-cell ring
  float4 hx[TZ][TX + 2];      // quarter x differences of d
  float4 hz[TZ + 2][TX];      // quarter z differences of d plus the reference part
  float2 tz[TZ][TX + 2];      // d/dz of (u, w)
  float2 tx[TZ + 2][TX];      // d/dx of (u, w)
  float4 fz[TZ + 1][TX];      // z face fluxes seen from above (rho, mu, mw, E order)
  float4 fxr[TZ];             // x face on the tile's right edge, per row
  float4 fg[TX];              // interface flux seen from fluid 1 (below)
  float rc[NROWC][TZ + 4];    // row constants of rows k0-2 ..
  double gam[4][TX + 2];      // sigma_xz, Pi_z, u_w, T_w per column i0-1 ..
};

// Lax–Friedrichs flux in the face frame from references and deviations.
// (r, mn, mt, E): reference of the side's row; (dr, dmn, dmt, dE): its
// reconstructed deviation; ke, pr: the row's reference kinetic energy and
// pressure. dq: q_left - q_right in the face frame. The normal-momentum flux
// carries p - p_ref only.
__device__ __forceinline__ void lf_face_dev(float rL, float mnL_, float mtL_, float EL_, float keL,
                                            float prL, float drL, float dmnL, float dmtL, float dEL,
                                            float rR, float mnR_, float mtR_, float ER_, float keR,
                                            float prR, float drR, float dmnR, float dmtR, float dER,
                                            const float dq[4], float gamma, float gm1,
                                            float out[4]) {
  const float lr = rL + drL, lmn = mnL_ + dmnL, lmt = mtL_ + dmtL, lE = EL_ + dEL;
  const float rr = rR + drR, rmn = mnR_ + dmnR, rmt = mtR_ + dmtR, rE = ER_ + dER;
  const float rsL = rsqrtf(lr), rsR = rsqrtf(rr);
  const float invL = rsL * rsL, invR = rsR * rsR;
  const float sL = lr * rsL, sR = rr * rsR;
  const float unL = lmn * invL, utL = lmt * invL;
  const float unR = rmn * invR, utR = rmt * invR;
  const float dpL = gm1 * (dEL - (0.5f * (lmn * unL + lmt * utL) - keL));
  const float dpR = gm1 * (dER - (0.5f * (rmn * unR + rmt * utR) - keR));
  const float pL = prL + dpL, pR = prR + dpR;
  const float XL = gamma * pL * invL, XR = gamma * pR * invR;
  const float cL = XL * rsqrtf(XL), cR = XR * rsqrtf(XR);
  const float HL = (lE + pL) * invL, HR = (rE + pR) * invR;
  const float den = __frcp_rn(sL + sR);
  const float un = (sL * unL + sR * unR) * den;
  const float ut = (sL * utL + sR * utR) * den;
  const float H = (sL * HL + sR * HR) * den;
  const float X = gm1 * (H - 0.5f * (un * un + ut * ut));
  const float c = X * rsqrtf(X);
  const float lam = fmaxf(fmaxf(fabsf(unL) + cL, fabsf(unR) + cR), fabsf(un) + c);
  const float hl = 0.5f * lam;
  out[0] = 0.5f * (lmn + rmn) + hl * dq[0];
  out[1] = 0.5f * ((lmn * unL + dpL) + (rmn * unR + dpR)) + hl * dq[1];
  out[2] = 0.5f * (lmt * unL + rmt * unR) + hl * dq[2];
  out[3] = 0.5f * (unL * (lE + pL) + unR * (rE + pR)) + hl * dq[3];
}

// One side of a z face in the face frame (normal = z: mn = rho w, mt = rho u).
struct SideZ {
  float r, mn, mt, E, ke, p;  // reference of the row
  float dr, dmn, dmt, dE;     // reconstructed deviation
};

__device__ __forceinline__ SideZ side_z(const MixedSmem& S, int rq, int rh, int cc, float sgn) {
  SideZ s;
  s.r = S.rc[0][rq];
  s.mt = S.rc[1][rq];
  s.mn = S.rc[2][rq];
  s.E = S.rc[3][rq];
  s.ke = S.rc[12][rq];
  s.p = S.rc[14][rq];
  const float4 q = S.q[rq][cc + 2];
  const float4 h = S.hz[rh][cc];
  s.dr = q.x + sgn * h.x;
  s.dmt = q.y + sgn * h.y;
  s.dmn = q.z + sgn * h.z;
  s.dE = q.w + sgn * h.w;
  return s;
}

// The z face f of the tile (between halo rows f+1 and f+2, i.e. rows k0+f-1
// and k0+f) in column cc: writes fz[f][cc], and fg[cc] at the interface.
__device__ __forceinline__ void z_face(const StageArgs& a, MixedSmem& S, int k0, int f, int cc) {
  const Geom& g = a.g;
  const int nz = g.nz, n1 = g.n1;
  const int ku = k0 + f, kd = ku - 1;
  const float gamma = g.gammaf, gm1 = g.gm1f;
  if (ku == 0 || ku == nz) {
    // outer wall: the boundary cell against its mirror (inviscid) and its
    // ghost 2*wall - interior (viscous); no-slip or slip, adiabatic
    const bool below = (ku == 0);
    const int rq = below ? f + 2 : f + 1, rh = below ? f + 1 : f, rv = below ? f + 1 : f;
    const SideZ s = side_z(S, rq, rh, cc, below ? -1.f : 1.f);
    const float dq[4] = {0.f, below ? -2.f * (s.mn + s.dmn) : 2.f * (s.mn + s.dmn), 0.f, 0.f};
    float FI[4], FV[4];
    if (below)
      lf_face_dev(s.r, -s.mn, s.mt, s.E, s.ke, s.p, s.dr, -s.dmn, s.dmt, s.dE, s.r, s.mn, s.mt, s.E, s.ke,
                  s.p, s.dr, s.dmn, s.dmt, s.dE, dq, gamma, gm1, FI);
    else
      lf_face_dev(s.r, s.mn, s.mt, s.E, s.ke, s.p, s.dr, s.dmn, s.dmt, s.dE, s.r, -s.mn, s.mt, s.E, s.ke,
                  s.p, s.dr, -s.dmn, s.dmt, s.dE, dq, gamma, gm1, FI);
    const float4 vv = S.v[rv][cc + 1];
    const float2 t = S.tx[rv][cc];
    const float un = vv.y, ut = vv.x, T = vv.z, gn = t.y, gt = t.x;
    const float utg = g.wall ? ut : -ut, gtg = g.wall ? gt : -gt;
    const int k = below ? ku : kd;
    const float mu = k < n1 ? g.mu1f : g.mu2f, kap = k < n1 ? g.kap1f : g.kap2f;
    const float inv_dn = k < n1 ? g.inv_dz1f : g.inv_dz2f;
    if (below) visc_face<float>(-un, utg, T, -gn, gtg, un, ut, T, gn, gt, inv_dn, mu, kap, FV);
    else visc_face<float>(un, ut, T, gn, gt, -un, utg, T, -gn, gtg, inv_dn, mu, kap, FV);
    S.fz[f][cc] = make_float4(FI[0] - FV[0], FI[2] - FV[2], FI[1] - FV[1], FI[3] - FV[3]);
  } else if (ku == n1) {
    // the interface: a rigid lid seen from each fluid (inviscid), the bulk
    // fluxes of App. B in double (viscous, shared by both fluids)
    const double sig = S.gam[0][cc + 1], Pi = S.gam[1][cc + 1], uw = S.gam[2][cc + 1];
    const float Vt = narrow(sig), VE = narrow(uw * sig - Pi);
    float FI[4];
    SideZ s = side_z(S, f + 2, f + 1, cc, -1.f);  // fluid 2, above
    float dq[4] = {0.f, -2.f * (s.mn + s.dmn), 0.f, 0.f};
    lf_face_dev(s.r, -s.mn, s.mt, s.E, s.ke, s.p, s.dr, -s.dmn, s.dmt, s.dE, s.r, s.mn, s.mt, s.E, s.ke, s.p,
                s.dr, s.dmn, s.dmt, s.dE, dq, gamma, gm1, FI);
    S.fz[f][cc] = make_float4(FI[0], FI[2] - Vt, FI[1], FI[3] - VE);
    s = side_z(S, f + 1, f, cc, 1.f);  // fluid 1, below
    dq[1] = 2.f * (s.mn + s.dmn);
    lf_face_dev(s.r, s.mn, s.mt, s.E, s.ke, s.p, s.dr, s.dmn, s.dmt, s.dE, s.r, -s.mn, s.mt, s.E, s.ke, s.p,
                s.dr, -s.dmn, s.dmt, s.dE, dq, gamma, gm1, FI);
    S.fg[cc] = make_float4(FI[0], FI[2] - Vt, FI[1], FI[3] - VE);
  } else {
    const SideZ L = side_z(S, f + 1, f, cc, 1.f), R = side_z(S, f + 2, f + 1, cc, -1.f);
    // q_left - q_right = q_ref(kd) - q_ref(ku) + (d_left - d_right)
    const float dq[4] = {S.rc[8][f + 1] + (L.dr - R.dr), S.rc[10][f + 1] + (L.dmn - R.dmn),
                         S.rc[9][f + 1] + (L.dmt - R.dmt), S.rc[11][f + 1] + (L.dE - R.dE)};
    float FI[4], FV[4];
    lf_face_dev(L.r, L.mn, L.mt, L.E, L.ke, L.p, L.dr, L.dmn, L.dmt, L.dE, R.r, R.mn, R.mt, R.E, R.ke, R.p,
                R.dr, R.dmn, R.dmt, R.dE, dq, gamma, gm1, FI);
    const float mu = kd < n1 ? g.mu1f : g.mu2f, kap = kd < n1 ? g.kap1f : g.kap2f;
    const float inv_dn = kd < n1 ? g.inv_dz1f : g.inv_dz2f;
    const float4 vL = S.v[f][cc + 1], vR = S.v[f + 1][cc + 1];
    const float2 tL = S.tx[f][cc], tR = S.tx[f + 1][cc];
    visc_face<float>(vL.y, vL.x, vL.z, tL.y, tL.x, vR.y, vR.x, vR.z, tR.y, tR.x, inv_dn, mu, kap, FV);
    S.fz[f][cc] = make_float4(FI[0] - FV[0], FI[2] - FV[2], FI[1] - FV[1], FI[3] - FV[3]);
  }
}

// The x face between ring columns f and f+1 (tile columns f-1 and f) of tile
// row rr; returns the flux in (rho, mu, mw, E) order.
__device__ __forceinline__ float4 x_face(const StageArgs& a, const MixedSmem& S, int rr, int f) {
  const Geom& g = a.g;
  const int rq = rr + 2;
  const float r0 = S.rc[0][rq], m0 = S.rc[1][rq], w0 = S.rc[2][rq], E0 = S.rc[3][rq];
  const float ke = S.rc[12][rq], pr = S.rc[14][rq];
  const float4 qL = S.q[rq][f + 1], qR = S.q[rq][f + 2];
  const float4 hL = S.hx[rr][f], hR = S.hx[rr][f + 1];
  const float dlr = qL.x + hL.x, dlmn = qL.y + hL.y, dlmt = qL.z + hL.z, dlE = qL.w + hL.w;
  const float drr = qR.x - hR.x, drmn = qR.y - hR.y, drmt = qR.z - hR.z, drE = qR.w - hR.w;
  const float dq[4] = {dlr - drr, dlmn - drmn, dlmt - drmt, dlE - drE};
  float FI[4];
  lf_face_dev(r0, m0, w0, E0, ke, pr, dlr, dlmn, dlmt, dlE, r0, m0, w0, E0, ke, pr, drr, drmn, drmt, drE, dq,
              g.gammaf, g.gm1f, FI);
  return make_float4(FI[0], FI[1], FI[2], FI[3]);
}

__device__ __forceinline__ float4 x_face_visc(const StageArgs& a, const MixedSmem& S, int rr, int f, float mu,
                                              float kap) {
  const float4 vL = S.v[rr + 1][f], vR = S.v[rr + 1][f + 1];
  const float2 tL = S.tz[rr][f], tR = S.tz[rr][f + 1];
  float FV[4];
  visc_face<float>(vL.x, vL.y, vL.z, tL.x, tL.y, vR.x, vR.y, vR.z, tR.x, tR.y, a.g.inv_dxf, mu, kap, FV);
  return make_float4(FV[0], FV[1], FV[2], FV[3]);
}

// Inlined into each kernel: launch constants then stay constant-bank
// operands. The single-instance and batch kernels may contract floating-point
// operations differently, so their results agree to float rounding (the
// FP32-flux tolerance), not bit for bit.
__device__ __forceinline__ void stage_tile_mixed(const StageArgs& a, int tile, MixedSmem& S) {
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int ty = tid / TX, tx = tid - ty * TX;  // owned cell
  const int tzi = tile / a.tiles_x;
  const int txi = tile - tzi * a.tiles_x;
  const int k0 = a.row0 + tzi * TZ;
  const int i0 = txi * TX;
  const int nz = g.nz, nx = g.nx, n1 = g.n1;
  const int row_hi = a.rhs_only ? a.rhs_hi : nz;
  const size_t plane = (size_t)nz * g.pitch;
  const bool odd_stage = !a.rhs_only && (a.stage & 1);
  const float* Ra = reinterpret_cast<const float*>(a.b.Ra);
  const float* rowc = a.b.rowc;

  // ---- 1. deviations of the stage state (tile + halo) and row constants --
  for (int e = tid; e < (TZ + 4) * (TX + 4); e += MIXED_THREADS) {
    const int rr = e / (TX + 4), cc = e - rr * (TX + 4);
    const int k = k0 - 2 + rr;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k >= 0 && k < nz) {
      int i = i0 - 2 + cc;
      if (i < 0) i += nx;
      if (i >= nx) i -= nx;
      if (i >= nx) i %= nx;  // only when nx is smaller than the tile
      const size_t off = (size_t)k * g.pitch + i;
      if (a.rhs_only) {
        val.x = narrow(a.rhs_in[off] - (double)rowc[k]);
        val.y = narrow(a.rhs_in[plane + off] - (double)rowc[nz + k]);
        val.z = narrow(a.rhs_in[2 * plane + off] - (double)rowc[2 * nz + k]);
        val.w = narrow(a.rhs_in[3 * plane + off] - (double)rowc[3 * nz + k]);
      } else {
        const float* base = (k < g.n1_r ? a.b.dA : a.dF) + off;
        val = make_float4(base[0], base[plane], base[2 * plane], base[3 * plane]);
        if (odd_stage) {
          const float h = k < g.n1_r ? g.dtf : g.hFf;
          const float* ra = Ra + off;
          val.x += h * ra[0];
          val.y += h * ra[plane];
          val.z += h * ra[2 * plane];
          val.w += h * ra[3 * plane];
        }
      }
    }
    S.q[rr][cc] = val;
  }
  if (tid < NROWC * (TZ + 4)) {
    const int j = tid / (TZ + 4), rr = tid - j * (TZ + 4);
    const int k = k0 - 2 + rr;
    S.rc[j][rr] = (k >= 0 && k < nz) ? rowc[j * nz + k] : 0.f;
  }
  const bool has_gamma = (n1 >= k0 && n1 <= k0 + TZ);
  __syncthreads();

  // ---- 2. u, w, T (full states) on the ring; interface state in double --
  const float gamma = g.gammaf, gm1 = g.gm1f;
  for (int e = tid; e < (TZ + 2) * (TX + 2); e += MIXED_THREADS) {
    const int rr = e / (TX + 2), cc = e - rr * (TX + 2);
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    const float4 d = S.q[rr + 1][cc + 1];
    const float r = S.rc[0][rr + 1] + d.x, mu_ = S.rc[1][rr + 1] + d.y, mw = S.rc[2][rr + 1] + d.z;
    const float inv = __frcp_rn(r);
    const float u = mu_ * inv, w = mw * inv;
    const float dp = gm1 * (d.w - (0.5f * (mu_ * u + mw * w) - S.rc[12][rr + 1]));
    S.v[rr][cc] = make_float4(u, w, gamma * (S.rc[14][rr + 1] + dp) * inv, 0.f);
  }
  if (has_gamma && tid < TX + 2) {
    int i = i0 - 1 + tid;
    if (i < 0) i += nx;
    if (i >= nx) i %= nx;
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
          qq[c] = base[off];
          if (odd_stage) qq[c] += (k < g.n1_r ? g.dt : g.hF) * widen(Ra[off]);
        }
      }
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
  const float hinv_dx = 0.5f * g.inv_dxf;
  for (int e = tid; e < TZ * (TX + 2); e += MIXED_THREADS) {
    const int rr = e / (TX + 2), cc = e - rr * (TX + 2);
    const int k = k0 + rr;
    if (k >= row_hi) continue;
    const float4 qe = S.q[rr + 2][cc + 2], qw = S.q[rr + 2][cc];
    S.hx[rr][cc] = make_float4(0.25f * (qe.x - qw.x), 0.25f * (qe.y - qw.y), 0.25f * (qe.z - qw.z),
                               0.25f * (qe.w - qw.w));
    const float4 vc = S.v[rr + 1][cc];
    float uu, wu, ud, wd;
    if (k + 1 == nz) { uu = g.wall ? vc.x : -vc.x; wu = -vc.y; }
    else if (k + 1 == n1) { uu = 2.0f * narrow(S.gam[2][cc]) - vc.x; wu = -vc.y; }
    else { const float4 vn = S.v[rr + 2][cc]; uu = vn.x; wu = vn.y; }
    if (k == 0) { ud = g.wall ? vc.x : -vc.x; wd = -vc.y; }
    else if (k == n1) { ud = 2.0f * narrow(S.gam[2][cc]) - vc.x; wd = -vc.y; }
    else { const float4 vs = S.v[rr][cc]; ud = vs.x; wd = vs.y; }
    const float hinv_dz = 0.5f * (k < n1 ? g.inv_dz1f : g.inv_dz2f);
    S.tz[rr][cc] = make_float2((uu - ud) * hinv_dz, (wu - wd) * hinv_dz);
  }
  for (int e = tid; e < (TZ + 2) * TX; e += MIXED_THREADS) {
    const int rr = e / TX, cc = e - rr * TX;
    const int k = k0 - 1 + rr;
    if (k < 0 || k >= nz) continue;
    const bool up_in = (k + 1 < nz) && ((k + 1 < n1) == (k < n1));
    const bool dn_in = (k - 1 >= 0) && ((k - 1 < n1) == (k < n1));
    const float4 own = S.q[rr + 1][cc + 2];
    const float4 mir = make_float4(own.x, own.y, -own.z, own.w);  // mirror ghost: rho w odd
    const float4 up = up_in ? S.q[rr + 2][cc + 2] : mir;
    const float4 dn = dn_in ? S.q[rr][cc + 2] : mir;
    S.hz[rr][cc] = make_float4(0.25f * (up.x - dn.x) + S.rc[4][rr + 1], 0.25f * (up.y - dn.y) + S.rc[5][rr + 1],
                               0.25f * (up.z - dn.z) + S.rc[6][rr + 1], 0.25f * (up.w - dn.w) + S.rc[7][rr + 1]);
    const float4 ve = S.v[rr][cc + 2], vw = S.v[rr][cc];
    S.tx[rr][cc] = make_float2((ve.x - vw.x) * hinv_dx, (ve.y - vw.y) * hinv_dx);
  }
  __syncthreads();

  // ---- 4. faces: own left x face (registers), own lower z face (shared) --
  const int k = k0 + ty;
  const bool live = ty < TZ && k < row_hi;
  float4 fxl = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ty < TZ) {
    if (live) {
      const float mu_c = k < n1 ? g.mu1f : g.mu2f, kap_c = k < n1 ? g.kap1f : g.kap2f;
      const float4 FI = x_face(a, S, ty, tx);
      const float4 FV = x_face_visc(a, S, ty, tx, mu_c, kap_c);
      fxl = make_float4(FI.x - FV.x, FI.y - FV.y, FI.z - FV.z, FI.w - FV.w);
    }
    // lower z face of the owned cell (needed by it, and by the cell below)
    if (k - 1 < row_hi) z_face(a, S, k0, ty, tx);
  } else {
    // warp 8: the z faces above the tile, then the x faces on its right edge
    if (k0 + TZ - 1 < row_hi) z_face(a, S, k0, TZ, tx);
    const int kr = k0 + tx;
    if (tx < TZ && kr < row_hi) {
      const float mu = kr < n1 ? g.mu1f : g.mu2f, kap = kr < n1 ? g.kap1f : g.kap2f;
      const float4 FI = x_face(a, S, tx, TX);
      const float4 FV = x_face_visc(a, S, tx, TX, mu, kap);
      S.fxr[tx] = make_float4(FI.x - FV.x, FI.y - FV.y, FI.z - FV.z, FI.w - FV.w);
    }
  }
  // right x face of the owned cell: the left face of the next lane
  float4 fxr;
  fxr.x = __shfl_down_sync(0xffffffffu, fxl.x, 1);
  fxr.y = __shfl_down_sync(0xffffffffu, fxl.y, 1);
  fxr.z = __shfl_down_sync(0xffffffffu, fxl.z, 1);
  fxr.w = __shfl_down_sync(0xffffffffu, fxl.w, 1);
  __syncthreads();
  if (tx == TX - 1 && ty < TZ) fxr = S.fxr[ty];

  // ---- 5. R (float) and the stage combination (double) -------------------
  const int i = i0 + tx;
  if (!live || i >= nx) return;
  const float inv_dx = g.inv_dxf;
  const float inv_dz = k < n1 ? g.inv_dz1f : g.inv_dz2f;
  const float4 fdn = S.fz[ty][tx];
  const float4 fup = (k == n1 - 1) ? S.fg[tx] : S.fz[ty + 1][tx];
  const float4 dc = S.q[ty + 2][tx + 2];
  float R[4];
  R[0] = (fxl.x - fxr.x) * inv_dx + (fdn.x - fup.x) * inv_dz;
  R[1] = (fxl.y - fxr.y) * inv_dx + (fdn.y - fup.y) * inv_dz;
  R[2] = (fxl.z - fxr.z) * inv_dx + (fdn.z - fup.z) * inv_dz;
  R[3] = (fxl.w - fxr.w) * inv_dx + (fdn.w - fup.w) * inv_dz;
  // gravity on the deviation; the reference part sits in the row constant
  R[2] += S.rc[13][ty + 2] - dc.x * g.Gf;
  R[3] -= (S.rc[2][ty + 2] + dc.z) * g.Gf;

  const size_t row_off = (size_t)k * g.pitch + i;
  if (a.rhs_only) {
#pragma unroll
    for (int c = 0; c < 4; c++) a.rhs_out[(size_t)c * plane + row_off] = widen(R[c]);
    return;
  }
  float* Ra_w = reinterpret_cast<float*>(a.b.Ra);
  const int st = a.stage;
  const double h2 = g.h2;
  if (k >= g.n1_r) {
    if (!(st & 1)) {
#pragma unroll
      for (int c = 0; c < 4; c++) Ra_w[(size_t)c * plane + row_off] = R[c];
    } else {
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const size_t o = (size_t)c * plane + row_off;
        const float s = Ra[o] + R[c];
        a.qF_next[o] = fma(h2, widen(s), a.qF[o]);
        a.dF_next[o] = a.dF[o] + g.h2f * s;  // float shadow; resynchronised each slow step
      }
    }
  } else if (k >= g.nS_r) {
    const size_t pb = (size_t)(g.n1_r - g.nS_r) * g.pitch;
    const size_t ob = (size_t)(k - g.nS_r) * g.pitch + i;
    const bool last = (st == 2 * g.m - 1);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const size_t o = (size_t)c * plane + row_off;
      double* acc = a.b.accB + (size_t)c * pb + ob;
      if (!(st & 1)) Ra_w[o] = R[c];
      const double r = widen(R[c]);
      if (st == 0) *acc = r;
      else if (last) *acc = fma(h2, *acc + r, a.b.qA[o]);
      else *acc = *acc + r;
    }
  } else {
    const size_t ps = (size_t)g.nS_r * g.pitch;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const size_t o = (size_t)c * plane + row_off;
      if (st == 0) Ra_w[o] = R[c];
      else a.b.accS[(size_t)c * ps + row_off] = fma(g.hdt, widen(Ra[o]) + widen(R[c]), a.b.qA[o]);
    }
  }
}

}  // namespace mprk
