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
// Layout for few instructions per cell: the halo tile is loaded once with
// u, w, T computed on the way in (float4 per cell in shared memory). One
// thread owns one cell of the TX x TZ tile and computes the x face on its
// left and the z face below it, taking slopes from the staged values as it
// goes; a ninth warp computes the faces on the tile's right and top edges.
// The right x face of a cell comes from the neighbouring lane by a warp
// shuffle. Two barriers per tile.
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

// Per-row constants: four float4 groups, group j of row k at [j * nz + k]:
//   A (j = 0)  q_ref (rho, rho u, rho w, rho E)
//   B (j = 1)  quarter z difference of q_ref with the mirror rule at walls and Gamma
//   C (j = 2)  q_ref(k) - q_ref(k+1)
//   D (j = 3)  (kinetic energy of q_ref, reference pressure divergence and
//              gravity for R(rho w), p_ref, 0)
constexpr int NROWC = 16;

// Nine warps: warps 0-7 own the TX x TZ cells, warp 8 computes the faces on
// the tile's top edge (one pass) and right edge (one pass), so every warp
// makes two face passes.
constexpr int MIXED_THREADS = NTHREADS + 32;

struct MixedSmem {
  float4 q[TZ + 4][TX + 4];  // deviation d of the stage state (rho, mu, mw, E) on the halo
  float4 v[TZ + 4][TX + 4];  // (u, w, T, -) full values on the halo
  float4 fz[TZ + 1][TX];     // z face fluxes seen from above (rho, mu, mw, E order)
  float4 fxr[TZ];            // x face on the tile's right edge, per row
  float4 fg[TX];             // interface flux seen from fluid 1 (below)
  float4 rcA[TZ + 4];        // q_ref per halo row
  float4 rcB[TZ + 4];        // quarter z difference of q_ref (mirror rule)
  float4 rcC[TZ + 4];        // q_ref(k) - q_ref(k+1)
  float4 rcD[TZ + 4];        // (kinetic energy of q_ref, R(rho w) constant, p_ref, -)
  double gam[4][TX + 2];     // sigma_xz, Pi_z, u_w, T_w per column i0-1 ..
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

// Geometry of a tile row: is the row above / below in the same fluid, and
// what lies beyond it (outer wall or Gamma).
struct RowNb {
  bool up_in, dn_in;      // neighbour row in the same fluid
  bool top_wall, top_gam; // row above is an outer wall / across Gamma
  bool bot_wall, bot_gam;
};

__device__ __forceinline__ RowNb row_nb(int k, int nz, int n1) {
  RowNb r;
  r.top_wall = (k + 1 == nz);
  r.top_gam = (k + 1 == n1);
  r.bot_wall = (k == 0);
  r.bot_gam = (k == n1);
  r.up_in = !r.top_wall && !r.top_gam;
  r.dn_in = !r.bot_wall && !r.bot_gam;
  return r;
}

__device__ __forceinline__ float4 mirror4(float4 q) { return make_float4(q.x, q.y, -q.z, q.w); }

constexpr int HW = TX + 4;  // halo row width: neighbours above and below are +-HW apart

// Quarter z difference of the deviation at the halo cell q (a pointer into
// S.q), mirror ghost beyond a wall or Gamma, plus the reference part rb of
// the row.
__device__ __forceinline__ float4 slope_z(const float4* q, float4 rb, const RowNb& nb) {
  const float4 own = q[0];
  const float4 up = nb.up_in ? q[HW] : mirror4(own);
  const float4 dn = nb.dn_in ? q[-HW] : mirror4(own);
  return make_float4(0.25f * (up.x - dn.x) + rb.x, 0.25f * (up.y - dn.y) + rb.y,
                     0.25f * (up.z - dn.z) + rb.z, 0.25f * (up.w - dn.w) + rb.w);
}

// d/dz of (u, w) at the halo cell v (a pointer into S.v): ghost
// 2*(wall state) - interior beyond a wall (no-slip or slip) or Gamma (the
// column's fluid-1 wall velocity uw).
__device__ __forceinline__ float2 dz_uw(const float4* v, const Geom& g, const RowNb& nb, float uw,
                                        float hinv_dz) {
  const float4 vc = v[0];
  float uu, wu, ud, wd;
  if (nb.up_in) { const float4 vn = v[HW]; uu = vn.x; wu = vn.y; }
  else if (nb.top_gam) { uu = 2.0f * uw - vc.x; wu = -vc.y; }
  else { uu = g.wall ? vc.x : -vc.x; wu = -vc.y; }
  if (nb.dn_in) { const float4 vs = v[-HW]; ud = vs.x; wd = vs.y; }
  else if (nb.bot_gam) { ud = 2.0f * uw - vc.x; wd = -vc.y; }
  else { ud = g.wall ? vc.x : -vc.x; wd = -vc.y; }
  return make_float2((uu - ud) * hinv_dz, (wu - wd) * hinv_dz);
}

// d/dx of (u, w) at the halo cell v.
__device__ __forceinline__ float2 dx_uw(const float4* v, float hinv_dx) {
  const float4 ve = v[1], vw = v[-1];
  return make_float2((ve.x - vw.x) * hinv_dx, (ve.y - vw.y) * hinv_dx);
}

// x face between tile columns f-1 and f (halo columns f+1, f+2) of halo row hr
// (grid row k): F* = F^{I*} - F^{V*}, in (rho, mu, mw, E) order.
__device__ __forceinline__ float4 x_face3(const MixedSmem& S, const Geom& g, int hr, int f, const RowNb& nb,
                                          float mu, float kap, float hinv_dz) {
  const float4* q = &S.q[hr][f];      // q[0..3]: halo columns f .. f+3
  const float4* v = &S.v[hr][f + 1];  // v[0], v[1]: the two cells
  const float4 qa = q[0], qb = q[1], qc = q[2], qd = q[3];
  const float4 ref = S.rcA[hr], rd = S.rcD[hr];
  // reconstructed deviations q + (q_{+1} - q_{-1})/4, q - (q_{+1} - q_{-1})/4
  const float dlr = qb.x + 0.25f * (qc.x - qa.x), dlm = qb.y + 0.25f * (qc.y - qa.y);
  const float dlw = qb.z + 0.25f * (qc.z - qa.z), dlE = qb.w + 0.25f * (qc.w - qa.w);
  const float drr = qc.x - 0.25f * (qd.x - qb.x), drm = qc.y - 0.25f * (qd.y - qb.y);
  const float drw = qc.z - 0.25f * (qd.z - qb.z), drE = qc.w - 0.25f * (qd.w - qb.w);
  const float dq[4] = {dlr - drr, dlm - drm, dlw - drw, dlE - drE};
  float FI[4], FV[4];
  lf_face_dev(ref.x, ref.y, ref.z, ref.w, rd.x, rd.z, dlr, dlm, dlw, dlE, ref.x, ref.y, ref.z, ref.w, rd.x, rd.z,
              drr, drm, drw, drE, dq, g.gammaf, g.gm1f, FI);
  float uwL = 0.f, uwR = 0.f;
  if (nb.top_gam || nb.bot_gam) {
    uwL = narrow(S.gam[2][f]);
    uwR = narrow(S.gam[2][f + 1]);
  }
  const float4 vL = v[0], vR = v[1];
  const float2 tL = dz_uw(v, g, nb, uwL, hinv_dz), tR = dz_uw(v + 1, g, nb, uwR, hinv_dz);
  visc_face<float>(vL.x, vL.y, vL.z, tL.x, tL.y, vR.x, vR.y, vR.z, tR.x, tR.y, g.inv_dxf, mu, kap, FV);
  return make_float4(FI[0] - FV[0], FI[1] - FV[1], FI[2] - FV[2], FI[3] - FV[3]);
}

// z face below grid row ku = k0+f (halo rows hd = f+1 below, hu = f+2 above)
// in tile column cc: writes fz[f][cc], and fg[cc] at the interface.
__device__ __forceinline__ void z_face3(MixedSmem& S, const Geom& g, int k0, int f, int cc) {
  const int nz = g.nz, n1 = g.n1;
  const int ku = k0 + f, kd = ku - 1;
  const int hd = f + 1, hu = f + 2, hc = cc + 2;
  const float4* qd = &S.q[hd][hc];  // cell below the face; the cell above is qd[HW]
  const float4* vd = &S.v[hd][hc];
  const float gamma = g.gammaf, gm1 = g.gm1f;
  const float hinv_dx = 0.5f * g.inv_dxf;
  if (ku == 0 || ku == nz) {
    // outer wall: the boundary cell against its mirror (inviscid) and its
    // ghost 2*wall - interior (viscous); no-slip or slip, adiabatic
    const bool below = (ku == 0);
    const int h = below ? hu : hd, k = below ? ku : kd;
    const float4* qc = below ? qd + HW : qd;
    const float4* vc = below ? vd + HW : vd;
    const RowNb nb = row_nb(k, nz, n1);
    const float4 q = qc[0], hz = slope_z(qc, S.rcB[h], nb);
    const float sg = below ? -1.f : 1.f;
    const float4 ref = S.rcA[h], rd = S.rcD[h];
    const float dr = q.x + sg * hz.x, dmt = q.y + sg * hz.y, dmn = q.z + sg * hz.z, dE = q.w + sg * hz.w;
    const float mn = ref.z + dmn;
    const float dq[4] = {0.f, below ? -2.f * mn : 2.f * mn, 0.f, 0.f};
    float FI[4], FV[4];
    if (below)
      lf_face_dev(ref.x, -ref.z, ref.y, ref.w, rd.x, rd.z, dr, -dmn, dmt, dE, ref.x, ref.z, ref.y, ref.w, rd.x,
                  rd.z, dr, dmn, dmt, dE, dq, gamma, gm1, FI);
    else
      lf_face_dev(ref.x, ref.z, ref.y, ref.w, rd.x, rd.z, dr, dmn, dmt, dE, ref.x, -ref.z, ref.y, ref.w, rd.x,
                  rd.z, dr, -dmn, dmt, dE, dq, gamma, gm1, FI);
    const float4 vv = vc[0];
    const float2 t = dx_uw(vc, hinv_dx);
    const float un = vv.y, ut = vv.x, T = vv.z, gn = t.y, gt = t.x;
    const float utg = g.wall ? ut : -ut, gtg = g.wall ? gt : -gt;
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
    {  // fluid 2, above: mirror below it
      const RowNb nb = row_nb(ku, nz, n1);
      const float4 q = qd[HW], hz = slope_z(qd + HW, S.rcB[hu], nb);
      const float4 ref = S.rcA[hu], rd = S.rcD[hu];
      const float dr = q.x - hz.x, dmt = q.y - hz.y, dmn = q.z - hz.z, dE = q.w - hz.w;
      const float dq[4] = {0.f, -2.f * (ref.z + dmn), 0.f, 0.f};
      lf_face_dev(ref.x, -ref.z, ref.y, ref.w, rd.x, rd.z, dr, -dmn, dmt, dE, ref.x, ref.z, ref.y, ref.w, rd.x,
                  rd.z, dr, dmn, dmt, dE, dq, gamma, gm1, FI);
      S.fz[f][cc] = make_float4(FI[0], FI[2] - Vt, FI[1], FI[3] - VE);
    }
    {  // fluid 1, below: mirror above it
      const RowNb nb = row_nb(kd, nz, n1);
      const float4 q = qd[0], hz = slope_z(qd, S.rcB[hd], nb);
      const float4 ref = S.rcA[hd], rd = S.rcD[hd];
      const float dr = q.x + hz.x, dmt = q.y + hz.y, dmn = q.z + hz.z, dE = q.w + hz.w;
      const float dq[4] = {0.f, 2.f * (ref.z + dmn), 0.f, 0.f};
      lf_face_dev(ref.x, ref.z, ref.y, ref.w, rd.x, rd.z, dr, dmn, dmt, dE, ref.x, -ref.z, ref.y, ref.w, rd.x,
                  rd.z, dr, -dmn, dmt, dE, dq, gamma, gm1, FI);
      S.fg[cc] = make_float4(FI[0], FI[2] - Vt, FI[1], FI[3] - VE);
    }
  } else {
    const RowNb nbd = row_nb(kd, nz, n1), nbu = row_nb(ku, nz, n1);
    const float4 qL = qd[0], qR = qd[HW];
    const float4 hL = slope_z(qd, S.rcB[hd], nbd), hR = slope_z(qd + HW, S.rcB[hu], nbu);
    const float4 refL = S.rcA[hd], rdL = S.rcD[hd], refR = S.rcA[hu], rdR = S.rcD[hu], dref = S.rcC[hd];
    // face frame: normal momentum rho w (.z), tangential rho u (.y)
    const float lr = qL.x + hL.x, lmt = qL.y + hL.y, lmn = qL.z + hL.z, lE = qL.w + hL.w;
    const float rr = qR.x - hR.x, rmt = qR.y - hR.y, rmn = qR.z - hR.z, rE = qR.w - hR.w;
    // q_left - q_right = q_ref(kd) - q_ref(ku) + (d_left - d_right)
    const float dq[4] = {dref.x + (lr - rr), dref.z + (lmn - rmn), dref.y + (lmt - rmt), dref.w + (lE - rE)};
    float FI[4], FV[4];
    lf_face_dev(refL.x, refL.z, refL.y, refL.w, rdL.x, rdL.z, lr, lmn, lmt, lE, refR.x, refR.z, refR.y, refR.w,
                rdR.x, rdR.z, rr, rmn, rmt, rE, dq, gamma, gm1, FI);
    const float mu = kd < n1 ? g.mu1f : g.mu2f, kap = kd < n1 ? g.kap1f : g.kap2f;
    const float inv_dn = kd < n1 ? g.inv_dz1f : g.inv_dz2f;
    const float4 vL = vd[0], vR = vd[HW];
    const float2 tL = dx_uw(vd, hinv_dx), tR = dx_uw(vd + HW, hinv_dx);
    visc_face<float>(vL.y, vL.x, vL.z, tL.y, tL.x, vR.y, vR.x, vR.z, tR.y, tR.x, inv_dn, mu, kap, FV);
    S.fz[f][cc] = make_float4(FI[0] - FV[0], FI[2] - FV[2], FI[1] - FV[1], FI[3] - FV[3]);
  }
}

// Inlined into each kernel: launch constants then stay constant-bank
// operands. The single-instance and batch kernels may contract floating-point
// operations differently, so their results agree to float rounding (the
// FP32-flux tolerance), not bit for bit.
__device__ __forceinline__ void stage_tile_mixed(const StageArgs& a, int tile, MixedSmem& S) {
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int ty = tid / TX, tx = tid - ty * TX;  // owned cell (warp 8: edge faces)
  const int tzi = tile / a.tiles_x;
  const int txi = tile - tzi * a.tiles_x;
  const int k0 = a.row0 + tzi * TZ;
  const int i0 = txi * TX;
  const int nz = g.nz, nx = g.nx, n1 = g.n1;
  const int row_hi = a.rhs_only ? a.rhs_hi : nz;
  const size_t plane = (size_t)nz * g.pitch;
  const bool odd_stage = !a.rhs_only && (a.stage & 1);
  const float* Ra = reinterpret_cast<const float*>(a.b.Ra);
  const float4* rowc = reinterpret_cast<const float4*>(a.b.rowc);
  const float gamma = g.gammaf, gm1 = g.gm1f;

  // ---- 1. stage-state deviations on the halo, with u, w, T per cell ------
  for (int e = tid; e < (TZ + 4) * (TX + 4); e += MIXED_THREADS) {
    const int rr = e / (TX + 4), cc = e - rr * (TX + 4);
    const int k = k0 - 2 + rr;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f), vv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k >= 0 && k < nz) {
      int i = i0 - 2 + cc;
      if (i < 0) i += nx;
      if (i >= nx) i -= nx;
      if (i >= nx) i %= nx;  // only when nx is smaller than the tile
      const size_t off = (size_t)k * g.pitch + i;
      const float4 ra4 = rowc[k], rd4 = rowc[3 * nz + k];
      const float r0 = ra4.x, m0 = ra4.y, w0 = ra4.z;
      if (a.rhs_only) {
        val.x = narrow(a.rhs_in[off] - (double)r0);
        val.y = narrow(a.rhs_in[plane + off] - (double)m0);
        val.z = narrow(a.rhs_in[2 * plane + off] - (double)w0);
        val.w = narrow(a.rhs_in[3 * plane + off] - (double)ra4.w);
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
      const float r = r0 + val.x, mu_ = m0 + val.y, mw = w0 + val.z;
      const float inv = __frcp_rn(r);
      const float u = mu_ * inv, w = mw * inv;
      const float dp = gm1 * (val.w - (0.5f * (mu_ * u + mw * w) - rd4.x));
      vv = make_float4(u, w, gamma * (rd4.z + dp) * inv, 0.f);
    }
    S.q[rr][cc] = val;
    S.v[rr][cc] = vv;
  }
  if (tid < 4 * (TZ + 4)) {
    const int j = tid / (TZ + 4), rr = tid - j * (TZ + 4);
    const int k = k0 - 2 + rr;
    const float4 c = (k >= 0 && k < nz) ? rowc[j * nz + k] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (j == 0) S.rcA[rr] = c;
    else if (j == 1) S.rcB[rr] = c;
    else if (j == 2) S.rcC[rr] = c;
    else S.rcD[rr] = c;
  }
  const bool has_gamma = (n1 >= k0 && n1 <= k0 + TZ);
  if (has_gamma && tid >= MIXED_THREADS - 64 && tid - (MIXED_THREADS - 64) < TX + 2) {
    // interface state of column i0-1+j in double from the two cells touching
    // Gamma (App. B, Eq. bulk-flux and the wall states)
    const int j = tid - (MIXED_THREADS - 64);
    int i = i0 - 1 + j;
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
    S.gam[0][j] = sig;
    S.gam[1][j] = Pi;
    S.gam[2][j] = u[0] + sig * g.cu1;
    S.gam[3][j] = T[0] - Pi * g.cT1;
  }
  __syncthreads();

  // ---- 2. faces: own left x face (registers), own lower z face (shared) --
  const int k = k0 + ty;
  const bool live = ty < TZ && k < row_hi;
  float4 fxl = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ty < TZ) {
    if (live) {
      const RowNb nb = row_nb(k, nz, n1);
      const float mu_c = k < n1 ? g.mu1f : g.mu2f, kap_c = k < n1 ? g.kap1f : g.kap2f;
      const float hinv_dz = 0.5f * (k < n1 ? g.inv_dz1f : g.inv_dz2f);
      fxl = x_face3(S, g, ty + 2, tx, nb, mu_c, kap_c, hinv_dz);
    }
    // lower z face of the owned cell (needed by it, and by the cell below)
    if (k - 1 < row_hi) z_face3(S, g, k0, ty, tx);
  } else {
    // warp 8: the z faces above the tile, then the x faces on its right edge
    if (k0 + TZ - 1 < row_hi) z_face3(S, g, k0, TZ, tx);
    const int kr = k0 + tx;
    if (tx < TZ && kr < row_hi) {
      const RowNb nb = row_nb(kr, nz, n1);
      const float mu = kr < n1 ? g.mu1f : g.mu2f, kap = kr < n1 ? g.kap1f : g.kap2f;
      const float hinv_dz = 0.5f * (kr < n1 ? g.inv_dz1f : g.inv_dz2f);
      S.fxr[tx] = x_face3(S, g, tx + 2, TX, nb, mu, kap, hinv_dz);
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

  // ---- 3. R (float) and the stage combination (double) -------------------
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
  R[2] += S.rcD[ty + 2].y - dc.x * g.Gf;
  R[3] -= (S.rcA[ty + 2].z + dc.z) * g.Gf;

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
