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
// A tile is TX x MTZ (32 x 16) cells and takes one of two paths:
//
// * Interior tiles (no wall, no interface and no F-row bound within two
//   rows) take the pair path. Each thread carries the cells of
//   rows k and k + TZ of one column. Shared memory interleaves the two
//   cells' values, so every float operation of the flux is one packed
//   f32x2 instruction (sm_100 and later) for both. The tile has no branch on
//   geometry.
// * Other tiles run the general path twice, on two TX x TZ halves, one cell
//   per thread, with the ghost rules of walls and the interface.
//
// Both paths lay out the work the same way. The halo tile is loaded once,
// with u, w and T computed on the way in. A thread computes the x face on
// its cell's left and the z face below it, taking slopes from the staged
// values as it goes. A ninth warp computes the faces on the tile's right and
// top edges, and the right x face of a cell comes from the neighbouring lane
// by a warp shuffle. There are two barriers per tile.
//
// The GB300 converts between float and double at the FP64 rate (2 per clock
// per SM, measured). The general path converts with integer bit operations
// (IEEE-754 round-to-nearest-even; exact widening). The pair path converts
// only once per component per combination, in hardware (also exact).
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

// Per-row constants (NROWC floats per row): float4 group j of row k at
// [j * nz + k].
//   A (j = 0)  q_ref (rho, rho u, rho w, rho E)
//   B (j = 1)  quarter z difference of q_ref with the mirror rule at walls and Gamma
//   C (j = 2)  q_ref(k) - q_ref(k+1)
//   D (j = 3)  (kinetic energy of q_ref, reference pressure divergence and
//              gravity for R(rho w), p_ref, 0)
// The same values paired for rows (k, k + TZ) for the pair path, each float4
// holding two pairs:
//   j = 4, 5   A (rho, rho u), (rho w, rho E)      j = 6, 7   B likewise
//   j = 8, 9   C likewise                          j = 10     (D.x, D.z) = (ke, p_ref)
//   j = 11     (D.y, 0): the R(rho w) constant
constexpr int RC_PAIR = 4;  // first paired group


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

// Whether this stage writes the step's F-row result into the state buffer:
// its last stage with an even number of fast substeps (the F rows ping-pong
// between the two state buffers and end where they started). The step
// completion then rebuilds the float shadow of every row from the double
// state, so this stage does not write the F rows' shadow.
__device__ __forceinline__ bool shadow_by_completion(const StageArgs& a) {
  return !a.rhs_only && a.stage == 2 * a.g.m - 1 && (a.g.m & 1) == 0;
}

// PAR: a launch's stage parity when the kernel is compiled for it (0 even,
// 1 odd; the batch kernel picks one per work item), or PAR_RT to read the
// parity and the right-hand-side hook from the arguments at run time.
constexpr int PAR_RT = 2;
template <int PAR>
__device__ __forceinline__ bool rhs_mode(const StageArgs& a) {
  return PAR == PAR_RT ? a.rhs_only != 0 : false;
}
template <int PAR>
__device__ __forceinline__ bool odd_mode(const StageArgs& a) {
  return PAR == PAR_RT ? (!a.rhs_only && (a.stage & 1)) : PAR == 1;
}

// The general path on the TX x TZ cells from row k0, column i0.
template <int PAR>
__device__ __forceinline__ void mixed_subtile(const StageArgs& a, int k0, int i0, MixedSmem& S) {
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  const int ty = tid / TX, tx = tid - ty * TX;  // owned cell (warp 8: edge faces)
  const int nz = g.nz, nx = g.nx, n1 = g.n1;
  const int row_hi = rhs_mode<PAR>(a) ? a.rhs_hi : nz;
  const size_t plane = (size_t)nz * g.pitch;
  const bool odd_stage = odd_mode<PAR>(a);
  const float* Ra = reinterpret_cast<const float*>(a.b.Ra);
  const float4* rowc = reinterpret_cast<const float4*>(a.b.rowc);
  const float gamma = g.gammaf, gm1 = g.gm1f;

  // ---- 1. stage-state deviations on the halo, with u, w, T per cell ------
  for (int e = tid; e < (TZ + 4) * (TX + 4); e += MIXED_THREADS) {
    const int rr = e / (TX + 4), cc = e - rr * (TX + 4);
    const int k = k0 - 2 + rr;
    float4 val = make_float4(0.f, 0.f, 0.f, 0.f), vv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k >= 0 && k < nz) {
      bool gh;
      const int i = halo_col(i0 - 2 + cc, nx, g.xwall, &gh);
      const size_t off = (size_t)k * g.pitch + i;
      const float4 ra4 = rowc[k], rd4 = rowc[3 * nz + k];
      const float r0 = ra4.x, m0 = ra4.y, w0 = ra4.z;
      if (rhs_mode<PAR>(a)) {
        val.x = narrow(a.rhs_in[off] - (double)r0);
        val.y = narrow((gh ? -a.rhs_in[plane + off] : a.rhs_in[plane + off]) - (double)m0);
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
        // mirror state beyond an x wall: rho u = m0 + d flips
        if (gh) val.y = -val.y - 2.0f * m0;
      }
      const float r = r0 + val.x, mu_ = m0 + val.y, mw = w0 + val.z;
      const float inv = __frcp_rn(r);
      const float u = mu_ * inv, w = mw * inv;
      const float dp = gm1 * (val.w - (0.5f * (mu_ * u + mw * w) - rd4.x));
      // the mirror state's u is already flipped; a no-slip wall flips w too
      vv = make_float4(u, (gh && g.wall == 0) ? -w : w, gamma * (rd4.z + dp) * inv, 0.f);
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
    bool gh;
    const int i = halo_col(i0 - 1 + j, nx, g.xwall, &gh);
    double u[2], T[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const int k = n1 - 1 + s;
      double qq[4];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const size_t off = (size_t)c * plane + (size_t)k * g.pitch + i;
        if (rhs_mode<PAR>(a)) {
          qq[c] = a.rhs_in[off];
        } else {
          const double* base = k < g.n1_r ? a.b.qA : a.qF;
          qq[c] = base[off];
          if (odd_stage) qq[c] += (k < g.n1_r ? g.dt : g.hF) * widen(Ra[off]);
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
  if (rhs_mode<PAR>(a)) {
#pragma unroll
    for (int c = 0; c < 4; c++) a.rhs_out[(size_t)c * plane + row_off] = widen(R[c]);
    return;
  }
  float* Ra_w = reinterpret_cast<float*>(a.b.Ra);
  const int st = a.stage;
  const double h2 = g.h2;
  if (k >= g.n1_r) {
    if (!odd_stage) {
#pragma unroll
      for (int c = 0; c < 4; c++) Ra_w[(size_t)c * plane + row_off] = R[c];
    } else {
#pragma unroll
      const bool shadow = !shadow_by_completion(a);  // as in the pair path
      for (int c = 0; c < 4; c++) {
        const size_t o = (size_t)c * plane + row_off;
        const float s = Ra[o] + R[c];
        a.qF_next[o] = fma(h2, widen(s), a.qF[o]);
        if (shadow) a.dF_next[o] = a.dF[o] + g.h2f * s;  // float shadow
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
      if (!odd_stage) Ra_w[o] = R[c];
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
      // the two float right-hand sides are summed in float, then combined
      // with q_n in double (one DFMA)
      if (st == 0) Ra_w[o] = R[c];
      else a.b.accS[(size_t)c * ps + row_off] = fma(g.hdt, widen(Ra[o] + R[c]), a.b.qA[o]);
    }
  }
}

// ===========================================================================
// The pair path. A float2 holds one quantity of the two cells a thread
// carries: .x for row k, .y for row k + TZ (the "A" and "B" cells).
// ===========================================================================

// f32x2 arithmetic (sm_100 and later), round to nearest: one instruction
// for both cells.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\t"
      "sub.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 sp2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
// reciprocal and reciprocal square root: one MUFU operation each (relative
// error about 2^-23, far below the mode's tolerance)
__device__ __forceinline__ float rcp_a(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsq_a(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float2 rcp2(float2 x) { return make_float2(rcp_a(x.x), rcp_a(x.y)); }
__device__ __forceinline__ float2 rsq2(float2 x) { return make_float2(rsq_a(x.x), rsq_a(x.y)); }

constexpr int PHR = TZ + 4;  // halo pair rows: pair row r holds rows k0-2+r and k0-2+r+TZ

// A staging buffer that tensor copies (TMA) fill with the float planes of
// one interior tile: the box of columns i0-4 .. i0+TX+3 (160 bytes, so the
// box starts on a 16-byte boundary), rows k0-2 .. k0+MTZ+1 and the four
// components.
constexpr int SROWS = MTZ + 4;
constexpr int SCOLS = TX + 8;
struct __align__(128) Stage {
  float d[4][SROWS][SCOLS];   // float shadow of the stage's base state
  float ra[4][SROWS][SCOLS];  // R_a (odd stages only)
};

struct PairSmem {
  float4 qa[PHR][HW];      // deviations: (rho A, rho B, rho u A, rho u B)
  float4 qb[PHR][HW];      //             (rho w A, rho w B, rho E A, rho E B)
  float4 vw[PHR][HW];      // (u A, u B, w A, w B)
  float2 vt[PHR][HW];      // (T A, T B)
  float4 fza[TZ + 1][TX];  // z face fluxes (rho, rho u) below pair row p of the tile
  float4 fzb[TZ + 1][TX];  //               (rho w, rho E)
  float4 fxa[TZ], fxb[TZ]; // x face fluxes on the tile's right edge
  float4 rc[8][PHR];       // paired row constants (groups RC_PAIR ..) of the halo pair rows
};

// ---- bulk copies and their mbarriers (PTX) -------------------------------

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of the given parity to complete; gives up after about
// one second (2^31 clocks) and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
// Orders this thread's earlier shared-memory accesses before later bulk
// copies into shared memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One 3D tensor copy (tile mode) of the box at (x, y, z) of tmap into dst.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tmap, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Lax–Friedrichs flux of lf_face_dev for both cells' faces. Each side gives
// its row's reference (r, mn, mt, E), kinetic energy ke and pressure pr,
// and its reconstructed deviation. dq is q_left - q_right in the face frame.
__device__ __forceinline__ void lf_face2(float2 rL, float2 mnL_, float2 mtL_, float2 EL_, float2 keL,
                                         float2 prL, float2 drL, float2 dmnL, float2 dmtL, float2 dEL,
                                         float2 rR, float2 mnR_, float2 mtR_, float2 ER_, float2 keR,
                                         float2 prR, float2 drR, float2 dmnR, float2 dmtR, float2 dER,
                                         const float2 dq[4], float2 gamma, float2 gm1, float2 out[4]) {
  const float2 half = sp2(0.5f), mhalf = sp2(-0.5f);
  const float2 lr = add2(rL, drL), lmn = add2(mnL_, dmnL), lmt = add2(mtL_, dmtL), lE = add2(EL_, dEL);
  const float2 rr = add2(rR, drR), rmn = add2(mnR_, dmnR), rmt = add2(mtR_, dmtR), rE = add2(ER_, dER);
  const float2 rsL = rsq2(lr), rsR = rsq2(rr);
  const float2 invL = mul2(rsL, rsL), invR = mul2(rsR, rsR);
  const float2 sL = mul2(lr, rsL), sR = mul2(rr, rsR);
  const float2 unL = mul2(lmn, invL), utL = mul2(lmt, invL);
  const float2 unR = mul2(rmn, invR), utR = mul2(rmt, invR);
  // p - p_ref = (gamma - 1) (dE + ke_ref - |m|^2 / (2 rho))
  const float2 dpL = mul2(gm1, fma2(mhalf, fma2(lmn, unL, mul2(lmt, utL)), add2(dEL, keL)));
  const float2 dpR = mul2(gm1, fma2(mhalf, fma2(rmn, unR, mul2(rmt, utR)), add2(dER, keR)));
  const float2 pL = add2(prL, dpL), pR = add2(prR, dpR);
  const float2 XL = mul2(mul2(gamma, pL), invL), XR = mul2(mul2(gamma, pR), invR);
  const float2 cL = mul2(XL, rsq2(XL)), cR = mul2(XR, rsq2(XR));
  const float2 eL = add2(lE, pL), eR = add2(rE, pR);  // rho H on each side
  const float2 HL = mul2(eL, invL), HR = mul2(eR, invR);
  // Roe averages
  const float2 den = rcp2(add2(sL, sR));
  const float2 un = mul2(fma2(sL, unL, mul2(sR, unR)), den);
  const float2 ut = mul2(fma2(sL, utL, mul2(sR, utR)), den);
  const float2 H = mul2(fma2(sL, HL, mul2(sR, HR)), den);
  const float2 X = mul2(gm1, fma2(mhalf, fma2(un, un, mul2(ut, ut)), H));
  const float2 c = mul2(X, rsq2(X));
  const float2 lam = make_float2(fmaxf(fmaxf(fabsf(unL.x) + cL.x, fabsf(unR.x) + cR.x), fabsf(un.x) + c.x),
                                 fmaxf(fmaxf(fabsf(unL.y) + cL.y, fabsf(unR.y) + cR.y), fabsf(un.y) + c.y));
  const float2 hl = mul2(half, lam);
  out[0] = fma2(hl, dq[0], mul2(half, add2(lmn, rmn)));
  out[1] = fma2(hl, dq[1], mul2(half, add2(fma2(lmn, unL, dpL), fma2(rmn, unR, dpR))));
  out[2] = fma2(hl, dq[2], mul2(half, fma2(lmt, unL, mul2(rmt, unR))));
  out[3] = fma2(hl, dq[3], mul2(half, fma2(unL, eL, mul2(unR, eR))));
}

// Viscous flux of visc_face for both cells' faces; out = (normal momentum,
// tangential momentum, energy) (the mass flux is zero).
__device__ __forceinline__ void visc_face2(float2 unL, float2 utL, float2 TL, float2 gnL, float2 gtL,
                                           float2 unR, float2 utR, float2 TR, float2 gnR, float2 gtR,
                                           float2 inv_dn, float2 mu, float2 kap, float2 out[3]) {
  const float2 half = sp2(0.5f);
  const float2 un = mul2(half, add2(unL, unR)), ut = mul2(half, add2(utL, utR));
  const float2 dn_un = mul2(sub2(unR, unL), inv_dn);
  const float2 dn_ut = mul2(sub2(utR, utL), inv_dn);
  const float2 dn_T = mul2(sub2(TR, TL), inv_dn);
  const float2 dt_un = mul2(half, add2(gnL, gnR));
  const float2 dt_ut = mul2(half, add2(gtL, gtR));
  const float2 snn = mul2(mu, fma2(sp2(2.0f), dn_un, mul2(sp2(-2.0f / 3.0f), add2(dn_un, dt_ut))));
  const float2 snt = mul2(mu, add2(dn_ut, dt_un));
  out[0] = snn;
  out[1] = snt;
  out[2] = fma2(un, snn, fma2(ut, snt, mul2(kap, dn_T)));
}

// Constants of an interior tile, the same for all its cells.
struct PairConst {
  float2 gamma, gm1, mu, kap, inv_dx, inv_dz, hinv_dx, hinv_dz;
};

// x face on the left of tile column f (halo columns f+1 | f+2) in halo pair
// row hr, whose paired reference rows give ref01, ref23 and kp.
// F = F^{I*} - F^{V*} in (rho, rho u, rho w, rho E) order.
__device__ __forceinline__ void pair_x_face(const PairSmem& S, const PairConst& C, int hr, int f, float4 ref01,
                                            float4 ref23, float4 kp, float2 F[4]) {
  const float2 q25 = sp2(0.25f), m25 = sp2(-0.25f);
  const float4 a0 = S.qa[hr][f], a1 = S.qa[hr][f + 1], a2 = S.qa[hr][f + 2], a3 = S.qa[hr][f + 3];
  const float4 b0 = S.qb[hr][f], b1 = S.qb[hr][f + 1], b2 = S.qb[hr][f + 2], b3 = S.qb[hr][f + 3];
  // reconstructed deviations: left d1 + (d2 - d0)/4, right d2 - (d3 - d1)/4
  const float2 lr = fma2(q25, sub2(lo2(a2), lo2(a0)), lo2(a1)), rr = fma2(m25, sub2(lo2(a3), lo2(a1)), lo2(a2));
  const float2 lm = fma2(q25, sub2(hi2(a2), hi2(a0)), hi2(a1)), rm = fma2(m25, sub2(hi2(a3), hi2(a1)), hi2(a2));
  const float2 lw = fma2(q25, sub2(lo2(b2), lo2(b0)), lo2(b1)), rw = fma2(m25, sub2(lo2(b3), lo2(b1)), lo2(b2));
  const float2 lE = fma2(q25, sub2(hi2(b2), hi2(b0)), hi2(b1)), rE = fma2(m25, sub2(hi2(b3), hi2(b1)), hi2(b2));
  const float2 dq[4] = {sub2(lr, rr), sub2(lm, rm), sub2(lw, rw), sub2(lE, rE)};
  float2 FI[4], FV[3];
  // face frame: normal momentum rho u, tangential rho w
  lf_face2(lo2(ref01), hi2(ref01), lo2(ref23), hi2(ref23), lo2(kp), hi2(kp), lr, lm, lw, lE, lo2(ref01),
           hi2(ref01), lo2(ref23), hi2(ref23), lo2(kp), hi2(kp), rr, rm, rw, rE, dq, C.gamma, C.gm1, FI);
  // z derivatives of (u, w) at the two cells, central
  const float4 vL = S.vw[hr][f + 1], vR = S.vw[hr][f + 2];
  const float4 uL = S.vw[hr + 1][f + 1], dL = S.vw[hr - 1][f + 1];
  const float4 uR = S.vw[hr + 1][f + 2], dR = S.vw[hr - 1][f + 2];
  const float2 gnL = mul2(sub2(lo2(uL), lo2(dL)), C.hinv_dz), gtL = mul2(sub2(hi2(uL), hi2(dL)), C.hinv_dz);
  const float2 gnR = mul2(sub2(lo2(uR), lo2(dR)), C.hinv_dz), gtR = mul2(sub2(hi2(uR), hi2(dR)), C.hinv_dz);
  visc_face2(lo2(vL), hi2(vL), S.vt[hr][f + 1], gnL, gtL, lo2(vR), hi2(vR), S.vt[hr][f + 2], gnR, gtR, C.inv_dx,
             C.mu, C.kap, FV);
  F[0] = FI[0];
  F[1] = sub2(FI[1], FV[0]);
  F[2] = sub2(FI[2], FV[1]);
  F[3] = sub2(FI[3], FV[2]);
}

// z face below halo pair row hu (rows of pair row hu - 1 below it) in tile
// column cc: writes fza / fzb [hu - 2][cc]. The paired row constants of both
// pair rows come from S.rc.
__device__ __forceinline__ void pair_z_face(PairSmem& S, const PairConst& C, int hu, int cc) {
  const int hd = hu - 1, c = cc + 2;
  const float2 q25 = sp2(0.25f);
  const float4 ref01d = S.rc[0][hd], ref23d = S.rc[1][hd], kpd = S.rc[6][hd];
  const float4 ref01u = S.rc[0][hu], ref23u = S.rc[1][hu], kpu = S.rc[6][hu];
  const float4 sb01d = S.rc[2][hd], sb23d = S.rc[3][hd];
  const float4 sb01u = S.rc[2][hu], sb23u = S.rc[3][hu];
  const float4 dc01 = S.rc[4][hd], dc23 = S.rc[5][hd];
  const float4 am = S.qa[hd - 1][c], ad = S.qa[hd][c], au = S.qa[hu][c], ap = S.qa[hu + 1][c];
  const float4 bm = S.qb[hd - 1][c], bd = S.qb[hd][c], bu = S.qb[hu][c], bp = S.qb[hu + 1][c];
  // below the face: d + (d_up - d_down)/4 + the reference's quarter difference;
  // above: d - (...)/4 - (...)
  const float2 lr = add2(lo2(ad), fma2(q25, sub2(lo2(au), lo2(am)), lo2(sb01d)));
  const float2 lm = add2(hi2(ad), fma2(q25, sub2(hi2(au), hi2(am)), hi2(sb01d)));
  const float2 lw = add2(lo2(bd), fma2(q25, sub2(lo2(bu), lo2(bm)), lo2(sb23d)));
  const float2 lE = add2(hi2(bd), fma2(q25, sub2(hi2(bu), hi2(bm)), hi2(sb23d)));
  const float2 rr = sub2(lo2(au), fma2(q25, sub2(lo2(ap), lo2(ad)), lo2(sb01u)));
  const float2 rm = sub2(hi2(au), fma2(q25, sub2(hi2(ap), hi2(ad)), hi2(sb01u)));
  const float2 rw = sub2(lo2(bu), fma2(q25, sub2(lo2(bp), lo2(bd)), lo2(sb23u)));
  const float2 rE = sub2(hi2(bu), fma2(q25, sub2(hi2(bp), hi2(bd)), hi2(sb23u)));
  // q_left - q_right = q_ref(kd) - q_ref(ku) + (d_left - d_right); face frame
  // (rho, rho w, rho u, rho E)
  const float2 dq[4] = {add2(lo2(dc01), sub2(lr, rr)), add2(lo2(dc23), sub2(lw, rw)),
                        add2(hi2(dc01), sub2(lm, rm)), add2(hi2(dc23), sub2(lE, rE))};
  float2 FI[4], FV[3];
  lf_face2(lo2(ref01d), lo2(ref23d), hi2(ref01d), hi2(ref23d), lo2(kpd), hi2(kpd), lr, lw, lm, lE, lo2(ref01u),
           lo2(ref23u), hi2(ref01u), hi2(ref23u), lo2(kpu), hi2(kpu), rr, rw, rm, rE, dq, C.gamma, C.gm1, FI);
  // x derivatives of (w, u) at the two cells, central
  const float4 vL = S.vw[hd][c], vR = S.vw[hu][c];
  const float4 eL = S.vw[hd][c + 1], wL = S.vw[hd][c - 1], eR = S.vw[hu][c + 1], wR = S.vw[hu][c - 1];
  const float2 gnL = mul2(sub2(hi2(eL), hi2(wL)), C.hinv_dx), gtL = mul2(sub2(lo2(eL), lo2(wL)), C.hinv_dx);
  const float2 gnR = mul2(sub2(hi2(eR), hi2(wR)), C.hinv_dx), gtR = mul2(sub2(lo2(eR), lo2(wR)), C.hinv_dx);
  visc_face2(hi2(vL), lo2(vL), S.vt[hd][c], gnL, gtL, hi2(vR), lo2(vR), S.vt[hu][c], gnR, gtR, C.inv_dz, C.mu,
             C.kap, FV);
  S.fza[hu - 2][cc] = cat2(FI[0], sub2(FI[2], FV[1]));
  S.fzb[hu - 2][cc] = cat2(sub2(FI[1], FV[0]), sub2(FI[3], FV[2]));
}

// An interior tile needs none of the ghost rules: rows k0-2 .. k0+MTZ+1 lie
// inside the grid and inside one fluid, and with x walls its halo columns
// i0-2 .. i0+TX+1 lie between them. For a stage (not the right-hand-side
// hook) they also lie on one side of the F-row bound.
__device__ __forceinline__ bool pair_interior(const StageArgs& a, int k0, int i0) {
  const Geom& g = a.g;
  const int hi = a.rhs_only ? a.rhs_hi : g.nz;
  const int lo_h = k0 - 2, hi_h = k0 + MTZ + 2;  // halo rows [lo_h, hi_h)
  if (lo_h < 0 || hi_h > g.nz || k0 + MTZ > hi || !(g.n1 <= lo_h || g.n1 >= hi_h)) return false;
  if (g.xwall && (i0 < 2 || i0 + TX + 2 > g.nx)) return false;  // halo columns inside the walls
  if (a.rhs_only) return true;
  // S and B rows may share a tile (the combination picks per cell, and both
  // take their stage values from q_n with dt); the F rows' state and step
  // differ, so no F row lies within the halo of a tile with S or B rows
  return g.n1_r <= lo_h || g.n1_r >= hi_h;
}

// Stage combination of one cell outside the F rows (B and S rows), the
// general path's arithmetic with R in float.
template <int PAR>
__device__ __forceinline__ void combine_slow_cell(const StageArgs& a, int k, size_t row_off, const float R[4]) {
  const Geom& g = a.g;
  const size_t plane = (size_t)g.nz * g.pitch;
  const float* Ra = reinterpret_cast<const float*>(a.b.Ra);
  float* Ra_w = reinterpret_cast<float*>(a.b.Ra);
  const int st = a.stage;
  if (k >= g.nS_r) {
    const size_t pb = (size_t)(g.n1_r - g.nS_r) * g.pitch;
    const size_t ob = row_off - (size_t)g.nS_r * g.pitch;
    const bool last = (st == 2 * g.m - 1);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const size_t o = (size_t)c * plane + row_off;
      double* acc = a.b.accB + (size_t)c * pb + ob;
      if (!odd_mode<PAR>(a)) Ra_w[o] = R[c];
      const double r = (double)R[c];
      if (st == 0) *acc = r;
      else if (last) *acc = fma(g.h2, *acc + r, a.b.qA[o]);
      else *acc = *acc + r;
    }
  } else {
    const size_t ps = (size_t)g.nS_r * g.pitch;
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const size_t o = (size_t)c * plane + row_off;
      if (st == 0) Ra_w[o] = R[c];
      else a.b.accS[(size_t)c * ps + row_off] = fma(g.hdt, (double)(Ra[o] + R[c]), a.b.qA[o]);
    }
  }
}

// L2 prefetch of the 128-byte line holding p: an ordinary load-store
// instruction, one per thread with the thread's own address (a bulk
// prefetch with per-thread addresses runs once per thread in turn).
__device__ __forceinline__ void prefetch_line_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 prefetch of the double rows that the stage combination of the tile's
// rows k0 .. k0+MTZ-1, columns i0 .. i0+TX-1 will read after the tile's
// second barrier: q_F (F rows, odd stages), the buffer accumulator (B rows,
// every stage but the first) and q_n (S rows at the second stage, B rows at
// the last). The last 8 MTZ threads (which stage one pair row rather than
// two) each prefetch one 128-byte half of a row's TX doubles: thread t
// counted from there takes row t / 8, component (t / 2) % 4, half t % 2.
// Every address lies inside its row's pitch. Issued as the tile starts, so
// that those loads find L2. The run-time form (the right-hand-side hook)
// does not prefetch.
template <int PAR>
__device__ __forceinline__ void prefetch_combination(const StageArgs& a, int k0, int i0) {
  const int t = (int)threadIdx.x - (MIXED_THREADS - 8 * MTZ);
  if (PAR == PAR_RT || t < 0) return;
  const Geom& g = a.g;
  const int k = k0 + t / 8, c = (t / 2) % 4, col = i0 + (t % 2) * (TX / 2);
  if (k >= g.nz) return;
  const size_t off = (size_t)c * g.nz * g.pitch + (size_t)k * g.pitch + col;
  const int st = a.stage;
  if (k >= g.n1_r) {
    if (odd_mode<PAR>(a)) prefetch_line_l2(a.qF + off);
  } else if (k >= g.nS_r) {
    if (st > 0) prefetch_line_l2(a.b.accB + ((size_t)c * (g.n1_r - g.nS_r) + (k - g.nS_r)) * g.pitch + col);
    if (st == 2 * g.m - 1) prefetch_line_l2(a.b.qA + off);
  } else if (st == 1) {
    prefetch_line_l2(a.b.qA + off);
  }
}

// The pair path on the TX x MTZ interior tile from row k0, column i0. stg,
// when not null, receives the tile's float planes by tensor copies that
// complete on bar (phase 0). Returns false if the wait for them gave up.
template <int PAR>
__device__ __forceinline__ bool pair_tile(const StageArgs& a, int k0, int i0, PairSmem& S, const Stage* stg,
                                          unsigned long long* bar) {
  const Geom& g = a.g;
  const int tid = threadIdx.x;
  prefetch_combination<PAR>(a, k0, i0);
  const int nz = g.nz, nx = g.nx;
  const size_t plane = (size_t)nz * g.pitch;
  const size_t pstep = (size_t)TZ * g.pitch;  // row k -> row k + TZ
  const float4* __restrict__ rowp = reinterpret_cast<const float4*>(a.b.rowc) + RC_PAIR * nz;
  const bool fluid1 = k0 < g.n1;
  bool ok = true;
  PairConst C;
  C.gamma = sp2(g.gammaf);
  C.gm1 = sp2(g.gm1f);
  C.mu = sp2(fluid1 ? g.mu1f : g.mu2f);
  C.kap = sp2(fluid1 ? g.kap1f : g.kap2f);
  C.inv_dx = sp2(g.inv_dxf);
  C.inv_dz = sp2(fluid1 ? g.inv_dz1f : g.inv_dz2f);
  C.hinv_dx = sp2(0.5f * g.inv_dxf);
  C.hinv_dz = sp2(0.5f * (fluid1 ? g.inv_dz1f : g.inv_dz2f));

  // ---- 1. deviations on the halo with u, w, T (pair rows r and r + 8 of a thread)
  {
    const int r0 = tid / HW, cc = tid - r0 * HW;
    int i = i0 - 2 + cc;
    if (i < 0) i += nx;
    if (i >= nx) i -= nx;
    if (i >= nx) i %= nx;  // only when nx is smaller than the tile
    const bool f_rows = k0 >= g.n1_r;
    const float* __restrict__ dsrc = f_rows ? a.dF : a.b.dA;
    const float* __restrict__ Ra = reinterpret_cast<const float*>(a.b.Ra);
    const float2 h = sp2(f_rows ? g.hFf : g.dtf);
    const bool odd_stage = odd_mode<PAR>(a);
    // a thread stages pair rows r0 and r0 + 8 (the second only when r0 < 4);
    // every global load is issued before the arithmetic
    constexpr int RSTEP = MIXED_THREADS / HW;
    const bool two = r0 + RSTEP < PHR;
    float2 d[2][4];
    float4 ref01[2], ref23[2], kp[2];
#pragma unroll
    for (int e = 0; e < 2; e++) {
      if (e == 1 && !two) break;
      const int kA = k0 - 2 + r0 + e * RSTEP;
      ref01[e] = rowp[kA];
      ref23[e] = rowp[nz + kA];
      kp[e] = rowp[6 * nz + kA];
    }
    // the paired row constants of the halo pair rows, which the face and
    // combination phases read from shared memory; the last threads, which
    // stage one pair row instead of two, load them
    const int t2 = tid - (MIXED_THREADS - 8 * PHR);
    if (t2 >= 0) {
      const int j = t2 / PHR, r = t2 - j * PHR;
      S.rc[j][r] = rowp[j * nz + k0 - 2 + r];
    }
    if (stg) ok = mbar_wait(bar, 0);  // the row constants above are in flight meanwhile
#pragma unroll
    for (int e = 0; e < 2; e++) {
      if (e == 1 && !two) break;
      const int kA = k0 - 2 + r0 + e * RSTEP;
      const size_t oA = (size_t)kA * g.pitch + i, oB = oA + pstep;
      if (stg) {
        // staged row of halo pair row r: r (A) and r + TZ (B); column cc + 2
        const int r = r0 + e * RSTEP;
#pragma unroll
        for (int c = 0; c < 4; c++) d[e][c] = make_float2(stg->d[c][r][cc + 2], stg->d[c][r + TZ][cc + 2]);
        if (odd_stage) {
#pragma unroll
          for (int c = 0; c < 4; c++)
            d[e][c] = fma2(h, make_float2(stg->ra[c][r][cc + 2], stg->ra[c][r + TZ][cc + 2]), d[e][c]);
        }
      } else if (rhs_mode<PAR>(a)) {
        const float refA[4] = {ref01[e].x, ref01[e].z, ref23[e].x, ref23[e].z};
        const float refB[4] = {ref01[e].y, ref01[e].w, ref23[e].y, ref23[e].w};
#pragma unroll
        for (int c = 0; c < 4; c++)
          d[e][c] = make_float2(__double2float_rn(a.rhs_in[c * plane + oA] - (double)refA[c]),
                                __double2float_rn(a.rhs_in[c * plane + oB] - (double)refB[c]));
      } else {
#pragma unroll
        for (int c = 0; c < 4; c++) d[e][c] = make_float2(dsrc[c * plane + oA], dsrc[c * plane + oB]);
        if (odd_stage) {
          float2 ra[4];
#pragma unroll
          for (int c = 0; c < 4; c++) ra[c] = make_float2(Ra[c * plane + oA], Ra[c * plane + oB]);
#pragma unroll
          for (int c = 0; c < 4; c++) d[e][c] = fma2(h, ra[c], d[e][c]);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 2; e++) {
      if (e == 1 && !two) break;
      const int r = r0 + e * RSTEP;
      const float2 rho = add2(lo2(ref01[e]), d[e][0]), mu_ = add2(hi2(ref01[e]), d[e][1]);
      const float2 mw = add2(lo2(ref23[e]), d[e][2]);
      const float2 inv = rcp2(rho);
      const float2 u = mul2(mu_, inv), w = mul2(mw, inv);
      const float2 dp = mul2(C.gm1, fma2(sp2(-0.5f), fma2(mu_, u, mul2(mw, w)), add2(d[e][3], lo2(kp[e]))));
      S.qa[r][cc] = cat2(d[e][0], d[e][1]);
      S.qb[r][cc] = cat2(d[e][2], d[e][3]);
      S.vw[r][cc] = cat2(u, w);
      S.vt[r][cc] = mul2(mul2(C.gamma, add2(hi2(kp[e]), dp)), inv);
    }
  }
  if (__syncthreads_or(!ok)) return false;

  // ---- 2. faces: own left x face (registers), own lower z face (shared) ----
  const int p = tid / TX, tx = tid - p * TX;  // pair row of the tile (warp 8: edges)
  float2 fxl[4];
  if (p < TZ) {
    pair_z_face(S, C, p + 2, tx);
    pair_x_face(S, C, p + 2, tx, S.rc[0][p + 2], S.rc[1][p + 2], S.rc[6][p + 2], fxl);
  } else {
    // warp 8: the z faces below pair row TZ (its B half is the tile's top
    // face), then the x faces on the tile's right edge
    pair_z_face(S, C, TZ + 2, tx);
    if (tx < TZ) {
      float2 F[4];
      pair_x_face(S, C, tx + 2, TX, S.rc[0][tx + 2], S.rc[1][tx + 2], S.rc[6][tx + 2], F);
      S.fxa[tx] = cat2(F[0], F[1]);
      S.fxb[tx] = cat2(F[2], F[3]);
    }
#pragma unroll
    for (int c = 0; c < 4; c++) fxl[c] = make_float2(0.f, 0.f);
  }
  // right x face of the owned cells: the left face of the next lane
  float2 fxr[4];
#pragma unroll
  for (int c = 0; c < 4; c++) {
    fxr[c].x = __shfl_down_sync(0xffffffffu, fxl[c].x, 1);
    fxr[c].y = __shfl_down_sync(0xffffffffu, fxl[c].y, 1);
  }
  // the combination's double operands (F rows of an odd stage), loaded
  // before the barrier so that their latency overlaps the wait
  const int kA = k0 + p;
  const int i = i0 + tx;
  const bool own = p < TZ && i < nx;
  const size_t offA = (size_t)kA * g.pitch + i, offB = offA + pstep;
  const bool f_odd = odd_mode<PAR>(a) && kA >= g.n1_r;
  double qa[4], qb[4];
  if (own && f_odd) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
      qa[c] = a.qF[c * plane + offA];
      qb[c] = a.qF[c * plane + offB];
    }
  }
  __syncthreads();
  if (!own) return true;
  if (tx == TX - 1) {
    const float4 ea = S.fxa[p], eb = S.fxb[p];
    fxr[0] = lo2(ea);
    fxr[1] = hi2(ea);
    fxr[2] = lo2(eb);
    fxr[3] = hi2(eb);
  }

  // ---- 3. R (float pairs) and the stage combination (double) -------------
  const float4 da = S.fza[p][tx], db = S.fzb[p][tx], ua = S.fza[p + 1][tx], ub = S.fzb[p + 1][tx];
  const float2 fdn[4] = {lo2(da), hi2(da), lo2(db), hi2(db)};
  const float2 fup[4] = {lo2(ua), hi2(ua), lo2(ub), hi2(ub)};
  float2 R[4];
#pragma unroll
  for (int c = 0; c < 4; c++) R[c] = fma2(sub2(fxl[c], fxr[c]), C.inv_dx, mul2(sub2(fdn[c], fup[c]), C.inv_dz));
  // gravity on the deviation; the reference part sits in the row constant
  const float4 dca = S.qa[p + 2][tx + 2], dcb = S.qb[p + 2][tx + 2];
  const float2 mG = sp2(-g.Gf);
  R[2] = add2(R[2], fma2(mG, lo2(dca), lo2(S.rc[7][p + 2])));
  R[3] = fma2(mG, add2(lo2(S.rc[1][p + 2]), lo2(dcb)), R[3]);

  if (rhs_mode<PAR>(a)) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
      a.rhs_out[c * plane + offA] = (double)R[c].x;
      a.rhs_out[c * plane + offB] = (double)R[c].y;
    }
    return true;
  }
  if (f_odd) {
    // R_a and the float shadow of the two cells: the staged rows p + 2 and
    // p + 2 + TZ, column tx + 4 (the staging buffer is not written again
    // in this tile), else global memory
    const float* Ra = reinterpret_cast<const float*>(a.b.Ra);
    float2 ra[4], dfo[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
      if (stg) {
        ra[c] = make_float2(stg->ra[c][p + 2][tx + 4], stg->ra[c][p + 2 + TZ][tx + 4]);
        dfo[c] = make_float2(stg->d[c][p + 2][tx + 4], stg->d[c][p + 2 + TZ][tx + 4]);
      } else {
        ra[c] = make_float2(Ra[c * plane + offA], Ra[c * plane + offB]);
        dfo[c] = make_float2(a.dF[c * plane + offA], a.dF[c * plane + offB]);
      }
    }
    const float2 h2f = sp2(g.h2f);
    // the float shadow follows the double state in float, except where the
    // step completion rebuilds it anyway (the last stage, even m)
    const bool shadow = !shadow_by_completion(a);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const size_t oA = c * plane + offA, oB = c * plane + offB;
      const float2 s = add2(ra[c], R[c]);
      a.qF_next[oA] = fma(g.h2, (double)s.x, qa[c]);
      a.qF_next[oB] = fma(g.h2, (double)s.y, qb[c]);
      if (shadow) {
        const float2 dn = fma2(h2f, s, dfo[c]);
        a.dF_next[oA] = dn.x;
        a.dF_next[oB] = dn.y;
      }
    }
  } else if (kA >= g.n1_r) {
    float* Ra_w = reinterpret_cast<float*>(a.b.Ra);
#pragma unroll
    for (int c = 0; c < 4; c++) {
      Ra_w[c * plane + offA] = R[c].x;
      Ra_w[c * plane + offB] = R[c].y;
    }
  } else {
    const float RA[4] = {R[0].x, R[1].x, R[2].x, R[3].x}, RB[4] = {R[0].y, R[1].y, R[2].y, R[3].y};
    combine_slow_cell<PAR>(a, kA, offA, RA);
    combine_slow_cell<PAR>(a, kA + TZ, offB, RB);
  }
  return true;
}

// One tile of the FP32-flux stage kernel: TX x MTZ cells from row k0,
// column i0. Inlined into each kernel: launch constants then stay
// constant-bank operands. The single-instance and batch kernels may contract
// floating-point operations differently, so their results agree to float
// rounding (the FP32-flux tolerance), not bit for bit. stg and bar as for
// pair_tile (stg only for tiles that tile_bulk_ok accepts); returns false if
// the wait for the tensor copies gave up.
union MixedTileSmem {
  MixedSmem gen;
  PairSmem pair;
};

template <int PAR>
__device__ __forceinline__ bool stage_tile_mixed(const StageArgs& a, int k0, int i0, MixedTileSmem& S,
                                                 const Stage* stg, unsigned long long* bar) {
  if (pair_interior(a, k0, i0)) return pair_tile<PAR>(a, k0, i0, S.pair, stg, bar);
  mixed_subtile<PAR>(a, k0, i0, S.gen);
  const int hi = rhs_mode<PAR>(a) ? a.rhs_hi : a.g.nz;
  if (k0 + TZ < hi) {
    __syncthreads();  // the first half's phase 3 reads shared memory
    mixed_subtile<PAR>(a, k0 + TZ, i0, S.gen);
  }
  return true;
}

// The same by linear tile index (row-major over tiles_x), without staging.
template <int PAR>
__device__ __forceinline__ void stage_tile_mixed(const StageArgs& a, int tile, MixedTileSmem& S) {
  const int tzi = tile / a.tiles_x;
  const int txi = tile - tzi * a.tiles_x;
  (void)stage_tile_mixed<PAR>(a, a.row0 + tzi * MTZ, txi * TX, S, nullptr, nullptr);
}

// Tiles whose float planes are tensor-copied: interior tiles of a stage
// away from the x wrap (the 40 staged columns lie inside the row).
__device__ __forceinline__ bool tile_bulk_ok(const StageArgs& a, int k0, int i0) {
  return a.bulk && !a.rhs_only && i0 >= 4 && i0 + TX + 4 <= a.g.nx && pair_interior(a, k0, i0);
}

// Issued by one thread: the tensor copies of the tile's float planes into B
// (the shadow box, and R_a's on odd stages), completing on bar. tm_sb / tm_f
// map the shadow of the S and B rows / of the F rows, tm_ra R_a.
__device__ __forceinline__ void stage_issue(const StageArgs& a, int k0, int i0, Stage& B, unsigned long long* bar,
                                            const CUtensorMap* tm_sb, const CUtensorMap* tm_f,
                                            const CUtensorMap* tm_ra) {
  const bool odd = a.stage & 1;
  mbar_expect_tx(bar, (unsigned)((odd ? 2 : 1) * sizeof(B.d)));
  tma_load_3d(&B.d[0][0][0], k0 >= a.g.n1_r ? tm_f : tm_sb, i0 - 4, k0 - 2, 0, bar);
  if (odd) tma_load_3d(&B.ra[0][0][0], tm_ra, i0 - 4, k0 - 2, 0, bar);
}

// Shared memory of the single-instance FP32-flux kernel: the tile's working
// set, the staging buffer's mbarrier and the staging buffer. The buffer
// comes last, so that even stages (no R_a box) launch without its second
// half.
struct MixedKernelSmem {
  MixedTileSmem work;
  unsigned long long bar;
  Stage stg;
};
// Dynamic shared memory of a launch of the stage kernel for stage parity odd.
constexpr size_t mixed_kernel_smem(bool odd) {
  return odd ? sizeof(MixedKernelSmem) : offsetof(MixedKernelSmem, stg) + sizeof(Stage::d);
}

}  // namespace mprk
