// physics.cuh -- per-cell and per-face device arithmetic of the FVCW scheme
// (Guo, Xiong & Shi): WENO-Z weights and compact rows (Sec. 2.2), the
// explicit WENO5-Z closure of bounded lines, the Zhang-Shu limiter and the
// HLLC flux with Batten's wave speeds (Sec. 2.4).
//
// Line variables are ordered (rho, m_n, [m_t,] E): m_n is the momentum
// normal to the faces of the line, m_t (2-D only) the tangential one.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace ppk {

template <typename real>
__device__ __forceinline__ real sqr(real x) { return x * x; }

// Sec. 2.2, eq. (weight): Jiang-Shu indicators of the three sub-stencils of
// cell i and the WENO-Z ratios q_k = (tau5 / (beta_k + eps))^2 they feed.
// The minus side (face i+1/2) uses (q0, q1, q2) with c = (0.2, 0.5, 0.3);
// the mirrored plus side (face i-1/2) uses (q2, q1, q0).
template <typename real>
__device__ __forceinline__ void zratios(real um2, real um1, real u0, real up1, real up2,
                                        real eps, real &q0, real &q1, real &q2) {
  const real c13 = real(13.0) / real(12.0);
  real b0 = c13 * sqr(um2 - real(2) * um1 + u0) + real(0.25) * sqr(um2 - real(4) * um1 + real(3) * u0);
  real b1 = c13 * sqr(um1 - real(2) * u0 + up1) + real(0.25) * sqr(um1 - up1);
  real b2 = c13 * sqr(u0 - real(2) * up1 + up2) + real(0.25) * sqr(real(3) * u0 - real(4) * up1 + up2);
  real tau = fabs(b2 - b0);
  real d0 = b0 + eps, d1 = b1 + eps, d2 = b2 + eps;
  real ti = tau / (d0 * d1 * d2);   // one division for the three ratios
  q0 = sqr(ti * d1 * d2);
  q1 = sqr(ti * d0 * d2);
  q2 = sqr(ti * d0 * d1);
}

// FP32 form of the same ratios, scaled so nothing overflows: with
// d_k = beta_k + eps and dmin = min d_k, when tau > dmin the returned values
// are (dmin/tau)^2 q_k = (dmin/d_k)^2 and the constant 1 of eq. (weight)
// becomes s = (dmin/tau)^2; the normalised weights are unchanged
// (near a jump of 3e6 the plain q_k reaches 1e52, beyond FP32's range).
//
// eps is lifted to the FP32 noise floor of the indicators.  The FP32
// averages the indicators are computed from carry, besides their own
// rounding (up to u max|ubar|, u = 2^-24), the rounding noise the FP32
// fluxes leave in the state step after step: a random walk of about
// cfl u |F| per step, tens to hundreds of u max|ubar| after 10^4 steps.
// eps of eq. (weight), meant to sit above the indicators' zero level and
// below every real one, becomes eps + 2^20 (u max|ubar|)^2 over the stencil:
// above 33 (150 u max|ubar|)^2, the indicators of a flat stencil carrying
// that noise, and still about 4e-9 max|ubar|^2, below the indicators of
// any feature the FP32 form resolves.  With the FP64 value alone, or a
// floor that the accumulated noise overtakes, the weights follow rounding
// noise where the solution is flat to FP32 precision and a grid-scale mode
// that the nonlinear weights otherwise damp grows from it (isentropic
// vortex on 1024^2 to t = 10: density L1 1.9e-4 with the floor at
// 4096 (u max|ubar|)^2, 1.7e-6 at 2^20 (u max|ubar|)^2).
constexpr float FP32_BETA_FLOOR = 1048576.0f * 5.9604645e-08f * 5.9604645e-08f;

__device__ __forceinline__ void zratios_scaled(float um2, float um1, float u0, float up1, float up2,
                                               float eps, float &q0, float &q1, float &q2,
                                               float &one) {
  const float c13 = 13.0f / 12.0f;
  float b0 = c13 * sqr(um2 - 2.0f * um1 + u0) + 0.25f * sqr(um2 - 4.0f * um1 + 3.0f * u0);
  float b1 = c13 * sqr(um1 - 2.0f * u0 + up1) + 0.25f * sqr(um1 - up1);
  float b2 = c13 * sqr(u0 - 2.0f * up1 + up2) + 0.25f * sqr(3.0f * u0 - 4.0f * up1 + up2);
  float tau = fabsf(b2 - b0);
  const float umax = fmaxf(fmaxf(fmaxf(fabsf(um2), fabsf(um1)), fmaxf(fabsf(up1), fabsf(up2))),
                           fabsf(u0));
  eps = fmaf(FP32_BETA_FLOOR * umax, umax, eps);
  float d0 = b0 + eps, d1 = b1 + eps, d2 = b2 + eps;
  float dmin = fminf(fminf(d0, d1), d2);
  // branch-free: the numerator is min(tau, dmin); the constant term is 1
  // while tau <= dmin (no rescaling), else (dmin/tau)^2
  const float r = fminf(tau, dmin);
  const float sc = dmin / tau;
  one = tau <= dmin ? 1.0f : sc * sc;
  q0 = sqr(r / d0);
  q1 = sqr(r / d1);
  q2 = sqr(r / d2);
}

// normalised weights from linear weights (d0, d1, d2) and ratios (q0, q1, q2);
// one is the scaled constant term (1 unless the ratios were rescaled)
template <typename real>
__device__ __forceinline__ void zweights(real d0, real d1, real d2, real q0, real q1, real q2,
                                         real &w0, real &w1, real &w2, real one = real(1)) {
  real a0 = d0 * (one + q0), a1 = d1 * (one + q1), a2 = d2 * (one + q2);
  real is = real(1) / (a0 + a1 + a2);
  w0 = a0 * is;
  w1 = a1 * is;
  w2 = a2 * is;
}

// ratios in the arithmetic of the line: plain in FP64, scaled in FP32
template <typename real>
__device__ __forceinline__ void zratios_any(real um2, real um1, real u0, real up1, real up2,
                                            real eps, real &q0, real &q1, real &q2, real &one) {
  if constexpr (sizeof(real) == 4) {
    zratios_scaled(um2, um1, u0, up1, up2, eps, q0, q1, q2, one);
  } else {
    zratios(um2, um1, u0, up1, up2, eps, q0, q1, q2);
    one = real(1);
  }
}

// One tridiagonal row in elimination order: a on the previously eliminated
// neighbour, b on the unknown, c on the next one, r the right-hand side.
template <typename real>
struct Row {
  real a, b, c, r;
};

// eq. (CWENO-FV) with weights (w0, w1, w2): the row for the unknown u~ at
// the face this cell reconstructs; uprev / unext are the neighbour averages
// on the side of the previously / next eliminated unknown.  The plus side
// is the mirror image, so the same formula serves both sides.
template <typename real>
__device__ __forceinline__ Row<real> compact_row(real w0, real w1, real w2, real uprev, real u0,
                                                  real unext) {
  const real third = real(1.0 / 3.0), sixth = real(1.0 / 6.0);
  Row<real> row;
  row.a = (real(2) * w0 + w1) * third;
  row.b = (w0 + real(2) * (w1 + w2)) * third;
  row.c = w2 * third;
  row.r = (w0 * uprev + (real(5) * (w0 + w1) + w2) * u0 + (w1 + real(5) * w2) * unext) * sixth;
  return row;
}

// the same row from (w0, w2) alone, using w0 + w1 + w2 = 1:
// a = (1 + w0 - w2)/3, b = (2 - w0)/3, c = w2/3,
// r = (w0 uprev + (5 - 4 w2) u0 + (1 - w0 + 4 w2) unext) / 6
template <typename real>
__device__ __forceinline__ Row<real> compact_row02(real w0, real w2, real uprev, real u0,
                                                    real unext) {
  const real third = real(1.0 / 3.0), sixth = real(1.0 / 6.0);
  Row<real> row;
  row.a = (real(1) + w0 - w2) * third;
  row.b = (real(2) - w0) * third;
  row.c = w2 * third;
  row.r = (w0 * uprev + (real(5) - real(4) * w2) * u0 + (real(1) - w0 + real(4) * w2) * unext) * sixth;
  return row;
}

// explicit fifth-order WENO-Z value at the face on the "next" side of the
// centre cell u0, from the five cells ordered from the far "previous" side
// (closure rows of bounded lines)
template <typename real>
__device__ __forceinline__ real weno5z_face(real um2, real um1, real u0, real up1, real up2,
                                            real eps) {
  real q0, q1, q2, w0, w1, w2, one;
  zratios_any(um2, um1, u0, up1, up2, eps, q0, q1, q2, one);
  zweights(real(0.1), real(0.6), real(0.3), q0, q1, q2, w0, w1, w2, one);
  const real sixth = real(1.0 / 6.0);
  real p0 = real(2) * um2 - real(7) * um1 + real(11) * u0;
  real p1 = -um1 + real(5) * u0 + real(2) * up1;
  real p2 = real(2) * u0 + real(5) * up1 - up2;
  return (w0 * p0 + w1 * p1 + w2 * p2) * sixth;
}

// ---------------------------------------------------------------- Euler
template <typename real, int NV>
__device__ __forceinline__ real kin2(const real *U) {  // |m|^2
  real m2 = U[1] * U[1];
  if (NV == 4) m2 += U[2] * U[2];
  return m2;
}

template <typename real, int NV>
__device__ __forceinline__ real pressure(const real *U, real gamma) {
  return (gamma - real(1)) * (U[NV - 1] - real(0.5) * kin2<real, NV>(U) / U[0]);
}

// specific internal energy e = E/rho - |u|^2 / 2
template <typename real, int NV>
__device__ __forceinline__ real spec_e(const real *U) {
  return U[NV - 1] / U[0] - real(0.5) * kin2<real, NV>(U) / (U[0] * U[0]);
}

template <typename real, int NV>
__device__ __forceinline__ void phys_flux(const real *U, real p, real *F) {
  real un = U[1] / U[0];
  F[0] = U[1];
  F[1] = U[1] * un + p;
  if (NV == 4) F[2] = U[2] * un;
  F[NV - 1] = un * (U[NV - 1] + p);
}

// the same with the normal velocity un = m_n / rho already known
template <typename real, int NV>
__device__ __forceinline__ void phys_flux_u(const real *U, real un, real p, real *F) {
  F[0] = U[1];
  F[1] = U[1] * un + p;
  if (NV == 4) F[2] = U[2] * un;
  F[NV - 1] = un * (U[NV - 1] + p);
}

// HLLC flux (Sec. 2.4, eqs. (HLLC), (contact-v), (star-l), (acoustic ws)).
// S_M's denominator uses rho_r on the right-state term, S_R is the max of
// the two estimates and the right star flux uses S_R.  In 2-D the
// tangential velocity is carried by the contact.  smax receives the larger
// |u| + a of the two face states (the speed eq. (CFL-CD) bounds).
// Four divisions per face (1/(rho_l rho_r) for both inverse densities,
// 1/(1 + R) for the Roe averages, S_M, and the star state's 1/(S_K - S_M)):
// in FP64 each one expands to a sequence on the FP64 pipe.
template <typename real, int NV>
__device__ __forceinline__ void hllc(const real *Ul, const real *Ur, real gamma, real *F,
                                     real &smax) {
  const real rl = Ul[0], rr = Ur[0];
  const real irr_irl = real(1) / (rl * rr);
  const real irl = rr * irr_irl, irr = rl * irr_irl;
  const real ml = Ul[1], mr = Ur[1];
  const real ul = ml * irl, ur = mr * irr;
  const real vl = NV == 4 ? Ul[2] * irl : real(0), vr = NV == 4 ? Ur[2] * irr : real(0);
  const real El = Ul[NV - 1], Er = Ur[NV - 1];
  // p = (gamma - 1)(E - |m|^2 / (2 rho)) with |m|^2 / rho = m . u
  real pl = (gamma - real(1)) * (El - real(0.5) * (ml * ul + (NV == 4 ? Ul[2] * vl : real(0))));
  real pr = (gamma - real(1)) * (Er - real(0.5) * (mr * ur + (NV == 4 ? Ur[2] * vr : real(0))));
  if constexpr (sizeof(real) == 4) {   // FP32 form: never a NaN sound speed from rounding
    pl = fmaxf(pl, 0.0f);
    pr = fmaxf(pr, 0.0f);
  }
  const real al = sqrt(gamma * pl * irl), ar = sqrt(gamma * pr * irr);
  smax = fmax(fabs(ul) + al, fabs(ur) + ar);
  const real Hl = (El + pl) * irl, Hr = (Er + pr) * irr;
  const real R = sqrt(rr * irl);
  const real iR = real(1) / (real(1) + R);
  const real ut = (ul + ur * R) * iR;
  const real vt = (vl + vr * R) * iR;
  const real Ht = (Hl + Hr * R) * iR;
  const real at = sqrt((gamma - real(1)) * (Ht - real(0.5) * (ut * ut + vt * vt)));
  const real SL = fmin(ul - al, ut - at);
  const real SR = fmax(ur + ar, ut + at);
  if (SL > real(0)) {
    phys_flux_u<real, NV>(Ul, ul, pl, F);
    return;
  }
  const real SM = (rr * ur * (SR - ur) - rl * ul * (SL - ul) + pl - pr) / (rr * (SR - ur) - rl * (SL - ul));
  const bool left = SM > real(0);
  if (!left && !(SR >= real(0))) {
    phys_flux_u<real, NV>(Ur, ur, pr, F);
    return;
  }
  // the star state of side K (K = l if S_M > 0, else r) and F = F_K + S_K (U*_K - U_K)
  real UK[NV];   // element-wise selects: no run-time indexing of the arrays
#pragma unroll
  for (int k = 0; k < NV; ++k) UK[k] = left ? Ul[k] : Ur[k];
  const real rK = left ? rl : rr, uK = left ? ul : ur, pK = left ? pl : pr;
  const real SK = left ? SL : SR, EK = left ? El : Er, vK = left ? vl : vr;
  real Fk[NV], Us[NV];
  const real ps = rK * (uK - SK) * (uK - SM) + pK;
  const real inv = real(1) / (SK - SM);
  Us[0] = rK * (SK - uK) * inv;
  Us[1] = ((SK - uK) * rK * uK + (ps - pK)) * inv;
  if (NV == 4) Us[2] = Us[0] * vK;
  Us[NV - 1] = ((SK - uK) * EK - pK * uK + ps * SM) * inv;
  phys_flux_u<real, NV>(UK, uK, pK, Fk);
#pragma unroll
  for (int k = 0; k < NV; ++k) F[k] = Fk[k] + SK * (Us[k] - UK[k]);
}

// The HLLC flux of the same two face states relative to a reference state
// R (FP32, the mixed form): returns F_HLLC(U_l, U_r) - F(R) from the full
// states U_K (wave speeds, signal speed smax) and their differences
// d_K = U_K - R, arranged so that every term that reaches the result is a
// product of a difference with an O(1) factor: its rounding is relative to
// |U - R|, not to |F|.  With u_K - u_R = (dm_K - u_R drho_K) / rho_K and
// p_K - p_R from (gamma-1)(dE - d(m.u)/2), the physical flux difference is
//   d(rho u) = dm, d(rho u^2 + p) = dm u + m_R du + dp,
//   d(rho u v) = dt u + t_R du, d((E+p) u) = (dE + dp) u + (E_R + p_R) du,
// and the star-state jump of eq. (star-l) is proportional to S_M - u_K,
//   S_M - u_l = (p_r - p_l - rho_r (S_R - u_r)(u_r - u_l)) / den,
//   S_M - u_r = (p_r - p_l - rho_l (S_L - u_l)(u_r - u_l)) / den,
// with den the denominator of S_M, p_r - p_l and u_r - u_l again from the
// differences.  R carries (rho, m_n, [m_t,] E) and rp = (u_R, v_R, p_R,
// E_R + p_R).  The branches and wave speeds are those of hllc().
template <int NV>
__device__ __forceinline__ void hllc_delta(const float *Ul, const float *Ur, const float *dl,
                                           const float *dr, const float *R, const float *rp,
                                           float gamma, float *dF, float &smax) {
  const float rl = Ul[0], rr = Ur[0];
  const float ipair = 1.0f / (rl * rr);
  const float irl = rr * ipair, irr = rl * ipair;
  const float ul = Ul[1] * irl, ur = Ur[1] * irr;
  const float vl = NV == 4 ? Ul[2] * irl : 0.0f, vr = NV == 4 ? Ur[2] * irr : 0.0f;
  const float El = Ul[NV - 1], Er = Ur[NV - 1];
  const float g1 = gamma - 1.0f;
  const float uR = rp[0], vR = rp[1], pR = rp[2], HR = rp[3];
  // differences of the primitive quantities from the reference
  const float dul = (dl[1] - uR * dl[0]) * irl, dur = (dr[1] - uR * dr[0]) * irr;
  const float dvl = NV == 4 ? (dl[2] - vR * dl[0]) * irl : 0.0f;
  const float dvr = NV == 4 ? (dr[2] - vR * dr[0]) * irr : 0.0f;
  const float dmul = dl[1] * ul + R[1] * dul + (NV == 4 ? dl[2] * vl + R[2] * dvl : 0.0f);
  const float dmur = dr[1] * ur + R[1] * dur + (NV == 4 ? dr[2] * vr + R[2] * dvr : 0.0f);
  const float dpl = g1 * (dl[NV - 1] - 0.5f * dmul), dpr = g1 * (dr[NV - 1] - 0.5f * dmur);
  const float pl = fmaxf(pR + dpl, 0.0f), pr = fmaxf(pR + dpr, 0.0f);
  const float al = sqrtf(gamma * pl * irl), ar = sqrtf(gamma * pr * irr);
  smax = fmaxf(fabsf(ul) + al, fabsf(ur) + ar);
  const float Hl = (El + pl) * irl, Hr = (Er + pr) * irr;
  const float Rq = sqrtf(rr * irl);
  const float iR = 1.0f / (1.0f + Rq);
  const float ut = (ul + ur * Rq) * iR, vt = (vl + vr * Rq) * iR, Ht = (Hl + Hr * Rq) * iR;
  const float at = sqrtf(g1 * (Ht - 0.5f * (ut * ut + vt * vt)));
  const float SL = fminf(ul - al, ut - at);
  const float SR = fmaxf(ur + ar, ut + at);
  // the physical flux difference of side K
  auto dphys = [&](const float *d, float u, float du, float dp, float *o) {
    o[0] = d[1];
    o[1] = d[1] * u + R[1] * du + dp;
    if (NV == 4) o[2] = d[2] * u + R[2] * du;
    o[NV - 1] = (d[NV - 1] + dp) * u + HR * du;
  };
  if (SL > 0.0f) {
    dphys(dl, ul, dul, dpl, dF);
    return;
  }
  const float den = rl * (SL - ul) - rr * (SR - ur);
  const float dpn = dpr - dpl, dun = dur - dul;
  const float sml = (dpn - rr * (SR - ur) * dun) / den;   // S_M - u_l
  const float SM = ul + sml;
  const bool left = SM > 0.0f;
  if (!left && !(SR >= 0.0f)) {
    dphys(dr, ur, dur, dpr, dF);
    return;
  }
  const float d = left ? sml : (dpn - rl * (SL - ul) * dun) / den;   // S_M - u_K
  const float rK = left ? rl : rr, uK = left ? ul : ur, pK = left ? pl : pr, SK = left ? SL : SR;
  const float vK = left ? vl : vr, EKr = left ? El * irl : Er * irr;
  float dK[NV];   // element-wise selects: no run-time indexing of the arrays
#pragma unroll
  for (int k = 0; k < NV; ++k) dK[k] = left ? dl[k] : dr[k];
  const float iss = 1.0f / (SK - SM);
  const float Jr = rK * d * iss;                 // rho*_K - rho_K
  const float chi = (SK - uK) * iss;
  float J[NV];
  J[0] = Jr;
  J[1] = Jr * SM + rK * d;
  if (NV == 4) J[2] = Jr * vK;
  J[NV - 1] = EKr * Jr + chi * d * (rK * SM + pK / (SK - uK));
  dphys(dK, uK, left ? dul : dur, left ? dpl : dpr, dF);
#pragma unroll
  for (int k = 0; k < NV; ++k) dF[k] += SK * J[k];
}

// Local Lax-Friedrichs flux, the alternative Sec. 3 names for the
// near-vacuum double rarefaction: the mean of the two physical fluxes minus
// alpha/2 times the jump, alpha the larger signal speed |u| + a of the two
// face states (also returned in smax, the speed eq. (CFL-CD) bounds)
template <typename real, int NV>
__device__ __forceinline__ void llf(const real *Ul, const real *Ur, real gamma, real *F,
                                    real &smax) {
  real pl = pressure<real, NV>(Ul, gamma), pr = pressure<real, NV>(Ur, gamma);
  if constexpr (sizeof(real) == 4) {
    pl = fmaxf(pl, 0.0f);
    pr = fmaxf(pr, 0.0f);
  }
  real al = fabs(Ul[1] / Ul[0]) + sqrt(gamma * pl / Ul[0]);
  real ar = fabs(Ur[1] / Ur[0]) + sqrt(gamma * pr / Ur[0]);
  smax = fmax(al, ar);
  real ha = real(0.5) * smax;
  real Fl[NV], Fr[NV];
  phys_flux<real, NV>(Ul, pl, Fl);
  phys_flux<real, NV>(Ur, pr, Fr);
#pragma unroll
  for (int k = 0; k < NV; ++k) F[k] = real(0.5) * (Fl[k] + Fr[k]) - ha * (Ur[k] - Ul[k]);
}

template <typename real>
__device__ __forceinline__ constexpr real unit_roundoff() {
  return sizeof(real) == 8 ? real(1.1102230246251565e-16) : real(5.9604645e-08);
}

// g(W) = rho E - |m|^2 / 2 - eps rho^2: for rho > 0, e(W) >= eps iff g >= 0
template <typename real, int NV>
__device__ __forceinline__ real energy_form(const real *w, real eps) {
  return w[0] * w[NV - 1] - real(0.5) * kin2<real, NV>(w) - eps * w[0] * w[0];
}

// round-off allowance of g along the segment from Ubar to W: forming
// (1-t) Ubar + t W costs a few ulps of |Ubar| + |W| per component, which
// moves the bilinear form g by at most a small multiple of
// u [(|E|+|E_w|)(|rho|+|rho_w|) + (|m|+|m_w|)^2]; the limiter asks g >= eta
// so that the rounded limited states stay inside G
template <typename real, int NV>
__device__ __forceinline__ real energy_allowance(const real *ub, const real *w, real uu) {
  real sm = real(0);
#pragma unroll
  for (int k = 1; k < NV - 1; ++k) sm += sqr(fabs(ub[k]) + fabs(w[k]));
  return real(16) * uu *
         ((fabs(ub[NV - 1]) + fabs(w[NV - 1])) * (fabs(ub[0]) + fabs(w[0])) + sm);
}

// root t in (0, 1] of g((1 - t) Ubar + t W) = eta: the quadratic
// A t^2 + B t + (C - eta) = 0 with C - eta > 0; the cancellation-free form
// 2C' / (-B + sqrt(B^2 - 4AC')) picks the root in (0, 1)
template <typename real, int NV>
__device__ __forceinline__ real energy_root(const real *ub, const real *w, real eps, real eta) {
  real dr = w[0] - ub[0], dE = w[NV - 1] - ub[NV - 1];
  real dm1 = w[1] - ub[1], dm2 = NV == 4 ? w[2] - ub[2] : real(0);
  real m1 = ub[1], m2 = NV == 4 ? ub[2] : real(0);
  real A = dE * dr - real(0.5) * (dm1 * dm1 + dm2 * dm2) - eps * dr * dr;
  real B = ub[NV - 1] * dr + dE * ub[0] - (m1 * dm1 + m2 * dm2) - real(2) * eps * ub[0] * dr;
  real C = ub[NV - 1] * ub[0] - real(0.5) * (m1 * m1 + m2 * m2) - eps * ub[0] * ub[0] - eta;
  if (!(C > real(0))) return real(0);
  real D = fmax(B * B - real(4) * A * C, real(0));
  real den = -B + sqrt(D);
  real t = den > real(0) ? real(2) * C / den : real(0);
  if (!(t >= real(0))) t = real(0);
  return fmin(t, real(1));
}

// Zhang-Shu limiter of one cell (Sec. 2.4, steps 1-4).  um = U^-_{i+1/2},
// up = U^+_{i-1/2} are limited in place.  Returns bit 0 if theta_1 < 1 and
// bit 1 if theta_2 < 1.  theta = 1 leaves the values untouched.  Both
// thresholds carry the round-off allowance that keeps the rounded limited
// states in G.
// uu is the unit round-off of the arithmetic in which the limited faces are
// stored and used (FP64 for the plain form, FP32 for the mixed form)
template <typename real, int NV>
__device__ __forceinline__ int limit_cell(const real *ub, real *um, real *up, real wgl, real eps,
                                          real uu) {
  int flags = 0;
  real inv12 = real(1) / (real(1) - real(2) * wgl);
  real rho_star = (ub[0] - wgl * up[0] - wgl * um[0]) * inv12;
  real rho_min = fmin(fmin(um[0], up[0]), rho_star);
  real eps_r = eps + real(8) * uu * (fabs(ub[0]) + fabs(rho_min));
  if (rho_min < eps_r) {
    real th1 = fmin(fmax((ub[0] - eps_r) / (ub[0] - rho_min), real(0)), real(1));
    um[0] = th1 * (um[0] - ub[0]) + ub[0];
    up[0] = th1 * (up[0] - ub[0]) + ub[0];
    flags |= 1;
  }
  real th2 = real(1);
  real w3[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) w3[k] = (ub[k] - wgl * up[k] - wgl * um[k]) * inv12;
  {
    real eta = energy_allowance<real, NV>(ub, um, uu);
    if (energy_form<real, NV>(um, eps) < eta) th2 = fmin(th2, energy_root<real, NV>(ub, um, eps, eta));
  }
  {
    real eta = energy_allowance<real, NV>(ub, up, uu);
    if (energy_form<real, NV>(up, eps) < eta) th2 = fmin(th2, energy_root<real, NV>(ub, up, eps, eta));
  }
  {
    real eta = energy_allowance<real, NV>(ub, w3, uu);
    if (energy_form<real, NV>(w3, eps) < eta) th2 = fmin(th2, energy_root<real, NV>(ub, w3, eps, eta));
  }
  if (th2 < real(1)) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      um[k] = th2 * (um[k] - ub[k]) + ub[k];
      up[k] = th2 * (up[k] - ub[k]) + ub[k];
    }
    flags |= 2;
  }
  return flags;
}

// Mixed form: an FP32 test of the limiter's conditions with doubled
// allowances; only cells that may need limiting compute the scaling factors
// theta_1, theta_2 in FP64 (with the FP32 allowance, since the limited faces
// are stored in FP32).  Returns the limiter flags.
// FP32 pretest of a cell: true when the exact (FP64) limiter might change
// its face values; the caller then runs the exact limiter on it.  Used by
// both forms (the FP64 form passes its values rounded to FP32).
template <int NV>
__device__ __forceinline__ bool limit_need_mixed(const float *ub, const float *um, const float *up,
                                                 float wgl, float inv12, float eps) {
  const float uf = 5.9604645e-08f;
  float w3[NV];   // the interior quadrature point implied by the cell average
#pragma unroll
  for (int k = 0; k < NV; ++k) w3[k] = (ub[k] - wgl * up[k] - wgl * um[k]) * inv12;
  const float rho_min = fminf(fminf(um[0], up[0]), w3[0]);
  bool need = rho_min < 2.0f * (eps + 8.0f * uf * (fabsf(ub[0]) + fabsf(rho_min)));
  // one allowance for the three points, with each magnitude replaced by the
  // largest over them: it bounds the three allowances, so the test (doubled
  // for FP32) flags every cell the exact test would (a superset; the FP64
  // pass decides)
  const float rmx = fmaxf(fmaxf(fabsf(um[0]), fabsf(up[0])), fabsf(w3[0]));
  const float emx = fmaxf(fmaxf(fabsf(um[NV - 1]), fabsf(up[NV - 1])), fabsf(w3[NV - 1]));
  float sm = 0.0f;
#pragma unroll
  for (int k = 1; k < NV - 1; ++k) {
    const float mk = fmaxf(fmaxf(fabsf(um[k]), fabsf(up[k])), fabsf(w3[k]));
    sm += sqr(fabsf(ub[k]) + mk);
  }
  const float eta2 =
      32.0f * uf * ((fabsf(ub[NV - 1]) + emx) * (fabsf(ub[0]) + rmx) + sm);
  need = need | (energy_form<float, NV>(um, eps) < eta2) |
         (energy_form<float, NV>(up, eps) < eta2) | (energy_form<float, NV>(w3, eps) < eta2);
  // magnitudes beyond FP32's range (or NaN) make the allowance non-finite:
  // such a cell always goes to the exact test
  return need | !(eta2 <= 3.0e38f);
}

// The FP64 limiter of a flagged cell of the mixed form, on FP32 face values
// limited in place (with the FP32 round-off allowance: the limited faces are
// stored in FP32).  Returns the limiter flags.
template <int NV>
__device__ __forceinline__ int limit_cell_mixed_fp64(const float *ub, float *um, float *up,
                                                     float wgl, float eps) {
  const double uf = 5.9604645e-08;
  double b[NV], m[NV], p[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    b[k] = ub[k];
    m[k] = um[k];
    p[k] = up[k];
  }
  const int f = limit_cell<double, NV>(b, m, p, (double)wgl, (double)eps, uf);
  if (f) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      um[k] = (float)m[k];
      up[k] = (float)p[k];
    }
  }
  return f;
}

}  // namespace ppk
