// xf_adjoint.cuh -- reverse mode (vector-Jacobian product) of the RHS stage.
//
// Ubar += scale * (dL/dU)^T Rbar, written by hand in the reverse order of the
// forward kernels in xf_device.cuh:
//   k_face_adj<D>: per face, recompute the forward face quantities, then walk
//     back through the back-projection (Eq. 15), the two WENO5-JS
//     reconstructions of every field (weights included), the PER projection
//     and LLF splitting (Eq. 14, alpha through the arg-max cell, first maximum
//     on ties, d|x|/dx = 0 at 0), the Roe-averaged face state and its thermo,
//     and the viscous face flux; adjoints of the per-cell fields are
//     scattered with atomicAdd into Qbar (same layout as Q).
//   k_grad_adj: gather form of the nodal-derivative adjoint (no atomics).
//   k_prim_adj: per padded cell, the adjoint of primitive recovery: transport
//     (Eq. 29, Wilke Eq. 22), EOS (Eq. 7), sound speed, and the Newton
//     temperature through the implicit-function theorem (dT = (de - sum_s e_s
//     dY_s)/c_v); scattered into Ubar through the boundary mapping.
#pragma once
#include "xf_device.cuh"

namespace xf {

// ------------------------------------------------------------ WENO5 adjoint
// Forward intermediates of one WENO5-JS reconstruction, computed exactly as
// weno5_nd (indicators scaled by 12 c_k with the linear weights folded in, as
// the sums of squares 16 A^2 + 39/4 x^2 of their LDL^T forms, candidates as
// 6 (q_k - f2)), kept for its reverse. F = f2 + num/den with the factor 6
// carried by den.
struct W5 {
  double a, b, c, d, A0, B1, D2, s0, s1, s2, p12, p02, p01, w0, w1, w2, q0, q1, q2;
  double num, den;
};

// K = Params::kface in registers, E = {12 eps c_k} in device memory (as
// weno5_nd)
__device__ __forceinline__ void w5_fwd(double f0, double f1, double f2, double f3, double f4,
                                       const double* K, const double* E, W5& r) {
  r.a = f1 - f0; r.b = f2 - f1; r.c = f3 - f2; r.d = f4 - f3;
  r.A0 = fma(K[0], r.b, r.a); r.B1 = fma(K[1], r.c, r.b); r.D2 = fma(K[0], r.c, r.d);
  const double cc = r.c * r.c;
  r.s0 = fma(r.A0, r.A0, fma(K[2] * r.b, r.b, __ldcg(E + 0)));  // 16 c_0 = 1
  r.s1 = fma(K[3] * r.B1, r.B1, fma(K[4], cc, __ldcg(E + 1)));
  r.s2 = fma(K[5] * r.D2, r.D2, fma(K[6], cc, __ldcg(E + 2)));
  r.p12 = r.s1 * r.s2; r.p02 = r.s0 * r.s2; r.p01 = r.s0 * r.s1;
  r.w0 = r.p12 * r.p12; r.w1 = r.p02 * r.p02; r.w2 = r.p01 * r.p01;
  r.q0 = fma(K[7], r.A0, K[8] * r.b);
  r.q1 = fma(K[9], r.c, r.b);
  r.q2 = fma(K[10], r.c, -r.d);
  r.num = fma(r.w0, r.q0, fma(r.w1, r.q1, r.w2 * r.q2));
  r.den = K[22] * ((r.w0 + r.w1) + r.w2);
}

// Reverse of one reconstruction: (nbar, dbar) for (num, den) -> fb[0..4] (added).
__device__ __forceinline__ void w5_rev(const W5& r, double nbar, double dbar, const double* K,
                                       double* fb) {
  const double d6 = K[22] * dbar;
  const double w0b = fma(nbar, r.q0, d6), w1b = fma(nbar, r.q1, d6), w2b = fma(nbar, r.q2, d6);
  const double q0b = nbar * r.w0, q1b = nbar * r.w1, q2b = nbar * r.w2;
  const double p12b = (w0b + w0b) * r.p12, p02b = (w1b + w1b) * r.p02, p01b = (w2b + w2b) * r.p01;
  const double s0b = fma(p02b, r.s2, p01b * r.s1);
  const double s1b = fma(p12b, r.s2, p01b * r.s0);
  const double s2b = fma(p12b, r.s1, p02b * r.s0);
  // s_k = 16 c_k L_k^2 + 39/4 c_k x_k^2 + e; A0 = a - 11/8 b, B1 = b - 5/8 c,
  // D2 = d - 11/8 c; q0 = 9/4 b - 2 A0, q1 = 2c + b, q2 = 4c - d
  // (K: 32 c_0 = 2, -1.375, -0.625, -2, 2.25, 2, 4, 32 c_1, 32 c_2, 19.5 c_k)
  const double A0b = fma(r.A0 + r.A0, s0b, K[7] * q0b);
  const double B1b = K[23] * r.B1 * s1b;
  const double D2b = K[24] * r.D2 * s2b;
  const double ab = A0b;
  const double bb = fma(K[25] * r.b, s0b, fma(K[8], q0b, fma(K[0], A0b, B1b + q1b)));
  const double cb = fma(r.c, fma(K[26], s1b, K[27] * s2b),
                        fma(K[9], q1b, fma(K[10], q2b, fma(K[1], B1b, K[0] * D2b))));
  const double db = D2b - q2b;
  fb[0] -= ab;
  fb[1] += ab - bb;
  fb[2] += bb - cb;
  fb[3] += cb - db;
  fb[4] += db;
}

// One field's F = F^+ + F^- (as rec_nd with WENO5) and its reverse: returns F
// and adds Fb dF/dw to wpb[0..5], wmb[0..5].
__device__ __forceinline__ double weno5_pair_fwd_adj(const double* wp, const double* wm,
                                                     const double* K, const double* E, double Fb,
                                                     double* wpb, double* wmb) {
  W5 P, M;
  w5_fwd(wp[0], wp[1], wp[2], wp[3], wp[4], K, E, P);
  w5_fwd(wm[5], wm[4], wm[3], wm[2], wm[1], K, E, M);
  // both reciprocals from one division; F from them
  const double rpm = rcp_nr1(P.den * M.den, K[13]);
  const double idp = rpm * M.den, idm = rpm * P.den;
  const double F = (wp[2] + wm[3]) + fma(P.num, idp, M.num * idm);
  double fb[5] = {-0.0, -0.0, -0.0, -0.0, -0.0};
  w5_rev(P, Fb * idp, -Fb * P.num * idp * idp, K, fb);
#pragma unroll
  for (int k = 0; k < 5; ++k) wpb[k] += fb[k];
  wpb[2] += Fb;
  double gb[5] = {-0.0, -0.0, -0.0, -0.0, -0.0};
  w5_rev(M, Fb * idm, -Fb * M.num * idm * idm, K, gb);
  wmb[5] += gb[0];
  wmb[4] += gb[1];
  wmb[3] += gb[2] + Fb;
  wmb[2] += gb[3];
  wmb[1] += gb[4];
  return F;
}

// ---------------------------------------------------------- WENO-CU6 adjoint
// Forward intermediates of one CU6 reconstruction exactly as cu6_nd (12 beta
// with beta_0..2 and beta_6 as LDL^T sums of squares, weights d_k (C s_k +
// 12 tau) times the other s_j, candidates 6 (q_k - f2)), and the reverse. den
// carries the 6.
struct C6 {
  double a, b, c, d, e, A0, B1, D2, y0, y1, y2, y3, y4;
  double s0, s1, s2, s3, p01, p23, g0, g1, g2, g3, w0, w1, w2, w3, q0, q1, q2, q3;
  double num, den;
};

__device__ __forceinline__ void c6_fwd(double f0, double f1, double f2, double f3, double f4,
                                       double f5, double e12, C6& r) {
  r.a = f1 - f0; r.b = f2 - f1; r.c = f3 - f2; r.d = f4 - f3; r.e = f5 - f4;
  r.A0 = fma(-1.375, r.b, r.a); r.B1 = fma(-0.625, r.c, r.b); r.D2 = fma(-1.375, r.c, r.d);
  const double c975 = 9.75 * r.c * r.c;
  const double b0 = fma(16.0 * r.A0, r.A0, (9.75 * r.b) * r.b);
  const double b1 = fma(16.0 * r.B1, r.B1, c975);
  const double b2 = fma(16.0 * r.D2, r.D2, c975);
  r.y4 = r.e;
  r.y3 = fma(kB6L43, r.e, r.d);
  r.y2 = fma(kB6L42, r.e, fma(kB6L32, r.d, r.c));
  r.y1 = fma(kB6L41, r.e, fma(kB6L31, r.d, fma(kB6L21, r.c, r.b)));
  r.y0 = fma(kB6L40, r.e, fma(kB6L30, r.d, fma(kB6L20, r.c, fma(kB6L10, r.b, r.a))));
  const double b6 = fma(kB6D[0] * r.y0, r.y0, fma(kB6D[1] * r.y1, r.y1, fma(kB6D[2] * r.y2, r.y2,
                    fma(kB6D[3] * r.y3, r.y3, kB6D[4] * r.y4 * r.y4))));
  const double tau = b6 - (b0 + b2 + 4.0 * b1) * (1.0 / 6.0);
  r.s0 = b0 + e12; r.s1 = b1 + e12; r.s2 = b2 + e12; r.s3 = b6 + e12;
  r.p01 = r.s0 * r.s1; r.p23 = r.s2 * r.s3;
  const double t05 = 0.05 * tau, t45 = 0.45 * tau;
  r.g0 = fma(0.05 * 20.0, r.s0, t05); r.g1 = fma(0.45 * 20.0, r.s1, t45);
  r.g2 = fma(0.45 * 20.0, r.s2, t45); r.g3 = fma(0.05 * 20.0, r.s3, t05);
  r.w0 = r.g0 * (r.s1 * r.p23); r.w1 = r.g1 * (r.s0 * r.p23);
  r.w2 = r.g2 * (r.p01 * r.s3); r.w3 = r.g3 * (r.p01 * r.s2);
  r.q0 = fma(-2.0, r.A0, 2.25 * r.b); r.q1 = fma(2.0, r.c, r.b); r.q2 = fma(4.0, r.c, -r.d);
  r.q3 = fma(6.0, r.c, fma(-5.0, r.d, 2.0 * r.e));
  r.num = fma(r.w0, r.q0, fma(r.w1, r.q1, fma(r.w2, r.q2, r.w3 * r.q3)));
  r.den = 6.0 * ((r.w0 + r.w1) + (r.w2 + r.w3));
}

// (nbar, dbar) for (num, den) -> fb[0..5] (added)
__device__ __forceinline__ void c6_rev(const C6& r, double nbar, double dbar, double* fb) {
  const double d6 = 6.0 * dbar;
  const double w0b = fma(nbar, r.q0, d6), w1b = fma(nbar, r.q1, d6);
  const double w2b = fma(nbar, r.q2, d6), w3b = fma(nbar, r.q3, d6);
  const double q0b = nbar * r.w0, q1b = nbar * r.w1, q2b = nbar * r.w2, q3b = nbar * r.w3;
  const double g0b = w0b * (r.s1 * r.p23), g1b = w1b * (r.s0 * r.p23);
  const double g2b = w2b * (r.p01 * r.s3), g3b = w3b * (r.p01 * r.s2);
  double s0b = fma(w1b * r.g1, r.p23, g0b), s1b = fma(w0b * r.g0, r.p23, 9.0 * g1b);
  double s2b = fma(w3b * r.g3, r.p01, 9.0 * g2b), s3b = fma(w2b * r.g2, r.p01, g3b);
  const double p23b = fma(w0b * r.g0, r.s1, w1b * r.g1 * r.s0);
  const double p01b = fma(w2b * r.g2, r.s3, w3b * r.g3 * r.s2);
  s0b = fma(p01b, r.s1, s0b); s1b = fma(p01b, r.s0, s1b);
  s2b = fma(p23b, r.s3, s2b); s3b = fma(p23b, r.s2, s3b);
  const double taub = fma(0.05, g0b + g3b, 0.45 * (g1b + g2b));
  // s_k = b_k + e12; tau = b6 - (b0 + b2 + 4 b1)/6
  const double b6b = s3b + taub;
  const double b0b = s0b - taub * (1.0 / 6.0), b2b = s2b - taub * (1.0 / 6.0);
  const double b1b = s1b - taub * (4.0 / 6.0);
  const double y0b = 2.0 * kB6D[0] * r.y0 * b6b, y1b = 2.0 * kB6D[1] * r.y1 * b6b;
  const double y2b = 2.0 * kB6D[2] * r.y2 * b6b, y3b = 2.0 * kB6D[3] * r.y3 * b6b;
  const double y4b = 2.0 * kB6D[4] * r.y4 * b6b;
  // b0 = 16 A0^2 + 39/4 b^2, b1 = 16 B1^2 + 39/4 c^2, b2 = 16 D2^2 + 39/4 c^2;
  // A0 = a - 11/8 b, B1 = b - 5/8 c, D2 = d - 11/8 c; q0 = 9/4 b - 2 A0
  const double A0b = fma(32.0 * r.A0, b0b, -2.0 * q0b);
  const double B1b = 32.0 * r.B1 * b1b, D2b = 32.0 * r.D2 * b2b;
  const double ab = y0b + A0b;
  const double bb = kB6L10 * y0b + y1b + fma(19.5 * r.b, b0b, fma(2.25, q0b, fma(-1.375, A0b, B1b))) +
                    q1b;
  const double cb = kB6L20 * y0b + kB6L21 * y1b + y2b +
                    fma(19.5 * r.c, b1b + b2b, fma(-0.625, B1b, -1.375 * D2b)) + 2.0 * q1b +
                    4.0 * q2b + 6.0 * q3b;
  const double db = kB6L30 * y0b + kB6L31 * y1b + kB6L32 * y2b + y3b + D2b - q2b - 5.0 * q3b;
  const double eb = kB6L40 * y0b + kB6L41 * y1b + kB6L42 * y2b + kB6L43 * y3b + y4b + 2.0 * q3b;
  fb[0] -= ab;
  fb[1] += ab - bb;
  fb[2] += bb - cb;
  fb[3] += cb - db;
  fb[4] += db - eb;
  fb[5] += eb;
}

// ------------------------------------------------------------ WENO7 adjoint
// Forward intermediates of one WENO7 reconstruction exactly as weno7_nd, and
// the reverse (den without a scale factor).
struct W7 {
  double x0, x1, x2, x3, x4, x5, A[4], B[4], s0, s1, s2, s3, p01, p23, r0, r1, r2, r3;
  double w0, w1, w2, w3, q0, q1, q2, q3, num, den;
};

__device__ __forceinline__ void w7_fwd(double f0, double f1, double f2, double f3, double f4,
                                       double f5, double f6, const double* ec, W7& r) {
  r.x0 = f1 - f0; r.x1 = f2 - f1; r.x2 = f3 - f2; r.x3 = f4 - f3; r.x4 = f5 - f4; r.x5 = f6 - f5;
  const double z2 = kW7D3 * r.x2 * r.x2, z3 = kW7D3 * r.x3 * r.x3;
  // A, B of Q0(x0, x1, x2), Q1(x1, x2, x3), Q1(x4, x3, x2), Q0(x5, x4, x3)
  r.A[0] = fma(1.6946983546617915, r.x2, fma(-2.5484460694698354, r.x1, r.x0));
  r.B[0] = fma(-1.4896519285042333, r.x2, r.x1);
  r.A[1] = fma(0.92509363295880154, r.x3, fma(-2.0749063670411987, r.x2, r.x1));
  r.B[1] = fma(-0.6326434619002822, r.x3, r.x2);
  r.A[2] = fma(0.92509363295880154, r.x2, fma(-2.0749063670411987, r.x3, r.x4));
  r.B[2] = fma(-0.6326434619002822, r.x2, r.x3);
  r.A[3] = fma(1.6946983546617915, r.x3, fma(-2.5484460694698354, r.x4, r.x5));
  r.B[3] = fma(-1.4896519285042333, r.x3, r.x4);
  const double Q0 = fma(547.0 * r.A[0], r.A[0], fma(155.46617915904935 * r.B[0], r.B[0], z2));
  const double Q1 = fma(267.0 * r.A[1], r.A[1], fma(318.50187265917606 * r.B[1], r.B[1], z3));
  const double Q2 = fma(267.0 * r.A[2], r.A[2], fma(318.50187265917606 * r.B[2], r.B[2], z2));
  const double Q3 = fma(547.0 * r.A[3], r.A[3], fma(155.46617915904935 * r.B[3], r.B[3], z3));
  r.s0 = fma(kW7c0, Q0, ec[0]); r.s1 = fma(kW7c1, Q1, ec[1]);
  r.s2 = fma(kW7c2, Q2, ec[2]); r.s3 = fma(kW7c3, Q3, ec[3]);
  r.p01 = r.s0 * r.s1; r.p23 = r.s2 * r.s3;
  r.r0 = r.s1 * r.p23; r.r1 = r.s0 * r.p23; r.r2 = r.p01 * r.s3; r.r3 = r.p01 * r.s2;
  r.w0 = r.r0 * r.r0; r.w1 = r.r1 * r.r1; r.w2 = r.r2 * r.r2; r.w3 = r.r3 * r.r3;
  r.q0 = fma(0.25, r.x0, fma(-5.0 / 6.0, r.x1, (13.0 / 12.0) * r.x2));
  r.q1 = fma(-1.0 / 12.0, r.x1, fma(1.0 / 3.0, r.x2, 0.25 * r.x3));
  r.q2 = fma(1.0 / 12.0, r.x2, fma(0.5, r.x3, (-1.0 / 12.0) * r.x4));
  r.q3 = fma(0.75, r.x3, fma(-1.0 / 3.0, r.x4, (1.0 / 12.0) * r.x5));
  r.num = fma(r.w0, r.q0, fma(r.w1, r.q1, fma(r.w2, r.q2, r.w3 * r.q3)));
  r.den = (r.w0 + r.w1) + (r.w2 + r.w3);
}

// (nbar, dbar) for (num, den) -> fb[0..6] (added)
__device__ __forceinline__ void w7_rev(const W7& r, double nbar, double dbar, double* fb) {
  const double w0b = fma(nbar, r.q0, dbar), w1b = fma(nbar, r.q1, dbar);
  const double w2b = fma(nbar, r.q2, dbar), w3b = fma(nbar, r.q3, dbar);
  const double q0b = nbar * r.w0, q1b = nbar * r.w1, q2b = nbar * r.w2, q3b = nbar * r.w3;
  const double r0b = 2.0 * r.r0 * w0b, r1b = 2.0 * r.r1 * w1b;
  const double r2b = 2.0 * r.r2 * w2b, r3b = 2.0 * r.r3 * w3b;
  const double p23b = fma(r0b, r.s1, r1b * r.s0), p01b = fma(r2b, r.s3, r3b * r.s2);
  const double s0b = fma(r1b, r.p23, p01b * r.s1), s1b = fma(r0b, r.p23, p01b * r.s0);
  const double s2b = fma(r3b, r.p01, p23b * r.s3), s3b = fma(r2b, r.p01, p23b * r.s2);
  const double Qb[4] = {kW7c0 * s0b, kW7c1 * s1b, kW7c2 * s2b, kW7c3 * s3b};
  double xb[6] = {-0.0, -0.0, -0.0, -0.0, -0.0, -0.0};
  // z2 (indicators 0 and 2), z3 (1 and 3)
  xb[2] += 2.0 * kW7D3 * r.x2 * (Qb[0] + Qb[2]);
  xb[3] += 2.0 * kW7D3 * r.x3 * (Qb[1] + Qb[3]);
  {  // Q0(x0, x1, x2)
    const double Ab = 2.0 * 547.0 * r.A[0] * Qb[0], Bb = 2.0 * 155.46617915904935 * r.B[0] * Qb[0];
    xb[0] += Ab; xb[1] += fma(-2.5484460694698354, Ab, Bb);
    xb[2] += fma(1.6946983546617915, Ab, -1.4896519285042333 * Bb);
  }
  {  // Q1(x1, x2, x3)
    const double Ab = 2.0 * 267.0 * r.A[1] * Qb[1], Bb = 2.0 * 318.50187265917606 * r.B[1] * Qb[1];
    xb[1] += Ab; xb[2] += fma(-2.0749063670411987, Ab, Bb);
    xb[3] += fma(0.92509363295880154, Ab, -0.6326434619002822 * Bb);
  }
  {  // Q1(x4, x3, x2)
    const double Ab = 2.0 * 267.0 * r.A[2] * Qb[2], Bb = 2.0 * 318.50187265917606 * r.B[2] * Qb[2];
    xb[4] += Ab; xb[3] += fma(-2.0749063670411987, Ab, Bb);
    xb[2] += fma(0.92509363295880154, Ab, -0.6326434619002822 * Bb);
  }
  {  // Q0(x5, x4, x3)
    const double Ab = 2.0 * 547.0 * r.A[3] * Qb[3], Bb = 2.0 * 155.46617915904935 * r.B[3] * Qb[3];
    xb[5] += Ab; xb[4] += fma(-2.5484460694698354, Ab, Bb);
    xb[3] += fma(1.6946983546617915, Ab, -1.4896519285042333 * Bb);
  }
  xb[0] += 0.25 * q0b;
  xb[1] += (-5.0 / 6.0) * q0b + (-1.0 / 12.0) * q1b;
  xb[2] += (13.0 / 12.0) * q0b + (1.0 / 3.0) * q1b + (1.0 / 12.0) * q2b;
  xb[3] += 0.25 * q1b + 0.5 * q2b + 0.75 * q3b;
  xb[4] += (-1.0 / 12.0) * q2b + (-1.0 / 3.0) * q3b;
  xb[5] += (1.0 / 12.0) * q3b;
#pragma unroll
  for (int j = 0; j < 6; ++j) { fb[j] -= xb[j]; fb[j + 1] += xb[j]; }
}

// One field's F = F^+ + F^- with the reconstruction REC and its reverse:
// returns F and adds Fb dF/dw to wpb[0..SW-1], wmb[0..SW-1] (w^- mirrored).
// e4, K and E as in rec_nd.
template <int REC>
__device__ __forceinline__ double rec_pair_fwd_adj(const double* wp, const double* wm,
                                                   const double* e4, const double* K,
                                                   const double* E, double Fb, double* wpb,
                                                   double* wmb) {
  if constexpr (REC == 5) {
    return weno5_pair_fwd_adj(wp, wm, K, E, Fb, wpb, wmb);
  } else if constexpr (REC == 6) {
    C6 P, M;
    c6_fwd(wp[0], wp[1], wp[2], wp[3], wp[4], wp[5], e4[3], P);
    c6_fwd(wm[5], wm[4], wm[3], wm[2], wm[1], wm[0], e4[3], M);
    const double rpm = rcp_nr(P.den * M.den);
    const double idp = rpm * M.den, idm = rpm * P.den;
    const double F = (wp[2] + wm[3]) + fma(P.num, idp, M.num * idm);
    double fb[6] = {-0.0, -0.0, -0.0, -0.0, -0.0, -0.0}, gb[6] = {-0.0, -0.0, -0.0, -0.0, -0.0, -0.0};
    c6_rev(P, Fb * idp, -Fb * P.num * idp * idp, fb);
    c6_rev(M, Fb * idm, -Fb * M.num * idm * idm, gb);
#pragma unroll
    for (int k = 0; k < 6; ++k) { wpb[k] += fb[k]; wmb[5 - k] += gb[k]; }
    wpb[2] += Fb;
    wmb[3] += Fb;
    return F;
  } else {
    W7 P, M;
    w7_fwd(wp[0], wp[1], wp[2], wp[3], wp[4], wp[5], wp[6], e4, P);
    w7_fwd(wm[7], wm[6], wm[5], wm[4], wm[3], wm[2], wm[1], e4, M);
    const double rpm = rcp_nr(P.den * M.den);
    const double idp = rpm * M.den, idm = rpm * P.den;
    const double F = (wp[3] + wm[4]) + fma(P.num, idp, M.num * idm);
    double fb[7] = {-0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0}, gb[7] = {-0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0};
    w7_rev(P, Fb * idp, -Fb * P.num * idp * idp, fb);
    w7_rev(M, Fb * idm, -Fb * M.num * idm * idm, gb);
#pragma unroll
    for (int k = 0; k < 7; ++k) { wpb[k] += fb[k]; wmb[7 - k] += gb[k]; }
    wpb[3] += Fb;
    wmb[4] += Fb;
    return F;
  }
}

// d c_p,s / dT at a clamped tau (0 outside the polynomial range)
__device__ __forceinline__ double dcp_s(const Params& p, int s, double T) {
  const double tau = fma(T, p.inv_span, p.tau0);  // as tau_of
  if (!(tau > 0.0 && tau < 1.0)) return 0.0;
  const double* a = p.rcp[s];
  return fma(fma(fma(4.0 * a[4], tau, 3.0 * a[3]), tau, 2.0 * a[2]), tau, a[1]) * p.inv_span;
}

// Reverse-mode accumulators below start at -0.0, not +0.0: -0.0 + x is x for
// every x (both zeros included), so the first accumulation folds away, while
// +0.0 + x would have to be computed (it turns -0 into +0).

// Atomic scatter that skips exact zeros (+0 and -0: the bit pattern shifted
// left by one is zero), tested on the integer pipe rather than with an FP64
// compare.
__device__ __forceinline__ void aadd(double* p, double v) {
  if ((__double_as_longlong(v) << 1) != 0) atomicAdd(p, v);
}

// a > b for non-negative doubles, on their bit patterns (integer pipe)
__device__ __forceinline__ bool gt_nn(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}


// ------------------------------------------------- positivity blend adjoint
// Reverse of pos_blend (Eq. 17-20) for one face inside an RK stage of step dt:
// recomputes the face's convective flux F_hat (conv_flux, WENO5) and the
// blend; with theta < 1, F* = F_LF + theta (F_hat - F_LF), so F_hat gets
// theta Gb and F_LF (1 - theta) Gb, and theta's adjoint goes to the binding
// partial-density condition (the first one reaching the minimum; none when
// theta is clipped at 0 or eps = lo, where theta is locally constant) and
// through F_LF of Eq. 19 (alpha through the cell with the larger |u_d| + c)
// to U, u_d, p and c of the two cells (scattered into Qb). Gc returns the
// adjoint of F_hat (Gb itself when the blend is inactive). With fh given,
// F_hat is read from the flux tape (fh[v * fstride], written by the forward
// step's k_face_tape) instead of being recomputed.
template <int DIM, int NS, int D, int REC>
__device__ __forceinline__ void pos_blend_adj(const Params& p, const double* __restrict__ q0,
                                              double* __restrict__ qb0, long long PC, long long sd,
                                              double dt, const double* Gb, double* Gc,
                                              const double* __restrict__ fh = nullptr,
                                              long long fstride = 0) {
  using L = Lay<DIM, NS>;
  constexpr int NV = L::NV;
  constexpr int IE = DIM + 1;
#define QF(field, m) ld(q0 + (long long)(field) * PC + (long long)(m) * sd)
#define QB(field, m, val) aadd(qb0 + (long long)(field) * PC + (long long)(m) * sd, (val))
  double Gh[NV];
  if (fh) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Gh[v] = ld(fh + v * fstride);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) Gh[v] = 0.0;
    uint32_t st = 0;
    conv_flux<DIM, NS, D, REC>(p, q0, PC, sd, Gh, st);
  }
  const double lam2 = 2.0 * DIM * dt * p.inv_dx[D];
  double Ua[NV], Ub[NV], Fa[NV], Fb[NV], Flf[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { Ua[v] = QF(L::U + v, 0); Ub[v] = QF(L::U + v, 1); }
  const double una = QF(L::UN + D, 0), unb = QF(L::UN + D, 1);
  const double pa = QF(L::P, 0), pb = QF(L::P, 1);
  const double ca = QF(L::C, 0), cb = QF(L::C, 1);
#pragma unroll
  for (int v = 0; v < NV; ++v) { Fa[v] = una * Ua[v]; Fb[v] = unb * Ub[v]; }
  Fa[1 + D] += pa; Fb[1 + D] += pb;
  Fa[IE] += pa * una; Fb[IE] += pb * unb;
  const double sa = fabs(una) + ca, sbv = fabs(unb) + cb;
  const double al = fmax(sa, sbv);
#pragma unroll
  for (int v = 0; v < NV; ++v) Flf[v] = 0.5 * (Fa[v] + Fb[v] + al * (Ua[v] - Ub[v]));
  // theta and its binding condition
  double theta = 1.0, lo_s = 0.0, hi_s = 0.0, eps_s = 0.0;
  int s_s = -1, side_s = 0;
  bool live = false;  // theta depends on (lo, hi) there
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double qa, qb, fh, fl;
    if (s < NS - 1) {
      qa = Ua[IE + 1 + s]; qb = Ub[IE + 1 + s]; fh = Gh[IE + 1 + s]; fl = Flf[IE + 1 + s];
    } else {
      qa = Ua[0]; qb = Ub[0]; fh = Gh[0]; fl = Flf[0];
#pragma unroll
      for (int k = 0; k < NS - 1; ++k) {
        qa -= Ua[IE + 1 + k]; qb -= Ub[IE + 1 + k]; fh -= Gh[IE + 1 + k]; fl -= Flf[IE + 1 + k];
      }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const double sg = side == 0 ? -lam2 : lam2;
      const double q = side == 0 ? qa : qb;
      const double hi = fma(sg, fh, q), lo = fma(sg, fl, q);
      const double eps = fmin(lo, p.pos_eps);
      if (hi < eps) {
        const double cand = (lo - eps) / (lo - hi);
        const double th = fmax(cand, 0.0);
        if (th < theta) {
          theta = th;
          s_s = s; side_s = side; lo_s = lo; hi_s = hi; eps_s = eps;
          live = cand > 0.0 && lo >= p.pos_eps;
        }
      }
    }
  }
  if (!(theta < 1.0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Gc[v] = Gb[v];
    return;
  }
  double thetab = -0.0, Flfb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    thetab = fma(Gh[v] - Flf[v], Gb[v], thetab);
    Gc[v] = theta * Gb[v];
    Flfb[v] = (1.0 - theta) * Gb[v];
  }
  double Uab[NV], Ubb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { Uab[v] = -0.0; Ubb[v] = -0.0; }
  if (live) {
    // theta = (lo - eps)/(lo - hi) with eps = pos_eps
    const double r = 1.0 / (lo_s - hi_s);
    const double lob = thetab * (eps_s - hi_s) * r * r;
    const double hib = thetab * (lo_s - eps_s) * r * r;
    const double sg = side_s == 0 ? -lam2 : lam2;
    const double qbar = lob + hib, flb = sg * lob, fhb = sg * hib;
    double* Ut = side_s == 0 ? Uab : Ubb;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (s != s_s) continue;
      if (s < NS - 1) {
        Ut[IE + 1 + s] += qbar;
        Flfb[IE + 1 + s] += flb;
        Gc[IE + 1 + s] += fhb;
      } else {
        Ut[0] += qbar; Flfb[0] += flb; Gc[0] += fhb;
#pragma unroll
        for (int k = 0; k < NS - 1; ++k) {
          Ut[IE + 1 + k] -= qbar; Flfb[IE + 1 + k] -= flb; Gc[IE + 1 + k] -= fhb;
        }
      }
    }
  }
  // F_LF = (F_a + F_b + alpha (U_a - U_b)) / 2
  double alb = -0.0, unab = -0.0, unbb = -0.0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const double h = 0.5 * Flfb[v];
    alb = fma(h, Ua[v] - Ub[v], alb);
    Uab[v] = fma(h, al + una, Uab[v]);
    Ubb[v] = fma(h, unb - al, Ubb[v]);
    unab = fma(h, Ua[v], unab);
    unbb = fma(h, Ub[v], unbb);
  }
  // pressure terms of the physical fluxes
  const double hm = 0.5 * Flfb[1 + D], he = 0.5 * Flfb[IE];
  const double pab = fma(he, una, hm), pbb = fma(he, unb, hm);
  unab = fma(he, pa, unab);
  unbb = fma(he, pb, unbb);
  // alpha = max(|u_a| + c_a, |u_b| + c_b)
  double cab = -0.0, cbb = -0.0;
  if (sa >= sbv) {
    unab += una > 0.0 ? alb : (una < 0.0 ? -alb : 0.0);
    cab = alb;
  } else {
    unbb += unb > 0.0 ? alb : (unb < 0.0 ? -alb : 0.0);
    cbb = alb;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) { QB(L::U + v, 0, Uab[v]); QB(L::U + v, 1, Ubb[v]); }
  QB(L::UN + D, 0, unab);
  QB(L::UN + D, 1, unbb);
  QB(L::P, 0, pab);
  QB(L::P, 1, pbb);
  QB(L::C, 0, cab);
  QB(L::C, 1, cbb);
#undef QF
#undef QB
}

// ================================================================ k_face_adj
// Per face of direction D: Gbar = scale (Rbar_right - Rbar_left)/dx (Rbar = 0
// outside the interior), then the reverse of face_one.
template <int DIM, int NS, int D, bool POS = false, int REC = 5>
__device__ __forceinline__ void face_adj(const Params& p, int fi, int fj, int fk,
                                         const double* __restrict__ Q,
                                         const double* __restrict__ Rbar, double scale,
                                         double* __restrict__ Qb, double dt = 0.0,
                                         const double* __restrict__ Fh = nullptr) {
  using L = Lay<DIM, NS>;
  constexpr int NV = L::NV;
  constexpr int IE = DIM + 1;
  constexpr int SO = REC == 7 ? 3 : 2;  // stencil cells left of the left cell
  constexpr int SW = 2 * SO + 2;        // stencil width
  int id[3] = {fi, fj, fk};
  id[D] -= 1;  // left cell
  const long long PC = p.pcells;
  const long long sy = p.np[0], sz = (long long)p.np[0] * p.np[1];
  const long long c0 = (id[2] + p.go[2]) * sz + (id[1] + p.go[1]) * sy + (id[0] + p.go[0]);
  const long long sd = D == 0 ? 1 : (D == 1 ? sy : sz);
  // ---- Gbar from the residual adjoint of the two neighbouring cells
  double Gb[NV];
  {
    const long long C = p.cells;
    const long long ci = ((long long)id[2] * p.n[1] + id[1]) * p.n[0] + id[0];
    const long long cstep = D == 0 ? 1 : (D == 1 ? p.n[0] : (long long)p.n[0] * p.n[1]);
    const bool lin = id[D] >= 0, rin = id[D] + 1 < p.n[D];
    const double w = scale * p.inv_dx[D];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double rr = rin ? Rbar[v * C + ci + cstep] : 0.0;
      const double rl = lin ? Rbar[v * C + ci] : 0.0;
      Gb[v] = (rr - rl) * w;
    }
  }
  const double* q0 = Q + c0;
  double* qb0 = Qb + c0;
#define QF(field, m) ld(q0 + (long long)(field) * PC + (long long)(m) * sd)
#define QB(field, m, val) aadd(qb0 + (long long)(field) * PC + (long long)(m) * sd, (val))
  if (p.convective) {
    // adjoint of the convective flux: Gbar itself, or its share through the
    // positivity-preserving blend inside an RK stage
    double Gc[NV];
    if constexpr (POS) {
      const long long nf0 = p.n[0] + (D == 0), nf1 = p.n[1] + (D == 1), nf2 = p.n[2] + (D == 2);
      const long long f = ((long long)fk * nf1 + fj) * nf0 + fi;
      pos_blend_adj<DIM, NS, D, REC>(p, q0, qb0, PC, sd, dt, Gb, Gc, Fh ? Fh + f : nullptr,
                                     nf0 * nf1 * nf2);
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) Gc[v] = Gb[v];
    }
    // ================= forward recomputation =================
    const double sL = QF(L::SR, 0), sR = QF(L::SR, 1);
    const double iw = rcp_nr(sL + sR);
    const double tL = sL * iw, tR = sR * iw;
    double uL[DIM], uR[DIM], ub[DIM], q2 = -0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      uL[a] = QF(L::UN + a, 0);
      uR[a] = QF(L::UN + a, 1);
      ub[a] = fma(tL, uL[a], tR * uR[a]);
      q2 = fma(ub[a], ub[a], q2);
    }
    const double HL = QF(L::H, 0), HR = QF(L::H, 1), TL = QF(L::T, 0), TR = QF(L::T, 1);
    const double Hb = fma(tL, HL, tR * HR);
    const double Tb = fma(tL, TL, tR * TR);
    double YL[NS], YR[NS], Yb[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      YL[s] = QF(L::Y + s, 0);
      YR[s] = QF(L::Y + s, 1);
      Yb[s] = fma(tL, YL[s], tR * YR[s]);
    }
    const TauPt tp = tau_of(p, Tb);
    double es[NS], cps[NS], Rb = -0.0, cvb = -0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      cps[s] = cp_s(p, s, tp.tc);
      es[s] = h_s(p, s, tp, cps[s]) - p.r[s] * Tb;
      Rb = fma(Yb[s], p.r[s], Rb);
      cvb = fma(Yb[s], cps[s] - p.r[s], cvb);
    }
    const double rRc = rcp_nr(Rb * cvb);
    const double Gam = Rb * Rb * rRc;
    const double hq2 = 0.5 * q2;
    double phi[NS], c2 = -0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      phi[s] = fma(p.r[s], Tb, -Gam * (es[s] - hq2));
      c2 = fma(Yb[s], phi[s], c2);
    }
    c2 = fma(Gam, Hb - q2, c2);
    bool fallback = false;
    double cl = 0.0, cr = 0.0;
    if (!(c2 > 0.0)) {
      fallback = true;
      cl = QF(L::C, 0);
      cr = QF(L::C, 1);
      c2 = 0.5 * (cl * cl + cr * cr);
    }
    const double rsc = rsqrt(c2);
    const double c = c2 * rsc;
    const double ic2 = rsc * rsc;
    const double hic2 = 0.5 * ic2;
    const double iGam = cvb * cvb * rRc;
    const double un = ub[D];
    const double phiN = phi[NS - 1];
    double gm[DIM], dphi[NS > 1 ? NS - 1 : 1], gs[NS > 1 ? NS - 1 : 1];
#pragma unroll
    for (int a = 0; a < DIM; ++a) gm[a] = -Gam * ub[a] * hic2;
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) { dphi[s] = phi[s] - phiN; gs[s] = dphi[s] * hic2; }
    const double gr = phiN * hic2, gE = Gam * hic2;
    // the LLF maxima from the halves |u - c|/2, |u + c|/2, u/2 that primitive
    // recovery stores (exact halves: the same arg-max cells and, halved, the
    // same maxima as from |u - c|, |u + c|, |u|)
    double rho_m[SW], p_m[SW], hun[SW], gUh[SW], unm[SW], cmv[SW];
    double ha_m = 0.0, ha_p = 0.0, ha0 = 0.0;
    int im = 0, ipp = 0, i0 = 0;
#pragma unroll
    for (int m = 0; m < SW; ++m) {
      const int o = m - SO;
      rho_m[m] = QF(L::U, o);
      unm[m] = QF(L::UN + D, o);
      p_m[m] = QF(L::P, o);
      cmv[m] = QF(L::C, o);
      hun[m] = QF(L::HU + D, o);
      const double xm = QF(L::AM + D, o), xp = QF(L::AP + D, o), x0 = fabs(hun[m]);
      if (m == 0 || gt_nn(xm, ha_m)) { ha_m = xm; im = m; }
      if (m == 0 || gt_nn(xp, ha_p)) { ha_p = xp; ipp = m; }
      if (m == 0 || gt_nn(x0, ha0)) { ha0 = x0; i0 = m; }
      double g = gr * rho_m[m];
#pragma unroll
      for (int a = 0; a < DIM; ++a) g = fma(gm[a], QF(L::U + 1 + a, o), g);
      g = fma(gE, QF(L::U + IE, o), g);
#pragma unroll
      for (int s = 0; s < NS - 1; ++s) g = fma(gs[s], QF(L::U + IE + 1 + s, o), g);
      gUh[m] = g;
    }
    const double e12c[4] = {p.wenoe[0], p.wenoe[1], p.wenoe[2], p.wenoe[3]};
    // the reconstruction's coefficients as register operands (Params::dev)
    double K[28];
#pragma unroll
    for (int j = 0; j < 28; ++j) K[j] = __ldcg(p.dev->kface + j);
    const double* Ec = p.dev->wenoe;
    const double chc = c * hic2;
    // the pressure terms p_m (l[m_n]/2 + (u_m/2) l[E]) of the dense rows, as in
    // conv_flux: one product pV per cell, -+ dl p_m for u -+ c, -2 pV for the
    // entropy row; nUv (the normal momentum relative to the face velocity) is
    // shared by u -+ c
    const double lE = Gam * hic2, hl0 = -0.5 * Gam * un * hic2, dl = 0.5 * chc;
    double nUv[SW], base[SW], pV[SW];
#pragma unroll
    for (int m = 0; m < SW; ++m) {
      nUv[m] = fma(-un, rho_m[m], QF(L::U + 1 + D, m - SO));
      base[m] = fma(hun[m], lE, hl0);
      pV[m] = p_m[m] * base[m];
    }
    double wp[SW], wm[SW];
    // ================= reverse =================
    // back-projection of the dense columns: adjoints of the reconstructed
    // fields depend on Gbar and the face state only
    double Sb = Gc[0] + Hb * Gc[IE];
#pragma unroll
    for (int a = 0; a < DIM; ++a) Sb = fma(ub[a], Gc[1 + a], Sb);
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) Sb = fma(Yb[s], Gc[IE + 1 + s], Sb);
    const double Dlb = c * Gc[1 + D] + un * c * Gc[IE];
    double ubb[DIM], Ybb[NS];
#pragma unroll
    for (int a = 0; a < DIM; ++a) ubb[a] = -0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) Ybb[s] = -0.0;
    double cb = -0.0, Hbb = -0.0, unb = -0.0, c2b = -0.0, iGamb = -0.0;
    const double Fmb = Sb - Dlb, Fpb = Sb + Dlb, Feb = Sb - c2 * iGam * Gc[IE];
    double Fm = 0.0, Fp = 0.0, Fe = 0.0;
    // per-field reverse; stencil adjoints accumulated here
    double rhob[SW], pb[SW], hunb[SW], gUhb[SW], mnb[SW];
#pragma unroll
    for (int m = 0; m < SW; ++m) { rhob[m] = -0.0; pb[m] = -0.0; hunb[m] = -0.0; gUhb[m] = -0.0; mnb[m] = -0.0; }
    double hamb = -0.0, hapb = -0.0, ha0b = -0.0, chcb = -0.0, Gamb = -0.0, hic2b = -0.0, ic2b = -0.0;
    double pVb[SW], nUb[SW], dlb = -0.0;
#pragma unroll
    for (int m = 0; m < SW; ++m) { pVb[m] = -0.0; nUb[m] = -0.0; }
#pragma unroll
    for (int fld = 0; fld < 3; ++fld) {
      const double ha = fld == 0 ? ha_m : (fld == 1 ? ha_p : ha0);
      const double Fb = fld == 0 ? Fmb : (fld == 1 ? Fpb : Feb);
      const double schc = fld == 0 ? -chc : chc;
      double LUv[SW];
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        double LU, pq;
        if (fld == 2) {
          LU = fma(-2.0, gUh[m], rho_m[m]);
          pq = -2.0 * pV[m];
        } else {
          LU = fma(schc, nUv[m], gUh[m]);
          pq = fma(fld == 0 ? -dl : dl, p_m[m], pV[m]);
        }
        LUv[m] = LU;
        wp[m] = fma(hun[m] + ha, LU, pq);
        wm[m] = fma(hun[m] - ha, LU, pq);
      }
      double wpb[SW], wmb[SW];
#pragma unroll
      for (int m = 0; m < SW; ++m) { wpb[m] = -0.0; wmb[m] = -0.0; }
      const double F = rec_pair_fwd_adj<REC>(wp, wm, e12c, K, Ec, Fb, wpb, wmb);
      if (fld == 0) Fm = F; else if (fld == 1) Fp = F; else Fe = F;
      double hab = -0.0;
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        // w+- = (hun +- ha) LU + pq: with s = wb+ + wb-, d = wb+ - wb-,
        // LUb = hun s + ha d, hunb += s LU, hab += d LU, and pq takes s
        const double sb = wpb[m] + wmb[m], db = wpb[m] - wmb[m];
        const double LUb = fma(hun[m], sb, ha * db);
        hunb[m] = fma(sb, LUv[m], hunb[m]);
        hab = fma(db, LUv[m], hab);
        if (fld == 2) {
          pVb[m] = fma(-2.0, sb, pVb[m]);
          rhob[m] += LUb;
          gUhb[m] = fma(-2.0, LUb, gUhb[m]);
        } else {
          const double sdl = fld == 0 ? -dl : dl;
          pVb[m] += sb;
          pb[m] = fma(sdl, sb, pb[m]);
          dlb = fma(fld == 0 ? -p_m[m] : p_m[m], sb, dlb);
          gUhb[m] += LUb;
          chcb = fma(fld == 0 ? -LUb : LUb, nUv[m], chcb);
          nUb[m] = fma(schc, LUb, nUb[m]);
        }
      }
      if (fld == 2) ha0b += hab;
      else if (fld == 0) hamb += hab;
      else hapb += hab;
    }
    // reverse of the shared terms: nU = m_n - u_n rho, pV = p base with
    // base = hun lE + hl0; lE = Gam hic2, hl0 = -Gam un hic2 / 2, dl = chc / 2
    {
      double lEb = -0.0, hl0b = -0.0;
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        mnb[m] += nUb[m];
        unb = fma(-nUb[m], rho_m[m], unb);
        rhob[m] = fma(-nUb[m], un, rhob[m]);
        pb[m] = fma(pVb[m], base[m], pb[m]);
        const double bb = pVb[m] * p_m[m];
        hunb[m] = fma(bb, lE, hunb[m]);
        lEb = fma(bb, hun[m], lEb);
        hl0b += bb;
      }
      Gamb = fma(lEb, hic2, fma(hl0b, -0.5 * un * hic2, Gamb));
      hic2b = fma(lEb, Gam, fma(hl0b, -0.5 * Gam * un, hic2b));
      unb = fma(hl0b, -0.5 * Gam * hic2, unb);
      chcb = fma(0.5, dlb, chcb);
    }
    // the back-projection terms that involve the reconstructed dense fields
    {
      const double S = Fm + Fp + Fe, Dl = Fp - Fm;
#pragma unroll
      for (int a = 0; a < DIM; ++a) ubb[a] += S * Gc[1 + a];
#pragma unroll
      for (int s = 0; s < NS - 1; ++s) Ybb[s] += S * Gc[IE + 1 + s];
      cb += Dl * Gc[1 + D] + un * Dl * Gc[IE];
      Hbb += S * Gc[IE];
      unb += c * Dl * Gc[IE];
      c2b -= iGam * Fe * Gc[IE];
      iGamb -= c2 * Fe * Gc[IE];
    }
    // tangential momenta and species (eigenvalue u, no pressure term)
    double hp0b[SW], hm0b[SW];
#pragma unroll
    for (int m = 0; m < SW; ++m) { hp0b[m] = -0.0; hm0b[m] = -0.0; }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (a == D) continue;
      const double Fb = Gc[1 + a] + ub[a] * Gc[IE];
      double LUv[SW];
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        LUv[m] = fma(-ub[a], rho_m[m], QF(L::U + 1 + a, m - SO));
        wp[m] = (hun[m] + ha0) * LUv[m];
        wm[m] = (hun[m] - ha0) * LUv[m];
      }
      double wpb[SW], wmb[SW];
#pragma unroll
      for (int m = 0; m < SW; ++m) { wpb[m] = -0.0; wmb[m] = -0.0; }
      const double Fk = rec_pair_fwd_adj<REC>(wp, wm, e12c, K, Ec, Fb, wpb, wmb);
      ubb[a] += Fk * Gc[IE];
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        const double LUb = wpb[m] * (hun[m] + ha0) + wmb[m] * (hun[m] - ha0);
        hp0b[m] += wpb[m] * LUv[m];
        hm0b[m] += wmb[m] * LUv[m];
        QB(L::U + 1 + a, m - SO, LUb);
        ubb[a] -= LUb * rho_m[m];
        rhob[m] -= LUb * ub[a];
      }
    }
    double dphib[NS > 1 ? NS - 1 : 1];
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
      const double Fb = Gc[IE + 1 + s] - dphi[s] * iGam * Gc[IE];
      double LUv[SW];
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        LUv[m] = fma(-Yb[s], rho_m[m], QF(L::U + IE + 1 + s, m - SO));
        wp[m] = (hun[m] + ha0) * LUv[m];
        wm[m] = (hun[m] - ha0) * LUv[m];
      }
      double wpb[SW], wmb[SW];
#pragma unroll
      for (int m = 0; m < SW; ++m) { wpb[m] = -0.0; wmb[m] = -0.0; }
      const double Fk = rec_pair_fwd_adj<REC>(wp, wm, e12c, K, Ec, Fb, wpb, wmb);
      dphib[s] = -iGam * Fk * Gc[IE];
      iGamb -= dphi[s] * Fk * Gc[IE];
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        const double LUb = wpb[m] * (hun[m] + ha0) + wmb[m] * (hun[m] - ha0);
        hp0b[m] += wpb[m] * LUv[m];
        hm0b[m] += wmb[m] * LUv[m];
        QB(L::U + IE + 1 + s, m - SO, LUb);
        Ybb[s] -= LUb * rho_m[m];
        rhob[m] -= LUb * Yb[s];
      }
    }
#pragma unroll
    for (int m = 0; m < SW; ++m) {
      hunb[m] += hp0b[m] + hm0b[m];
      ha0b += hp0b[m] - hm0b[m];
    }
    // stencil preparation
    cb += chcb * hic2;
    hic2b += chcb * c;
    double grb = -0.0, gEb = -0.0, gmb[DIM], gsb[NS > 1 ? NS - 1 : 1];
#pragma unroll
    for (int a = 0; a < DIM; ++a) gmb[a] = -0.0;
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) gsb[s] = -0.0;
#pragma unroll
    for (int m = 0; m < SW; ++m) {
      const int o = m - SO;
      const double g = gUhb[m];
      grb += g * rho_m[m];
      rhob[m] += g * gr;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        gmb[a] += g * QF(L::U + 1 + a, o);
        double v = g * gm[a];
        if (a == D) v += mnb[m];
        QB(L::U + 1 + a, o, v);
      }
      gEb += g * QF(L::U + IE, o);
      QB(L::U + IE, o, g * gE);
#pragma unroll
      for (int s = 0; s < NS - 1; ++s) {
        gsb[s] += g * QF(L::U + IE + 1 + s, o);
        QB(L::U + IE + 1 + s, o, g * gs[s]);
      }
      QB(L::U, o, rhob[m]);
      QB(L::P, o, pb[m]);
      double unmb = 0.5 * hunb[m];
      double cmb = -0.0;
      if (m == im) { const double sg = unm[m] - cmv[m] > 0.0 ? 1.0 : (unm[m] - cmv[m] < 0.0 ? -1.0 : 0.0); unmb += 0.5 * hamb * sg; cmb -= 0.5 * hamb * sg; }
      if (m == ipp) { const double sg = unm[m] + cmv[m] > 0.0 ? 1.0 : (unm[m] + cmv[m] < 0.0 ? -1.0 : 0.0); unmb += 0.5 * hapb * sg; cmb += 0.5 * hapb * sg; }
      if (m == i0) { const double sg = unm[m] > 0.0 ? 1.0 : (unm[m] < 0.0 ? -1.0 : 0.0); unmb += 0.5 * ha0b * sg; }
      QB(L::UN + D, o, unmb);
      QB(L::C, o, cmb);
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      Gamb -= gmb[a] * ub[a] * hic2;
      ubb[a] -= gmb[a] * Gam * hic2;
      hic2b -= gmb[a] * Gam * ub[a];
    }
    double phib[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) phib[s] = -0.0;
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
      const double db = dphib[s] + gsb[s] * hic2;
      hic2b += gsb[s] * dphi[s];
      phib[s] += db;
      phib[NS - 1] -= db;
    }
    phib[NS - 1] += grb * hic2;
    hic2b += grb * phiN + gEb * Gam;
    Gamb += gEb * hic2;
    // Roe state
    ic2b += 0.5 * hic2b;
    c2b -= ic2b * ic2 * ic2;
    const double iRb = cvb * rRc, icv = Rb * rRc;  // 1/R, 1/c_v
    double cvbb = iGamb * iRb, Rbb = -iGamb * iGam * iRb;
    c2b += cb * 0.5 * rsc;
    ubb[D] += unb;
    double Tbb = -0.0, q2b = -0.0;
    if (fallback) {
      QB(L::C, 0, c2b * cl);
      QB(L::C, 1, c2b * cr);
    } else {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        Ybb[s] += c2b * phi[s];
        phib[s] += c2b * Yb[s];
      }
      Gamb += c2b * (Hb - q2);
      Hbb += c2b * Gam;
      q2b -= c2b * Gam;
    }
    double hq2b = -0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Tbb += phib[s] * p.r[s];
      Gamb -= phib[s] * (es[s] - hq2);
      hq2b += phib[s] * Gam;
      const double esb = -phib[s] * Gam;
      Tbb += esb * (cps[s] - p.r[s]);
    }
    q2b += 0.5 * hq2b;
    Rbb += Gamb * icv;
    cvbb -= Gamb * Gam * icv;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Ybb[s] += Rbb * p.r[s] + cvbb * (cps[s] - p.r[s]);
      Tbb += cvbb * Yb[s] * dcp_s(p, s, Tb);
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) ubb[a] += 2.0 * ub[a] * q2b;
    double tLb = -0.0, tRb = -0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      QB(L::UN + a, 0, tL * ubb[a]);
      QB(L::UN + a, 1, tR * ubb[a]);
      tLb += ubb[a] * uL[a];
      tRb += ubb[a] * uR[a];
    }
    QB(L::H, 0, tL * Hbb);
    QB(L::H, 1, tR * Hbb);
    tLb += Hbb * HL;
    tRb += Hbb * HR;
    QB(L::T, 0, tL * Tbb);
    QB(L::T, 1, tR * Tbb);
    tLb += Tbb * TL;
    tRb += Tbb * TR;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      QB(L::Y + s, 0, tL * Ybb[s]);
      QB(L::Y + s, 1, tR * Ybb[s]);
      tLb += Ybb[s] * YL[s];
      tRb += Ybb[s] * YR[s];
    }
    const double iwb = tLb * sL + tRb * sR;
    QB(L::SR, 0, tLb * iw - iwb * iw * iw);
    QB(L::SR, 1, tRb * iw - iwb * iw * iw);
  }

  if (p.viscous) {
    const double wi = 1.0 / 16.0;
    const double wd = p.inv_dx[D] * (1.0 / 12.0);
#define FI(field) ((9.0 * (QF(field, 0) + QF(field, 1)) - (QF(field, -1) + QF(field, 2))) * wi)
#define FD(field) ((15.0 * (QF(field, 1) - QF(field, 0)) - (QF(field, 2) - QF(field, -1))) * wd)
// adjoints of FI / FD scattered to cells -1..2 (the stencils are symmetric
// up to sign, so two products serve the four cells)
#define BI(field, val) { const double a_ = wi * (val), b_ = 9.0 * a_; \
    QB(field, -1, -a_); QB(field, 0, b_); QB(field, 1, b_); QB(field, 2, -a_); }
#define BD(field, val) { const double a_ = wd * (val), b_ = 15.0 * a_; \
    QB(field, -1, a_); QB(field, 0, -b_); QB(field, 1, b_); QB(field, 2, -a_); }
    const double mu = FI(L::MU), ka = FI(L::KA), Df = FI(L::DF), rf = FI(L::U), Tf = FI(L::T);
    double uf[DIM], gr[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      uf[a] = FI(L::UN + a);
#pragma unroll
      for (int b = 0; b < DIM; ++b) gr[a][b] = (b == D) ? FD(L::UN + a) : FI(L::GU + a * DIM + b);
    }
    double div = -0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) div += gr[a][a];
    double tau[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      tau[a] = mu * (gr[D][a] + gr[a][D]);
      if (a == D) tau[a] = fma(-2.0 / 3.0 * mu, div, tau[a]);
    }
    // species diffusivities at the face: the common D, or each species' D_sm
    // (mixture-averaged model). With the common D the mixture correction
    // D Y_s sum_t dY_t vanishes identically (sum_t Y_t = 1), as in the
    // forward face, and is neither formed nor reversed.
    const bool dsm = p.diffusion == 1;
    double dY[NS], Yf[NS], Dsf[NS], corr = -0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      // the last species' flux enters neither a species row nor, in the
      // difference form below, the heat flux: its gradient is needed only
      // for the mixture correction
      dY[s] = (dsm || s < NS - 1) ? FD(L::Y + s) : -0.0;
      Dsf[s] = dsm ? FI(L::DS + s) : Df;
      if (dsm) {
        Yf[s] = FI(L::Y + s);
        corr = fma(Dsf[s], dY[s], corr);
      } else {
        Yf[s] = -0.0;
      }
    }
    const TauPt tp = tau_of(p, Tf);
    const double dT = FD(L::T);
    // reverse: Gout[IE] -= ka dT + work - qd; Gout[1+a] -= tau_a; Gout[IE+1+s] += J_s.
    // As in the forward face, qd = sum_{s<N} (h_s - h_N) J_s (sum_s J_s = 0),
    // so the last species' J has no adjoint.
    const double workb = -Gb[IE], kab = -Gb[IE] * dT, dTb = -Gb[IE] * ka, qdb = Gb[IE];
    double Tfb = -0.0, rfb = -0.0, corrb = -0.0, mub = -0.0, divb = -0.0;
    double dYb[NS], Yfb[NS], Dsfb[NS];
    Dsfb[NS - 1] = -0.0; dYb[NS - 1] = -0.0; Yfb[NS - 1] = -0.0;
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) {
      const double J = dsm ? -rf * fma(Dsf[s], dY[s], -Yf[s] * corr) : -rf * (Df * dY[s]);
      const double cpd = cpd_s_dev(p, s, tp.tc);
      const double hd = hd_s_dev(p, s, tp);
      double Jb = fma(qdb, hd, Gb[IE + 1 + s]);
      Tfb += qdb * J * cpd;
      rfb -= Jb * (dsm ? Dsf[s] * dY[s] - Yf[s] * corr : Df * dY[s]);
      Dsfb[s] = -Jb * rf * dY[s];
      dYb[s] = -Jb * rf * Dsf[s];
      if (dsm) {
        Yfb[s] = Jb * rf * corr;
        corrb += Jb * rf * Yf[s];
      } else {
        Yfb[s] = -0.0;
      }
    }
    // corr = sum_s D_s dY_s (mixture-averaged model only)
    if (dsm) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        Dsfb[s] = fma(corrb, dY[s], Dsfb[s]);
        dYb[s] = fma(corrb, Dsf[s], dYb[s]);
      }
    }
    double Dfb = -0.0;
    if (p.diffusion != 1) {
#pragma unroll
      for (int s = 0; s < NS; ++s) Dfb += Dsfb[s];
    }
    double grb[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) grb[a][b] = -0.0;
    double ufb[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const double taub = workb * uf[a] - Gb[1 + a];
      ufb[a] = workb * tau[a];
      mub += taub * (gr[D][a] + gr[a][D]);
      grb[D][a] += taub * mu;
      grb[a][D] += taub * mu;
      if (a == D) {
        mub -= (2.0 / 3.0) * taub * div;
        divb -= (2.0 / 3.0) * mu * taub;
      }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) grb[a][a] += divb;
    BI(L::MU, mub);
    BI(L::KA, kab);
    if (p.diffusion == 1) {
#pragma unroll
      for (int s = 0; s < NS; ++s) BI(L::DS + s, Dsfb[s]);
    } else {
      BI(L::DF, Dfb);
    }
    BI(L::U, rfb);
    BI(L::T, Tfb);
    BD(L::T, dTb);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      BI(L::UN + a, ufb[a]);
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        if (b == D) { BD(L::UN + a, grb[a][b]); }
        else { BI(L::GU + a * DIM + b, grb[a][b]); }
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      if (dsm || s < NS - 1) BD(L::Y + s, dYb[s]);
      if (dsm) BI(L::Y + s, Yfb[s]);
    }
#undef FI
#undef FD
#undef BI
#undef BD
  }
#undef QF
#undef QB
}

template <int DIM, int NS, int D, int REC = 5>
__global__ void __launch_bounds__(128)
k_face_adj(const __grid_constant__ Params p, const double* __restrict__ Q,
           const double* __restrict__ Rbar, double scale, double* __restrict__ Qb) {
  const int nf0 = p.n[0] + (D == 0), nf1 = p.n[1] + (D == 1), nf2 = p.n[2] + (D == 2);
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= (long long)nf0 * nf1 * nf2) return;
  face_adj<DIM, NS, D, false, REC>(p, (int)(f % nf0), (int)((f / nf0) % nf1),
                                   (int)(f / ((long long)nf0 * nf1)), Q, Rbar, scale, Qb);
}

// the same inside an RK stage of a handle with the positivity-preserving
// blend: dtp holds the stage's time step
template <int DIM, int NS, int D, int REC = 5>
__global__ void __launch_bounds__(128)
k_face_adj_pos(const __grid_constant__ Params p, const double* __restrict__ Q,
               const double* __restrict__ Rbar, double scale, double* __restrict__ Qb,
               const double* __restrict__ dtp) {
  const int nf0 = p.n[0] + (D == 0), nf1 = p.n[1] + (D == 1), nf2 = p.n[2] + (D == 2);
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= (long long)nf0 * nf1 * nf2) return;
  face_adj<DIM, NS, D, true, REC>(p, (int)(f % nf0), (int)((f / nf0) % nf1),
                                  (int)(f / ((long long)nf0 * nf1)), Q, Rbar, scale, Qb, *dtp);
}

// the same reading the unblended convective fluxes of the forward step from
// the flux tape Fh ([n_v][faces] of this direction and stage)
template <int DIM, int NS, int D, int REC = 5>
__global__ void __launch_bounds__(128)
k_face_adj_pos_tape(const __grid_constant__ Params p, const double* __restrict__ Q,
                    const double* __restrict__ Rbar, double scale, double* __restrict__ Qb,
                    const double* __restrict__ dtp, const double* __restrict__ Fh) {
  const int nf0 = p.n[0] + (D == 0), nf1 = p.n[1] + (D == 1), nf2 = p.n[2] + (D == 2);
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= (long long)nf0 * nf1 * nf2) return;
  face_adj<DIM, NS, D, true, REC>(p, (int)(f % nf0), (int)((f / nf0) % nf1),
                                  (int)(f / ((long long)nf0 * nf1)), Q, Rbar, scale, Qb, *dtp, Fh);
}

// ================================================================ k_prim_adj
// Per padded cell t: Qbar (all fields of this cell) -> Ubar of its interior
// source cell (with the symmetric-mirror sign flips).
template <int DIM, int NS>
__device__ __forceinline__ void prim_adj_cell(const Params& p, long long t,
                                              const double* __restrict__ Q,
                                              const double* __restrict__ Qb,
                                              double* __restrict__ Ubar) {
  using L = Lay<DIM, NS>;
  constexpr int NV = L::NV;
  const long long PC = p.pcells;
  const int ip = (int)(t % p.np[0]);
  const int jp = (int)((t / p.np[0]) % p.np[1]);
  const int kp = (int)(t / ((long long)p.np[0] * p.np[1]));
  const int i = ip - p.go[0], j = jp - p.go[1], k = kp - p.go[2];
  bool f0 = false, f1 = false, f2 = false;
  const int si = map_axis(i, p.n[0], p.bc[0][0], p.bc[0][1], &f0);
  const int sj = DIM > 1 ? map_axis(j, p.n[1], p.bc[1][0], p.bc[1][1], &f1) : 0;
  const int sk = DIM > 2 ? map_axis(k, p.n[2], p.bc[2][0], p.bc[2][1], &f2) : 0;
  const long long src = ((long long)sk * p.n[1] + sj) * p.n[0] + si;
  const double* q = Q + t;
  const double* qb = Qb + t;
  // forward values of this cell
  double u[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = q[(L::U + v) * PC];
  const double rho = u[0], E = u[DIM + 1];
  double vel[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) vel[a] = q[(L::UN + a) * PC];
  double Y[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) Y[s] = q[(L::Y + s) * PC];
  const double T = q[L::T * PC], pr = q[L::P * PC], c = q[L::C * PC];
  const TauPt tp = tau_of(p, T);
  double Rm = -0.0, cpm = -0.0, dcpm = -0.0, es[NS], cps[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    cps[s] = cp_s(p, s, tp.tc);
    es[s] = h_s(p, s, tp, cps[s]) - p.r[s] * T;
    Rm = fma(Y[s], p.r[s], Rm);
    cpm = fma(Y[s], cps[s], cpm);
    dcpm = fma(Y[s], dcp_s(p, s, T), dcpm);
  }
  const double cvm = cpm - Rm, RT = Rm * T;
  // reciprocals: 1/rho and 1/c_p from one division, 1/c_v from another
  const double irc = rcp_nr(rho * cpm);
  const double irho = cpm * irc, icpm = rho * irc;
  const double icvm = rcp_nr(cvm);
  // adjoint accumulators
  double ub[NV], Yb[NS], velb[DIM];
#pragma unroll
  for (int v = 0; v < NV; ++v) ub[v] = qb[(L::U + v) * PC];
#pragma unroll
  for (int s = 0; s < NS; ++s) Yb[s] = qb[(L::Y + s) * PC];
#pragma unroll
  for (int a = 0; a < DIM; ++a) velb[a] = qb[(L::UN + a) * PC];
  double Tb = qb[L::T * PC], prb = qb[L::P * PC], cb = qb[L::C * PC];
  double rhob = -0.0, Eb = -0.0, irhob = -0.0, cpmb = -0.0, Rmb = -0.0;
  if (p.viscous) {
    const double mub = qb[L::MU * PC], kab = qb[L::KA * PC], Db = qb[L::DF * PC];
    // D = ka / (Le rho cp)
    const double ka = q[L::KA * PC], Dd = q[L::DF * PC];
    double kabar = fma(Db * p.inv_lewis, irc, kab);
    rhob -= Db * Dd * irho;
    cpmb -= Db * Dd * icpm;
    // Wilke mixtures (Eq. 22), recomputed in k_prim's expanded form: with
    // r_s = sqrt(mu_s), d_s = S0_s + 2 r_s m1_s + r_s^2 m2_s, where
    // S0_s = X_s + sum_{t!=s} X_t A_st, m1_s = sum_{t!=s} X_t r_t^-1 A_st B_st
    // and m2_s = sum_{t!=s} X_t r_t^-2 A_st B_st^2 (Phi_ss = 1); the same with
    // sqrt(kappa_s) for kappa. The coefficients come from the parameters'
    // device copy (register operands), the exponentials from exp_k.
    const Params& pd = *p.dev;
    double KL[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) KL[j] = rd(pd.klog[j]);
    const double lnT = log_k(T, KL);
    double KX[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) KX[j] = rd(pd.kexp[j]);
    double smu[NS], ska[NS], ismu[NS], iska[NS], X[NS], xs = -0.0, dlm[NS], dlk[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double* fm = pd.lnmu[s];
      const double* fk = pd.lnka[s];
      const double lm = fma(fma(fma(rd(fm[3]), lnT, rd(fm[2])), lnT, rd(fm[1])), lnT, rd(fm[0]));
      const double lk = fma(fma(fma(rd(fk[3]), lnT, rd(fk[2])), lnT, rd(fk[1])), lnT, rd(fk[0]));
      dlm[s] = fma(fma(3.0 * rd(fm[3]), lnT, 2.0 * rd(fm[2])), lnT, rd(fm[1]));
      dlk[s] = fma(fma(3.0 * rd(fk[3]), lnT, 2.0 * rd(fk[2])), lnT, rd(fk[1]));
      smu[s] = exp_k(0.5 * lm, KX);
      ska[s] = exp_k(0.5 * lk, KX);
      X[s] = Y[s] * rd(pd.invW[s]);
      xs += X[s];
    }
    // the 2N reciprocals from one division (running products, as in k_prim)
    {
      double pre[2 * NS];
      pre[0] = smu[0];
#pragma unroll
      for (int k = 1; k < 2 * NS; ++k) pre[k] = pre[k - 1] * (k < NS ? smu[k] : ska[k - NS]);
      double inv = rcp_nr(pre[2 * NS - 1]);
#pragma unroll
      for (int k = 2 * NS - 1; k > 0; --k) {
        const double v = k < NS ? smu[k] : ska[k - NS];
        const double r = inv * pre[k - 1];
        if (k < NS) ismu[k] = r; else iska[k - NS] = r;
        inv *= v;
      }
      ismu[0] = inv;
    }
    const double ixs = rcp_nr(xs);
    double xm1[NS], xm2[NS], xk1[NS], xk2[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      X[s] *= ixs;
      xm1[s] = X[s] * ismu[s];
      xm2[s] = xm1[s] * ismu[s];
      xk1[s] = X[s] * iska[s];
      xk2[s] = xk1[s] * iska[s];
    }
    const double mtot = mub * p.fmu, ktot = kabar * p.fka;
    double Xb[NS], smub[NS], skab[NS], xm1b[NS], xm2b[NS], xk1b[NS], xk2b[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Xb[s] = -0.0; smub[s] = -0.0; skab[s] = -0.0;
      xm1b[s] = -0.0; xm2b[s] = -0.0; xk1b[s] = -0.0; xk2b[s] = -0.0;
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double s0 = X[s], am1 = -0.0, am2 = -0.0, ak1 = -0.0, ak2 = -0.0;
#pragma unroll
      for (int tt = 0; tt < NS; ++tt) {
        if (tt == s) continue;
        const double wab = rd(pd.wAB[s][tt]), wabb = rd(pd.wABB[s][tt]);
        s0 = fma(X[tt], rd(pd.wA[s][tt]), s0);
        am1 = fma(xm1[tt], wab, am1);
        am2 = fma(xm2[tt], wabb, am2);
        ak1 = fma(xk1[tt], wab, ak1);
        ak2 = fma(xk2[tt], wabb, ak2);
      }
      const double rs = smu[s], ks = ska[s];
      const double sm2 = rs * rs, sk2 = ks * ks;
      const double dm = fma(sm2, am2, fma(rs + rs, am1, s0));
      const double dk = fma(sk2, ak2, fma(ks + ks, ak1, s0));
      const double rdd = rcp_nr(dm * dk);
      const double idm = rdd * dk, idk = rdd * dm;
      // the mixture terms X_s a_s / d_s: their adjoints through X_s, r_s and d_s
      const double tm = X[s] * sm2 * idm, tk = X[s] * sk2 * idk;
      Xb[s] += fma(mtot * sm2, idm, ktot * sk2 * idk);
      const double dmb = -mtot * tm * idm, dkb = -ktot * tk * idk;
      // d term / d r_s = 2 X_s r_s / d_s, d d_s / d r_s = 2 (m1_s + r_s m2_s)
      smub[s] += 2.0 * fma(mtot * X[s], rs * idm, dmb * fma(rs, am2, am1));
      skab[s] += 2.0 * fma(ktot * X[s], ks * idk, dkb * fma(ks, ak2, ak1));
      const double s0b = dmb + dkb;
      const double m1b = 2.0 * dmb * rs, m2b = dmb * sm2;
      const double k1b = 2.0 * dkb * ks, k2b = dkb * sk2;
      Xb[s] += s0b;
#pragma unroll
      for (int tt = 0; tt < NS; ++tt) {
        if (tt == s) continue;
        const double wab = rd(pd.wAB[s][tt]), wabb = rd(pd.wABB[s][tt]);
        Xb[tt] = fma(s0b, rd(pd.wA[s][tt]), Xb[tt]);
        xm1b[tt] = fma(m1b, wab, xm1b[tt]);
        xm2b[tt] = fma(m2b, wabb, xm2b[tt]);
        xk1b[tt] = fma(k1b, wab, xk1b[tt]);
        xk2b[tt] = fma(k2b, wabb, xk2b[tt]);
      }
    }
    // xm1 = X r^-1, xm2 = xm1 r^-1 (and with sqrt(kappa)): adjoints of X and r^-1
    double ismub[NS], iskab[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const double x1 = fma(xm2b[t], ismu[t], xm1b[t]);
      const double y1 = fma(xk2b[t], iska[t], xk1b[t]);
      ismub[t] = fma(xm2b[t], xm1[t], x1 * X[t]);
      iskab[t] = fma(xk2b[t], xk1[t], y1 * X[t]);
      Xb[t] = fma(x1, ismu[t], fma(y1, iska[t], Xb[t]));
    }
    double lnTb = -0.0, xdot = -0.0;
    if (p.diffusion == 1) {
      // mixture-averaged D_sm (Eq. 25-26), recomputed as in k_prim, then reversed:
      // X~ = (max(X, 0) + 1e-12)/sum, W~ = sum X~ W, e_st = exp(-l_st(ln T)) = p D_st^-1 (SI),
      // den_s = sum_{t!=s} X~_t e_st, num_s = sum_{t!=s} X~_t W_t,
      // D_s = num_s / (W~ den_s p* fdsm)
      constexpr int NP = NS * (NS - 1) / 2;
      double m[NS], Xt[NS], XW[NS], den[NS], xts = -0.0, Wt = -0.0;
      double e[NP > 0 ? NP : 1], dl[NP > 0 ? NP : 1];
#pragma unroll
      for (int s = 0; s < NS; ++s) { m[s] = fmax(X[s], 0.0) + 1e-12; xts += m[s]; den[s] = -0.0; }
      const double ixts = rcp_nr(xts);
#pragma unroll
      for (int s = 0; s < NS; ++s) { Xt[s] = m[s] * ixts; XW[s] = Xt[s] * p.Wm[s]; Wt += XW[s]; }
      {
        int k = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int tt = s + 1; tt < NS; ++tt, ++k) {
            const double* bc = p.dbin[s][tt];
            const double l = fma(fma(fma(bc[3], lnT, bc[2]), lnT, bc[1]), lnT, bc[0]);
            dl[k] = fma(fma(3.0 * bc[3], lnT, 2.0 * bc[2]), lnT, bc[1]);
            e[k] = exp_k(-l, KX);
            den[s] = fma(Xt[tt], e[k], den[s]);
            den[tt] = fma(Xt[s], e[k], den[tt]);
          }
      }
      const double sc = rcp_nr(Wt * pr * p.fdsm);
      double numb[NS], denb[NS], nbs = -0.0, scb = -0.0;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        double num = -0.0;
#pragma unroll
        for (int tt = 0; tt < NS; ++tt)
          if (tt != s) num += XW[tt];
        const double iden = rcp_nr(den[s]);
        const double Dsb = qb[(L::DS + s) * PC];
        const double Ds = num * sc * iden;
        numb[s] = Dsb * sc * iden;
        scb = fma(Dsb, num * iden, scb);
        denb[s] = -Dsb * Ds * iden;
        nbs += numb[s];
      }
      const double Wtb = -scb * sc / Wt;
      prb -= scb * sc / pr;
      double Xtb[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) Xtb[s] = (nbs - numb[s] + Wtb) * p.Wm[s];
      {
        int k = 0;
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int tt = s + 1; tt < NS; ++tt, ++k) {
            Xtb[tt] = fma(denb[s], e[k], Xtb[tt]);
            Xtb[s] = fma(denb[tt], e[k], Xtb[s]);
            const double eb = fma(denb[s], Xt[tt], denb[tt] * Xt[s]);
            lnTb -= eb * e[k] * dl[k];
          }
      }
      double xtd = -0.0;
#pragma unroll
      for (int s = 0; s < NS; ++s) xtd = fma(Xtb[s], Xt[s], xtd);
#pragma unroll
      for (int s = 0; s < NS; ++s)
        if (X[s] > 0.0) Xb[s] += (Xtb[s] - xtd) * ixts;
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      smub[s] -= ismub[s] * ismu[s] * ismu[s];
      skab[s] -= iskab[s] * iska[s] * iska[s];
      lnTb += 0.5 * (smub[s] * smu[s] * dlm[s] + skab[s] * ska[s] * dlk[s]);
      xdot += Xb[s] * X[s];
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) Yb[s] += (Xb[s] - xdot) * ixs * p.invW[s];
    Tb += lnTb / T;
  }
  // H = (E + p) / rho; sqrt(rho)
  const double Hb = qb[L::H * PC];
  Eb += Hb * irho;
  prb += Hb * irho;
  irhob += Hb * (E + pr);
  rhob += qb[L::SR * PC] * 0.5 * q[L::SR * PC] * irho;   // d sqrt(rho) = 1/(2 sqrt(rho))
  // c = sqrt(cp R T / cv)
  const double c2b = cb * 0.5 / c;
  cpmb += c2b * (-RT * Rm * (icvm * icvm));
  Rmb += c2b * cpm * RT * (icvm * icvm);
  double RTb = c2b * cpm * icvm;
  // p = rho R T
  rhob += prb * RT;
  RTb += prb * rho;
  Rmb += RTb * T;
  Tb += RTb * Rm;
  // mixture cp and R
  Tb += cpmb * dcpm;
#pragma unroll
  for (int s = 0; s < NS; ++s) Yb[s] += cpmb * cps[s] + Rmb * p.r[s];
  // Newton temperature through the implicit-function theorem
  const double eb = Tb * icvm;
#pragma unroll
  for (int s = 0; s < NS; ++s) Yb[s] -= eb * es[s];
  // Y_N = 1 - sum_{s<N} Y_s
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) Yb[s] -= Yb[NS - 1];
  // e = E/rho - |u|^2/2
  Eb += eb * irho;
  irhob += eb * E;
#pragma unroll
  for (int a = 0; a < DIM; ++a) velb[a] -= eb * vel[a];
  // u_a = m_a / rho, Y_s = rhoY_s / rho
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    ub[1 + a] += velb[a] * irho;
    irhob += velb[a] * u[1 + a];
  }
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) {
    ub[DIM + 2 + s] += Yb[s] * irho;
    irhob += Yb[s] * u[DIM + 2 + s];
  }
  rhob -= irhob * irho * irho;
  ub[0] += rhob;
  ub[DIM + 1] += Eb;
  if (f0) ub[1] = -ub[1];
  if (DIM > 1 && f1) ub[2] = -ub[2];
  if (DIM > 2 && f2) ub[3] = -ub[3];
  const long long C = p.cells;
#pragma unroll
  for (int v = 0; v < NV; ++v) aadd(Ubar + v * C + src, ub[v]);
  (void)E;
}

template <int DIM, int NS>
__global__ void __launch_bounds__(128)
k_prim_adj(const __grid_constant__ Params p, const double* __restrict__ Q,
           const double* __restrict__ Qb, double* __restrict__ Ubar) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < p.pcells) prim_adj_cell<DIM, NS>(p, t, Q, Qb, Ubar);
}

// ================================================================ k_grad_adj
// Gather form: GU_ab[t] = w (u_a[t-2] - u_a[t+2] + 8 (u_a[t+1] - u_a[t-1])) along b,
// so ubar_a[t'] += sum_j coef_j GUbar_ab[t' - j] over the cells where GU was formed.
template <int DIM, int NS>
__global__ void __launch_bounds__(256)
k_grad_adj(const __grid_constant__ Params p, double* __restrict__ Qb) {
  using L = Lay<DIM, NS>;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.pcells) return;
  const long long PC = p.pcells;
  int idx[3];
  idx[0] = (int)(t % p.np[0]);
  idx[1] = (int)((t / p.np[0]) % p.np[1]);
  idx[2] = (int)(t / ((long long)p.np[0] * p.np[1]));
  const long long stride[3] = {1, p.np[0], (long long)p.np[0] * p.np[1]};
  const int js[4] = {-2, -1, 1, 2};
  const double cj[4] = {1.0, -8.0, 8.0, -1.0};  // coefficient of u[t + j] in GU[t]
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      const double w = p.inv_dx[b] * (1.0 / 12.0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int src = idx[b] - js[q];  // the GU cell whose stencil holds t at offset j
        if (src < 2 || src >= p.np[b] - 2) continue;
        acc = fma(cj[q] * w, Qb[(L::GU + a * DIM + b) * PC + t - js[q] * stride[b]], acc);
      }
    }
    Qb[(L::UN + a) * PC + t] += acc;
  }
}

// ============================================================ objective ===
// J = sum_cells Y_s (1 - Y_s) dV (the mixing measure); per-block partial sums
// (deterministic two-pass reduction) and the gradient dJ/dU.
template <int DIM, int NS>
__global__ void __launch_bounds__(256)
k_mixing(const __grid_constant__ Params p, const double* __restrict__ U, int sp, double dV,
         double* __restrict__ part, double* __restrict__ Ubar) {
  constexpr int NV = DIM + 1 + NS;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long C = p.cells;
  double j = 0.0;
  if (c < C) {
    const double rho = U[c], irho = rcp_nr(rho);
    double Y;
    if (sp < NS - 1) {
      Y = U[(DIM + 2 + sp) * C + c] * irho;
    } else {
      double ys = 0.0;
#pragma unroll
      for (int s = 0; s < NS - 1; ++s) ys += U[(DIM + 2 + s) * C + c];
      Y = 1.0 - ys * irho;
    }
    j = Y * (1.0 - Y) * dV;
    const double gY = (1.0 - 2.0 * Y) * dV;  // dJ/dY
#pragma unroll
    for (int v = 0; v < NV; ++v) Ubar[v * C + c] = 0.0;
    if (sp < NS - 1) {
      Ubar[(DIM + 2 + sp) * C + c] = gY * irho;
      Ubar[c] = -gY * Y * irho;
    } else {
#pragma unroll
      for (int s = 0; s < NS - 1; ++s) Ubar[(DIM + 2 + s) * C + c] = -gY * irho;
      Ubar[c] = gY * (1.0 - Y) * irho;
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = j;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}


// ====================================================== k_from_prim_adj ===
// Reverse of k_from_prim: Ubar -> Pbar (overwritten).
template <int DIM, int NS>
__global__ void __launch_bounds__(256)
k_from_prim_adj(const __grid_constant__ Params p, const double* __restrict__ P,
                const double* __restrict__ Ub, double* __restrict__ Pb) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.cells) return;
  const long long C = p.cells;
  const double rho = P[c];
  double Y[NS], ys = 0.0, Rm = 0.0;
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) { Y[s] = P[(DIM + 2 + s) * C + c]; ys += Y[s]; }
  Y[NS - 1] = 1.0 - ys;
#pragma unroll
  for (int s = 0; s < NS; ++s) Rm = fma(Y[s], p.r[s], Rm);
  const double pr = P[(DIM + 1) * C + c];
  const double T = pr / (rho * Rm);
  const TauPt tp = tau_of(p, T);
  double e = 0.0, cv = 0.0, es[NS], ke = 0.0, u[DIM];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const double cps = cp_s(p, s, tp.tc);
    es[s] = h_s(p, s, tp, cps) - p.r[s] * T;
    e = fma(Y[s], es[s], e);
    cv = fma(Y[s], cps - p.r[s], cv);
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) { u[a] = P[(1 + a) * C + c]; ke = fma(u[a], u[a], ke); }
  const double UbE = Ub[(DIM + 1) * C + c];
  double rhob = Ub[c] + UbE * fma(0.5, ke, e);
  double ub[DIM];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const double m = Ub[(1 + a) * C + c];
    rhob = fma(m, u[a], rhob);
    ub[a] = m * rho + UbE * rho * u[a];
  }
  double Yb[NS];
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) {
    const double g = Ub[(DIM + 2 + s) * C + c];
    rhob = fma(g, Y[s], rhob);
    Yb[s] = g * rho;
  }
  Yb[NS - 1] = 0.0;
  const double eb = UbE * rho;
#pragma unroll
  for (int s = 0; s < NS; ++s) Yb[s] += eb * es[s];
  const double Tb = eb * cv;
  const double prb = Tb / (rho * Rm);
  rhob -= Tb * T / rho;
  const double Rmb = -Tb * T / Rm;
#pragma unroll
  for (int s = 0; s < NS; ++s) Yb[s] += Rmb * p.r[s];
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) Yb[s] -= Yb[NS - 1];
  Pb[c] = rhob;
#pragma unroll
  for (int a = 0; a < DIM; ++a) Pb[(1 + a) * C + c] = ub[a];
  Pb[(DIM + 1) * C + c] = prb;
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) Pb[(DIM + 2 + s) * C + c] = Yb[s];
}


}  // namespace xf
