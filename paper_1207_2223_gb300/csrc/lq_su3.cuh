// 3x3 complex matrix helpers for the gauge-side kernels (FP64): products,
// the su(3) projection Im tr(t_a W), exp(i eps P) and reunitarisation.
#pragma once
#include "lq_device.cuh"

namespace lq {

struct M3 {
  cplx<double> m[9];   // row-major
};

__device__ __forceinline__ M3 load_m3(const double2* __restrict__ g64, int V, int mu, int s) {
  M3 r;
  const double2* p = g64 + (size_t)mu * 9 * V;
#pragma unroll
  for (int c = 0; c < 9; ++c) { double2 w = __ldg(p + (size_t)c * V + s); r.m[c] = {w.x, w.y}; }
  return r;
}
// coherent load, for kernels that also write the gauge field
__device__ __forceinline__ M3 load_m3_rw(const double2* g64, int V, int mu, int s) {
  M3 r;
  const double2* p = g64 + (size_t)mu * 9 * V;
#pragma unroll
  for (int c = 0; c < 9; ++c) { double2 w = p[(size_t)c * V + s]; r.m[c] = {w.x, w.y}; }
  return r;
}
__device__ __forceinline__ void store_m3(double2* g64, int V, int mu, int s, const M3& a) {
  double2* p = g64 + (size_t)mu * 9 * V;
#pragma unroll
  for (int c = 0; c < 9; ++c) p[(size_t)c * V + s] = make_double2(a.m[c].re, a.m[c].im);
}

// a b
__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<double> t = cmul(a.m[3 * i], b.m[j]);
      t = cmadd(t, a.m[3 * i + 1], b.m[3 + j]);
      r.m[3 * i + j] = cmadd(t, a.m[3 * i + 2], b.m[6 + j]);
    }
  return r;
}
// a b^dag
__device__ __forceinline__ M3 mul_dag(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // sum_k a_ik conj(b_jk)
      cplx<double> t = cjmul(b.m[3 * j], a.m[3 * i]);
      t = cjmadd(t, b.m[3 * j + 1], a.m[3 * i + 1]);
      r.m[3 * i + j] = cjmadd(t, b.m[3 * j + 2], a.m[3 * i + 2]);
    }
  return r;
}
// a^dag b
__device__ __forceinline__ M3 dag_mul(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // sum_k conj(a_ki) b_kj
      cplx<double> t = cjmul(a.m[i], b.m[j]);
      t = cjmadd(t, a.m[3 + i], b.m[3 + j]);
      r.m[3 * i + j] = cjmadd(t, a.m[6 + i], b.m[6 + j]);
    }
  return r;
}
__device__ __forceinline__ void add_to(M3& a, const M3& b) {
#pragma unroll
  for (int c = 0; c < 9; ++c) a.m[c] = a.m[c] + b.m[c];
}
__device__ __forceinline__ double re_trace(const M3& a) { return a.m[0].re + a.m[4].re + a.m[8].re; }
// Re tr(a b^dag) = Re sum_ij a_ij conj(b_ij)
__device__ __forceinline__ double re_tr_mul_dag(const M3& a, const M3& b) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 9; ++c) s += a.m[c].re * b.m[c].re + a.m[c].im * b.m[c].im;
  return s;
}

// f_a = Im tr(t_a W), t_a = lambda_a / sqrt(2), written out from the
// Gell-Mann matrices: tr(lambda_1 W) = W01 + W10, tr(lambda_2 W) = i (W01 - W10),
// tr(lambda_3 W) = W00 - W11, ... tr(lambda_8 W) = (W00 + W11 - 2 W22) / sqrt(3).
__device__ __forceinline__ void im_tr_ta(const M3& W, double f[8]) {
  const double r2 = 0.70710678118654752440;
  const double r6 = 0.40824829046386301637;   // 1 / sqrt(6)
  f[0] = r2 * (W.m[1].im + W.m[3].im);
  f[1] = r2 * (W.m[1].re - W.m[3].re);
  f[2] = r2 * (W.m[0].im - W.m[4].im);
  f[3] = r2 * (W.m[2].im + W.m[6].im);
  f[4] = r2 * (W.m[2].re - W.m[6].re);
  f[5] = r2 * (W.m[5].im + W.m[7].im);
  f[6] = r2 * (W.m[5].re - W.m[7].re);
  f[7] = r6 * (W.m[0].im + W.m[4].im - 2.0 * W.m[8].im);
}

// X = i eps sum_a p_a t_a (anti-Hermitian, traceless)
// eps P, P = sum_a p_a t_a (Hermitian, traceless)
__device__ __forceinline__ M3 eps_algebra(const double p[8], double eps) {
  const double r2 = 0.70710678118654752440 * eps;
  const double r6 = 0.40824829046386301637 * eps;
  M3 P;
  P.m[0] = {r2 * p[2] + r6 * p[7], 0.0};
  P.m[4] = {-r2 * p[2] + r6 * p[7], 0.0};
  P.m[8] = {-2.0 * r6 * p[7], 0.0};
  P.m[1] = {r2 * p[0], -r2 * p[1]};
  P.m[3] = {r2 * p[0], r2 * p[1]};
  P.m[2] = {r2 * p[3], -r2 * p[4]};
  P.m[6] = {r2 * p[3], r2 * p[4]};
  P.m[5] = {r2 * p[5], -r2 * p[6]};
  P.m[7] = {r2 * p[5], r2 * p[6]};
  return P;
}
// i eps P
__device__ __forceinline__ M3 i_eps_algebra(const double p[8], double eps) {
  const M3 P = eps_algebra(p, eps);
  M3 X;
#pragma unroll
  for (int c = 0; c < 9; ++c) X.m[c] = {-P.m[c].im, P.m[c].re};
  return X;
}

// exp(X) by scaling and squaring: X / 2^k has Frobenius norm <= 1/4, a Taylor
// series of 16 terms in Horner form (remainder < 0.25^17 / 17! ~ 6e-25), then
// k squarings.
__device__ __forceinline__ M3 expm3(const M3& X) {
  double n2 = 0.0;
#pragma unroll
  for (int c = 0; c < 9; ++c) n2 += norm2(X.m[c]);
  int k = 0;
  double nrm = sqrt(n2);
  while (nrm > 0.25 && k < 60) { nrm *= 0.5; ++k; }
  const double sc = ldexp(1.0, -k);
  M3 A;
#pragma unroll
  for (int c = 0; c < 9; ++c) A.m[c] = sc * X.m[c];
  // Horner: E = I + A/1 (I + A/2 (I + ... (I + A/16)))
  M3 E;
#pragma unroll
  for (int c = 0; c < 9; ++c) E.m[c] = {0.0, 0.0};
  E.m[0] = E.m[4] = E.m[8] = {1.0, 0.0};
  for (int j = 16; j >= 1; --j) {
    M3 T = mul(A, E);
    const double inv = 1.0 / j;
#pragma unroll
    for (int c = 0; c < 9; ++c) E.m[c] = inv * T.m[c];
    E.m[0].re += 1.0; E.m[4].re += 1.0; E.m[8].re += 1.0;
  }
  for (int i = 0; i < k; ++i) E = mul(E, E);
  return E;
}

// exp(i Q) for Hermitian traceless Q by the Cayley-Hamilton closed form of
// Morningstar and Peardon, PRD 69 (2004) 054501: exp(iQ) = f0 + f1 Q + f2 Q^2,
// where the f_j follow from the invariants c0 = det Q = tr(Q^3)/3 and
// c1 = tr(Q^2)/2 through the eigenvalues 2u, -u + w, -u - w of Q.  For c0 < 0
// the coefficients come from -Q: f_j(-c0) = (-1)^j conj(f_j(c0)).  With c0 >= 0
// the denominator 9u^2 - w^2 is at least c1, so the form is well conditioned;
// Q = 0 (c1 below 1e-12) goes to the Taylor series.  About a quarter of the FP64
// work of expm3 (one matrix product and a few sines and cosines instead of ~18
// products).
__device__ __forceinline__ M3 expi_hermitian(const M3& Q) {
  const M3 Q2 = mul(Q, Q);
  const double c1 = 0.5 * (Q2.m[0].re + Q2.m[4].re + Q2.m[8].re);
  if (!(c1 >= 1e-12)) {
    M3 X;
#pragma unroll
    for (int c = 0; c < 9; ++c) X.m[c] = {-Q.m[c].im, Q.m[c].re};
    return expm3(X);
  }
  double t3 = 0.0;   // Re tr(Q Q^2)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) t3 += Q.m[3 * i + k].re * Q2.m[3 * k + i].re - Q.m[3 * i + k].im * Q2.m[3 * k + i].im;
  const double c0s = t3 / 3.0;
  const bool neg = c0s < 0.0;
  const double c0 = fabs(c0s);
  const double r = sqrt(c1 / 3.0);
  const double c0max = 2.0 * r * r * r;
  const double theta = acos(fmin(1.0, c0 / c0max));
  double s3, c3;
  sincos(theta / 3.0, &s3, &c3);
  const double u = r * c3, w = sqrt(c1) * s3;
  const double u2 = u * u, w2 = w * w;
  double su, cu, sw, cw;
  sincos(u, &su, &cu);
  sincos(w, &sw, &cw);
  // sin(w)/w, by its series near w = 0
  const double xi0 = fabs(w) > 0.05 ? sw / w : 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0));
  const cplx<double> e2 = {cu * cu - su * su, 2.0 * su * cu};   // exp(2iu)
  const cplx<double> em = {cu, -su};                            // exp(-iu)
  const cplx<double> h0 = (u2 - w2) * e2 + cmul(em, cplx<double>{8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0});
  const cplx<double> h1 = (2.0 * u) * e2 - cmul(em, cplx<double>{2.0 * u * cw, -(3.0 * u2 - w2) * xi0});
  const cplx<double> h2 = e2 - cmul(em, cplx<double>{cw, 3.0 * u * xi0});
  const double inv = 1.0 / (9.0 * u2 - w2);
  cplx<double> f0 = inv * h0, f1 = inv * h1, f2 = inv * h2;
  if (neg) {
    f0 = conjg(f0);
    f1 = -conjg(f1);
    f2 = conjg(f2);
  }
  M3 E;
#pragma unroll
  for (int c = 0; c < 9; ++c) E.m[c] = cmul(f1, Q.m[c]) + cmul(f2, Q2.m[c]);
  E.m[0] = E.m[0] + f0;
  E.m[4] = E.m[4] + f0;
  E.m[8] = E.m[8] + f0;
  return E;
}

// Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1)
__device__ __forceinline__ void reunitarise(M3& U) {
  const double n0 = 1.0 / sqrt(norm2(U.m[0]) + norm2(U.m[1]) + norm2(U.m[2]));
  for (int j = 0; j < 3; ++j) U.m[j] = n0 * U.m[j];
  // <r0, r1> = sum conj(r0_j) r1_j
  cplx<double> d = cjmul(U.m[0], U.m[3]);
  d = cjmadd(d, U.m[1], U.m[4]);
  d = cjmadd(d, U.m[2], U.m[5]);
  for (int j = 0; j < 3; ++j) U.m[3 + j] = U.m[3 + j] - cmul(d, U.m[j]);
  const double n1 = 1.0 / sqrt(norm2(U.m[3]) + norm2(U.m[4]) + norm2(U.m[5]));
  for (int j = 0; j < 3; ++j) U.m[3 + j] = n1 * U.m[3 + j];
  U.m[6] = conjg(cmul(U.m[1], U.m[5]) - cmul(U.m[2], U.m[4]));
  U.m[7] = conjg(cmul(U.m[2], U.m[3]) - cmul(U.m[0], U.m[5]));
  U.m[8] = conjg(cmul(U.m[0], U.m[4]) - cmul(U.m[1], U.m[3]));
}

}  // namespace lq
