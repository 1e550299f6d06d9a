// Device-side counter-based random numbers for the HMC heat bath (paper
// Sec. 2 and Sec. 3 step 1: Gaussian momenta and the Gaussian pseudofermion
// noise chi at the start of every trajectory; the uniform of the Metropolis
// test at its end).
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds on a 4-word counter with a 2-word key;
// a round multiplies counter words 0 and 2 by two fixed odd constants, keeps
// the high and low 32 bits of both 64-bit products, xors the high halves with
// the other two counter words and the key, and permutes the words; the key is
// advanced by two Weyl increments between rounds.
//
// Uniforms carry 53 random bits; Gaussians come from the Box-Muller
// transform.  Its logarithm and sine / cosine are series written out with
// additions, multiplications, one division and one square root, each an
// explicitly rounded-to-nearest intrinsic (no contraction into fused
// multiply-adds), in the same order as the host-side generator that seeds
// the tests: both produce the same bits.
//   log v        v = f 2^e, f in [sqrt(1/2), sqrt(2)); log f = 2 atanh z,
//                z = (f-1)/(f+1), atanh z = z sum_{k<=10} z^2k / (2k+1);
//                e ln 2 with ln 2 = hi + lo, hi of 32 significant bits
//   sin, cos     of 2 pi u: quadrant n = floor(4u), remainder f (exact);
//                complementary angle for f > 1/2; Taylor series in
//                x = (pi/2) h, h <= 1/2, to the x^19 / x^18 terms
#pragma once
#include <stdint.h>

namespace lq {
namespace rng {

// Philox4x32 round constants: multipliers and the key increments (the
// golden-ratio and sqrt(3)-1 Weyl constants), as published.
constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

struct Words { uint32_t x, y, z, w; };

__host__ __device__ inline Words philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                               uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += kW0; k1 += kW1; }
    const uint64_t p0 = (uint64_t)kM0 * c0;
    const uint64_t p1 = (uint64_t)kM1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// Double in [0, 1) from two words: the top 27 bits of a and the top 26 of b.
__host__ __device__ inline double uniform53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

// Series constants, each the double nearest to the exact value:
// ln 2 split (hi: 32 significant bits), pi / 2, sqrt(1/2), 1 / (2k+1), (-1)^k / (2k+1)!, (-1)^k / (2k)!.
constexpr double kLn2Hi = 0x1.62e42fee00000p-1;
constexpr double kLn2Lo = 0x1.a39ef35793c76p-33;
constexpr double kPiHalf = 0x1.921fb54442d18p+0;
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double madd(double s, double w, double c) { return add(mul(s, w), c); }

// log v for positive normal v (the heat bath uses v in (0, 1]).
__device__ __forceinline__ double log_series(double v) {
  int e;
  double f = frexp(v, &e);               // v = f 2^e, f in [0.5, 1): exact
  if (f < kSqrtHalf) { f = mul(f, 2.0); e -= 1; }
  const double z = __ddiv_rn(add(f, -1.0), add(f, 1.0));
  const double w = mul(z, z);
  double s = madd(1.0 / 21.0, w, 1.0 / 19.0);
  s = madd(s, w, 1.0 / 17.0);
  s = madd(s, w, 1.0 / 15.0);
  s = madd(s, w, 1.0 / 13.0);
  s = madd(s, w, 1.0 / 11.0);
  s = madd(s, w, 1.0 / 9.0);
  s = madd(s, w, 1.0 / 7.0);
  s = madd(s, w, 1.0 / 5.0);
  s = madd(s, w, 1.0 / 3.0);
  s = madd(s, w, 1.0);
  const double q = mul(z, s);
  const double ed = (double)e;
  return add(mul(ed, kLn2Hi), add(mul(ed, kLn2Lo), add(q, q)));
}

// sin(2 pi u), cos(2 pi u) for u in [0, 1).
__device__ __forceinline__ void sincos_2pi(double u, double* sn, double* cs) {
  const double q4 = mul(u, 4.0);
  const double nq = floor(q4);
  const double f = add(q4, -nq);
  const bool hi = f > 0.5;
  const double h = hi ? add(1.0, -f) : f;
  const double x = mul(h, kPiHalf);
  const double w = mul(x, x);
  // (-1)^k / (2k+1)!, k = 9 .. 1
  double ps = madd(-1.0 / 121645100408832000.0, w, 1.0 / 355687428096000.0);
  ps = madd(ps, w, -1.0 / 1307674368000.0);
  ps = madd(ps, w, 1.0 / 6227020800.0);
  ps = madd(ps, w, -1.0 / 39916800.0);
  ps = madd(ps, w, 1.0 / 362880.0);
  ps = madd(ps, w, -1.0 / 5040.0);
  ps = madd(ps, w, 1.0 / 120.0);
  ps = madd(ps, w, -1.0 / 6.0);
  const double sx = add(x, mul(mul(x, w), ps));
  // (-1)^k / (2k)!, k = 9 .. 1
  double pc = madd(-1.0 / 6402373705728000.0, w, 1.0 / 20922789888000.0);
  pc = madd(pc, w, -1.0 / 87178291200.0);
  pc = madd(pc, w, 1.0 / 479001600.0);
  pc = madd(pc, w, -1.0 / 3628800.0);
  pc = madd(pc, w, 1.0 / 40320.0);
  pc = madd(pc, w, -1.0 / 720.0);
  pc = madd(pc, w, 1.0 / 24.0);
  pc = madd(pc, w, -1.0 / 2.0);
  const double cx = add(1.0, mul(w, pc));
  const double sf = hi ? cx : sx, cf = hi ? sx : cx;   // sin, cos of (pi/2) f
  switch ((int)nq) {
    case 0: *sn = sf; *cs = cf; break;
    case 1: *sn = cf; *cs = -sf; break;
    case 2: *sn = -sf; *cs = -cf; break;
    default: *sn = -cf; *cs = sf; break;
  }
}

// Two N(0,1) variates from one Philox output: Box-Muller on uniform53(x, y), uniform53(z, w).
__device__ __forceinline__ void gaussian_pair(const Words& r, double* z0, double* z1) {
  const double u1 = uniform53(r.x, r.y), u2 = uniform53(r.z, r.w);
  const double rad = __dsqrt_rn(mul(-2.0, log_series(add(1.0, -u1))));
  double s, c;
  sincos_2pi(u2, &s, &c);
  *z0 = mul(rad, c);
  *z1 = mul(rad, s);
}

}  // namespace rng
}  // namespace lq
