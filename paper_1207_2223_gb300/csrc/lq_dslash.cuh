// Wilson hopping stencil with fused epilogues (paper Sec. 3, kernel 1: the
// Dirac operator and its adjoint applied to the pseudofermion field inside
// the conjugate-gradient routine; Eq. 4 gives the operator M = D + m).
//
//   (H psi)(x) = sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
//   M psi = psi - kappa H psi,     M^dag: projector signs of the two hops swapped
//
// One thread per site.  Each of the 8 hops loads the neighbour spinor,
// projects it to two colour vectors with (1 -+ g_mu), multiplies them by
// the link (or its adjoint), and adds the rebuilt four-spinor to a
// register accumulator.  The neighbour indices are computed from the site
// coordinates, no neighbour table is stored (paper Sec. 3).  What happens
// to the result is an epilogue functor, so the CG vector updates and the
// FP64 norms fuse into the same pass over the lattice.
#pragma once
#include <algorithm>

#include "lq_device.cuh"

namespace lq {

// Device-resident scalars of one CG solve.  Kernels of an iteration read
// alpha / beta from here and the last block of a reducing kernel updates
// them, so an iteration needs no host round trip.
struct SolverState {
  double rr;          // |r|^2 of the iterated residual
  double rr_prev;     // |r|^2 of the previous iteration
  double tt;          // |M p|^2 = p^dag M^dag M p
  double alpha, beta;
  double phi2;        // |phi|^2
  double stop2;       // tol^2 |phi|^2
  double rr_ref;      // |r|^2 right after the last reliable update
  double delta2;      // reliable update when rr < delta2 * rr_ref
  double rr_true;     // |phi - M^dag M x|^2 of the last true-residual pass
  int iter;           // iterations done
  int iter_since_ru;  // iterations since the last reliable update
  int ru_every;       // reliable update at least this often (0: never)
  int maxiter;
  int halt;           // 1: the iteration kernels return at once
  int breakdown;      // 1: non-positive or non-finite p^dag A p, or a NaN
  int hist_len;       // capacity of hist
  int pad_;
  double* hist;       // relative iterated residual per iteration (may be null)
};

struct NoEpiState {};

// s * a; FP32 complex numbers with one packed FP32x2 multiply
template <typename T> __device__ __forceinline__ cplx<T> scale_c(T s, cplx<T> a) { return s * a; }
template <> __device__ __forceinline__ cplx<float> scale_c<float>(float s, cplx<float> a) {
  const float2 r = __fmul2_rn(make_float2(a.re, a.im), make_float2(s, s));
  return {r.x, r.y};
}

// Where the spinor of site n lives: element n of one field of V sites.
struct SingleIndex {
  int V;
  __device__ __forceinline__ int stride() const { return V; }
  __device__ __forceinline__ int operator()(int n) const { return n; }
};

// Both hops of direction MU at site s.  INIT: the forward hop is the site's first
// contribution and sets acc (the first direction of the stencil).  The antiperiodic
// sign of a hop across the time boundary is folded into the norm scale of 16-bit
// storage, which is multiplied anyway; for the other formats it flips sign bits.
template <int MU, bool DAG, GStore G, SStore SI, typename T, class IX = SingleIndex, bool INIT = false>
__device__ __forceinline__ void hop_dir(const Geom& geo, const GaugeRef& U, const SpinorRef& in, int s,
                                        const int c[4], cplx<T> acc[12], IX ix = IX{0}) {
  if constexpr (std::is_same<IX, SingleIndex>::value) ix.V = geo.V;
  constexpr int SF = DAG ? +1 : -1;   // forward hop uses (1 + SF g_mu)
  constexpr bool SCALED = SI == SStore::F16 || SI == SStore::BF16 || SI == SStore::I16 || G == GStore::I16_12;
  {
    const int n = nbr_fwd(geo, s, c, MU);
    cplx<T> p[12];
    T sc = load_spinor_raw<SI, T>(in, ix.stride(), ix(n), p);
    cplx<T> h0[3], h1[3];
    project<MU, SF>(p, h0, h1);
    const bool flip = MU == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1;
    if constexpr (SCALED) {
      if (flip) sc = -sc;
      if constexpr (G == GStore::I16_12) sc = sc * (T)kQ16Inv;   // links as raw integers
#pragma unroll
      for (int k = 0; k < 3; ++k) { h0[k] = scale_c(sc, h0[k]); h1[k] = scale_c(sc, h1[k]); }
    } else if (flip) {
      negate3(h0);
      negate3(h1);
    }
    cplx<T> u[9];
    if constexpr (G == GStore::I16_12) load_link_q16<T>(U, geo.V, MU, s, u);
    else load_link<G, T>(U, geo.V, MU, s, u);
    cplx<T> w0[3], w1[3];
    su3_mul(u, h0, w0);
    su3_mul(u, h1, w1);
    accumulate<MU, SF, T, INIT>(acc, w0, w1);
  }
  {
    const int n = nbr_bwd(geo, s, c, MU);
    cplx<T> p[12];
    T sc = load_spinor_raw<SI, T>(in, ix.stride(), ix(n), p);
    cplx<T> h0[3], h1[3];
    project<MU, -SF>(p, h0, h1);
    const bool flip = MU == 3 && geo.antiperiodic && c[3] == 0;
    if constexpr (SCALED) {
      if (flip) sc = -sc;
      if constexpr (G == GStore::I16_12) sc = sc * (T)kQ16Inv;   // links as raw integers
#pragma unroll
      for (int k = 0; k < 3; ++k) { h0[k] = scale_c(sc, h0[k]); h1[k] = scale_c(sc, h1[k]); }
    } else if (flip) {
      negate3(h0);
      negate3(h1);
    }
    cplx<T> u[9];
    if constexpr (G == GStore::I16_12) load_link_q16<T>(U, geo.V, MU, n, u);
    else load_link<G, T>(U, geo.V, MU, n, u);
    cplx<T> w0[3], w1[3];
    su3_dagmul(u, h0, w0);
    su3_dagmul(u, h1, w1);
    accumulate<MU, -SF>(acc, w0, w1);
  }
}

// Threads per block: 256 for FP32 arithmetic; 128 for FP64 and double-float,
// whose 190-250 registers per thread would otherwise leave one block per SM
// (the FP64 pipe, not occupancy, bounds the FP64 operator).
template <typename T> struct DslashBlock { static constexpr int value = 256; };
template <> struct DslashBlock<double> { static constexpr int value = 128; };
template <> struct DslashBlock<df64> { static constexpr int value = 128; };
// Minimum resident blocks per SM requested from the compiler (register cap).
#ifndef LQ_DSLASH_MIN_BLOCKS
#define LQ_DSLASH_MIN_BLOCKS 2
#endif

// Pass 1 of CG and the plain operator (no epilogue loads) are latency-bound:
// they may ask for more resident blocks than pass 2.
#ifndef LQ_K1_MIN_BLOCKS
#define LQ_K1_MIN_BLOCKS LQ_DSLASH_MIN_BLOCKS
#endif
template <typename T, class Epi> struct EpiMinBlocks { static constexpr int value = LQ_DSLASH_MIN_BLOCKS; };

// |v|^2 of one site in the kernel's arithmetic precision; the per-site sums
// are then accumulated in FP64 (one FP64 add per site: the FP64 pipe of this
// part is ~60x slower than its FP32 pipe).
template <typename T>
__device__ __forceinline__ double site_norm2(const cplx<T> v[12]) {
  T a = (T)0;
#pragma unroll
  for (int k = 0; k < 12; ++k) { a = fma(v[k].re, v[k].re, a); a = fma(v[k].im, v[k].im, a); }
  return (double)a;
}

// Grid-stride: the grid is one wave of resident blocks and every thread
// walks the lattice in steps of the grid size, so the halt check and the
// block reduction happen once per block rather than once per 256 sites.
template <typename T, GStore G, SStore SI, bool DAG, class Epi>
__global__ void __launch_bounds__(DslashBlock<T>::value, (EpiMinBlocks<T, Epi>::value)) dslash_kernel(Geom geo, GaugeRef U, SpinorRef in,
                                                                        T kappa, Epi epi, ReduceScratch rs) {
  if (epi.halted()) return;
  double red[Epi::NRED];
#pragma unroll
  for (int q = 0; q < Epi::NRED; ++q) red[q] = 0.0;
  const int stride = gridDim.x * blockDim.x;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < geo.V; s += stride) {
    int c[4];
    site_coords(geo, s, c);
    cplx<T> acc[12];
    hop_dir<0, DAG, G, SI, T, SingleIndex, true>(geo, U, in, s, c, acc);
    hop_dir<1, DAG, G, SI, T>(geo, U, in, s, c, acc);
    hop_dir<2, DAG, G, SI, T>(geo, U, in, s, c, acc);
    hop_dir<3, DAG, G, SI, T>(geo, U, in, s, c, acc);
    cplx<T> ctr[12];
    load_spinor<SI, T>(in, geo.V, s, ctr);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[k].re = fma(-kappa, acc[k].re, ctr[k].re);
      acc[k].im = fma(-kappa, acc[k].im, ctr[k].im);
    }
    epi.apply(geo.V, s, acc, red);
  }
  if constexpr (Epi::REDUCE) {
    double tot[Epi::NRED];
    if (grid_sum<Epi::NRED>(red, rs, tot)) epi.finalize(tot);
  }
}

// ------------------------------------------------------------ epilogues
template <SStore SO>
struct EpiStore {                       // out = M psi
  static constexpr int NRED = 1;
  static constexpr bool REDUCE = false;
  SpinorRef out;
  __device__ bool halted() const { return false; }
  template <typename T> __device__ void apply(int V, int s, cplx<T> v[12], double (&)[NRED]) const {
    store_spinor<SO, T>(out, V, s, v);
  }
  __device__ void finalize(double (&)[NRED]) const {}
};

template <SStore SO>
struct EpiStoreNorm {                   // out = M psi, *result = |out|^2
  static constexpr int NRED = 1;
  static constexpr bool REDUCE = true;
  SpinorRef out;
  double* result;
  __device__ bool halted() const { return false; }
  template <typename T> __device__ void apply(int V, int s, cplx<T> v[12], double (&red)[NRED]) const {
    store_spinor<SO, T>(out, V, s, v);
    red[0] += site_norm2(v);
  }
  __device__ void finalize(double (&tot)[NRED]) const { *result = tot[0]; }
};

// CG step 1:  t = M p, tt = |t|^2, alpha = rr / tt
template <SStore ST>
struct EpiCG1 {
  static constexpr int NRED = 1;
  static constexpr bool REDUCE = true;
  SpinorRef t;
  SolverState* st;
  __device__ bool halted() const { return *(volatile const int*)&st->halt; }
  template <typename T> __device__ void apply(int V, int s, cplx<T> v[12], double (&red)[NRED]) const {
    store_spinor<ST, T>(t, V, s, v);
    red[0] += site_norm2(v);
  }
  __device__ void finalize(double (&tot)[NRED]) const {
    const double tt = tot[0], rr = st->rr;
    st->tt = tt;
    if (!(tt > 0.0) || !isfinite(tt) || !isfinite(rr)) {
      st->breakdown = 1;
      st->halt = 1;
      st->alpha = 0.0;
    } else {
      st->alpha = rr / tt;
    }
  }
};

// CG step 2:  r <- r - alpha M^dag t,  x <- x + alpha p,  rr_new = |r|^2,
// beta = rr_new / rr; decides whether the iteration halts (converged
// estimate, reliable update due, or iteration limit).
template <SStore SR, SStore SX, SStore SP>
struct EpiCG2 {
  static constexpr int NRED = 1;
  static constexpr bool REDUCE = true;
  SpinorRef r, x, p;
  SolverState* st;
  __device__ bool halted() const { return *(volatile const int*)&st->halt; }
  template <typename T> __device__ void apply(int V, int s, cplx<T> v[12], double (&red)[NRED]) const {
    const T alpha = (T)st->alpha;
    cplx<T> rv[12], xv[12], pv[12];
    load_spinor<SR, T, false>(r, V, s, rv);
    load_spinor<SX, T, false>(x, V, s, xv);
    load_spinor<SP, T>(p, V, s, pv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k].re = fma(-alpha, v[k].re, rv[k].re);
      rv[k].im = fma(-alpha, v[k].im, rv[k].im);
      xv[k].re = fma(alpha, pv[k].re, xv[k].re);
      xv[k].im = fma(alpha, pv[k].im, xv[k].im);
    }
    store_spinor<SR, T>(r, V, s, rv);
    store_spinor<SX, T>(x, V, s, xv);
    red[0] += site_norm2(rv);
  }
  // One thread, at the end of the kernel's critical path: every field is read before
  // the first store (a store through st->hist could alias them and serialise the reads).
  __device__ void finalize(double (&tot)[NRED]) const {
    const double rr_new = tot[0];
    const int it = st->iter, since = st->iter_since_ru + 1, ru_every = st->ru_every, maxiter = st->maxiter;
    const int hist_len = st->hist_len;
    const double rr = st->rr, phi2 = st->phi2, stop2 = st->stop2, delta2 = st->delta2, rr_ref = st->rr_ref;
    double* hist = st->hist;
    const bool finite = isfinite(rr_new);
    const bool halt = !finite || rr_new <= stop2 || (ru_every > 0 && since >= ru_every) ||
                      (delta2 > 0.0 && rr_new < delta2 * rr_ref) || it + 1 >= maxiter;
    st->iter = it + 1;
    st->iter_since_ru = since;
    st->beta = rr_new / rr;
    st->rr_prev = rr;
    st->rr = rr_new;
    if (!finite) st->breakdown = 1;
    if (halt) st->halt = 1;
    if (hist != nullptr && it < hist_len) hist[it] = sqrt(rr_new / phi2);
  }
};

template <SStore S> struct EpiMinBlocks<float, EpiCG1<S>> { static constexpr int value = LQ_K1_MIN_BLOCKS; };
template <SStore S> struct EpiMinBlocks<float, EpiStore<S>> { static constexpr int value = LQ_K1_MIN_BLOCKS; };

// True residual in FP64:  v = M^dag (M x)  ->  r = phi - v, |r|^2.
// Optionally also stores r in a low-precision field (reliable update).
template <SStore SLO, bool STORE_LO>
struct EpiResidual {
  static constexpr int NRED = 1;
  static constexpr bool REDUCE = true;
  SpinorRef phi, r, r_lo;
  SolverState* st;
  __device__ bool halted() const { return false; }
  template <typename T> __device__ void apply(int V, int s, cplx<T> v[12], double (&red)[NRED]) const {
    cplx<double> ph[12];
    load_spinor<SStore::F64, double>(phi, V, s, ph);
    cplx<double> rv[12];
    double a = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k] = {ph[k].re - (double)v[k].re, ph[k].im - (double)v[k].im};
      a += rv[k].re * rv[k].re + rv[k].im * rv[k].im;
    }
    store_spinor<SStore::F64, double>(r, V, s, rv);
    if constexpr (STORE_LO) store_spinor<SLO, double>(r_lo, V, s, rv);
    red[0] += a;
  }
  __device__ void finalize(double (&tot)[NRED]) const { st->rr_true = tot[0]; }
};

inline int grid_for(int V, int bs) { return (V + bs - 1) / bs; }

// Resident blocks of one kernel on the current device (queried once per kernel).
int resident_grid(const void* kernel, int block);

// A lattice with fewer full blocks (one site per thread) than half a wave leaves SMs idle;
// it runs in blocks of half the size, which spread over twice as many SMs (measured: 8^4
// 5.2 -> 4.8 ms per mixed solve; at 16^4, with 256 blocks, the full blocks were faster).
template <typename T, GStore G, SStore SI, bool DAG, class Epi>
inline void launch_dslash(const Geom& geo, GaugeRef U, SpinorRef in, double kappa, const Epi& epi,
                          const ReduceScratch& rs, cudaStream_t stream) {
  constexpr int bs = DslashBlock<T>::value;
  const void* kern = reinterpret_cast<const void*>(&dslash_kernel<T, G, SI, DAG, Epi>);
  static const int wave = resident_grid(kern, bs);
  if (2 * grid_for(geo.V, bs) <= wave) {
    static const int wave_half = resident_grid(kern, bs / 2);
    const int grid = std::min(grid_for(geo.V, bs / 2), wave_half);
    dslash_kernel<T, G, SI, DAG, Epi><<<grid, bs / 2, 0, stream>>>(geo, U, in, (T)kappa, epi, rs);
    return;
  }
  const int grid = std::min(grid_for(geo.V, bs), wave);
  dslash_kernel<T, G, SI, DAG, Epi><<<grid, bs, 0, stream>>>(geo, U, in, (T)kappa, epi, rs);
}

}  // namespace lq
