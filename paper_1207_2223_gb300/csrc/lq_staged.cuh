// Wilson hopping stencil with in-block sharing of links through shared memory
// (the paper's kernel 1, Sec. 3, applied tile by tile).
//
// Every link U_mu(x) enters the operator twice: in the forward hop of x,
// U_mu(x) (1 -+ g_mu) psi(x+mu), and in the backward hop of x+mu,
// U_mu(x)^dag (1 +- g_mu) psi(x).  The plain kernel loads, decodes and (for
// 12-real storage) rebuilds every link twice, in two different threads.
// Here a block owns a tile of TILE consecutive sites; for mu = x, y the thread
// of site x decodes U_mu(x) once, applies it to its own forward hop, and when
// x+mu lies in the same tile it also forms the backward-hop term of x+mu,
//     W_mu(x) = U_mu(x)^dag (1 +- g_mu) psi(x)       (two colour vectors),
// from its own spinor and leaves it in shared memory.  After a barrier the
// thread of x+mu adds W_mu(x) instead of loading U_mu(x) and psi(x) and
// decoding them again.  Tiles follow the lattice order (x fastest), so with
// L_x dividing TILE every x hop and all but one row of y hops stay inside
// the tile; z and t hops, and hops that leave the tile, go through global
// memory as in the plain kernel.  Results equal the plain kernel's up to the
// order of the FP32 additions.  (Measured on GB300 at 32^3 x 64, 16-bit storage:
// slower than the plain kernel; the option stays off by default.)
#pragma once

#include "lq_dslash.cuh"

namespace lq {

constexpr int kStagedTile = 256;

template <int MU, bool DAG, GStore G, SStore SI, typename T>
__device__ __forceinline__ void load_link_any(const GaugeRef& U, int V, int s, cplx<T> u[9]) {
  if constexpr (G == GStore::I16_12) load_link_q16<T>(U, V, MU, s, u);
  else load_link<G, T>(U, V, MU, s, u);
}

// Scale of the half spinor of a hop: the site norm of 16-bit storage, the
// 1/32767 of raw fixed-point links; needed only when it differs from 1.
template <GStore G, SStore SI>
constexpr bool hop_scaled() {
  return SI == SStore::F16 || SI == SStore::BF16 || SI == SStore::I16 || G == GStore::I16_12;
}

// The forward hop of s in direction MU with the link u already decoded.
template <int MU, bool DAG, GStore G, SStore SI, typename T>
__device__ __forceinline__ void fwd_hop_with(const Geom& geo, const SpinorRef& in, int s, const int c[4],
                                             const cplx<T> u[9], cplx<T> acc[12]) {
  constexpr int SF = DAG ? +1 : -1;
  const int n = nbr_fwd(geo, s, c, MU);
  cplx<T> p[12];
  T sc = load_spinor_raw<SI, T>(in, geo.V, n, p);
  cplx<T> h0[3], h1[3];
  project<MU, SF>(p, h0, h1);
  if (MU == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1) sc = -sc;
  if constexpr (G == GStore::I16_12) sc = sc * (T)kQ16Inv;
  if (hop_scaled<G, SI>() || (MU == 3 && geo.antiperiodic)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) { h0[k] = scale_c(sc, h0[k]); h1[k] = scale_c(sc, h1[k]); }
  }
  cplx<T> w0[3], w1[3];
  su3_mul(u, h0, w0);
  su3_mul(u, h1, w1);
  accumulate<MU, SF>(acc, w0, w1);
}

// The backward hop of site f (= x + mu) formed at x = s from its own raw spinor p
// (scale sc) and the link u = U_mu(s): w = U^dag (1 +- g_mu) psi(s) (x, y hops carry no sign).
template <int MU, bool DAG, GStore G, typename T>
__device__ __forceinline__ void bwd_term(const cplx<T> p[12], T sc, const cplx<T> u[9], cplx<T> w0[3],
                                         cplx<T> w1[3]) {
  constexpr int SF = DAG ? +1 : -1;
  cplx<T> h0[3], h1[3];
  project<MU, -SF>(p, h0, h1);
#pragma unroll
  for (int k = 0; k < 3; ++k) { h0[k] = scale_c(sc, h0[k]); h1[k] = scale_c(sc, h1[k]); }
  su3_dagmul(u, h0, w0);
  su3_dagmul(u, h1, w1);
}

// The backward hop of s in direction MU through global memory (plain kernel's second half).
template <int MU, bool DAG, GStore G, SStore SI, typename T>
__device__ __forceinline__ void bwd_hop_global(const Geom& geo, const GaugeRef& U, const SpinorRef& in, int s,
                                               const int c[4], cplx<T> acc[12]) {
  constexpr int SF = DAG ? +1 : -1;
  const int n = nbr_bwd(geo, s, c, MU);
  cplx<T> p[12];
  T sc = load_spinor_raw<SI, T>(in, geo.V, n, p);
  cplx<T> h0[3], h1[3];
  project<MU, -SF>(p, h0, h1);
  if (MU == 3 && geo.antiperiodic && c[3] == 0) sc = -sc;
  if constexpr (G == GStore::I16_12) sc = sc * (T)kQ16Inv;
  if (hop_scaled<G, SI>() || (MU == 3 && geo.antiperiodic)) {
#pragma unroll
    for (int k = 0; k < 3; ++k) { h0[k] = scale_c(sc, h0[k]); h1[k] = scale_c(sc, h1[k]); }
  }
  cplx<T> u[9];
  load_link_any<MU, DAG, G, SI, T>(U, geo.V, n, u);
  cplx<T> w0[3], w1[3];
  su3_dagmul(u, h0, w0);
  su3_dagmul(u, h1, w1);
  accumulate<MU, -SF>(acc, w0, w1);
}

// Shared-memory slots of the backward-hop terms: [mu][12 reals][TILE], one
// float per bank-consecutive thread.
struct StagedSmem {
  float w[2][12][kStagedTile];
};

template <int MU, bool DAG, GStore G, SStore SI, typename T>
__device__ __forceinline__ void staged_first_half(const Geom& geo, const GaugeRef& U, const SpinorRef& in, int s,
                                                  const int c[4], int base, int end, const cplx<T> pown[12],
                                                  T scown, cplx<T> acc[12], StagedSmem& sm) {
  cplx<T> u[9];
  load_link_any<MU, DAG, G, SI, T>(U, geo.V, s, u);
  fwd_hop_with<MU, DAG, G, SI, T>(geo, in, s, c, u, acc);
  const int f = nbr_fwd(geo, s, c, MU);
  if (f >= base && f < end) {
    cplx<T> w0[3], w1[3];
    bwd_term<MU, DAG, G, T>(pown, scown, u, w0, w1);
    const int t = s - base;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sm.w[MU][4 * k + 0][t] = (float)w0[k].re;
      sm.w[MU][4 * k + 1][t] = (float)w0[k].im;
      sm.w[MU][4 * k + 2][t] = (float)w1[k].re;
      sm.w[MU][4 * k + 3][t] = (float)w1[k].im;
    }
  }
}

template <int MU, bool DAG, GStore G, SStore SI, typename T>
__device__ __forceinline__ void staged_second_half(const Geom& geo, const GaugeRef& U, const SpinorRef& in, int s,
                                                   const int c[4], int base, int end, cplx<T> acc[12],
                                                   const StagedSmem& sm) {
  constexpr int SF = DAG ? +1 : -1;
  const int b = nbr_bwd(geo, s, c, MU);
  if (b >= base && b < end) {
    const int t = b - base;
    cplx<T> w0[3], w1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      w0[k] = {(T)sm.w[MU][4 * k + 0][t], (T)sm.w[MU][4 * k + 1][t]};
      w1[k] = {(T)sm.w[MU][4 * k + 2][t], (T)sm.w[MU][4 * k + 3][t]};
    }
    accumulate<MU, -SF>(acc, w0, w1);
  } else {
    bwd_hop_global<MU, DAG, G, SI, T>(geo, U, in, s, c, acc);
  }
}

// Grid-stride over tiles (one wave of resident blocks).  Two shared-memory buffers
// alternate between consecutive tiles of a block, so one barrier per tile suffices:
// a buffer is written again only two tiles later, after every thread has passed the
// barrier of the tile in between and so has finished reading it.
template <typename T, GStore G, SStore SI, bool DAG, class Epi>
__global__ void __launch_bounds__(kStagedTile, (EpiMinBlocks<T, Epi>::value))
    dslash_staged_kernel(Geom geo, GaugeRef U, SpinorRef in, T kappa, Epi epi, ReduceScratch rs) {
  if (epi.halted()) return;
  extern __shared__ float4 staged_dyn[];
  StagedSmem* bufs = reinterpret_cast<StagedSmem*>(staged_dyn);
  int parity = 0;
  double red[Epi::NRED];
#pragma unroll
  for (int q = 0; q < Epi::NRED; ++q) red[q] = 0.0;
  const int ntiles = (geo.V + kStagedTile - 1) / kStagedTile;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int base = tile * kStagedTile;
    const int end = min(base + kStagedTile, geo.V);
    const int s = base + (int)threadIdx.x;
    const bool valid = s < geo.V;
    StagedSmem& sm = bufs[parity];
    parity ^= 1;
    int c[4] = {0, 0, 0, 0};
    cplx<T> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {(T)0, (T)0};
    if (valid) {
      site_coords(geo, s, c);
      cplx<T> pown[12];
      T scown = load_spinor_raw<SI, T>(in, geo.V, s, pown);
      if constexpr (G == GStore::I16_12) scown = scown * (T)kQ16Inv;
      staged_first_half<0, DAG, G, SI, T>(geo, U, in, s, c, base, end, pown, scown, acc, sm);
      staged_first_half<1, DAG, G, SI, T>(geo, U, in, s, c, base, end, pown, scown, acc, sm);
    }
    __syncthreads();
    if (valid) {
      staged_second_half<0, DAG, G, SI, T>(geo, U, in, s, c, base, end, acc, sm);
      staged_second_half<1, DAG, G, SI, T>(geo, U, in, s, c, base, end, acc, sm);
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
  }
  if constexpr (Epi::REDUCE) {
    double tot[Epi::NRED];
    if (grid_sum<Epi::NRED>(red, rs, tot)) epi.finalize(tot);
  }
}

constexpr size_t kStagedSmemBytes = 2 * sizeof(StagedSmem);   // 48 KiB: opted in below

// Resident blocks of the staged kernel with its dynamic shared memory (once per kernel).
template <typename T, GStore G, SStore SI, bool DAG, class Epi>
int staged_wave() {
  auto kern = &dslash_staged_kernel<T, G, SI, DAG, Epi>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStagedSmemBytes);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStagedTile, kStagedSmemBytes);
  return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

template <typename T, GStore G, SStore SI, bool DAG, class Epi>
inline void launch_dslash_staged(const Geom& geo, GaugeRef U, SpinorRef in, double kappa, const Epi& epi,
                                 const ReduceScratch& rs, cudaStream_t stream) {
  static const int wave = staged_wave<T, G, SI, DAG, Epi>();
  const int grid = std::min(grid_for(geo.V, kStagedTile), wave);
  dslash_staged_kernel<T, G, SI, DAG, Epi><<<grid, kStagedTile, kStagedSmemBytes, stream>>>(geo, U, in, (T)kappa,
                                                                                            epi, rs);
}

}  // namespace lq
