// Double-float reliable updates of the batched solver (the CG routine of
// Sec. 3 over a batch of systems, with the intermediate true residuals of the
// mixed-precision iteration in double-float arithmetic as for a single solve):
//   x_df += x_lo, x_lo = 0;   per column: tmp = M x_df, r = phi - M^dag tmp
// Each column is one launch of the two-threads-per-site double-float operator
// on its own lattice, its elements addressed through the batch layout (chunk
// stride = the batch's element count, sites from the column's first element).
// The column's |r|^2 goes through the same per-column rule as the FP64 update
// (freeze at the tolerance, restart on drift); a batch whose columns are all
// frozen is then certified in FP64, which reopens any column the double-float
// estimate froze too early.
#include "lq_batch.cuh"
#include "lq_dfsplit.cuh"

namespace lq {

namespace {

constexpr int kBS = 256;

// x_df += x_lo; x_lo = 0
template <SStore S>
__global__ void __launch_bounds__(kBS) batch_accumulate_df_kernel(int total, SpinorRef xlo, SpinorRef xdf) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    cplx<float> a[12], z[12];
    cplx<df64> b[12];
    load_spinor<xlo_store(S), float, false>(xlo, total, e, a);
    load_spinor<SStore::DF64, df64, false>(xdf, total, e, b);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      b[k] = {b[k].re + df64(a[k].re), b[k].im + df64(a[k].im)};
      z[k] = {0.f, 0.f};
    }
    store_spinor<SStore::DF64, df64>(xdf, total, e, b);
    store_spinor<xlo_store(S), float>(xlo, total, e, z);
  }
}

// a column's |r|^2 after its double-float update
struct DFFinBatch {
  BatchState* st;
  int col;
  __device__ void operator()(double rr) const {
    reliable_update_column(st, col, rr);
    st->iter_since_ru = 0;
    st->halt = 0;
  }
};

template <SStore S>
void tail(const BatchDfArgs& a, const BatchDesc& bd, cudaStream_t st) {
  const int grid = std::max(1, std::min((bd.total + kBS - 1) / kBS, a.flat_grid));
  if (a.accumulate) batch_accumulate_df_kernel<S><<<grid, kBS, 0, st>>>(bd.total, a.xlo, a.xdf);
  if (!a.residual) return;
  const ReduceScratch rs{a.br.partials, a.br.ticket, a.br.max_blocks};
  for (int k = 0; k < bd.nsys; ++k) {
    const SysDesc& sd = bd.sys[k];
    for (int r = 0; r < sd.R; ++r) {
      const int off = sd.off + r * sd.geo.V;
      launch_dslash_dfsplit<false>(sd.geo, a.gauge_df[k], a.xdf, sd.kappa, DFEpiStore{a.tmpdf}, rs, st, bd.total,
                                   off, a.prefetch);
      DFEpiResidual<S, DFFinBatch, false> e1{a.phidf, SpinorRef{nullptr, nullptr}, a.rlo,
                                             DFFinBatch{a.st, sd.col + r}};
      launch_dslash_dfsplit<true>(sd.geo, a.gauge_df[k], a.tmpdf, sd.kappa, e1, rs, st, bd.total, off, a.prefetch);
    }
  }
}

}  // namespace

void batch_df_tail(const BatchDfArgs& a, const BatchDesc& bd, SStore s, cudaStream_t st) {
  switch (s) {
    case SStore::F16: tail<SStore::F16>(a, bd, st); break;
    case SStore::BF16: tail<SStore::BF16>(a, bd, st); break;
    case SStore::I16: tail<SStore::I16>(a, bd, st); break;
    default: tail<SStore::F32>(a, bd, st); break;
  }
}

}  // namespace lq
