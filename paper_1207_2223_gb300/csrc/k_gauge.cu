// Gauge-side kernels of the molecular dynamics (paper Sec. 3, kernels 2 and 4;
// Eq. 5): plaquettes and the Wilson gauge action, the gauge force fused with
// the momentum update, the link update U <- exp(i eps p) U with
// reunitarisation, and the kinetic-energy difference.  All FP64.
//
// Momenta and forces are stored site-major as double [32][V], entry
// (4 mu + ... ) -> index (8 mu + a) * V + site, for su(3) coefficient a.
#include "lq_internal.h"
#include "lq_su3.cuh"

namespace lq {

static constexpr int kBS = 256;

__device__ __forceinline__ double site_plaquettes(const double2* g, const Geom& geo, int s, const int c[4]) {
  double sum = 0.0;
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    const int xm = nbr_fwd(geo, s, c, mu);
    const M3 Umu = load_m3(g, geo.V, mu, s);
#pragma unroll 1
    for (int nu = mu + 1; nu < 4; ++nu) {
      const int xn = nbr_fwd(geo, s, c, nu);
      // Re tr(U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag) = Re tr[(U_mu(x) U_nu(x+mu)) (U_nu(x) U_mu(x+nu))^dag]
      const M3 a = mul(Umu, load_m3(g, geo.V, nu, xm));
      const M3 b = mul(load_m3(g, geo.V, nu, s), load_m3(g, geo.V, mu, xn));
      sum += re_tr_mul_dag(a, b);
    }
  }
  return sum;
}

// red[0] = sum_x sum_{mu<nu} Re tr U_P (gauge a);  red[1] = same minus for gauge b (when given)
__global__ void __launch_bounds__(kBS) plaquette_kernel(Geom geo, const double2* ga, const double2* gb,
                                                        ReduceScratch rs, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double red[2] = {0.0, 0.0};
  if (s < geo.V) {
    int c[4];
    site_coords(geo, s, c);
    const double pa = site_plaquettes(ga, geo, s, c);
    red[0] = pa;
    if (gb) red[1] = pa - site_plaquettes(gb, geo, s, c);
  }
  double tot[2];
  if (grid_sum<2>(red, rs, tot)) { out[0] = tot[0]; out[1] = tot[1]; }
}

// F_a(x, mu) = (beta/3) Im tr(t_a U_mu(x) Sigma_mu(x)), Sigma the six staples.
// UPDATE: p -= eps F, otherwise F is stored.
template <bool UPDATE>
__global__ void __launch_bounds__(kBS) gauge_force_kernel(Geom geo, const double2* g, double* f, double beta,
                                                          double eps) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * geo.V) return;
  const int mu = idx / geo.V, s = idx - mu * geo.V;
  int c[4];
  site_coords(geo, s, c);
  const int xm = nbr_fwd(geo, s, c, mu);
  int cm[4] = {c[0], c[1], c[2], c[3]};
  cm[mu] = (c[mu] + 1) % geo.L[mu];
  M3 S;
#pragma unroll
  for (int k = 0; k < 9; ++k) S.m[k] = {0.0, 0.0};
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int xn = nbr_fwd(geo, s, c, nu);
    const int xmn = nbr_bwd(geo, s, c, nu);          // x - nu
    const int xpm_mn = nbr_bwd(geo, xm, cm, nu);     // x + mu - nu
    // upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    M3 up = mul_dag(load_m3(g, geo.V, nu, xm), load_m3(g, geo.V, mu, xn));
    up = mul_dag(up, load_m3(g, geo.V, nu, s));
    add_to(S, up);
    // lower: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) = (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu)
    M3 lo = mul(load_m3(g, geo.V, mu, xmn), load_m3(g, geo.V, nu, xpm_mn));
    lo = dag_mul(lo, load_m3(g, geo.V, nu, xmn));
    add_to(S, lo);
  }
  const M3 W = mul(load_m3(g, geo.V, mu, s), S);
  double fa[8];
  im_tr_ta(W, fa);
  const double sc = beta / 3.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double* q = f + ((size_t)mu * 8 + a) * geo.V + s;
    if (UPDATE) *q -= eps * sc * fa[a];
    else *q = sc * fa[a];
  }
}

// U_mu(x) <- reunitarise(exp(i eps P) U_mu(x)), P = sum_a p_a t_a; the exponential by
// the Cayley-Hamilton closed form (lq_su3.cuh)
__global__ void __launch_bounds__(kBS) link_update_kernel(Geom geo, double2* g, const double* p, double eps) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * geo.V) return;
  const int mu = idx / geo.V, s = idx - mu * geo.V;
  double pa[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) pa[a] = p[((size_t)mu * 8 + a) * geo.V + s];
  const M3 E = expi_hermitian(eps_algebra(pa, eps));
  M3 U = mul(E, load_m3_rw(g, geo.V, mu, s));
  reunitarise(U);
  store_m3(g, geo.V, mu, s, U);
}

__global__ void __launch_bounds__(kBS) pack_mom_kernel(int V, const double* canon, double* soa) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int k = 0; k < 32; ++k) soa[(size_t)k * V + s] = canon[(size_t)s * 32 + k];
}
__global__ void __launch_bounds__(kBS) unpack_mom_kernel(int V, const double* soa, double* canon) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int k = 0; k < 32; ++k) canon[(size_t)s * 32 + k] = soa[(size_t)k * V + s];
}

// out[0] = (1/2) sum (p^2 - p0^2), per element, then summed
__global__ void __launch_bounds__(kBS) kinetic_diff_kernel(int V, const double* p, const double* p0,
                                                           ReduceScratch rs, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double red[1] = {0.0};
  if (s < V) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const double a = p[(size_t)k * V + s], b = p0[(size_t)k * V + s];
      red[0] += 0.5 * (a - b) * (a + b);
    }
  }
  double tot[1];
  if (grid_sum<1>(red, rs, tot)) out[0] = tot[0];
}

void launch_plaquette(const Geom& g, const void* ga, const void* gb, const ReduceScratch& rs, double* out,
                      cudaStream_t st) {
  plaquette_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g, static_cast<const double2*>(ga),
                                                       static_cast<const double2*>(gb), rs, out);
}
void launch_gauge_force(const Geom& g, const void* gauge, double* f, double beta, double eps, bool update,
                        cudaStream_t st) {
  const int grid = grid_for(4 * g.V, kBS);
  if (update) gauge_force_kernel<true><<<grid, kBS, 0, st>>>(g, static_cast<const double2*>(gauge), f, beta, eps);
  else gauge_force_kernel<false><<<grid, kBS, 0, st>>>(g, static_cast<const double2*>(gauge), f, beta, eps);
}
void launch_link_update(const Geom& g, void* gauge, const double* p, double eps, cudaStream_t st) {
  link_update_kernel<<<grid_for(4 * g.V, kBS), kBS, 0, st>>>(g, static_cast<double2*>(gauge), p, eps);
}
void launch_pack_mom(const Geom& g, const double* canon, double* soa, cudaStream_t st) {
  pack_mom_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, canon, soa);
}
void launch_unpack_mom(const Geom& g, const double* soa, double* canon, cudaStream_t st) {
  unpack_mom_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, soa, canon);
}
void launch_kinetic_diff(const Geom& g, const double* p, const double* p0, const ReduceScratch& rs, double* out,
                         cudaStream_t st) {
  kinetic_diff_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, p, p0, rs, out);
}

}  // namespace lq
