// Fermion force (paper Sec. 3, kernel 3: the driving force of the fermion
// fields, fused with the momentum evolution), and the pseudofermion-action
// difference used in Delta H (Eq. 5).  FP64.
//
// With X = (M^dag M)^{-1} phi and Y = M X, the derivative of
// S_f = phi^dag (M^dag M)^{-1} phi under U_mu(x) -> exp(i w t_a) U_mu(x) is
//   F_a(x, mu) = 2 kappa s Im tr(t_a Q),
//   Q = sum_spin [ X(x) (U (1 + g_mu) Y(x+mu))^dag - U X(x+mu) ((1 - g_mu) Y(x))^dag ],
// s the sign of the hop x -> x+mu.  (1 -+ g_mu) has rank 2, so each spin sum
// reduces to two colour outer products of projected half spinors
// (sum_spin conj(((1+S g) a)_s) b_s = conj(h(a)_0) h(b)_0 + conj(h(a)_1) h(b)_1,
// h = the two independent components of the projection), which is the
// paper's observation that the gamma algebra leaves few non-zero terms.
#include "lq_internal.h"
#include "lq_su3.cuh"

namespace lq {

static constexpr int kBS = 256;

template <int MU>
__device__ __forceinline__ M3 force_matrix(const cplx<double> Xx[12], const cplx<double> Yx[12],
                                           const cplx<double> Xf[12], const cplx<double> Yf[12], const M3& U) {
  cplx<double> a0[3], a1[3], b0[3], b1[3];
  M3 Q;
#pragma unroll
  for (int k = 0; k < 9; ++k) Q.m[k] = {0.0, 0.0};
  // A = sum_k (U h(X(x+mu))_k) h(Y(x))_k^dag with (1 - g_mu)
  project<MU, -1>(Xf, a0, a1);
  project<MU, -1>(Yx, b0, b1);
  cplx<double> u0[3], u1[3];
  su3_mul(U.m, a0, u0);
  su3_mul(U.m, a1, u1);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<double> t = cjmul(b0[j], u0[i]);       // u0_i conj(b0_j)
      t = cjmadd(t, b1[j], u1[i]);
      Q.m[3 * i + j] = Q.m[3 * i + j] - t;
    }
  // B = sum_k h(X(x))_k (U h(Y(x+mu))_k)^dag with (1 + g_mu)
  project<MU, +1>(Xx, a0, a1);
  project<MU, +1>(Yf, b0, b1);
  su3_mul(U.m, b0, u0);
  su3_mul(U.m, b1, u1);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<double> t = cjmul(u0[j], a0[i]);       // a0_i conj((U b0)_j)
      t = cjmadd(t, u1[j], a1[i]);
      Q.m[3 * i + j] = Q.m[3 * i + j] + t;
    }
  return Q;
}

template <bool UPDATE>
__global__ void __launch_bounds__(kBS) fermion_force_kernel(Geom geo, const double2* g, SpinorRef X, SpinorRef Y,
                                                            double* f, double kappa, double eps) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * geo.V) return;
  const int mu = idx / geo.V, s = idx - mu * geo.V;
  int c[4];
  site_coords(geo, s, c);
  const int xf = nbr_fwd(geo, s, c, mu);
  const double sign = (mu == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1) ? -1.0 : 1.0;
  cplx<double> Xx[12], Yx[12], Xf[12], Yf[12];
  load_spinor<SStore::F64, double>(X, geo.V, s, Xx);
  load_spinor<SStore::F64, double>(Y, geo.V, s, Yx);
  load_spinor<SStore::F64, double>(X, geo.V, xf, Xf);
  load_spinor<SStore::F64, double>(Y, geo.V, xf, Yf);
  const M3 U = load_m3(g, geo.V, mu, s);
  M3 Q;
  switch (mu) {
    case 0: Q = force_matrix<0>(Xx, Yx, Xf, Yf, U); break;
    case 1: Q = force_matrix<1>(Xx, Yx, Xf, Yf, U); break;
    case 2: Q = force_matrix<2>(Xx, Yx, Xf, Yf, U); break;
    default: Q = force_matrix<3>(Xx, Yx, Xf, Yf, U); break;
  }
  double fa[8];
  im_tr_ta(Q, fa);
  const double sc = 2.0 * kappa * sign;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    double* q = f + ((size_t)mu * 8 + a) * geo.V + s;
    if (UPDATE) *q -= eps * sc * fa[a];
    else *q = sc * fa[a];
  }
}

// out[0] = sum_x [ Re phi(x)^dag X(x) - |chi(x)|^2 ]
__global__ void __launch_bounds__(kBS) fermion_action_diff_kernel(int V, SpinorRef phi, SpinorRef X, SpinorRef chi,
                                                                  ReduceScratch rs, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double red[1] = {0.0};
  if (s < V) {
    cplx<double> a[12], b[12], c[12];
    load_spinor<SStore::F64, double>(phi, V, s, a);
    load_spinor<SStore::F64, double>(X, V, s, b);
    load_spinor<SStore::F64, double>(chi, V, s, c);
#pragma unroll
    for (int k = 0; k < 12; ++k) red[0] += (a[k].re * b[k].re + a[k].im * b[k].im) - norm2(c[k]);
  }
  double tot[1];
  if (grid_sum<1>(red, rs, tot)) out[0] = tot[0];
}

// Complex gradient of S_f with respect to the entries of U_mu(x) in the
// convention dS = Re sum conj(G) dU (that of torch.autograd):
//   G = conj(2 kappa s C),  C_ij = sum_spin conj(((1 - g_mu) Y(x))_i) X(x+mu)_j
//                                + sum_spin conj(X(x)_i) ((1 + g_mu) Y(x+mu))_j,
// each spin sum again over the two half-spinor components.  G is written in
// the canonical layout [V][4][3][3] complex.
template <int MU>
__device__ __forceinline__ M3 grad_matrix(const cplx<double> Xx[12], const cplx<double> Yx[12],
                                          const cplx<double> Xf[12], const cplx<double> Yf[12]) {
  cplx<double> a0[3], a1[3], b0[3], b1[3];
  M3 C;
  project<MU, -1>(Yx, a0, a1);
  project<MU, -1>(Xf, b0, b1);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<double> t = cjmul(a0[i], b0[j]);
      C.m[3 * i + j] = cjmadd(t, a1[i], b1[j]);
    }
  project<MU, +1>(Xx, a0, a1);
  project<MU, +1>(Yf, b0, b1);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<double> t = cjmadd(C.m[3 * i + j], a0[i], b0[j]);
      C.m[3 * i + j] = cjmadd(t, a1[i], b1[j]);
    }
  return C;
}

__global__ void __launch_bounds__(kBS) fermion_grad_kernel(Geom geo, SpinorRef X, SpinorRef Y, double2* G,
                                                           double kappa) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * geo.V) return;
  const int mu = idx / geo.V, s = idx - mu * geo.V;
  int c[4];
  site_coords(geo, s, c);
  const int xf = nbr_fwd(geo, s, c, mu);
  const double sign = (mu == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1) ? -1.0 : 1.0;
  cplx<double> Xx[12], Yx[12], Xf[12], Yf[12];
  load_spinor<SStore::F64, double>(X, geo.V, s, Xx);
  load_spinor<SStore::F64, double>(Y, geo.V, s, Yx);
  load_spinor<SStore::F64, double>(X, geo.V, xf, Xf);
  load_spinor<SStore::F64, double>(Y, geo.V, xf, Yf);
  M3 C;
  switch (mu) {
    case 0: C = grad_matrix<0>(Xx, Yx, Xf, Yf); break;
    case 1: C = grad_matrix<1>(Xx, Yx, Xf, Yf); break;
    case 2: C = grad_matrix<2>(Xx, Yx, Xf, Yf); break;
    default: C = grad_matrix<3>(Xx, Yx, Xf, Yf); break;
  }
  const double sc = 2.0 * kappa * sign;
  double2* out = G + ((size_t)s * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) out[k] = make_double2(sc * C.m[k].re, -sc * C.m[k].im);
}

// out[0] = sum_x Re phi(x)^dag X(x)
__global__ void __launch_bounds__(kBS) dot_re_kernel(int V, SpinorRef a, SpinorRef b, ReduceScratch rs,
                                                     double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double red[1] = {0.0};
  if (s < V) {
    cplx<double> u[12], v[12];
    load_spinor<SStore::F64, double>(a, V, s, u);
    load_spinor<SStore::F64, double>(b, V, s, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) red[0] += u[k].re * v[k].re + u[k].im * v[k].im;
  }
  double tot[1];
  if (grid_sum<1>(red, rs, tot)) out[0] = tot[0];
}

void launch_fermion_grad(const Geom& g, SpinorRef X, SpinorRef Y, double* G, double kappa, cudaStream_t st) {
  fermion_grad_kernel<<<grid_for(4 * g.V, kBS), kBS, 0, st>>>(g, X, Y, reinterpret_cast<double2*>(G), kappa);
}
void launch_dot_re(const Geom& g, SpinorRef a, SpinorRef b, const ReduceScratch& rs, double* out, cudaStream_t st) {
  dot_re_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, a, b, rs, out);
}

void launch_fermion_force(const Geom& g, const void* gauge, SpinorRef X, SpinorRef Y, double* f, double kappa,
                          double eps, bool update, cudaStream_t st) {
  const int grid = grid_for(4 * g.V, kBS);
  const double2* gp = static_cast<const double2*>(gauge);
  if (update) fermion_force_kernel<true><<<grid, kBS, 0, st>>>(g, gp, X, Y, f, kappa, eps);
  else fermion_force_kernel<false><<<grid, kBS, 0, st>>>(g, gp, X, Y, f, kappa, eps);
}
void launch_fermion_action_diff(const Geom& g, SpinorRef phi, SpinorRef X, SpinorRef chi, const ReduceScratch& rs,
                                double* out, cudaStream_t st) {
  fermion_action_diff_kernel<<<grid_for(g.V, kBS), kBS, 0, st>>>(g.V, phi, X, chi, rs, out);
}

}  // namespace lq
