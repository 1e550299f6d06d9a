// A deliberately naive Wilson operator, for the ablation of the paper's
// central observation (Sec. 3 and 4: keeping run-time arrays in registers
// instead of global memory sped their kernels up about fivefold).  It is
// written the way a direct port of array-based CPU code runs on a GPU:
//   - the canonical array-of-structures layout ([site][mu][3][3] links,
//     [site][spin][colour] spinors), one thread per site;
//   - a neighbour table and its boundary signs stored in global memory;
//   - (1 -+ gamma_mu) applied as a dense 4x4 spin matrix, all 16 entries;
//   - the result accumulated through global memory (a volatile output
//     array), as the unscalarised arrays of the paper's first version were.
// It is correct (tested against the oracle) and only meant to be timed
// against dslash_kernel.
#include <cmath>

#include "lq_internal.h"

namespace lq {

// (1 - g_mu) and (1 + g_mu), DeGrand-Rossi basis, complex entries (re, im)
__constant__ double2 c_proj[2][4][16];

static const double kGamma[4][4][4][2] = {
    {{{0, 0}, {0, 0}, {0, 0}, {0, 1}}, {{0, 0}, {0, 0}, {0, 1}, {0, 0}},
     {{0, 0}, {0, -1}, {0, 0}, {0, 0}}, {{0, -1}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 0}, {-1, 0}}, {{0, 0}, {0, 0}, {1, 0}, {0, 0}},
     {{0, 0}, {1, 0}, {0, 0}, {0, 0}}, {{-1, 0}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {0, -1}},
     {{0, -1}, {0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 1}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {1, 0}},
     {{1, 0}, {0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {1, 0}, {0, 0}, {0, 0}}}};

__global__ void naive_neighbours_kernel(Geom geo, int* nbr, double* sgn) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= geo.V) return;
  int c[4];
  site_coords(geo, s, c);
  for (int mu = 0; mu < 4; ++mu) {
    nbr[(2 * mu) * geo.V + s] = nbr_fwd(geo, s, c, mu);
    nbr[(2 * mu + 1) * geo.V + s] = nbr_bwd(geo, s, c, mu);
    sgn[(2 * mu) * geo.V + s] = (mu == 3 && geo.antiperiodic && c[3] == geo.L[3] - 1) ? -1.0 : 1.0;
    sgn[(2 * mu + 1) * geo.V + s] = (mu == 3 && geo.antiperiodic && c[3] == 0) ? -1.0 : 1.0;
  }
}

__global__ void naive_dslash_kernel(int V, const int* nbr, const double* sgn, const double2* U, const double2* in,
                                    volatile double* out, double kappa, int dagger) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int k = 0; k < 12; ++k) {
    out[2 * ((size_t)s * 12 + k)] = in[(size_t)s * 12 + k].x;
    out[2 * ((size_t)s * 12 + k) + 1] = in[(size_t)s * 12 + k].y;
  }
  for (int mu = 0; mu < 4; ++mu) {
    for (int dir = 0; dir < 2; ++dir) {
      const int n = nbr[(2 * mu + dir) * V + s];
      const double eta = -kappa * sgn[(2 * mu + dir) * V + s];
      // forward hop: (1 - g) U_mu(x) psi(x+mu); backward: (1 + g) U_mu(x-mu)^dag psi(x-mu); dagger swaps
      const int which = (dir == 0) ? (dagger ? 1 : 0) : (dagger ? 0 : 1);
      const int lk = dir == 0 ? s : n;
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i)
          for (int b = 0; b < 4; ++b) {
            const double2 P = c_proj[which][mu][4 * a + b];
            if (P.x == 0.0 && P.y == 0.0) continue;
            for (int j = 0; j < 3; ++j) {
              const double2 u = dir == 0 ? U[((size_t)lk * 4 + mu) * 9 + 3 * i + j]
                                         : make_double2(U[((size_t)lk * 4 + mu) * 9 + 3 * j + i].x,
                                                        -U[((size_t)lk * 4 + mu) * 9 + 3 * j + i].y);
              const double2 v = in[(size_t)n * 12 + 3 * b + j];
              const double2 uv = make_double2(u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x);
              const double2 t = make_double2(P.x * uv.x - P.y * uv.y, P.x * uv.y + P.y * uv.x);
              const size_t o = 2 * ((size_t)s * 12 + 3 * a + i);
              out[o] = out[o] + eta * t.x;
              out[o + 1] = out[o + 1] + eta * t.y;
            }
          }
    }
  }
}

// t_a = lambda_a / sqrt(2) (Gell-Mann matrices), row-major complex entries
__constant__ double2 c_ta[8][9];

// The fermion force of k_force.cu written the same naive way, for the force half
// of the ablation: one thread per link (x, mu) in the canonical order, Y and X
// read as full four-spinors from the array-of-structures layout, (1 -+ g_mu)
// applied as dense 4x4 spin matrices, the colour matrix
//   Q = sum_spin [ X(x) (U (1 + g_mu) Y(x+mu))^dag - U X(x+mu) ((1 - g_mu) Y(x))^dag ]
// accumulated in a global scratch array, and F_a = 2 kappa s Im tr(t_a Q) formed
// with dense t_a.  F: canonical [V][4][8].
__global__ void naive_force_kernel(int V, const int* nbr, const double* sgn, const double2* U, const double2* X,
                                   const double2* Y, volatile double* Q, double* F, double kappa) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 4 * V) return;
  const int s = idx / 4, mu = idx - 4 * s;
  const int n = nbr[(2 * mu) * V + s];
  const double sign = sgn[(2 * mu) * V + s];
  volatile double* q = Q + (size_t)idx * 18;
  for (int k = 0; k < 18; ++k) q[k] = 0.0;
  const double2* u = U + ((size_t)s * 4 + mu) * 9;
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < 3; ++j) {
      // w = (U (1 + g_mu) Y(x+mu))_{a j}
      double2 w = make_double2(0.0, 0.0);
      for (int b = 0; b < 4; ++b) {
        const double2 P = c_proj[1][mu][4 * a + b];
        for (int k = 0; k < 3; ++k) {
          const double2 uk = u[3 * j + k], y = Y[(size_t)n * 12 + 3 * b + k];
          const double2 uy = make_double2(uk.x * y.x - uk.y * y.y, uk.x * y.y + uk.y * y.x);
          w.x += P.x * uy.x - P.y * uy.y;
          w.y += P.x * uy.y + P.y * uy.x;
        }
      }
      for (int i = 0; i < 3; ++i) {
        const double2 xv = X[(size_t)s * 12 + 3 * a + i];
        q[2 * (3 * i + j)] = q[2 * (3 * i + j)] + (xv.x * w.x + xv.y * w.y);
        q[2 * (3 * i + j) + 1] = q[2 * (3 * i + j) + 1] + (xv.y * w.x - xv.x * w.y);
      }
    }
  for (int a = 0; a < 4; ++a)
    for (int j = 0; j < 3; ++j) {
      // v = ((1 - g_mu) Y(x))_{a j}
      double2 v = make_double2(0.0, 0.0);
      for (int b = 0; b < 4; ++b) {
        const double2 P = c_proj[0][mu][4 * a + b], y = Y[(size_t)s * 12 + 3 * b + j];
        v.x += P.x * y.x - P.y * y.y;
        v.y += P.x * y.y + P.y * y.x;
      }
      for (int i = 0; i < 3; ++i) {
        double2 ux = make_double2(0.0, 0.0);   // (U X(x+mu))_{a i}
        for (int k = 0; k < 3; ++k) {
          const double2 uk = u[3 * i + k], xv = X[(size_t)n * 12 + 3 * a + k];
          ux.x += uk.x * xv.x - uk.y * xv.y;
          ux.y += uk.x * xv.y + uk.y * xv.x;
        }
        q[2 * (3 * i + j)] = q[2 * (3 * i + j)] - (ux.x * v.x + ux.y * v.y);
        q[2 * (3 * i + j) + 1] = q[2 * (3 * i + j) + 1] - (ux.y * v.x - ux.x * v.y);
      }
    }
  for (int b = 0; b < 8; ++b) {
    double im = 0.0;   // Im tr(t_b Q) = Im sum_ij t_ij Q_ji
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double2 t = c_ta[b][3 * i + j];
        im += t.x * q[2 * (3 * j + i) + 1] + t.y * q[2 * (3 * j + i)];
      }
    F[(size_t)idx * 8 + b] = 2.0 * kappa * sign * im;
  }
}

static bool g_proj_set[64] = {};

void naive_setup(lq_ctx* c, int** nbr, double** sgn) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_proj_set[dev]) {
    double2 h[2][4][16];
    for (int mu = 0; mu < 4; ++mu)
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          const double one = a == b ? 1.0 : 0.0;
          h[0][mu][4 * a + b] = make_double2(one - kGamma[mu][a][b][0], -kGamma[mu][a][b][1]);
          h[1][mu][4 * a + b] = make_double2(one + kGamma[mu][a][b][0], kGamma[mu][a][b][1]);
        }
    cudaMemcpyToSymbol(c_proj, h, sizeof(h));
    const double r = 1.0 / std::sqrt(2.0), r3 = 1.0 / std::sqrt(6.0);
    double2 t[8][9] = {};
    t[0][1] = t[0][3] = make_double2(r, 0.0);                                   // lambda_1
    t[1][1] = make_double2(0.0, -r); t[1][3] = make_double2(0.0, r);            // lambda_2
    t[2][0] = make_double2(r, 0.0); t[2][4] = make_double2(-r, 0.0);            // lambda_3
    t[3][2] = t[3][6] = make_double2(r, 0.0);                                   // lambda_4
    t[4][2] = make_double2(0.0, -r); t[4][6] = make_double2(0.0, r);            // lambda_5
    t[5][5] = t[5][7] = make_double2(r, 0.0);                                   // lambda_6
    t[6][5] = make_double2(0.0, -r); t[6][7] = make_double2(0.0, r);            // lambda_7
    t[7][0] = t[7][4] = make_double2(r3, 0.0); t[7][8] = make_double2(-2.0 * r3, 0.0);   // lambda_8
    cudaMemcpyToSymbol(c_ta, t, sizeof(t));
    g_proj_set[dev] = true;
  }
  naive_neighbours_kernel<<<grid_for(c->geo.V, 256), 256, 0, c->stream>>>(c->geo, *nbr, *sgn);
}

void launch_naive_dslash(lq_ctx* c, const int* nbr, const double* sgn, const double* Ucanon, const double* in,
                         double* out, double kappa, int dagger) {
  naive_dslash_kernel<<<grid_for(c->geo.V, 128), 128, 0, c->stream>>>(
      c->geo.V, nbr, sgn, reinterpret_cast<const double2*>(Ucanon), reinterpret_cast<const double2*>(in),
      reinterpret_cast<volatile double*>(out), kappa, dagger);
}

void launch_naive_force(lq_ctx* c, const int* nbr, const double* sgn, const double* Ucanon, const double* X,
                        const double* Y, double* Q, double* F, double kappa) {
  naive_force_kernel<<<grid_for(4 * c->geo.V, 128), 128, 0, c->stream>>>(
      c->geo.V, nbr, sgn, reinterpret_cast<const double2*>(Ucanon), reinterpret_cast<const double2*>(X),
      reinterpret_cast<const double2*>(Y), reinterpret_cast<volatile double*>(Q), F, kappa);
}

}  // namespace lq
