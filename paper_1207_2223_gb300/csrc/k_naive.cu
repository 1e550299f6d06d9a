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

}  // namespace lq
