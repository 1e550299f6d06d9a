"""Conventions of the oracle (parity unpinned only where a test says so).

The paper fixes none of these (Sec. 3 mentions only that the gamma
matrices have few non-zero entries).  The readings taken:

* lattice Lx x Ly x Lz x Lt, mu = 0..3 = x, y, z, t, site
  s = x + Lx (y + Ly (z + Lz t));
* fermion boundary conditions periodic in x, y, z and antiperiodic in t:
  a hop across the t boundary, in either direction, carries a factor -1;
  gauge links are always periodic;
* gamma matrices in the DeGrand-Rossi basis; gamma_5 = g_x g_y g_z g_t;
* su(3) generators t_a = lambda_a / sqrt(2) (Gell-Mann lambda), so
  tr(t_a t_b) = delta_ab and (1/2) tr p^2 = (1/2) sum_a p_a^2 (Eq. 5).
"""
import numpy as np

_i = 1j
GAMMA = np.array([
    # gamma_x
    [[0, 0, 0, _i], [0, 0, _i, 0], [0, -_i, 0, 0], [-_i, 0, 0, 0]],
    # gamma_y
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    # gamma_z
    [[0, 0, _i, 0], [0, 0, 0, -_i], [-_i, 0, 0, 0], [0, _i, 0, 0]],
    # gamma_t
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)

_s2 = 1.0 / np.sqrt(2.0)
_s6 = 1.0 / np.sqrt(6.0)
GELL_MANN = np.array([
    [[0, 1, 0], [1, 0, 0], [0, 0, 0]],
    [[0, -_i, 0], [_i, 0, 0], [0, 0, 0]],
    [[1, 0, 0], [0, -1, 0], [0, 0, 0]],
    [[0, 0, 1], [0, 0, 0], [1, 0, 0]],
    [[0, 0, -_i], [0, 0, 0], [_i, 0, 0]],
    [[0, 0, 0], [0, 0, 1], [0, 1, 0]],
    [[0, 0, 0], [0, 0, -_i], [0, _i, 0]],
    [[1, 0, 0], [0, 1, 0], [0, 0, -2]],
], dtype=np.complex128)
GELL_MANN[7] *= 1.0 / np.sqrt(3.0)
T = GELL_MANN * _s2          # t_a, a = 0..7


def volume(dims):
    return int(np.prod(dims))


def coords(dims):
    """(V, 4) coordinates of every site in canonical order."""
    Lx, Ly, Lz, Lt = dims
    s = np.arange(volume(dims))
    return np.stack([s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)], axis=1)


def site_index(c, dims):
    Lx, Ly, Lz, Lt = dims
    return c[..., 0] + Lx * (c[..., 1] + Ly * (c[..., 2] + Lz * c[..., 3]))


def neighbours(dims, t_antiperiodic=True):
    """Forward / backward neighbour indices and fermion hop signs.

    Returns (fwd, bwd, sf, sb), each (4, V): fwd[mu][s] is the index of
    s + mu-hat, bwd[mu][s] of s - mu-hat; sf, sb are the +-1 factors the
    fermion hop s -> s +- mu-hat carries (-1 only across the t boundary
    when t_antiperiodic).
    """
    c = coords(dims)
    V = c.shape[0]
    fwd = np.empty((4, V), dtype=np.int64)
    bwd = np.empty((4, V), dtype=np.int64)
    sf = np.ones((4, V))
    sb = np.ones((4, V))
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (c[:, mu] + 1) % dims[mu]
        cb = c.copy()
        cb[:, mu] = (c[:, mu] - 1) % dims[mu]
        fwd[mu] = site_index(cf, dims)
        bwd[mu] = site_index(cb, dims)
        if mu == 3 and t_antiperiodic:
            sf[mu, c[:, 3] == dims[3] - 1] = -1.0
            sb[mu, c[:, 3] == 0] = -1.0
    return fwd, bwd, sf, sb


def dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))
