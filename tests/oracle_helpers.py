"""Dense brute-force constructions used to pin the oracle on tiny lattices.

These build the Wilson matrix entry by entry from explicit coordinate
loops (independent of the vectorised oracle code) and provide dense
algebra for solves and spectra.
"""
import numpy as np

from oracle.conventions import GAMMA


def dense_wilson_loops(U, dims, kappa, t_antiperiodic=True):
    """Dense M = 1 - kappa H, index (site*12 + spin*3 + colour), built by loops."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    N = 12 * V
    M = np.eye(N, dtype=np.complex128)
    I4 = np.eye(4)

    def idx(x, y, z, t):
        return x + Lx * (y + Ly * (z + Lz * t))

    for t in range(Lt):
        for z in range(Lz):
            for y in range(Ly):
                for x in range(Lx):
                    s = idx(x, y, z, t)
                    c = [x, y, z, t]
                    for mu in range(4):
                        up = list(c)
                        up[mu] = (c[mu] + 1) % dims[mu]
                        dn = list(c)
                        dn[mu] = (c[mu] - 1) % dims[mu]
                        sf = -1.0 if (mu == 3 and t_antiperiodic and c[3] == Lt - 1) else 1.0
                        sb = -1.0 if (mu == 3 and t_antiperiodic and c[3] == 0) else 1.0
                        f = idx(*up)
                        b = idx(*dn)
                        M[12 * s:12 * s + 12, 12 * f:12 * f + 12] += \
                            -kappa * sf * np.kron(I4 - GAMMA[mu], U[s, mu])
                        M[12 * s:12 * s + 12, 12 * b:12 * b + 12] += \
                            -kappa * sb * np.kron(I4 + GAMMA[mu], np.conj(U[b, mu]).T)
    return M


def dense_from_operator(op, V):
    """Columns of a linear operator on (V, 4, 3) spinors."""
    N = 12 * V
    cols = []
    for j in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[j] = 1.0
        cols.append(op(e.reshape(V, 4, 3)).reshape(N))
    return np.array(cols).T
