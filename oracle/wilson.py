"""Wilson-Dirac operator in hopping-parameter form (Eq. 4, Sec. 3 kernel 1).

The paper writes M = D + m (Eq. 4) and applies M and M^dag to the
pseudofermion field inside CG (Sec. 3, kernel 1).  Reading taken (r = 1,
hopping-parameter normalisation, i.e. 2 kappa (D + m) with
m = 1/(2 kappa) - 4):

    (H psi)(x) = sum_mu [ (1 - g_mu) U_mu(x)        psi(x + mu) s_f
                        + (1 + g_mu) U_mu(x - mu)^dag psi(x - mu) s_b ]
    M = 1 - kappa H

and M^dag is the adjoint of that matrix: the projectors of the two hops
swap, (1 + g_mu) forward and (1 - g_mu) backward.  The overall scale of M
cancels from the HMC (phi = M^dag chi scales with it).
"""
import numpy as np

from .conventions import GAMMA, ONE4, neighbours, volume


def hopping(U, psi, dims, t_antiperiodic=True, dagger=False, sites=None, nbr=None):
    """H psi (or H^dag psi) at ``sites`` (all sites when None).

    U: complex (V, 4, 3, 3); psi: complex (V, 4, 3).  Returns (n, 4, 3).
    """
    fwd, bwd, sf, sb = nbr if nbr is not None else neighbours(dims, t_antiperiodic)
    if sites is None:
        sites = np.arange(volume(dims))
    out = np.zeros((len(sites), 4, 3), dtype=np.complex128)
    for mu in range(4):
        f = fwd[mu][sites]
        b = bwd[mu][sites]
        Uf = U[sites, mu]                       # U_mu(x)
        Ub = U[b, mu]                           # U_mu(x - mu)
        # U psi: sum_b U[a, b] psi[s, b]  ->  psi @ U^T
        hop_f = np.matmul(psi[f], np.swapaxes(Uf, -1, -2)) * sf[mu][sites][:, None, None]
        # U^dag psi: sum_b conj(U[b, a]) psi[s, b]  ->  psi @ conj(U)
        hop_b = np.matmul(psi[b], np.conj(Ub)) * sb[mu][sites][:, None, None]
        pm = ONE4 - GAMMA[mu]
        pp = ONE4 + GAMMA[mu]
        if not dagger:
            out += np.matmul(pm, hop_f) + np.matmul(pp, hop_b)
        else:
            out += np.matmul(pp, hop_f) + np.matmul(pm, hop_b)
    return out


def apply_M(U, psi, dims, kappa, t_antiperiodic=True, dagger=False, sites=None, nbr=None):
    """M psi = psi - kappa H psi   (M^dag psi when dagger)."""
    h = hopping(U, psi, dims, t_antiperiodic, dagger, sites, nbr)
    base = psi if sites is None else psi[sites]
    return base - kappa * h


def apply_MdagM(U, psi, dims, kappa, t_antiperiodic=True, nbr=None):
    nbr = nbr if nbr is not None else neighbours(dims, t_antiperiodic)
    t = apply_M(U, psi, dims, kappa, t_antiperiodic, False, None, nbr)
    return apply_M(U, t, dims, kappa, t_antiperiodic, True, None, nbr)


def apply_MdagM_sites(U, psi, dims, kappa, sites, t_antiperiodic=True):
    """(M^dag M psi) at ``sites`` only, shape (n, 4, 3).

    M^dag M psi at x needs M psi at x and at its eight neighbours, and those need
    psi up to two hops away.  M psi is evaluated on that one-hop neighbourhood
    only (by ``apply_M`` with ``sites``), placed in an otherwise zero field, and
    M^dag is applied to it at ``sites``: the same numbers as the full-lattice
    ``apply_MdagM`` at those sites, at a cost that grows with the sample, not
    with the lattice.
    """
    nbr = neighbours(dims, t_antiperiodic)
    fwd, bwd = nbr[0], nbr[1]
    sites = np.asarray(sites)
    ring = np.unique(np.concatenate([sites] + [fwd[mu][sites] for mu in range(4)] +
                                    [bwd[mu][sites] for mu in range(4)]))
    t = np.zeros_like(psi)
    t[ring] = apply_M(U, psi, dims, kappa, t_antiperiodic, False, ring, nbr)
    return apply_M(U, t, dims, kappa, t_antiperiodic, True, sites, nbr)
