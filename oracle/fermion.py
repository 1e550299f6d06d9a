"""Pseudofermion action and fermion force (Eq. 3-5; Sec. 3 kernel 3).

S_f = phi^dag (M^dag M)^{-1} phi (Eq. 4, 5).  With X = (M^dag M)^{-1} phi
and Y = M X, differentiating under U_mu(x) -> exp(i omega_a t_a) U_mu(x)
gives dS_f = -X^dag d(M^dag M) X = -2 Re Y^dag dM X = 2 kappa Re Y^dag dH X,
and only the two hops through link (x, mu) depend on it:

  F_a(x, mu) = 2 kappa Re[ i Y(x)^dag (1 - g_mu) t_a U_mu(x) X(x+mu) s
                         - i Y(x+mu)^dag (1 + g_mu) U_mu(x)^dag t_a X(x) s ]

with s the fermion sign of the hop x -> x+mu.  ``fermion_force_from_X``
takes X as given; ``fermion_force`` solves for it first.

The complex gradient of S_f with respect to the entries of U (the
convention of torch.autograd for a real function of complex inputs,
dS = Re sum conj(G) dU) is G = conj(C),
C = 2 kappa s [ ((1 - g_mu) Y(x))^H X(x+mu) + X(x)^H ((1 + g_mu) Y(x+mu)) ]
as 3x3 colour matrices (spin summed).
"""
import numpy as np

from .cg import cg_MdagM
from .conventions import GAMMA, ONE4, T, neighbours
from .wilson import apply_M


def pseudofermion_action(U, phi, dims, kappa, tol=1e-10, t_antiperiodic=True):
    X, _, _ = cg_MdagM(U, phi, dims, kappa, tol, t_antiperiodic=t_antiperiodic)
    return float(np.vdot(phi, X).real)


def fermion_force_from_X(U, X, dims, kappa, t_antiperiodic=True, sites=None):
    """F_a(x, mu) at ``sites`` (all sites when None), shape (n, 4, 8), given X = (M^dag M)^{-1} phi."""
    nbr = neighbours(dims, t_antiperiodic)
    fwd, _, sf, _ = nbr
    x = np.arange(U.shape[0]) if sites is None else np.asarray(sites)
    F = np.zeros((len(x), 4, 8))
    # Y = M X, needed at x and at x + mu only
    Y = apply_M(U, X, dims, kappa, t_antiperiodic, sites=x, nbr=nbr)
    for mu in range(4):
        s = sf[mu][x][:, None]
        xf = fwd[mu][x]
        Yf = apply_M(U, X, dims, kappa, t_antiperiodic, sites=xf, nbr=nbr)
        Xf = X[xf]
        Um = U[x, mu]
        Yp = np.matmul(ONE4 - GAMMA[mu], Y)            # (1 - g_mu) Y(x)
        Ym = np.matmul(ONE4 + GAMMA[mu], Yf)           # (1 + g_mu) Y(x+mu)
        UXf = np.matmul(Xf, np.swapaxes(Um, -1, -2))   # U X(x+mu), spin-major
        # term 1: Y(x)^dag (1-g) t_a U X(x+mu) = sum_{s,i,j} conj(Yp[s,i]) t_a[i,j] (U Xf)[s,j]
        t1 = np.einsum("vsi,aij,vsj->va", np.conj(Yp), T, UXf)
        # term 2: Y(x+mu)^dag (1+g) U^dag t_a X(x) = sum conj(Ym[s,i]) conj(U[j,i]) t_a[j,k] X[s,k]
        t2 = np.einsum("vsi,vji,ajk,vsk->va", np.conj(Ym), np.conj(Um), T, X[x])
        F[:, mu] = 2.0 * kappa * s * (1j * t1 - 1j * t2).real
    return F


def fermion_force(U, phi, dims, kappa, tol=1e-10, t_antiperiodic=True):
    X, it, res = cg_MdagM(U, phi, dims, kappa, tol, t_antiperiodic=t_antiperiodic)
    return fermion_force_from_X(U, X, dims, kappa, t_antiperiodic), X, it, res


def fermion_grad_from_X(U, X, dims, kappa, t_antiperiodic=True):
    """Complex gradient G = dS_f/dconj(U) in the torch convention, shape (V, 4, 3, 3)."""
    fwd, _, sf, _ = neighbours(dims, t_antiperiodic)
    Y = apply_M(U, X, dims, kappa, t_antiperiodic)
    G = np.zeros_like(U)
    for mu in range(4):
        s = sf[mu][:, None, None]
        Yp = np.matmul(ONE4 - GAMMA[mu], Y)
        Ym = np.matmul(ONE4 + GAMMA[mu], Y[fwd[mu]])
        C = np.einsum("vsi,vsj->vij", np.conj(Yp), X[fwd[mu]]) + \
            np.einsum("vsj,vsi->vji", np.conj(X), Ym)
        G[:, mu] = np.conj(2.0 * kappa * s * C)
    return G
