"""Wilson plaquette gauge action and its force (Eq. 1 "S_g"; Sec. 3 kernel 2).

The paper names S_g only as a discretisation of (1/2) tr F^2 (Eq. 1) and
lists the gauge force as kernel 2 of Sec. 3.  Reading taken: the Wilson
plaquette action

    S_g = beta * sum_{x, mu<nu} (1 - Re tr U_{mu nu}(x) / 3),
    U_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag,

and the force F_a(x, mu) = dS_g / d omega_a under U_mu(x) -> exp(i omega_a t_a) U_mu(x),
which equals (beta / 3) Im tr(t_a U_mu(x) Sigma_mu(x)) with the staple sum
Sigma_mu(x) = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
                             + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) ].
"""
import numpy as np

from .conventions import T, dagger, neighbours


def plaquette_field(U, dims):
    """Re tr U_{mu nu}(x) for the six planes mu < nu, shape (6, V)."""
    fwd, _, _, _ = neighbours(dims, False)
    out = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = U[:, mu] @ U[fwd[mu], nu] @ dagger(U[fwd[nu], mu]) @ dagger(U[:, nu])
            out.append(np.trace(P, axis1=-2, axis2=-1).real)
    return np.array(out)


def plaquette(U, dims):
    """Average of Re tr U_P / 3 over the 6 V plaquettes (1 for U = 1)."""
    return float(np.mean(plaquette_field(U, dims)) / 3.0)


def gauge_action(U, dims, beta):
    return float(beta * np.sum(1.0 - plaquette_field(U, dims) / 3.0))


def staple_sum(U, dims, sites=None):
    """Sigma_mu(x) at ``sites`` (all sites when None), shape (n, 4, 3, 3)."""
    fwd, bwd, _, _ = neighbours(dims, False)
    x = np.arange(U.shape[0]) if sites is None else np.asarray(sites)
    S = np.zeros((len(x), 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            xm, xn, xb = fwd[mu][x], fwd[nu][x], bwd[nu][x]
            upper = U[xm, nu] @ dagger(U[xn, mu]) @ dagger(U[x, nu])
            xmn = bwd[nu][xm]                        # x + mu - nu
            lower = dagger(U[xmn, nu]) @ dagger(U[xb, mu]) @ U[xb, nu]
            S[:, mu] += upper + lower
    return S


def gauge_force(U, dims, beta, sites=None):
    """F_a(x, mu) = (beta/3) Im tr(t_a U_mu(x) Sigma_mu(x)) at ``sites``, shape (n, 4, 8)."""
    x = np.arange(U.shape[0]) if sites is None else np.asarray(sites)
    W = U[x] @ staple_sum(U, dims, sites)
    tr = np.einsum("aij,...ji->...a", T, W)
    return (beta / 3.0) * tr.imag
