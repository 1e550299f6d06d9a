"""su(3) algebra, exp(i eps p) and reunitarisation (Sec. 2; Sec. 3 kernel 4).

The paper evolves the links with the momenta, U and exp(i p) being
conjugate (Sec. 2 after Eq. 5), as kernel 4 of Sec. 3.  Reading taken:
U <- exp(i eps P) U with P = sum_a p_a t_a, followed by reunitarisation
(Gram-Schmidt on rows 1 and 2, row 3 = conj(row1 x row2)).

The exponential is the Taylor series summed to convergence after scaling
by 2^-s, then squared s times (scaling and squaring).
"""
import numpy as np

from .conventions import T


def algebra_matrix(p):
    """P = sum_a p_a t_a from coefficients (..., 8) -> (..., 3, 3) Hermitian."""
    return np.einsum("...a,aij->...ij", p, T)


def algebra_coeffs(P):
    """p_a = tr(t_a P) for Hermitian traceless P."""
    return np.einsum("aij,...ji->...a", T, P).real


def expm(X):
    """exp(X) for a stack of 3x3 complex matrices, scaling and squaring + Taylor."""
    X = np.asarray(X, dtype=np.complex128)
    nrm = np.max(np.sqrt(np.sum(np.abs(X) ** 2, axis=(-2, -1)))) if X.size else 0.0
    s = 0
    while nrm / (2 ** s) > 0.25:
        s += 1
    A = X / (2 ** s)
    E = np.broadcast_to(np.eye(3, dtype=np.complex128), X.shape).copy()
    term = E.copy()
    for k in range(1, 60):
        term = term @ A / k
        E = E + term
        if np.max(np.abs(term)) < 1e-30:
            break
    for _ in range(s):
        E = E @ E
    return E


def reunitarise(U):
    """Project to SU(3): normalise row 1, orthonormalise row 2, row 3 = conj(r1 x r2)."""
    U = np.array(U, dtype=np.complex128, copy=True)
    r1 = U[..., 0, :]
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1))[..., None]
    r2 = U[..., 1, :]
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1)[..., None] * r1
    r2 = r2 / np.sqrt(np.sum(np.abs(r2) ** 2, axis=-1))[..., None]
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def link_update(U, p, eps):
    """U <- reunitarise(exp(i eps P) U), P = sum_a p_a t_a, per link."""
    return reunitarise(expm(1j * eps * algebra_matrix(p)) @ U)
