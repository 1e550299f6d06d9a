"""Conjugate gradient on M^dag M (Sec. 1 after Eq. 3; Sec. 3 "conjugate gradient routine").

The paper inverts M^dag M on the pseudofermion field with CG (Eq. 4 and
the text after Eq. 3).  This is textbook Hestenes-Stiefel CG from x0 = 0.
Stopping rule (the paper only quotes a "limit"): stop once the relative
true residual ||phi - M^dag M x|| / ||phi|| <= tol, recomputed in FP64;
if the recursive residual has met the tolerance but the true one has not,
restart from the true residual.
"""
import numpy as np

from .conventions import neighbours
from .wilson import apply_MdagM


def cg_MdagM(U, phi, dims, kappa, tol=1e-10, maxiter=100000, t_antiperiodic=True, history=None):
    """Solve M^dag M x = phi.  Returns (x, iterations, true relative residual)."""
    nbr = neighbours(dims, t_antiperiodic)
    A = lambda v: apply_MdagM(U, v, dims, kappa, t_antiperiodic, nbr)   # noqa: E731
    phinorm = np.sqrt(np.vdot(phi, phi).real)
    x = np.zeros_like(phi)
    if phinorm == 0.0:
        return x, 0, 0.0
    r = phi.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    true_rel = 1.0
    for it in range(1, maxiter + 1):
        Ap = A(p)
        pAp = np.vdot(p, Ap).real
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        if history is not None:
            history.append(np.sqrt(rr_new) / phinorm)
        if rr_new <= (tol * phinorm) ** 2:
            rt = phi - A(x)
            true_rel = np.sqrt(np.vdot(rt, rt).real) / phinorm
            if true_rel <= tol:
                return x, it, true_rel
            r = rt
            p = r.copy()
            rr = np.vdot(r, r).real
            continue
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    rt = phi - A(x)
    return x, maxiter, np.sqrt(np.vdot(rt, rt).real) / phinorm
