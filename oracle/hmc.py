"""Hybrid Monte Carlo trajectory (Eq. 5; Sec. 2; Sec. 3 trajectory steps).

Hamiltonian (Eq. 5):  H = (1/2) sum tr p^2 + S_g(U) + phi^dag (M^dag M)^{-1} phi.
One trajectory (Sec. 3, the three steps of the evolution):
  1. heat bath: p with N(0,1) coefficients, phi = M^dag chi with chi complex
     Gaussian of density exp(-chi^dag chi) (Sec. 2); both are passed in;
     S_f at the start equals chi^dag chi exactly;
  2. leapfrog (reading: momentum half steps at both ends)
        p <- p - eps/2 F(U)
        repeat n: U <- exp(i eps p) U ; p <- p - eps F(U)  (eps/2 on the last)
     with F = dS/d omega (gauge + fermion, each solve from x0 = 0);
  3. Metropolis: accept iff u < exp(-Delta H), u uniform in [0, 1), passed in.
Delta H is summed as per-element differences (kinetic), per-plaquette
differences (gauge) and phi^dag X - chi^dag chi (fermion), with math.fsum.
"""
import math
import numpy as np

from .cg import cg_MdagM
from .fermion import fermion_force_from_X
from .gauge import gauge_force, plaquette, plaquette_field
from .su3 import link_update
from .wilson import apply_M


def total_force(U, phi, dims, beta, kappa, tol, t_antiperiodic=True, stats=None):
    X, it, res = cg_MdagM(U, phi, dims, kappa, tol, t_antiperiodic=t_antiperiodic)
    if stats is not None:
        stats.append((it, res))
    return gauge_force(U, dims, beta) + fermion_force_from_X(U, X, dims, kappa, t_antiperiodic)


def leapfrog(U, p, phi, dims, beta, kappa, n_steps, tau, tol, t_antiperiodic=True, stats=None):
    eps = tau / n_steps
    p = p - 0.5 * eps * total_force(U, phi, dims, beta, kappa, tol, t_antiperiodic, stats)
    for i in range(n_steps):
        U = link_update(U, p, eps)
        step = eps if i < n_steps - 1 else 0.5 * eps
        p = p - step * total_force(U, phi, dims, beta, kappa, tol, t_antiperiodic, stats)
    return U, p


def trajectory(U0, p0, chi, u, dims, beta, kappa, n_steps, tau=1.0, tol=1e-10, t_antiperiodic=True):
    """One HMC trajectory; returns a dict with the proposal, Delta H and the decision."""
    stats = []
    phi = apply_M(U0, chi, dims, kappa, t_antiperiodic, dagger=True)
    U1, p1 = leapfrog(U0, p0, phi, dims, beta, kappa, n_steps, tau, tol, t_antiperiodic, stats)
    X, it, res = cg_MdagM(U1, phi, dims, kappa, tol, t_antiperiodic=t_antiperiodic)
    stats.append((it, res))
    dK = 0.5 * math.fsum((p1 * p1 - p0 * p0).ravel())
    dSg = (beta / 3.0) * math.fsum((plaquette_field(U0, dims) - plaquette_field(U1, dims)).ravel())
    dSf = math.fsum((np.conj(phi) * X).real.ravel()) - math.fsum((np.abs(chi) ** 2).ravel())
    dH = dK + dSg + dSf
    accept = bool(u < math.exp(-dH)) if dH > -700 else True
    U_out = U1 if accept else U0
    return {"U": U_out, "U_proposed": U1, "p": p1, "phi": phi, "dH": dH, "dK": dK, "dSg": dSg,
            "dSf": dSf, "accept": accept, "plaquette": plaquette(U_out, dims), "solves": stats}
