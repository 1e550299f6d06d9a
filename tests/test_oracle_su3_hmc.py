"""Pins of the oracle's link update and HMC trajectory (Eq. 5; Sec. 2; Sec. 3 kernel 4)."""
import math
import numpy as np
import pytest

from oracle.conventions import T
from oracle.gauge import plaquette
from oracle.hmc import leapfrog, trajectory
from oracle.su3 import algebra_coeffs, algebra_matrix, expm, link_update, reunitarise
from oracle.wilson import apply_M
from synth import Lattice, gauge_exp_iA, momenta, chi_noise, metropolis_uniform


def test_expm_matches_eigendecomposition():
    rng = np.random.default_rng(0)
    p = rng.normal(size=(50, 8)) * 2.0
    P = algebra_matrix(p)
    w, v = np.linalg.eigh(P)
    ref = np.einsum("nij,nj,nkj->nik", v, np.exp(1j * w), v.conj())
    assert np.max(np.abs(expm(1j * P) - ref)) < 1e-13


def test_expm_small_argument_taylor():
    X = 1j * algebra_matrix(np.full(8, 1e-4))
    # the remainder after the cubic term is O(|X|^4) ~ 1e-15
    assert np.max(np.abs(expm(X) - (np.eye(3) + X + X @ X / 2 + X @ X @ X / 6))) < 1e-15


def test_algebra_roundtrip():
    p = np.random.default_rng(1).normal(size=(10, 8))
    assert np.max(np.abs(algebra_coeffs(algebra_matrix(p)) - p)) < 1e-14
    assert np.allclose(0.5 * np.einsum("nij,nji->n", algebra_matrix(p), algebra_matrix(p)).real,
                       0.5 * np.sum(p * p, -1))


def test_reunitarise():
    lat = Lattice((2, 2, 2, 2))
    U = gauge_exp_iA(lat, 0.5, 1)
    assert np.max(np.abs(reunitarise(U) - U)) < 1e-14
    W = U + 1e-3 * np.random.default_rng(2).normal(size=U.shape)
    R = reunitarise(W)
    assert np.max(np.abs(R @ np.conj(np.swapaxes(R, -1, -2)) - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(R) - 1)) < 1e-14


def test_link_update_group_and_composition():
    lat = Lattice((2, 2, 2, 2))
    U = gauge_exp_iA(lat, 0.3, 2)
    p = momenta(lat, 2)
    U1 = link_update(U, p, 0.05)
    assert np.max(np.abs(np.linalg.det(U1) - 1)) < 1e-14
    # exp(i a P) exp(i b P) = exp(i (a + b) P)
    assert np.max(np.abs(link_update(link_update(U, p, 0.03), p, 0.02) - U1)) < 1e-13
    assert np.max(np.abs(link_update(U1, p, -0.05) - U)) < 1e-13


SMALL = dict(dims=(2, 2, 2, 4), beta=5.6, kappa=0.12)


def _start(seed=0):
    lat = Lattice(SMALL["dims"])
    U = gauge_exp_iA(lat, 0.3, seed)
    return lat, U, momenta(lat, seed), chi_noise(lat, seed)


def test_leapfrog_reversible():
    lat, U, p, chi = _start()
    d, b, k = SMALL["dims"], SMALL["beta"], SMALL["kappa"]
    phi = apply_M(U, chi, d, k, dagger=True)
    U1, p1 = leapfrog(U, p, phi, d, b, k, 6, 0.6, 1e-14)
    U2, p2 = leapfrog(U1, -p1, phi, d, b, k, 6, 0.6, 1e-14)
    assert np.max(np.abs(U2 - U)) < 1e-10
    assert np.max(np.abs(p2 + p)) < 1e-10


def test_delta_H_scales_as_eps_squared():
    lat, U, p, chi = _start(1)
    d, b, k = SMALL["dims"], SMALL["beta"], SMALL["kappa"]
    dh = [abs(trajectory(U, p, chi, 0.5, d, b, k, n, tau=0.5, tol=1e-13)["dH"]) for n in (5, 10, 20)]
    assert 3.3 < dh[0] / dh[1] < 4.7
    assert 3.3 < dh[1] / dh[2] < 4.7


def test_metropolis_decision():
    lat, U, p, chi = _start(2)
    d, b, k = SMALL["dims"], SMALL["beta"], SMALL["kappa"]
    r = trajectory(U, p, chi, 0.0, d, b, k, 4, tau=0.4, tol=1e-12)
    assert r["accept"]                                   # u = 0 always accepts
    assert np.array_equal(r["U"], r["U_proposed"])
    u = min(0.999999, math.exp(-r["dH"]) * 1.0001) if r["dH"] > 0 else None
    if u is not None:
        r2 = trajectory(U, p, chi, u, d, b, k, 4, tau=0.4, tol=1e-12)
        assert not r2["accept"] and np.array_equal(r2["U"], U)
    # the Hamiltonian pieces add up
    assert r["dH"] == pytest.approx(r["dK"] + r["dSg"] + r["dSf"], abs=1e-12)


@pytest.mark.slow
def test_small_preset_trajectory_eps_squared():
    """4^4, beta 5.6, kappa 0.15, tau 1 from the rough exp(iA) start (sigma 0.3): the start is far
    from equilibrium, so Delta H is large at 10 steps, but it falls as eps^2 with 20 steps."""
    lat = Lattice((4, 4, 4, 4))
    U = gauge_exp_iA(lat, 0.3, 0)
    p = momenta(lat, 0)
    chi = chi_noise(lat, 0)
    r10 = trajectory(U, p, chi, metropolis_uniform(0), lat.dims, 5.6, 0.15, 10, 1.0, 1e-10)
    r20 = trajectory(U, p, chi, metropolis_uniform(0), lat.dims, 5.6, 0.15, 20, 1.0, 1e-10)
    assert 3.0 < r10["dH"] / r20["dH"] < 5.0
    assert 0.0 < r10["plaquette"] < 1.0
    assert all(res <= 1e-10 for _, res in r10["solves"])
