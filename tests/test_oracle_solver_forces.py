"""Pins of the oracle's CG, actions and forces (Eq. 4-5; Sec. 3 kernels 2 and 3)."""
import numpy as np
import pytest
from scipy.linalg import expm as scipy_expm

from oracle.cg import cg_MdagM
from oracle.conventions import T, neighbours
from oracle.fermion import fermion_force_from_X, fermion_grad_from_X
from oracle.gauge import gauge_action, gauge_force, plaquette, plaquette_field, staple_sum
from oracle.wilson import apply_M, apply_MdagM
from synth import Lattice, gauge_exp_iA, gauge_transform, source, identity_gauge, plane_wave
from tests.oracle_helpers import dense_wilson_loops


def test_cg_matches_dense_solve():
    dims = (2, 2, 2, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.35, 5)
    phi = source(lat, 5)
    k = 0.15
    M = dense_wilson_loops(U, dims, k)
    x_dense = np.linalg.solve(M.conj().T @ M, phi.reshape(-1)).reshape(phi.shape)
    x, it, res = cg_MdagM(U, phi, dims, k, tol=1e-13)
    assert res <= 1e-13
    assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) < 1e-11


def test_free_spectrum_of_MdagM():
    """U = 1: the dense spectrum of M^dag M is the closed form (1 - 2k sum cos p)^2 + 4k^2 sum sin^2 p,
    each value 12-fold (4 spins x 3 colours)."""
    dims = (2, 2, 2, 4)
    lat = Lattice(dims)
    k = 0.12
    M = dense_wilson_loops(identity_gauge(lat), dims, k)
    ev = np.sort(np.linalg.eigvalsh(M.conj().T @ M))
    vals = []
    for nx in range(2):
        for ny in range(2):
            for nz in range(2):
                for nt in range(4):
                    _, p = plane_wave(lat, (nx, ny, nz, nt), np.ones((4, 3)))
                    a = 1 - 2 * k * np.sum(np.cos(p))
                    vals += [a * a + 4 * k * k * np.sum(np.sin(p) ** 2)] * 12
    assert np.max(np.abs(ev - np.sort(vals))) < 1e-13


def test_cg_true_residual_and_history():
    dims = (4, 4, 2, 2)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 2)
    phi = source(lat, 1)
    hist = []
    x, it, res = cg_MdagM(U, phi, dims, 0.15, tol=1e-10, history=hist)
    r = phi - apply_MdagM(U, x, dims, 0.15)
    assert np.linalg.norm(r) / np.linalg.norm(phi) == pytest.approx(res, rel=1e-6)
    assert res <= 1e-10 and len(hist) == it


def test_plaquette_unit_and_gauge_invariance():
    dims = (2, 4, 2, 4)
    lat = Lattice(dims)
    assert plaquette(identity_gauge(lat), dims) == pytest.approx(1.0, abs=1e-15)
    U = gauge_exp_iA(lat, 0.4, 9)
    g = gauge_transform(lat, 10)
    fwd, _, _, _ = neighbours(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd[mu]], -1, -2))
    assert np.max(np.abs(plaquette_field(Ug, dims) - plaquette_field(U, dims))) < 1e-13


def test_staples_count_each_plaquette_four_times():
    """sum_{x,mu} Re tr(U_mu(x) Sigma_mu(x)) = 4 sum_P Re tr U_P (each plaquette has 4 links)."""
    dims = (2, 2, 4, 2)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.5, 4)
    lhs = np.trace(U @ staple_sum(U, dims), axis1=-2, axis2=-1).real.sum()
    assert lhs == pytest.approx(4.0 * plaquette_field(U, dims).sum(), rel=1e-13)


def _perturb(U, site, mu, a, eta):
    Up = U.copy()
    Up[site, mu] = scipy_expm(1j * eta * T[a]) @ U[site, mu]
    return Up


def test_gauge_force_finite_differences():
    dims = (2, 2, 2, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.4, 6)
    beta = 5.6
    F = gauge_force(U, dims, beta)
    assert np.max(np.abs(gauge_force(identity_gauge(lat), dims, beta))) < 1e-14
    rng = np.random.default_rng(0)
    eta = 1e-5
    for _ in range(24):
        s, mu, a = rng.integers(lat.V), rng.integers(4), rng.integers(8)
        fd = (gauge_action(_perturb(U, s, mu, a, eta), dims, beta) -
              gauge_action(_perturb(U, s, mu, a, -eta), dims, beta)) / (2 * eta)
        assert abs(fd - F[s, mu, a]) < 1e-6 * max(1.0, abs(F[s, mu, a]))


def _dense_Sf(U, phi, dims, k):
    M = dense_wilson_loops(U, dims, k)
    return np.vdot(phi.reshape(-1), np.linalg.solve(M.conj().T @ M, phi.reshape(-1))).real


def test_fermion_force_finite_differences():
    """F_f against central differences of S_f computed by dense solves; links across
    the antiperiodic t boundary included."""
    dims = (2, 2, 2, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.35, 7)
    phi = source(lat, 3)
    k = 0.14
    X, _, _ = cg_MdagM(U, phi, dims, k, tol=1e-14)
    F = fermion_force_from_X(U, X, dims, k)
    eta = 1e-5
    t_boundary = [s for s in range(lat.V) if s // 8 == 3]          # t = Lt - 1
    checks = [(t_boundary[0], 3, 2), (t_boundary[1], 3, 7), (0, 0, 0), (5, 1, 4), (17, 2, 6),
              (t_boundary[2], 0, 3), (30, 3, 1)]
    for s, mu, a in checks:
        fd = (_dense_Sf(_perturb(U, s, mu, a, eta), phi, dims, k) -
              _dense_Sf(_perturb(U, s, mu, a, -eta), phi, dims, k)) / (2 * eta)
        assert abs(fd - F[s, mu, a]) < 2e-6 * max(1.0, abs(F[s, mu, a])), (s, mu, a, fd, F[s, mu, a])


def test_fermion_gradient_torch_convention_and_projection():
    """G = dS_f/dconj(U): dS/dRe U_ij = Re G_ij and dS/dIm U_ij = Im G_ij; and the
    su(3) force is F_a = -Im tr(t_a U G^dag)."""
    dims = (2, 2, 2, 2)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.35, 8)
    phi = source(lat, 4)
    k = 0.13
    X, _, _ = cg_MdagM(U, phi, dims, k, tol=1e-14)
    G = fermion_grad_from_X(U, X, dims, k)
    eta = 1e-6
    for (s, mu, i, j) in [(0, 0, 0, 1), (3, 3, 2, 2), (9, 1, 1, 0), (15, 2, 0, 2)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            Up = U.copy(); Up[s, mu, i, j] += unit * eta
            Um = U.copy(); Um[s, mu, i, j] -= unit * eta
            fd = (_dense_Sf(Up, phi, dims, k) - _dense_Sf(Um, phi, dims, k)) / (2 * eta)
            assert abs(fd - part(G[s, mu, i, j])) < 1e-6 * max(1.0, abs(G[s, mu, i, j]))
    F = fermion_force_from_X(U, X, dims, k)
    Fp = -np.einsum("aij,vmjk,vmik->vma", T, U, np.conj(G)).imag
    assert np.max(np.abs(F - Fp)) < 1e-12


def test_pseudofermion_heatbath_identity():
    """phi = M^dag chi  =>  phi^dag (M^dag M)^{-1} phi = chi^dag chi."""
    dims = (4, 2, 2, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 12)
    chi = source(lat, 12)
    phi = apply_M(U, chi, dims, 0.15, dagger=True)
    X, _, _ = cg_MdagM(U, phi, dims, 0.15, tol=1e-12)
    assert np.vdot(phi, X).real == pytest.approx(np.vdot(chi, chi).real, rel=1e-11)


def test_fermion_force_gauge_covariant():
    """Under U -> g U g'^dag, X -> g X: the Lie-algebra force rotates as F -> g F g^dag,
    so sum_a F_a^2 at each link is invariant."""
    dims = (2, 2, 2, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.35, 13)
    X = source(lat, 13)
    g = gauge_transform(lat, 14)
    fwd, _, _, _ = neighbours(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd[mu]], -1, -2))
    Xg = np.matmul(X, np.swapaxes(g, -1, -2))
    F = fermion_force_from_X(U, X, dims, 0.15)
    Fg = fermion_force_from_X(Ug, Xg, dims, 0.15)
    assert np.max(np.abs(np.sum(F ** 2, -1) - np.sum(Fg ** 2, -1))) < 1e-12


def test_forces_at_sampled_sites_equal_full_evaluation():
    """The site-sampled evaluation used for full-size parity equals the full one."""
    dims = (4, 2, 4, 6)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.4, 21)
    X = source(lat, 21)
    sites = np.array([0, 7, 19, 33, lat.V - 1, 100])
    assert np.array_equal(gauge_force(U, dims, 5.6, sites=sites), gauge_force(U, dims, 5.6)[sites])
    full = fermion_force_from_X(U, X, dims, 0.15)
    part = fermion_force_from_X(U, X, dims, 0.15, sites=sites)
    assert np.max(np.abs(part - full[sites])) < 1e-14
