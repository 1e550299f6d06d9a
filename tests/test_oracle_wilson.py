"""Pins of the oracle's Dirac operator (Eq. 4; Sec. 3 kernel 1) against mathematics
that does not depend on the implementation."""
import numpy as np
import pytest

from oracle.conventions import GAMMA, GAMMA5, T, neighbours
from oracle.wilson import apply_M, apply_MdagM, hopping
from synth import Lattice, gauge_exp_iA, gauge_transform, source, plane_wave, identity_gauge
from tests.oracle_helpers import dense_wilson_loops, dense_from_operator


def test_gamma_clifford_and_hermitian():
    for m in range(4):
        assert np.allclose(GAMMA[m], GAMMA[m].conj().T)
        for n in range(4):
            ac = GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m]
            assert np.allclose(ac, 2.0 * (m == n) * np.eye(4))
        assert np.allclose(GAMMA5 @ GAMMA[m] + GAMMA[m] @ GAMMA5, 0)
    # DeGrand-Rossi: gamma_5 = diag(1, 1, -1, -1)
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


def test_su3_generators():
    tr = np.einsum("aij,bji->ab", T, T)
    assert np.allclose(tr, np.eye(8))
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T) and abs(np.trace(T[a])) < 1e-15
    # completeness: sum_a t_a[i,j] t_a[k,l] = d_il d_jk - d_ij d_kl / 3
    lhs = np.einsum("aij,akl->ijkl", T, T)
    d = np.eye(3)
    rhs = np.einsum("il,jk->ijkl", d, d) - np.einsum("ij,kl->ijkl", d, d) / 3.0
    assert np.allclose(lhs, rhs)


def test_neighbours_inverse():
    dims = (2, 3, 4, 5)
    fwd, bwd, sf, sb = neighbours(dims, True)
    for mu in range(4):
        assert np.array_equal(fwd[mu][bwd[mu]], np.arange(120))
        # the sign of the hop x -> x+mu equals that of x+mu -> x
        assert np.array_equal(sb[mu][fwd[mu]], sf[mu])


@pytest.mark.parametrize("dims", [(4, 2, 6, 8), (2, 2, 2, 2), (3, 4, 2, 6)])
@pytest.mark.parametrize("dagger", [False, True])
def test_free_field_closed_form(dims, dagger):
    """U = 1: a plane wave e^{ip.x} u is an eigenvector with
    M = 1 - 2 kappa sum cos p + 2 i kappa sum gamma sin p  (sign of the gamma term flips for M^dag)."""
    lat = Lattice(dims)
    U = identity_gauge(lat)
    kappa = 0.137
    rng = np.random.default_rng(1)
    for n in [(0, 0, 0, 0), (1, 0, 1, 2), (dims[0] - 1, 1, 0, dims[3] - 1)]:
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        psi, p = plane_wave(lat, n, u)
        a = 1.0 - 2.0 * kappa * np.sum(np.cos(p))
        G = sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
        K = a * np.eye(4) + (-1 if dagger else 1) * 2j * kappa * G
        expect = np.matmul(K, psi)
        got = apply_M(U, psi, dims, kappa, dagger=dagger)
        assert np.max(np.abs(got - expect)) < 1e-13
        mdm = apply_MdagM(U, psi, dims, kappa)
        lam = a * a + 4 * kappa ** 2 * np.sum(np.sin(p) ** 2)
        assert np.max(np.abs(mdm - lam * psi)) < 1e-13


def test_free_field_periodic_time():
    lat = Lattice((2, 4, 2, 4))
    U = identity_gauge(lat)
    u = np.ones((4, 3))
    psi, p = plane_wave(lat, (1, 1, 0, 1), u, t_antiperiodic=False)
    a = 1.0 - 2.0 * 0.1 * np.sum(np.cos(p))
    K = a * np.eye(4) + 2j * 0.1 * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    got = apply_M(U, psi, lat.dims, 0.1, t_antiperiodic=False)
    assert np.max(np.abs(got - np.matmul(K, psi))) < 1e-13


def _random_setup(dims, seed=3, sigma=0.4):
    lat = Lattice(dims)
    return lat, gauge_exp_iA(lat, sigma, seed), source(lat, seed, 0), source(lat, seed, 1)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 6)])
def test_adjoint_and_gamma5_hermiticity(dims):
    lat, U, a, b = _random_setup(dims)
    k = 0.15
    lhs = np.vdot(a, apply_M(U, b, dims, k))
    rhs = np.vdot(apply_M(U, a, dims, k, dagger=True), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    g5b = np.matmul(GAMMA5, b)
    assert np.max(np.abs(apply_M(U, b, dims, k, dagger=True) -
                         np.matmul(GAMMA5, apply_M(U, g5b, dims, k)))) < 1e-13


def test_gauge_covariance():
    dims = (2, 4, 2, 4)
    lat, U, psi, _ = _random_setup(dims)
    g = gauge_transform(lat, 11)
    fwd, _, _, _ = neighbours(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fwd[mu]], -1, -2))
    psig = np.matmul(psi, np.swapaxes(g, -1, -2))         # colour rotation at every spin
    for dag in (False, True):
        lhs = apply_M(Ug, psig, dims, 0.15, dagger=dag)
        rhs = np.matmul(apply_M(U, psi, dims, 0.15, dagger=dag), np.swapaxes(g, -1, -2))
        assert np.max(np.abs(lhs - rhs)) < 1e-13


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 3, 4)])
def test_dense_matrix_matches_loop_construction(dims):
    """Columns of the oracle's M equal an entry-by-entry loop construction;
    the columns of M^dag equal the conjugate transpose."""
    lat, U, _, _ = _random_setup(dims)
    k = 0.13
    Mloop = dense_wilson_loops(U, dims, k)
    Mcols = dense_from_operator(lambda v: apply_M(U, v, dims, k), lat.V)
    assert np.max(np.abs(Mcols - Mloop)) < 1e-14
    Mdcols = dense_from_operator(lambda v: apply_M(U, v, dims, k, dagger=True), lat.V)
    assert np.max(np.abs(Mdcols - Mloop.conj().T)) < 1e-14


def test_sampled_sites_match_full():
    dims = (4, 2, 2, 6)
    lat, U, psi, _ = _random_setup(dims)
    full = apply_M(U, psi, dims, 0.15, dagger=True)
    sites = np.array([0, 5, 17, lat.V - 1, 40])
    part = apply_M(U, psi, dims, 0.15, dagger=True, sites=sites)
    assert np.array_equal(part, full[sites])


def test_sampled_MdagM_matches_dense_loop_matrix():
    """M^dag M at a few sites, evaluated from the one-hop neighbourhood only, equals the
    rows of the dense (M^dag M) built from the entry-by-entry loop construction (L = 2 in
    two directions, so neighbours coincide), and the full-lattice M^dag M at those sites."""
    from oracle.wilson import apply_MdagM, apply_MdagM_sites
    dims = (2, 3, 2, 4)
    lat, U, psi, _ = _random_setup(dims)
    k = 0.14
    Mloop = dense_wilson_loops(U, dims, k)
    dense = (Mloop.conj().T @ Mloop) @ psi.reshape(-1)
    sites = np.array([0, 7, 13, lat.V - 1])
    part = apply_MdagM_sites(U, psi, dims, k, sites)
    assert np.max(np.abs(part - dense.reshape(lat.V, 4, 3)[sites])) < 1e-13
    assert np.max(np.abs(part - apply_MdagM(U, psi, dims, k)[sites])) < 1e-14


def test_linearity():
    dims = (2, 2, 2, 4)
    lat, U, a, b = _random_setup(dims)
    c = 0.3 - 1.7j
    lhs = hopping(U, a + c * b, dims)
    rhs = hopping(U, a, dims) + c * hopping(U, b, dims)
    assert np.max(np.abs(lhs - rhs)) < 1e-13
