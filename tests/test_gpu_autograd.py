"""The differentiable pseudofermion action S_f = phi^dag (M^dag M)^{-1} phi (Eq. 4, 5):
library gradient against the oracle, against finite differences, and torch's gradcheck."""
import numpy as np
import pytest

from oracle.cg import cg_MdagM
from oracle.conventions import T
from oracle.fermion import fermion_grad_from_X
from synth import Lattice, gauge_exp_iA, source
from tests.gpu_common import require_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (3, 5, 2, 7)])
def test_fermion_grad_matches_oracle(lq, dims):
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.35, 8)
    X = source(lat, 9)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        G = torch.empty_like(dev(U))
        lq.lq_fermion_grad(ctx, G, dev(X), 0.15)
        got = host(G)
    finally:
        lq.lq_destroy(ctx)
    ref = fermion_grad_from_X(U, X, dims, 0.15)
    assert rel_err(got, ref) < 1e-12


def test_action_value_matches_oracle(lq):
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 8)
    phi = source(lat, 8)
    x_ref, _, _ = cg_MdagM(U, phi, dims, 0.15, 1e-13)
    S_ref = np.vdot(phi, x_ref).real
    from paper_1207_2223_gb300.autograd import pseudofermion_action
    S = pseudofermion_action(dev(U), dev(phi), dims, 0.15, 1e-12)
    assert float(S) == pytest.approx(S_ref, rel=1e-11)


def _fd_check(dims, kappa, seed, samples, tol_solve, eps=1e-5):
    from paper_1207_2223_gb300.autograd import pseudofermion_action
    lat = Lattice(dims)
    U0 = dev(gauge_exp_iA(lat, 0.3, seed))
    phi = dev(source(lat, seed))
    U = U0.clone().requires_grad_(True)
    S = pseudofermion_action(U, phi, dims, kappa, tol_solve)
    S.backward()
    G = U.grad.detach()
    rng = np.random.default_rng(seed)
    worst = 0.0
    scale = float(G.abs().max())
    for _ in range(samples):
        s, mu, i, j = int(rng.integers(lat.V)), int(rng.integers(4)), int(rng.integers(3)), int(rng.integers(3))
        for unit, part in ((1.0, "real"), (1j, "imag")):
            Up = U0.clone(); Up[s, mu, i, j] += unit * eps
            Um = U0.clone(); Um[s, mu, i, j] -= unit * eps
            fd = (float(pseudofermion_action(Up, phi, dims, kappa, tol_solve)) -
                  float(pseudofermion_action(Um, phi, dims, kappa, tol_solve))) / (2 * eps)
            g = float(getattr(G[s, mu, i, j], part))
            worst = max(worst, abs(fd - g) / scale)
    return worst


def test_backward_against_central_differences_4x4x4x4(lq):
    """Central differences with eps = 1e-5 in FP64, solves to 1e-13."""
    assert _fd_check((4, 4, 4, 4), 0.15, 8, 8, 1e-13) < 1e-5


def test_backward_against_central_differences_16x16x16x16(lq):
    """The 16^4 workload (kappa 0.15, seed 8): 8 sampled entries (real and imaginary parts)
    against central differences."""
    assert _fd_check((16, 16, 16, 16), 0.15, 8, 8, 1e-12) < 1e-4


def test_backward_matches_oracle_gradient_16x16x16x16(lq):
    """The 16^4 workload (kappa 0.15, seed 8): the autograd backward equals, on every link,
    the oracle's gradient evaluated from a solution X that the oracle itself certifies
    (its FP64 M^dag M X reproduces phi to 1e-10).  The backward recomputes X with the same
    deterministic solver, so it works from the same X."""
    from oracle.wilson import apply_MdagM
    from paper_1207_2223_gb300.autograd import pseudofermion_action
    dims, kappa = (16, 16, 16, 16), 0.15
    lat = Lattice(dims)
    U_h = gauge_exp_iA(lat, 0.3, 8)
    phi_h = source(lat, 8)
    U = dev(U_h).requires_grad_(True)
    phi = dev(phi_h)
    S = pseudofermion_action(U, phi, dims, kappa, 1e-10)
    S.backward()
    G = host(U.grad)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U_h))
        X = torch.empty_like(phi)
        lq.lq_solve_MdagM(ctx, X, phi, kappa, 1e-10, 100000, lq.LQ_F64, 50)
        X_h = host(X)
    finally:
        lq.lq_destroy(ctx)
    res = np.linalg.norm(phi_h - apply_MdagM(U_h, X_h, dims, kappa)) / np.linalg.norm(phi_h)
    assert res <= 1.01e-10, res
    assert float(S.detach()) == pytest.approx(np.vdot(phi_h, X_h).real, rel=1e-12)
    G_ref = fermion_grad_from_X(U_h, X_h, dims, kappa)
    assert rel_err(G, G_ref) < 1e-12
    assert np.max(np.abs(G - G_ref)) < 1e-12 * np.max(np.abs(G_ref))


def test_gradient_consistent_with_su3_force_16x16x16x16(lq):
    """F_a = -Im tr(t_a U G^dag) ties the complex gradient to the su(3) force kernel."""
    dims = (16, 16, 16, 16)
    lat = Lattice(dims)
    U = dev(gauge_exp_iA(lat, 0.3, 8))
    phi = dev(source(lat, 8))
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, U)
        X = torch.empty_like(phi)
        lq.lq_solve_MdagM(ctx, X, phi, 0.15, 1e-10)
        G = torch.empty_like(U)
        lq.lq_fermion_grad(ctx, G, X, 0.15)
        F = torch.empty((lat.V, 4, 8), dtype=torch.float64, device="cuda")
        lq.lq_fermion_force(ctx, F, X, 0.15)
    finally:
        lq.lq_destroy(ctx)
    Tt = torch.from_numpy(T).cuda()
    Fp = -torch.einsum("aij,vmjk,vmik->vma", Tt, U, G.conj()).imag
    assert float((Fp - F).abs().max()) < 1e-12 * float(F.abs().max())


def test_gradient_of_phi_and_gradcheck(lq):
    """dS/dphi = 2 X, and torch.autograd.gradcheck on a 2^4 lattice (solves to 1e-14)."""
    from paper_1207_2223_gb300.autograd import pseudofermion_action
    dims = (2, 2, 2, 2)
    lat = Lattice(dims)
    U = dev(gauge_exp_iA(lat, 0.3, 3)).requires_grad_(True)
    phi = dev(source(lat, 3)).requires_grad_(True)
    f = lambda u, p: pseudofermion_action(u, p, dims, 0.13, 1e-14)   # noqa: E731
    assert torch.autograd.gradcheck(f, (U, phi), eps=1e-6, atol=1e-6, rtol=1e-4)


def test_cached_context_loop_allocates_once_16x16x16x16(lq):
    """A forward + backward loop at 16^4 reuses one cached context: after the first step the
    device's free memory does not move (no allocation by the library), every step loads the
    links (forward and backward) and gives the same gradient, and a change of the links made
    through .data, which torch's version counter does not see, is picked up."""
    from paper_1207_2223_gb300 import autograd as ag
    ag.release_contexts()
    dims, kappa = (16, 16, 16, 16), 0.15
    lat = Lattice(dims)
    U = dev(gauge_exp_iA(lat, 0.3, 8)).requires_grad_(True)
    phi = dev(source(lat, 8))
    free, g0, same = [], None, []
    for step in range(4):
        U.grad = None
        S = ag.pseudofermion_action(U, phi, dims, kappa, 1e-10)
        S.backward()
        torch.cuda.synchronize()
        if g0 is None:
            g0 = U.grad.clone()
        else:
            same.append(bool(torch.equal(U.grad, g0)))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    key = (dims, True, U.device.index)
    assert ag.cached_context_stats()[key] == 8
    assert len(set(free[1:])) == 1, free
    assert all(same)
    S0 = float(ag.pseudofermion_action(U.detach(), phi, dims, kappa, 1e-10))
    U.data[0, 0] *= -1.0                    # bypasses the version counter
    S1 = float(ag.pseudofermion_action(U.detach(), phi, dims, kappa, 1e-10))
    U.data[0, 0] *= -1.0
    assert S1 != S0
    assert float(ag.pseudofermion_action(U.detach(), phi, dims, kappa, 1e-10)) == S0
    ag.release_contexts()
    assert ag.cached_context_stats() == {}
