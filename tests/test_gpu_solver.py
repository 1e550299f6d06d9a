"""CG on M^dag M (Sec. 1 after Eq. 3; Sec. 3) on the GPU against the oracle's solve."""
import numpy as np
import pytest

from oracle.cg import cg_MdagM
from synth import Lattice, gauge_exp_iA, source
from tests.gpu_common import require_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


# The oracle solves to 1e-13; the GPU to 1e-10.  The solution error is at
# most cond(M^dag M) times the residual; cond stays below ~1e3 for these
# lattices (CG converges in < 300 iterations), so 1e-6 is a safe bound.
X_TOL = 1e-6


@pytest.mark.parametrize("dims,kappa,sigma", [((4, 4, 4, 4), 0.15, 0.3), ((6, 4, 2, 6), 0.155, 0.3),
                                              ((8, 8, 8, 8), 0.156, 0.25)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4, 6])
def test_solve_matches_oracle(lq, dims, kappa, sigma, prec):
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, sigma, 2)
    phi = source(lat, 7)
    ohist = []
    x_ref, it_ref, res_ref = cg_MdagM(U, phi, dims, kappa, tol=1e-13, history=ohist)
    # iterations the oracle's recursion needed to reach 1e-10
    it_ref10 = 1 + int(np.argmax(np.array(ohist) <= 1e-10))
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        x = torch.zeros_like(dev(phi))
        hist = np.zeros(5000)
        status, st = lq.lq_solve_MdagM(ctx, x, dev(phi), kappa, 1e-10, 5000, prec, 50, hist=hist)
        got = host(x)
        # residual recomputed independently through the FP64 operator
        r = torch.empty_like(x)
        lq.lq_apply_MdagM(ctx, r, x, kappa, lq.LQ_F64)
        res = np.linalg.norm(phi - host(r)) / np.linalg.norm(phi)
    finally:
        lq.lq_destroy(ctx)
    assert status == lq.LQ_OK and st["converged"] == 1
    assert st["true_rel_resid"] <= 1e-10 and res <= 1e-10
    assert rel_err(got, x_ref) < X_TOL
    n = st["iterations"]
    assert n > 0 and np.all(hist[:n] > 0)
    if prec == 0:
        # same algorithm and stopping rule: the iteration count agrees up to rounding drift
        assert abs(n - it_ref10) <= max(3, it_ref10 // 20), (n, it_ref10)


@pytest.mark.parametrize("df_updates", [0, 1])
def test_mixed_solve_with_and_without_double_float_updates(lq, df_updates):
    """Reliable updates in FP64 or in double-float (certified in FP64 at the end): same
    iteration count on a well-conditioned system, both to a 1e-10 FP64 residual."""
    dims = (6, 4, 4, 8)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 5)
    phi = source(lat, 5)
    x_ref, _, _ = cg_MdagM(U, phi, dims, 0.15, tol=1e-13)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_set_option(ctx, lq.LQ_OPT_DF64_UPDATES, df_updates)
        lq.lq_gauge_set(ctx, dev(U))
        x = torch.zeros_like(dev(phi))
        status, st = lq.lq_solve_MdagM(ctx, x, dev(phi), 0.15, 1e-10, 5000, lq.LQ_F32_12, 20)
        got = host(x)
    finally:
        lq.lq_destroy(ctx)
    assert status == lq.LQ_OK and st["true_rel_resid"] <= 1e-10
    assert rel_err(got, x_ref) < X_TOL
    assert st["reliable_updates"] >= 2


def test_kappa_zero_is_identity(lq):
    """kappa = 0: M = 1, so M^dag M x = phi gives x = phi in one iteration."""
    dims = (4, 2, 2, 6)
    lat = Lattice(dims)
    phi = source(lat, 4)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(gauge_exp_iA(lat, 0.3, 4)))
        for prec in (lq.LQ_F64, lq.LQ_I16_12):
            x = torch.zeros_like(dev(phi))
            status, st = lq.lq_solve_MdagM(ctx, x, dev(phi), 0.0, 1e-10, 100, prec, 50)
            # FP64: one iteration; 16-bit storage: a few, each removing the rounding of the last
            assert status == lq.LQ_OK and st["iterations"] <= (1 if prec == lq.LQ_F64 else 8)
            assert rel_err(host(x), phi) < 1e-10
    finally:
        lq.lq_destroy(ctx)


def test_zero_source_and_errors(lq):
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 1)
    ctx = lq.lq_create(dims)
    try:
        x = torch.ones((lat.V, 4, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(lq.LQError) as e:
            lq.lq_solve_MdagM(ctx, x, torch.zeros_like(x), 0.15)
        assert e.value.status == lq.LQ_ERR_STATE         # no gauge field yet
        lq.lq_gauge_set(ctx, dev(U))
        status, st = lq.lq_solve_MdagM(ctx, x, torch.zeros_like(x), 0.15)
        assert status == lq.LQ_OK and st["iterations"] == 0
        assert float(x.abs().max()) == 0.0
        phi = dev(source(lat, 3))
        status, st = lq.lq_solve_MdagM(ctx, x, phi, 0.15, 1e-10, 5)
        assert status == lq.LQ_ERR_NOT_CONVERGED and st["iterations"] == 5 and st["true_rel_resid"] > 1e-10
        bad = phi.clone()
        bad[3, 1, 2] = complex(float("nan"), 0.0)
        with pytest.raises(lq.LQError) as e:
            lq.lq_solve_MdagM(ctx, x, bad, 0.15)
        assert e.value.status == lq.LQ_ERR_NAN
        with pytest.raises(lq.LQError):
            lq.lq_solve_MdagM(ctx, x, phi, 0.15, -1.0)
        with pytest.raises(lq.LQError):
            lq.lq_solve_MdagM(ctx, x, phi, 0.15, 1e-10, 100, lq.LQ_DF64)   # operator-only precision
    finally:
        lq.lq_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 6])
def test_graphs_and_direct_launches_give_identical_solves(lq, prec):
    """The CUDA-graph replay launches the same kernels in the same order as direct
    launches, and every reduction has a fixed order: the solution, the iteration count
    and the residual agree bit for bit.  An unknown option is refused."""
    dims = (6, 4, 4, 8)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 4)
    phi = source(lat, 9)
    out = {}
    for graphs in (1, 0):
        ctx = lq.lq_create(dims)
        try:
            lq.lq_set_option(ctx, lq.LQ_OPT_CUDA_GRAPHS, graphs)
            lq.lq_gauge_set(ctx, dev(U))
            x = torch.zeros_like(dev(phi))
            status, st = lq.lq_solve_MdagM(ctx, x, dev(phi), 0.155, 1e-10, 5000, prec, 50)
            assert status == lq.LQ_OK
            out[graphs] = (host(x), st["iterations"], st["true_rel_resid"])
            if graphs == 0:
                with pytest.raises(lq.LQError) as e:
                    lq.lq_set_option(ctx, 99, 1)
                assert e.value.status == lq.LQ_ERR_ARG
        finally:
            lq.lq_destroy(ctx)
    assert np.array_equal(out[1][0], out[0][0])
    assert out[1][1:] == out[0][1:]


def test_16bit_solves_keep_the_fp64_iteration_count(lq):
    """With the low-precision solution accumulated in FP32, 16-bit storage of the iteration
    vectors costs (almost) no iterations against plain FP64 CG (8^4, kappa 0.156)."""
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.25, 2)
    phi = source(lat, 7)
    ctx = lq.lq_create(dims)
    its = {}
    try:
        lq.lq_gauge_set(ctx, dev(U))
        for prec in (0, 3, 4, 6):
            x = torch.zeros_like(dev(phi))
            status, st = lq.lq_solve_MdagM(ctx, x, dev(phi), 0.156, 1e-10, 5000, prec, 50)
            assert status == lq.LQ_OK and st["true_rel_resid"] <= 1e-10
            its[prec] = st["iterations"]
    finally:
        lq.lq_destroy(ctx)
    assert its[3] <= 1.05 * its[0] + 5, its      # FP16-12
    assert its[6] <= 1.05 * its[0] + 5, its      # 16-bit fixed point
    assert its[4] <= 1.3 * its[0] + 5, its       # BF16-12 (8-bit significand)


def test_full_size_mixed_and_f64_solves(lq):
    """32^3 x 64, sigma 0.25, seed 2, kappa 0.156: FP16, BF16, fixed-point and FP64 solves all
    reach a 1e-10 FP64 true residual, and agree with each other within the conditioning bound.
    The oracle checks each solution independently: it evaluates M^dag M x at ~200 sampled
    sites from their neighbourhoods (no GPU arithmetic involved), which must agree element by
    element with the GPU's FP64 M^dag M x there, and the residual phi - M^dag M x over the
    sample must be of the size the solver certified."""
    from oracle.wilson import apply_MdagM_sites
    dims = (32, 32, 32, 64)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.25, 2)
    phi_h = source(lat, 2)
    phi = dev(phi_h)
    rng = np.random.default_rng(5)
    sites = np.unique(np.concatenate([rng.integers(0, lat.V, 200), [0, lat.V - 1, 32 ** 3 * 63]]))
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        xs = {}
        for prec in (lq.LQ_F16_12, lq.LQ_BF16_12, lq.LQ_I16_12, lq.LQ_F64):
            x = torch.zeros_like(phi)
            status, st = lq.lq_solve_MdagM(ctx, x, phi, 0.156, 1e-10, 20000, prec, 50)
            assert status == lq.LQ_OK and st["true_rel_resid"] <= 1e-10, st
            r = torch.empty_like(x)
            lq.lq_apply_MdagM(ctx, r, x, 0.156, lq.LQ_F64)
            assert float(torch.linalg.vector_norm(phi - r) / torch.linalg.vector_norm(phi)) <= 1e-10
            xh = host(x)
            Ax = apply_MdagM_sites(U, xh, dims, 0.156, sites)
            assert rel_err(host(r)[sites], Ax) < 1e-13, prec
            res = np.linalg.norm(phi_h[sites] - Ax) / np.linalg.norm(phi_h[sites])
            assert res <= 3e-10, (prec, res)
            xs[prec] = x
        for prec in (lq.LQ_F16_12, lq.LQ_BF16_12, lq.LQ_I16_12):
            d = float(torch.linalg.vector_norm(xs[prec] - xs[lq.LQ_F64]) / torch.linalg.vector_norm(xs[lq.LQ_F64]))
            assert d < X_TOL, (prec, d)
    finally:
        lq.lq_destroy(ctx)
