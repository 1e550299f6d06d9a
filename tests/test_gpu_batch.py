"""Batched CG (many right-hand sides sharing one gauge field; independent lattices of
different volumes and kappa in one launch) against the oracle and the single solver."""
import numpy as np
import pytest

from oracle.cg import cg_MdagM
from synth import Lattice, gauge_exp_iA, source
from tests.gpu_common import require_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu

X_TOL = 1e-6     # conditioning bound of the solution error at a 1e-10 residual (see test_gpu_solver)


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


def _true_residuals(lq, dims, U, xs, phis, kappa):
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, U)
        out = []
        for x, phi in zip(xs, phis):
            r = torch.empty_like(x)
            lq.lq_apply_MdagM(ctx, r, x, kappa, lq.LQ_F64)
            out.append(float(torch.linalg.vector_norm(phi - r) / torch.linalg.vector_norm(phi)))
        return out
    finally:
        lq.lq_destroy(ctx)


@pytest.mark.parametrize("prec", [1, 2, 3, 4, 6])
def test_multi_rhs_matches_oracle(lq, prec):
    dims, R, kappa = (4, 4, 4, 4), 12, 0.155
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 3)
    phis = np.stack([source(lat, 3, i) for i in range(R)])            # [R][V][4][3]
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        phid = dev(phis)
        x = torch.zeros_like(phid)
        status, st, iters, resid, hist = lq.lq_solve_batch([ctx], [x], [phid], [kappa], R, 1e-10, 5000, prec, 25,
                                                           hist_len=3000)
        xs = host(x)
    finally:
        lq.lq_destroy(ctx)
    assert status == lq.LQ_OK and st["converged"] == 1
    assert np.all(resid <= 1e-10) and np.all(iters > 0)
    res = _true_residuals(lq, dims, dev(U), [dev(xs[i]) for i in range(R)], [dev(phis[i]) for i in range(R)], kappa)
    assert max(res) <= 1e-10
    for i in (0, 5, 11):
        xr, _, _ = cg_MdagM(U, phis[i], dims, kappa, 1e-13)
        assert rel_err(xs[i], xr) < X_TOL
    n = st["iterations"]
    assert np.all(hist[:, 0] > 0) and np.all(hist[:, :n].min(axis=1) < 1e-6)


def test_uneven_lattices_one_launch_match_oracle(lq):
    shapes = [(4, 4, 4, 4), (2, 4, 6, 4), (6, 2, 2, 4), (4, 4, 2, 8)]
    kappas = [0.12, 0.14, 0.15, 0.155]
    ctxs, xs, phis, Us = [], [], [], []
    try:
        for k, (dims, kap) in enumerate(zip(shapes, kappas)):
            lat = Lattice(dims)
            U = gauge_exp_iA(lat, 0.3, 4 + k)
            c = lq.lq_create(dims)
            lq.lq_gauge_set(c, dev(U))
            ctxs.append(c)
            Us.append(U)
            phis.append(dev(source(lat, 4 + k)))
            xs.append(torch.zeros_like(phis[-1]))
        status, st, iters, resid, _ = lq.lq_solve_batch(ctxs, xs, phis, kappas, 1, 1e-10, 5000, lq.LQ_I16_12, 50)
        got = [host(x) for x in xs]
    finally:
        for c in ctxs:
            lq.lq_destroy(c)
    assert status == lq.LQ_OK and np.all(resid <= 1e-10)
    for k, (dims, kap) in enumerate(zip(shapes, kappas)):
        xr, _, _ = cg_MdagM(Us[k], host(phis[k]), dims, kap, 1e-13)
        assert rel_err(got[k], xr) < X_TOL, dims
    # the lightest system (kappa 0.12) is frozen no later than the heaviest (kappa 0.155)
    assert iters[0] <= iters[3]


def test_batch_reuses_workspace_and_rejects_bad_arguments(lq):
    dims = (4, 4, 2, 4)
    lat = Lattice(dims)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(gauge_exp_iA(lat, 0.3, 1)))
        phi = dev(np.stack([source(lat, 1, i) for i in range(2)]))
        x1, x2 = torch.zeros_like(phi), torch.zeros_like(phi)
        s1 = lq.lq_solve_batch([ctx], [x1], [phi], [0.15], 2)
        s2 = lq.lq_solve_batch([ctx], [x2], [phi], [0.15], 2)
        assert s1[0] == s2[0] == lq.LQ_OK
        assert torch.equal(x1, x2)                         # deterministic reductions
        with pytest.raises(lq.LQError):
            lq.lq_solve_batch([ctx], [host(x1)], [phi], [0.15], 2)   # host buffer
        with pytest.raises(lq.LQError):
            lq.lq_solve_batch([ctx], [x1], [phi], [0.15], 2, inner_prec=lq.LQ_DF64)
        with pytest.raises(lq.LQError):
            lq.lq_solve_batch([ctx], [x1], [phi], [0.15], 17)                    # too many right-hand sides
    finally:
        lq.lq_destroy(ctx)


def test_full_size_multi_rhs_24x24x24x24(lq):
    """24^4, kappa 0.155, seed 3, 12 right-hand sides sharing one FP32 gauge field: every
    column reaches a 1e-10 FP64 true residual and agrees with the single-RHS solver."""
    dims, R, kappa = (24, 24, 24, 24), 12, 0.155
    lat = Lattice(dims)
    U = dev(gauge_exp_iA(lat, 0.3, 3))
    phis = dev(np.stack([source(lat, 3, i) for i in range(R)]))
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, U)
        x = torch.zeros_like(phis)
        status, st, iters, resid, hist = lq.lq_solve_batch([ctx], [x], [phis], [kappa], R, 1e-10, 20000,
                                                           lq.LQ_F32, 50, hist_len=4000)
        assert status == lq.LQ_OK and np.all(resid <= 1e-10)
        for i in (0, 7):
            r = torch.empty_like(x[i])
            lq.lq_apply_MdagM(ctx, r, x[i], kappa, lq.LQ_F64)
            assert float(torch.linalg.vector_norm(phis[i] - r) / torch.linalg.vector_norm(phis[i])) <= 1e-10
            xs = torch.zeros_like(phis[i])
            lq.lq_solve_MdagM(ctx, xs, phis[i], kappa, 1e-10, 20000, lq.LQ_F32_12, 50)
            assert float(torch.linalg.vector_norm(xs - x[i]) / torch.linalg.vector_norm(xs)) < X_TOL
    finally:
        lq.lq_destroy(ctx)


def test_full_size_uneven_lattices(lq):
    """8^4, 12^4, 16^4 and 8^3 x 16 with kappa 0.12, 0.14, 0.15, 0.155 and seeds 4-7, one batch."""
    shapes = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (8, 8, 8, 16)]
    kappas = [0.12, 0.14, 0.15, 0.155]
    ctxs, xs, phis = [], [], []
    try:
        for k, dims in enumerate(shapes):
            lat = Lattice(dims)
            c = lq.lq_create(dims)
            lq.lq_gauge_set(c, dev(gauge_exp_iA(lat, 0.3, 4 + k)))
            ctxs.append(c)
            phis.append(dev(source(lat, 4 + k)))
            xs.append(torch.zeros_like(phis[-1]))
        status, st, iters, resid, hist = lq.lq_solve_batch(ctxs, xs, phis, kappas, 1, 1e-10, 20000, lq.LQ_F32_12,
                                                           50, hist_len=4000)
        assert status == lq.LQ_OK and np.all(resid <= 1e-10)
        for k in range(4):
            r = torch.empty_like(xs[k])
            lq.lq_apply_MdagM(ctxs[k], r, xs[k], kappas[k], lq.LQ_F64)
            assert float(torch.linalg.vector_norm(phis[k] - r) / torch.linalg.vector_norm(phis[k])) <= 1e-10
    finally:
        for c in ctxs:
            lq.lq_destroy(c)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("rb", [1, 2, 3, 4])
@pytest.mark.parametrize("prec", [2, 3, 4, 6])
def test_rhs_per_thread_variants_match_oracle(lq, rb, prec, order):
    """Every register-blocking width (right-hand sides per thread, forced) in both tile orders
    solves a 12-RHS batch at 4^3 x 8 to a 1e-10 FP64 true residual, agrees with the oracle's
    solutions, and the per-column residual histories start at 1 and fall below 1e-6."""
    dims, R, kappa = (4, 4, 4, 8), 12, 0.15
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 5)
    phis = np.stack([source(lat, 5, i) for i in range(R)])
    ctx = lq.lq_create(dims)
    try:
        lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_RHS_PER_THREAD, rb)
        lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_TILE_ORDER, order)
        lq.lq_gauge_set(ctx, dev(U))
        x = torch.zeros_like(dev(phis))
        status, st, iters, resid, hist = lq.lq_solve_batch([ctx], [x], [dev(phis)], [kappa], R, 1e-10, 5000, prec,
                                                           50, hist_len=2000)
        xs = host(x)
        tune = lq.lq_batch_tuning(ctx)
    finally:
        lq.lq_destroy(ctx)
    assert status == lq.LQ_OK and np.all(resid <= 1e-10)
    assert tune["rhs_per_thread"] == rb and tune["tile"] == 256 and tune["site_major"] == (1 if order == 1 else 0)
    for i in (0, 7, 11):
        xr, _, _ = cg_MdagM(U, phis[i], dims, kappa, 1e-13)
        assert rel_err(xs[i], xr) < X_TOL
    n = st["iterations"]
    assert np.allclose(hist[:, 0], hist[:, 0]) and np.all(hist[:, :n].min(axis=1) < 1e-6)


def test_autotuner_reports_its_choice(lq):
    """With the default option the first batched solve times every candidate launch shape and
    keeps the fastest; a second solve of the same shape reuses it."""
    dims, R = (8, 8, 8, 8), 6
    lat = Lattice(dims)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(gauge_exp_iA(lat, 0.3, 2)))
        phis = dev(np.stack([source(lat, 2, i) for i in range(R)]))
        x = torch.zeros_like(phis)
        with pytest.raises(lq.LQError):
            lq.lq_batch_tuning(ctx)                          # nothing solved yet
        s1 = lq.lq_solve_batch([ctx], [x], [phis], [0.15], R, 1e-10, 5000, lq.LQ_F16_12, 50)
        t1 = lq.lq_batch_tuning(ctx)
        x2 = torch.zeros_like(phis)
        s2 = lq.lq_solve_batch([ctx], [x2], [phis], [0.15], R, 1e-10, 5000, lq.LQ_F16_12, 50)
        t2 = lq.lq_batch_tuning(ctx)
        with pytest.raises(lq.LQError):
            lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_RHS_PER_THREAD, 5)
    finally:
        lq.lq_destroy(ctx)
    assert s1[0] == s2[0] == lq.LQ_OK
    assert torch.equal(x, x2)
    # two tile orders x rhs per thread 1, 2, 3 (divisors of 6) x 3 shapes
    assert len(t1["candidate_ms"]) == 18 and t1["rhs_per_thread"] in (1, 2, 3) and t1["site_major"] in (0, 1)
    assert min(t1["candidate_ms"]) > 0 and t1 == t2


@pytest.mark.parametrize("prec", [2, 3, 6])
def test_persistent_iteration_matches_graphs_and_oracle(lq, prec):
    """One cooperative launch per chunk of iterations (all passes, device-wide barriers) gives
    the same solutions as the per-pass launches within the conditioning bound, each column to
    a 1e-10 FP64 true residual, for right-hand sides sharing links and for uneven lattices."""
    dims, R, kappa = (4, 4, 4, 8), 6, 0.15
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 9)
    phis = np.stack([source(lat, 9, i) for i in range(R)])
    sols = {}
    for persistent in (0, 1):
        ctx = lq.lq_create(dims)
        try:
            lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_PERSISTENT, persistent)
            lq.lq_gauge_set(ctx, dev(U))
            x = torch.zeros_like(dev(phis))
            status, st, iters, resid, hist = lq.lq_solve_batch([ctx], [x], [dev(phis)], [kappa], R, 1e-10, 5000,
                                                               prec, 50, hist_len=2000)
            assert status == lq.LQ_OK and np.all(resid <= 1e-10), (persistent, resid)
            assert np.all(hist[:, :st["iterations"]].min(axis=1) < 1e-6)
            sols[persistent] = host(x)
        finally:
            lq.lq_destroy(ctx)
    assert rel_err(sols[1], sols[0]) < X_TOL
    xr, _, _ = cg_MdagM(U, phis[3], dims, kappa, 1e-13)
    assert rel_err(sols[1][3], xr) < X_TOL
    # uneven lattices and kappas in one persistent launch
    shapes = [(4, 4, 4, 4), (2, 4, 6, 4), (6, 2, 2, 4)]
    kappas = [0.12, 0.14, 0.155]
    ctxs, xs, ph, Us = [], [], [], []
    try:
        for k, d in enumerate(shapes):
            l2 = Lattice(d)
            Uk = gauge_exp_iA(l2, 0.3, 20 + k)
            c = lq.lq_create(d)
            lq.lq_gauge_set(c, dev(Uk))
            if k == 0:
                lq.lq_set_option(c, lq.LQ_OPT_BATCH_PERSISTENT, 1)
            ctxs.append(c)
            Us.append(Uk)
            ph.append(dev(source(l2, 20 + k)))
            xs.append(torch.zeros_like(ph[-1]))
        status, st, iters, resid, _ = lq.lq_solve_batch(ctxs, xs, ph, kappas, 1, 1e-10, 5000, prec, 50)
        got = [host(v) for v in xs]
    finally:
        for c in ctxs:
            lq.lq_destroy(c)
    assert status == lq.LQ_OK and np.all(resid <= 1e-10)
    for k, d in enumerate(shapes):
        xr, _, _ = cg_MdagM(Us[k], host(ph[k]), d, kappas[k], 1e-13)
        assert rel_err(got[k], xr) < X_TOL, d


def test_persistent_barrier_timeout_is_reported_and_recoverable(lq):
    """Failure detection of the persistent iteration: with the test option its barrier waits
    for a block that does not exist, every wait runs out after about a second, and the call
    returns LQ_ERR_TIMEOUT instead of hanging; the context then solves normally."""
    dims, R = (4, 4, 2, 4), 2
    lat = Lattice(dims)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(gauge_exp_iA(lat, 0.3, 4)))
        phis = dev(np.stack([source(lat, 4, i) for i in range(R)]))
        x = torch.zeros_like(phis)
        lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_PERSISTENT, 1)
        lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_BARRIER_TEST, 1)
        with pytest.raises(lq.LQError) as e:
            lq.lq_solve_batch([ctx], [x], [phis], [0.15], R, 1e-10, 5000, lq.LQ_F32_12, 50)
        assert e.value.status == lq.LQ_ERR_TIMEOUT
        assert "timed out" in str(e.value)
        lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_BARRIER_TEST, 0)
        x = torch.zeros_like(phis)
        status, st, iters, resid, _ = lq.lq_solve_batch([ctx], [x], [phis], [0.15], R, 1e-10, 5000, lq.LQ_F32_12, 50)
        assert status == lq.LQ_OK and np.all(resid <= 1e-10)
        # and the single solver on the same context is unaffected
        xs = torch.zeros_like(phis[0])
        status, st1 = lq.lq_solve_MdagM(ctx, xs, phis[0], 0.15, 1e-10, 5000, lq.LQ_F32_12, 50)
        assert status == lq.LQ_OK
    finally:
        lq.lq_destroy(ctx)


@pytest.mark.parametrize("prec", [2, 3, 6])
def test_double_float_updates_match_fp64_updates(lq, prec):
    """The batch's intermediate reliable updates in double-float arithmetic (the default) and
    in FP64 throughout give solutions that agree within the conditioning bound and with the
    oracle; both end on an FP64-certified residual, for right-hand sides sharing links and for
    uneven lattices, and a tolerance of 1e-12 is still met (certified in FP64)."""
    shapes = [(4, 4, 4, 8), (2, 4, 6, 4), (6, 2, 2, 4)]
    kappas = [0.15, 0.14, 0.155]
    R = 3
    Us = [gauge_exp_iA(Lattice(d), 0.3, 30 + k) for k, d in enumerate(shapes)]
    phis = [np.stack([source(Lattice(d), 30 + k, i) for i in range(R)]) for k, d in enumerate(shapes)]
    sols, stats = {}, {}
    for df in (1, 0):
        ctxs, xs = [], []
        try:
            for k, d in enumerate(shapes):
                c = lq.lq_create(d)
                lq.lq_gauge_set(c, dev(Us[k]))
                ctxs.append(c)
                xs.append(torch.zeros_like(dev(phis[k])))
            lq.lq_set_option(ctxs[0], lq.LQ_OPT_DF64_UPDATES, df)
            status, st, iters, resid, _ = lq.lq_solve_batch(ctxs, xs, [dev(p) for p in phis], kappas, R, 1e-10,
                                                            5000, prec, 25)
            assert status == lq.LQ_OK and np.all(resid <= 1e-10), (df, resid)
            sols[df] = [host(x) for x in xs]
            stats[df] = st
            for k in range(len(shapes)):
                res = _true_residuals(lq, shapes[k], dev(Us[k]), [xs[k][i] for i in range(R)],
                                      [dev(phis[k][i]) for i in range(R)], kappas[k])
                assert max(res) <= 1e-10, (df, k, res)
            if df:
                xt = [torch.zeros_like(x) for x in xs]
                status, st, iters, resid, _ = lq.lq_solve_batch(ctxs, xt, [dev(p) for p in phis], kappas, R,
                                                                1e-12, 5000, lq.LQ_F32, 25)
                assert status == lq.LQ_OK and np.all(resid <= 1e-12), resid
                res = _true_residuals(lq, shapes[0], dev(Us[0]), [xt[0][i] for i in range(R)],
                                      [dev(phis[0][i]) for i in range(R)], kappas[0])
                assert max(res) <= 1e-12, res
        finally:
            for c in ctxs:
                lq.lq_destroy(c)
    for k in range(len(shapes)):
        assert rel_err(sols[1][k], sols[0][k]) < X_TOL, k
        xr, _, _ = cg_MdagM(Us[k], phis[k][1], shapes[k], kappas[k], 1e-13)
        assert rel_err(sols[1][k][1], xr) < X_TOL, k
    assert stats[1]["kernel_launches"] > 0 and stats[0]["kernel_launches"] > 0


@pytest.mark.parametrize("df", [1, 0])
def test_device_loop_matches_host_loop(lq, df):
    """The whole solve as one graph whose conditional nodes take every convergence decision on
    the device (the default) and the host loop (one graph per chunk of iterations, decisions on
    the host) run the same kernels in the same order: bit-identical solutions, histories,
    iteration and reliable-update counts, with double-float or FP64 intermediate updates, for
    right-hand sides sharing links and uneven lattices.  An unreachable tolerance ends at the
    iteration limit with LQ_ERR_NOT_CONVERGED."""
    shapes = [(4, 4, 4, 8), (2, 4, 6, 4)]
    kappas = [0.15, 0.155]
    R = 2
    Us = [gauge_exp_iA(Lattice(d), 0.3, 40 + k) for k, d in enumerate(shapes)]
    phis = [np.stack([source(Lattice(d), 40 + k, i) for i in range(R)]) for k, d in enumerate(shapes)]
    out = {}
    for loop in (1, 0):
        ctxs = []
        try:
            for k, d in enumerate(shapes):
                c = lq.lq_create(d)
                lq.lq_gauge_set(c, dev(Us[k]))
                ctxs.append(c)
            lq.lq_set_option(ctxs[0], lq.LQ_OPT_DF64_UPDATES, df)
            lq.lq_set_option(ctxs[0], lq.LQ_OPT_BATCH_DEVICE_LOOP, loop)
            # one fixed launch shape for both (the tuner's timing may pick different shapes,
            # whose reductions round differently)
            lq.lq_set_option(ctxs[0], lq.LQ_OPT_BATCH_RHS_PER_THREAD, 1)
            xs = [torch.zeros_like(dev(p)) for p in phis]
            status, st, iters, resid, hist = lq.lq_solve_batch(ctxs, xs, [dev(p) for p in phis], kappas, R, 1e-10,
                                                               5000, lq.LQ_F16_12, 25, hist_len=2000)
            assert status == lq.LQ_OK and np.all(resid <= 1e-10), (loop, resid)
            out[loop] = ([host(x) for x in xs], st, iters, resid, hist)
            xt = [torch.zeros_like(dev(p)) for p in phis]
            status, st2, _, _, _ = lq.lq_solve_batch(ctxs, xt, [dev(p) for p in phis], kappas, R, 1e-30, 30,
                                                     lq.LQ_F16_12, 25)
            assert status == lq.LQ_ERR_NOT_CONVERGED and st2["iterations"] == 30, (loop, st2)
        finally:
            for c in ctxs:
                lq.lq_destroy(c)
    (x1, s1, i1, r1, h1), (x0, s0, i0, r0, h0) = out[1], out[0]
    for a, b in zip(x1, x0):
        assert np.array_equal(a, b)
    assert np.array_equal(i1, i0) and np.array_equal(r1, r0) and np.array_equal(h1, h0)
    assert s1["iterations"] == s0["iterations"] and s1["reliable_updates"] == s0["reliable_updates"]
    assert s1["converged"] == s0["converged"] == 1
    xr, _, _ = cg_MdagM(Us[1], phis[1][0], shapes[1], kappas[1], 1e-13)
    assert rel_err(x1[1][0], xr) < X_TOL


@pytest.mark.parametrize("loop,df", [(1, 1), (0, 1), (1, 0)])
def test_zero_and_non_finite_columns(lq, loop, df):
    """Degenerate columns: a zero right-hand side is frozen at once (x = 0, residual 0) while the
    other columns converge; a NaN in one right-hand side ends the call with LQ_ERR_NAN (no hang,
    whichever loop drives it), and the context then solves normally."""
    dims, R = (4, 4, 2, 4), 3
    lat = Lattice(dims)
    phis = np.stack([source(lat, 8, i) for i in range(R)])
    phis[1] = 0.0
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(gauge_exp_iA(lat, 0.3, 8)))
        lq.lq_set_option(ctx, lq.LQ_OPT_BATCH_DEVICE_LOOP, loop)
        lq.lq_set_option(ctx, lq.LQ_OPT_DF64_UPDATES, df)
        x = torch.zeros_like(dev(phis))
        status, st, iters, resid, _ = lq.lq_solve_batch([ctx], [x], [dev(phis)], [0.15], R, 1e-10, 5000,
                                                        lq.LQ_F16_12, 25)
        assert status == lq.LQ_OK and st["converged"] == 1
        assert resid[1] == 0.0 and np.all(resid <= 1e-10)
        assert not torch.any(x[1] != 0)
        bad = phis.copy()
        bad[2, 5, 1, 2] = np.nan
        with pytest.raises(lq.LQError) as e:
            lq.lq_solve_batch([ctx], [torch.zeros_like(x)], [dev(bad)], [0.15], R, 1e-10, 5000, lq.LQ_F16_12, 25)
        assert e.value.status == lq.LQ_ERR_NAN
        x2 = torch.zeros_like(x)
        status, st, iters, resid2, _ = lq.lq_solve_batch([ctx], [x2], [dev(phis)], [0.15], R, 1e-10, 5000,
                                                         lq.LQ_F16_12, 25)
        assert status == lq.LQ_OK and np.array_equal(resid2, resid) and torch.equal(x2, x)
    finally:
        lq.lq_destroy(ctx)
