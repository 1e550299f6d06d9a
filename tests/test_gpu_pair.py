"""The two-site packed stencil for 16-bit fixed-point storage (sites x and x + L_t/2
per thread, FP32x2 arithmetic) against the FP64 oracle (Eq. 4; Sec. 3 kernel 1),
next to the one-site kernel it replaces (LQ_OPT_PAIR_SITES 0)."""
import numpy as np
import pytest

from oracle.wilson import apply_M as o_apply_M
from synth import Lattice, gauge_exp_iA, source
from tests.gpu_common import require_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu

# 16-bit fixed point: rounding 2^-16 of the site maximum for spinors and of 1 for links
TOL_I16 = 2e-4

# L_t = 2 (every time hop wraps), odd extents elsewhere, an odd L_t (one-site fallback),
# a ragged volume that is not a multiple of the block size
SHAPES = [(2, 2, 2, 2), (4, 4, 4, 4), (3, 5, 2, 6), (6, 4, 2, 7), (8, 8, 8, 16), (5, 3, 7, 10)]


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


def _apply(lq, dims, U, psi, kappa, dagger, pair, antiperiodic=True):
    ctx = lq.lq_create(dims, t_antiperiodic=antiperiodic)
    try:
        lq.lq_set_option(ctx, lq.LQ_OPT_PAIR_SITES, pair)
        lq.lq_gauge_set(ctx, dev(U))
        out = torch.empty_like(dev(psi))
        lq.lq_apply_M(ctx, out, dev(psi), kappa, dagger, lq.LQ_I16_12)
        return host(out)
    finally:
        lq.lq_destroy(ctx)


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("antiperiodic", [True, False])
def test_pair_operator_matches_oracle(lq, dims, dagger, antiperiodic):
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 3)
    psi = source(lat, 4)
    ref = o_apply_M(U, psi, dims, 0.155, t_antiperiodic=antiperiodic, dagger=dagger)
    got_pair = _apply(lq, dims, U, psi, 0.155, dagger, 1, antiperiodic)
    got_one = _apply(lq, dims, U, psi, 0.155, dagger, 0, antiperiodic)
    assert rel_err(got_pair, ref) < TOL_I16
    assert rel_err(got_one, ref) < TOL_I16
    # the two kernels compute the same quantised operator up to FP32 rounding and
    # one quantisation step of the 16-bit output
    scale = np.max(np.abs(ref), axis=(1, 2), keepdims=True)
    assert np.max(np.abs(got_pair - got_one) / scale) < 4.0 / 32767


def test_pair_operator_zero_and_sparse_input(lq):
    """A zero field stays zero (zero site norms encode as zero) and a single point
    source spreads to exactly its eight neighbours and itself."""
    dims = (4, 4, 4, 6)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 5)
    zero = np.zeros((lat.V, 4, 3), complex)
    assert np.all(_apply(lq, dims, U, zero, 0.15, False, 1) == 0)
    pt = zero.copy()
    s0 = 1 + 4 * (2 + 4 * (3 + 4 * 5))          # (1, 2, 3, 5): the last time slice
    pt[s0] = np.arange(12).reshape(4, 3) * (0.3 - 0.1j) + 0.5
    got = _apply(lq, dims, U, pt, 0.15, True, 1)
    ref = o_apply_M(U, pt, dims, 0.15, dagger=True)
    assert set(np.flatnonzero(np.abs(got).sum(axis=(1, 2)))) == set(np.flatnonzero(np.abs(ref).sum(axis=(1, 2))))
    assert rel_err(got, ref) < TOL_I16


@pytest.mark.parametrize("pair", [1, 0])
def test_pair_mixed_solve(lq, pair):
    """The 16-bit mixed solve through either kernel reaches the FP64 residual 1e-10 with
    a similar iteration count."""
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.25, 2)
    phi = source(lat, 7)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_set_option(ctx, lq.LQ_OPT_PAIR_SITES, pair)
        lq.lq_gauge_set(ctx, dev(U))
        x = torch.zeros_like(dev(phi))
        status, st = lq.lq_solve_MdagM(ctx, x, dev(phi), 0.156, 1e-10, 5000, lq.LQ_I16_12, 50)
        r = torch.empty_like(x)
        lq.lq_apply_MdagM(ctx, r, x, 0.156, lq.LQ_F64)
        res = np.linalg.norm(phi - host(r)) / np.linalg.norm(phi)
    finally:
        lq.lq_destroy(ctx)
    assert status == lq.LQ_OK and st["converged"] == 1
    assert st["true_rel_resid"] <= 1e-10 and res <= 1e-10
    assert st["iterations"] < 400


def test_pair_full_size_sampled_sites(lq):
    """32^3 x 64 (sigma 0.25, seed 2, kappa 0.156), the launch configuration of the
    benchmark: sampled output sites of the paired operator against the oracle, including
    both time boundaries and the two halves' seam (t = 31, 32)."""
    dims = (32, 32, 32, 64)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.25, 2)
    psi = source(lat, 2)
    rng = np.random.default_rng(1)
    slab = 32 * 32 * 32
    sites = np.unique(np.concatenate([rng.integers(0, lat.V, 200),
                                      [0, lat.V - 1, 31 * slab, 32 * slab, 31 * slab + 5, 32 * slab - 1]]))
    ctx = lq.lq_create(dims)
    try:
        Ud = dev(U)
        lq.lq_gauge_set(ctx, Ud)
        del Ud
        pin = dev(psi)
        out = torch.empty_like(pin)
        for d in (False, True):
            ref = o_apply_M(U, psi, dims, 0.156, dagger=d, sites=sites)
            lq.lq_apply_M(ctx, out, pin, 0.156, d, lq.LQ_I16_12)
            assert rel_err(host(out)[sites], ref) < TOL_I16, d
    finally:
        lq.lq_destroy(ctx)
