"""Parity of the CUDA Wilson operator (Eq. 4; Sec. 3 kernel 1) with the FP64 oracle."""
import numpy as np
import pytest

from oracle.wilson import apply_M as o_apply_M, apply_MdagM as o_apply_MdagM
from synth import Lattice, gauge_exp_iA, source, identity_gauge, plane_wave
from tests.gpu_common import require_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu

# FP64 bound: relative 1e-12.  Lower precisions: relative error of the
# storage format (FP32 2^-24, FP16 2^-11 relative to the site norm, BF16
# 2^-8) times a small factor for the ~100 operations per output.
# Double-float (LQ_DF64, ~48-bit significands): 1e-12 as for FP64.  16-bit fixed point
# (LQ_I16_12): rounding 2^-16 of the site maximum for spinors and of 1 for links.
TOL = {0: 1e-12, 1: 2e-6, 2: 2e-6, 3: 2e-3, 4: 1.5e-2, 5: 1e-12, 6: 2e-4}

SHAPES = [(4, 4, 4, 4), (2, 2, 2, 2), (6, 4, 2, 6), (3, 5, 2, 7), (8, 8, 8, 16)]

# Element-by-element bounds.  Output site s of M psi reads psi at s and its eight
# neighbours, each rounded to the storage format relative to its own site maximum
# (spinors) or to 1 (links), then about 100 arithmetic operations, and the output is
# rounded to the format again; the error of every component is bounded by a small
# multiple of the format's unit roundoff times the local scale L(s) = max |psi| over
# those nine sites (the links are unitary).  Unit roundoffs: FP32 2^-24, FP16 2^-11,
# BF16 2^-8, 16-bit fixed point 2^-15 (2^-16 on the links), double-float ~2^-48
# (given as 2^-46), FP64 2^-53 (given as 2^-50: ~100 roundings); the factor 16 covers
# the nine inputs, the link rounding, the arithmetic and the rounding of the output.
UNIT = {0: 2.0 ** -50, 1: 2.0 ** -24, 2: 2.0 ** -24, 3: 2.0 ** -11, 4: 2.0 ** -8, 5: 2.0 ** -46, 6: 2.0 ** -15}
ELEM_FACTOR = 16.0


def local_scale(psi, dims, sites=None):
    """max |psi| (real or imaginary part) over each site and its eight neighbours."""
    from oracle.conventions import neighbours
    fwd, bwd, _, _ = neighbours(dims, True)
    m = np.maximum(np.abs(psi.real), np.abs(psi.imag)).reshape(psi.shape[0], -1).max(axis=1)
    idx = np.arange(psi.shape[0]) if sites is None else np.asarray(sites)
    L = m[idx]
    for mu in range(4):
        L = np.maximum(L, np.maximum(m[fwd[mu][idx]], m[bwd[mu][idx]]))
    return L


def elementwise_ratio(got, ref, L):
    """max over sites of (largest component error at the site) / (local scale at the site)."""
    d = np.abs(got - ref).reshape(got.shape[0], -1).max(axis=1)
    return float(np.max(d / L))


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


def _setup(dims, seed=1, sigma=0.3):
    lat = Lattice(dims)
    return lat, gauge_exp_iA(lat, sigma, seed), source(lat, seed, 0)


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_M_f64(lq, dims, dagger):
    lat, U, psi = _setup(dims)
    kappa = 0.155
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        out = torch.empty_like(dev(psi))
        lq.lq_apply_M(ctx, out, dev(psi), kappa, dagger, lq.LQ_F64)
        got = host(out)
    finally:
        lq.lq_destroy(ctx)
    ref = o_apply_M(U, psi, dims, kappa, dagger=dagger)
    assert rel_err(got, ref) < TOL[0]
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_M_low_precision(lq, prec, dagger):
    dims = (4, 4, 6, 8)
    lat, U, psi = _setup(dims, seed=2)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        out = torch.empty_like(dev(psi))
        lq.lq_apply_M(ctx, out, dev(psi), 0.15, dagger, prec)
        got = host(out)
    finally:
        lq.lq_destroy(ctx)
    ref = o_apply_M(U, psi, dims, 0.15, dagger=dagger)
    assert rel_err(got, ref) < TOL[prec]
    # every site, every component, against the format's bound relative to the local scale
    ratio = elementwise_ratio(got, ref, local_scale(psi, dims))
    assert ratio < ELEM_FACTOR * UNIT[prec], (prec, ratio, ELEM_FACTOR * UNIT[prec])


def test_apply_MdagM_f64_and_host_buffers(lq):
    """Host (numpy) buffers go through the same call; results equal the device path bit for bit."""
    dims = (4, 2, 4, 6)
    lat, U, psi = _setup(dims, seed=3)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, U)                    # host buffer
        out_h = np.empty_like(psi)
        lq.lq_apply_MdagM(ctx, out_h, psi, 0.14)
        out_d = torch.empty_like(dev(psi))
        lq.lq_apply_MdagM(ctx, out_d, dev(psi), 0.14)
        got_d = host(out_d)
        Uback = np.empty_like(U)
        lq.lq_gauge_get(ctx, Uback)
    finally:
        lq.lq_destroy(ctx)
    ref = o_apply_MdagM(U, psi, dims, 0.14)
    assert rel_err(out_h, ref) < 1e-12
    assert np.array_equal(out_h, got_d)
    assert np.array_equal(Uback, U)


@pytest.mark.parametrize("dims", [(4, 2, 4, 6), (5, 3, 7, 5)])
def test_page_locked_host_buffers_in_place(lq, dims):
    """With LQ_OPT_HOST_DIRECT the packing kernels read and write page-locked host buffers in
    place: gauge in and out, right-hand side in, result out, and a solve, all bit-identical
    to the staged path; pageable host buffers are still staged.  Volumes that are not a
    multiple of the packing tiles (64 sites for links, 128 for spinors) cover the ragged
    tile."""
    lat, U, psi = _setup(dims, seed=4)
    Up, psip = torch.from_numpy(U).pin_memory(), torch.from_numpy(psi).pin_memory()
    res = {}
    for direct in (0, 1):
        ctx = lq.lq_create(dims)
        try:
            lq.lq_set_option(ctx, lq.LQ_OPT_HOST_DIRECT, direct)
            lq.lq_gauge_set(ctx, Up)
            out_p = torch.empty_like(psip).pin_memory()
            lq.lq_apply_MdagM(ctx, out_p, psip, 0.14)
            out_n = np.empty_like(psi)
            lq.lq_apply_MdagM(ctx, out_n, psi, 0.14)                    # pageable: staged
            Ub = torch.empty_like(Up).pin_memory()
            lq.lq_gauge_get(ctx, Ub)
            x = torch.zeros_like(psip).pin_memory()
            status, st = lq.lq_solve_MdagM(ctx, x, psip, 0.14, 1e-10, 5000, lq.LQ_F16_12, 50)
            assert status == lq.LQ_OK
            res[direct] = (out_p.numpy().copy(), out_n, Ub.numpy().copy(), x.numpy().copy())
        finally:
            lq.lq_destroy(ctx)
    ref = o_apply_MdagM(U, psi, dims, 0.14)
    assert rel_err(res[1][0], ref) < 1e-12
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)
    assert np.array_equal(res[1][2], U)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 2, 7), (2, 2, 2, 2), (8, 8, 8, 16)])
def test_double_float_prefetch_variant_is_identical(lq, dims):
    """The double-float operator that prefetches the next hop's operands into shared memory
    (LQ_OPT_DF64_PREFETCH) computes the same arithmetic in the same order: M and M^dag equal the
    plain variant bit for bit (and the FP64 oracle within 1e-12), and so do a mixed solve with
    double-float reliable updates and a batched solve of two right-hand sides."""
    lat, U, psi = _setup(dims, seed=6)
    res = {}
    for pf in (0, 1):
        ctx = lq.lq_create(dims)
        try:
            lq.lq_set_option(ctx, lq.LQ_OPT_DF64_PREFETCH, pf)
            lq.lq_gauge_set(ctx, dev(U))
            outs = []
            for d in (False, True):
                out = torch.empty_like(dev(psi))
                lq.lq_apply_M(ctx, out, dev(psi), 0.15, d, lq.LQ_DF64)
                outs.append(host(out))
            x = torch.zeros_like(dev(psi))
            status, st = lq.lq_solve_MdagM(ctx, x, dev(psi), 0.15, 1e-10, 5000, lq.LQ_F16_12, 25)
            assert status == lq.LQ_OK
            phis = dev(np.stack([psi, source(lat, 6, 1)]))
            xb = torch.zeros_like(phis)
            bstatus, bst, _, bres, _ = lq.lq_solve_batch([ctx], [xb], [phis], [0.15], 2, 1e-10, 5000,
                                                         lq.LQ_F16_12, 25)
            assert bstatus == lq.LQ_OK and np.all(bres <= 1e-10)
            res[pf] = outs + [host(x), host(xb)]
        finally:
            lq.lq_destroy(ctx)
    for d, k in ((False, 0), (True, 1)):
        assert rel_err(res[1][k], o_apply_M(U, psi, dims, 0.15, dagger=d)) < 1e-12
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


def test_free_field_plane_wave(lq):
    """U = 1: the GPU operator reproduces the closed form on a plane wave."""
    dims = (4, 6, 2, 8)
    lat = Lattice(dims)
    u = np.arange(12).reshape(4, 3) * (0.1 + 0.2j) + 1
    psi, p = plane_wave(lat, (1, 2, 1, 3), u)
    from oracle.conventions import GAMMA
    kappa = 0.12
    a = 1 - 2 * kappa * np.sum(np.cos(p))
    K = a * np.eye(4) + 2j * kappa * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(identity_gauge(lat)))
        out = torch.empty_like(dev(psi))
        lq.lq_apply_M(ctx, out, dev(psi), kappa, False, lq.LQ_F64)
        got = host(out)
    finally:
        lq.lq_destroy(ctx)
    assert np.max(np.abs(got - np.matmul(K, psi))) < 1e-13


def test_periodic_time_option(lq):
    dims = (2, 4, 2, 4)
    lat, U, psi = _setup(dims, seed=4)
    ctx = lq.lq_create(dims, t_antiperiodic=False)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        out = torch.empty_like(dev(psi))
        lq.lq_apply_M(ctx, out, dev(psi), 0.13, True, lq.LQ_F64)
        got = host(out)
    finally:
        lq.lq_destroy(ctx)
    ref = o_apply_M(U, psi, dims, 0.13, t_antiperiodic=False, dagger=True)
    assert rel_err(got, ref) < 1e-12


def test_full_size_sampled_sites(lq):
    """32^3 x 64 (sigma 0.25, seed 2, kappa 0.156): sampled output sites against the
    oracle evaluated site by site, in every precision."""
    dims = (32, 32, 32, 64)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.25, 2)
    psi = source(lat, 2)
    rng = np.random.default_rng(0)
    sites = np.unique(np.concatenate([rng.integers(0, lat.V, 200), [0, lat.V - 1, 31, 32 * 32 * 32 * 63]]))
    ref = {d: o_apply_M(U, psi, dims, 0.156, dagger=d, sites=sites) for d in (False, True)}
    L = local_scale(psi, dims, sites)
    ctx = lq.lq_create(dims)
    try:
        Ud = dev(U)
        lq.lq_gauge_set(ctx, Ud)
        del Ud
        pin = dev(psi)
        out = torch.empty_like(pin)
        for prec in (0, 1, 2, 3, 4, 5, 6):
            for d in (False, True):
                lq.lq_apply_M(ctx, out, pin, 0.156, d, prec)
                got = host(out)[sites]
                assert rel_err(got, ref[d]) < TOL[prec], (prec, d)
                ratio = elementwise_ratio(got, ref[d], L)
                assert ratio < ELEM_FACTOR * UNIT[prec], (prec, d, ratio)
    finally:
        lq.lq_destroy(ctx)


# Lattices where hops stay inside and leave the 256-site tiles of the staged stencil:
# L_x = 32 (every x hop in the tile, y hops leave it once per 8 rows), L_x = 2 (forward and
# backward x neighbour coincide), odd extents (tiles cut rows), a partial last tile.
STAGED_SHAPES = [(32, 8, 2, 4), (4, 4, 4, 4), (3, 5, 2, 7), (2, 2, 2, 2), (6, 4, 2, 6), (16, 4, 4, 6)]


@pytest.mark.parametrize("dims", STAGED_SHAPES)
@pytest.mark.parametrize("prec", [1, 2, 3, 4, 6])
def test_staged_stencil_matches_oracle(lq, dims, prec):
    """The stencil that shares x and y links in-block through shared memory equals the
    oracle element by element within the format's bound, for M and M^dag."""
    lat, U, psi = _setup(dims, seed=6)
    ref = {d: o_apply_M(U, psi, dims, 0.152, dagger=d) for d in (False, True)}
    L = local_scale(psi, dims)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_set_option(ctx, lq.LQ_OPT_STAGED, 1)
        lq.lq_gauge_set(ctx, dev(U))
        out = torch.empty_like(dev(psi))
        for d in (False, True):
            lq.lq_apply_M(ctx, out, dev(psi), 0.152, d, prec)
            got = host(out)
            assert rel_err(got, ref[d]) < TOL[prec], (dims, prec, d)
            assert elementwise_ratio(got, ref[d], L) < ELEM_FACTOR * UNIT[prec], (dims, prec, d)
    finally:
        lq.lq_destroy(ctx)


@pytest.mark.parametrize("prec", [3, 6])
def test_staged_cg_passes_and_solve(lq, prec):
    """With the staged stencil the mixed solve at 8^3 x 16 still reaches an FP64 true residual
    of 1e-10 and agrees with the plain-stencil solve within the conditioning bound."""
    dims = (8, 8, 8, 16)
    lat, U, psi = _setup(dims, seed=7)
    xs = {}
    for staged in (0, 1):
        ctx = lq.lq_create(dims)
        try:
            lq.lq_set_option(ctx, lq.LQ_OPT_STAGED, staged)
            lq.lq_gauge_set(ctx, dev(U))
            x = torch.zeros_like(dev(psi))
            status, st = lq.lq_solve_MdagM(ctx, x, dev(psi), 0.155, 1e-10, 5000, prec, 50)
            assert status == lq.LQ_OK and st["true_rel_resid"] <= 1e-10
            xs[staged] = host(x)
        finally:
            lq.lq_destroy(ctx)
    assert rel_err(xs[1], xs[0]) < 1e-6
