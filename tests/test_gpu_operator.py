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
    ctx = lq.lq_create(dims)
    try:
        Ud = dev(U)
        lq.lq_gauge_set(ctx, Ud)
        del Ud
        pin = dev(psi)
        out = torch.empty_like(pin)
        for prec in (0, 1, 3, 5, 6):
            for d in (False, True):
                lq.lq_apply_M(ctx, out, pin, 0.156, d, prec)
                got = host(out)[sites]
                assert rel_err(got, ref[d]) < TOL[prec], (prec, d)
    finally:
        lq.lq_destroy(ctx)
