"""The naive global-memory Wilson operator and fermion force used for the register
ablation are correct."""
import numpy as np
import pytest

from oracle.fermion import fermion_force_from_X
from oracle.wilson import apply_M
from synth import Lattice, gauge_exp_iA, source
from tests.gpu_common import require_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 5, 2, 7)])
@pytest.mark.parametrize("dagger", [False, True])
def test_naive_operator_matches_oracle(lq, dims, dagger):
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 2)
    psi = source(lat, 2)
    ctx = lq.lq_create(dims)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        out = torch.empty_like(dev(psi))
        lq.lq_apply_M_naive(ctx, out, dev(psi), 0.15, dagger)
        got = host(out)
    finally:
        lq.lq_destroy(ctx)
    assert rel_err(got, apply_M(U, psi, dims, 0.15, dagger=dagger)) < 1e-12


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2), (3, 5, 2, 7)])
@pytest.mark.parametrize("antiperiodic", [True, False])
def test_naive_force_matches_oracle(lq, dims, antiperiodic):
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.35, 5)
    X = source(lat, 6)
    ctx = lq.lq_create(dims, t_antiperiodic=antiperiodic)
    try:
        lq.lq_gauge_set(ctx, dev(U))
        F = torch.empty((lat.V, 4, 8), dtype=torch.float64, device="cuda")
        ms = lq.lq_fermion_force_naive(ctx, F, dev(X), 0.15, 2)
        got = host(F)
        ms_opt = lq.lq_time_fermion_force(ctx, dev(X), 0.15, 2)
    finally:
        lq.lq_destroy(ctx)
    ref = fermion_force_from_X(U, X, dims, 0.15, antiperiodic)
    assert rel_err(got, ref) < 1e-12
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    assert ms > 0 and ms_opt > 0


def test_fma_peak_probe(lq):
    """The measured FP64 and FP32 multiply-add rates are positive and ordered as on any
    part with a reduced FP64 pipe (FP32 at least 4x FP64); both are finite."""
    ctx = lq.lq_create((2, 2, 2, 2))
    try:
        f64 = lq.lq_time_fma_peak(ctx, lq.LQ_F64)
        f32 = lq.lq_time_fma_peak(ctx, lq.LQ_F32)
        with pytest.raises(lq.LQError):
            lq.lq_time_fma_peak(ctx, lq.LQ_F16_12)
    finally:
        lq.lq_destroy(ctx)
    assert 0.05 < f64 < 200.0 and 1.0 < f32 < 1000.0
    assert f32 > 4.0 * f64
