"""The naive global-memory Wilson operator used for the register ablation is correct."""
import pytest

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
