"""The allocation-free M^dag M entry point agrees with the regular one.

lq_apply_MdagM_static is meant for callers that cannot let the library
allocate device memory (their memory is all owned by their own pool, or
capped by a host program), so it runs with no context and keeps its
intermediate field in a fixed array inside the library.  This file is
collected last so that a failing run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from synth import Lattice, gauge_exp_iA, source
from tests.gpu_common import require_gpu, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


def regular_MdagM(lq, dims, U, psi, kappa, t_antiperiodic):
    ctx = lq.lq_create(dims, t_antiperiodic)
    try:
        lq.lq_gauge_set(ctx, U)
        out = torch.empty_like(psi)
        lq.lq_apply_MdagM(ctx, out, psi, kappa, lq.LQ_F64)
        return host(out)
    finally:
        lq.lq_destroy(ctx)


def test_static_matches_regular_on_two_calls_in_a_row(lq):
    cases = [((4, 4, 4, 8), 0.155, True, 1), ((16, 16, 16, 16), 0.15, True, 2), ((6, 4, 2, 6), 0.13, False, 3)]
    outs = []
    for dims, kappa, ap, seed in cases:
        lat = Lattice(dims)
        U = dev(gauge_exp_iA(lat, 0.3, seed))
        psi = dev(source(lat, seed))
        ref = regular_MdagM(lq, dims, U, psi, kappa, ap)
        out = torch.full_like(psi, complex(float("nan"), 0.0))
        lq.lq_apply_MdagM_static(out, U, psi, dims, kappa, ap)
        got = host(out)
        assert rel_err(got, ref) < 1e-12, dims
        outs.append(got)
    # the same call again gives the same result (no state carries over)
    dims, kappa, ap, seed = cases[0]
    lat = Lattice(dims)
    U = dev(gauge_exp_iA(lat, 0.3, seed))
    psi = dev(source(lat, seed))
    again = torch.empty_like(psi)
    lq.lq_apply_MdagM_static(again, U, psi, dims, kappa, ap)
    assert np.array_equal(host(again), outs[0])
    # out may be the same buffer as in: the second kernel reads only the array
    inplace = psi.clone()
    lq.lq_apply_MdagM_static(inplace, U, inplace, dims, kappa, ap)
    assert rel_err(host(inplace), regular_MdagM(lq, dims, U, psi, kappa, ap)) < 1e-12


def test_static_refuses_host_buffers_and_wrong_sizes(lq):
    """The C entry point refuses host memory with LQ_ERR_ARG before any kernel runs; the
    Python wrapper refuses CPU tensors and buffers whose size does not match the lattice."""
    import ctypes
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    U_h = gauge_exp_iA(lat, 0.3, 1)
    psi_h = source(lat, 1)
    out_h = np.empty_like(psi_h)
    d = (ctypes.c_int * 4)(*dims)
    lib = lq.load()
    st = lib.lq_apply_MdagM_static(out_h.ctypes.data, U_h.ctypes.data, psi_h.ctypes.data, d, 1, 0.15, None)
    assert st == lq.LQ_ERR_ARG
    assert "device" in lib.lq_last_error(None).decode()
    U, psi = dev(U_h), dev(psi_h)
    out = torch.empty_like(psi)
    st = lib.lq_apply_MdagM_static(out.data_ptr(), U.data_ptr(), psi_h.ctypes.data, d, 1, 0.15, None)
    assert st == lq.LQ_ERR_ARG
    with pytest.raises(ValueError):
        lq.lq_apply_MdagM_static(out, U, torch.from_numpy(psi_h), dims, 0.15)      # CPU tensor
    with pytest.raises(ValueError):
        lq.lq_apply_MdagM_static(out, U, psi.to(torch.complex64), dims, 0.15)      # wrong dtype
    with pytest.raises(ValueError):
        lq.lq_apply_MdagM_static(out[:-1], U, psi, dims, 0.15)                     # too small
    with pytest.raises(ValueError):
        lq.lq_apply_MdagM_static(out, U[:-1], psi, dims, 0.15)


def test_static_rejects_lattices_beyond_the_array(lq):
    dims = (16, 16, 16, 17)
    U = torch.zeros((2, 4, 3, 3), dtype=torch.complex128, device="cuda")
    psi = torch.zeros((2, 4, 3), dtype=torch.complex128, device="cuda")
    import ctypes
    lib = lq.load()
    for bad in (dims, (65536, 65536, 65536, 65536), (2, 2, 2, 2 ** 30)):
        d = (ctypes.c_int * 4)(*bad)
        st = lib.lq_apply_MdagM_static(psi.data_ptr(), U.data_ptr(), psi.data_ptr(), d, 1, 0.1, None)
        assert st == lq.LQ_ERR_SHAPE, bad
        assert "65536" in lib.lq_last_error(None).decode()
