"""The heat bath drawn on the device (Sec. 2; Sec. 3 step 1): the CUDA generator reproduces
the seeded host generator bit for bit, and a trajectory with its heat bath on the device is
the trajectory with the host's draws passed in."""
import os

import numpy as np
import pytest

from synth import Lattice, gauge_exp_iA, momenta, chi_noise, metropolis_uniform, philox4x32_10
from tests.gpu_common import require_gpu, dev, host, torch

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lq():
    return require_gpu()


def test_device_philox_known_answers_and_host_words(lq):
    """The published known-answer vectors, then 2^20 random (counter, key) sets against the
    host generator: every output word equal."""
    rows = [[int(w, 16) for w in ln.split()] for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    rng = np.random.default_rng(4)
    rand = rng.integers(0, 2 ** 32, size=(1 << 20, 6), dtype=np.uint64)
    inp = np.concatenate([np.array([r[:6] for r in rows], dtype=np.uint64), rand])
    ctx = lq.lq_create((2, 2, 2, 2))
    try:
        d_in = dev(inp.astype(np.uint32).view(np.int32))
        d_out = torch.empty((inp.shape[0], 4), dtype=torch.int32, device="cuda")
        lq.lq_philox4x32_10(ctx, d_in, d_out)
        got = host(d_out).view(np.uint32)
    finally:
        lq.lq_destroy(ctx)
    for i, r in enumerate(rows):
        assert [int(v) for v in got[i]] == r[6:]
    ref = np.stack(philox4x32_10(*[inp[:, k] for k in range(6)]), axis=1)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("seed,traj", [(8, 0), (11, 37), (0xFFFFFFFF, (1 << 30) - 1)])
def test_device_heatbath_bit_exact(lq, seed, traj):
    """16^4: 2,097,152 momentum coefficients and 1,572,864 noise reals drawn on the device
    equal the host generator's bit for bit (Box-Muller included), and so does u."""
    dims = (16, 16, 16, 16)
    lat = Lattice(dims)
    ctx = lq.lq_create(dims)
    try:
        p = torch.empty((lat.V, 4, 8), dtype=torch.float64, device="cuda")
        chi = torch.empty((lat.V, 4, 3), dtype=torch.complex128, device="cuda")
        u = lq.lq_heatbath_draw(ctx, seed, traj, p, chi)
        ph = np.empty((lat.V, 4, 8))                    # host buffers take the staged path
        chih = np.empty((lat.V, 4, 3), dtype=np.complex128)
        lq.lq_heatbath_draw(ctx, seed, traj, ph, chih)
        got_p, got_chi = host(p), host(chi)
    finally:
        lq.lq_destroy(ctx)
    ref_p, ref_chi = momenta(lat, seed, traj), chi_noise(lat, seed, traj)
    assert np.array_equal(got_p.view(np.uint64), ref_p.view(np.uint64))
    assert np.array_equal(got_chi.view(np.uint64), ref_chi.view(np.uint64))
    assert np.array_equal(ph, ref_p) and np.array_equal(chih, ref_chi)
    assert u == metropolis_uniform(seed, traj)


def test_heatbath_rejects_counters_out_of_range(lq):
    ctx = lq.lq_create((2, 2, 2, 2))
    try:
        with pytest.raises(lq.LQError) as e:
            lq.lq_heatbath_draw(ctx, 1 << 32, 0)
        assert e.value.status == lq.LQ_ERR_ARG
        with pytest.raises(lq.LQError):
            lq.lq_heatbath_draw(ctx, 1, 1 << 30)
    finally:
        lq.lq_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 3])
def test_seeded_trajectory_equals_trajectory_with_host_draws(lq, prec):
    """4^4 (beta 5.6, kappa 0.15, 10 steps): the trajectory whose heat bath runs on the device
    gives, bit for bit, the Delta H, decision, plaquette, final momenta and links of the
    trajectory given the host generator's draws; two trajectories in a row as well."""
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    U = gauge_exp_iA(lat, 0.3, 0)
    out = {}
    for mode in ("seeded", "host"):
        ctx = lq.lq_create(dims)
        try:
            lq.lq_gauge_set(ctx, dev(U))
            rs, ps = [], []
            for traj in (0, 1):
                if mode == "seeded":
                    p = torch.empty((lat.V, 4, 8), dtype=torch.float64, device="cuda")
                    r = lq.lq_hmc_trajectory_seeded(ctx, 0, traj, 5.6, 0.15, 10, 1.0, 1e-10, 10000, prec, 50,
                                                    p_out=p)
                else:
                    p = dev(momenta(lat, 0, traj))
                    r = lq.lq_hmc_trajectory(ctx, p, dev(chi_noise(lat, 0, traj)), metropolis_uniform(0, traj),
                                             5.6, 0.15, 10, 1.0, 1e-10, 10000, prec, 50)
                rs.append(r)
                ps.append(host(p))
            Ug = np.empty_like(U)
            lq.lq_gauge_get(ctx, Ug)
            out[mode] = (rs, ps, Ug)
        finally:
            lq.lq_destroy(ctx)
    for a, b in zip(out["seeded"][0], out["host"][0]):
        for k in ("dH", "dK", "dSg", "dSf", "accepted", "plaquette", "cg_iterations"):
            assert a[k] == b[k], k
    for a, b in zip(out["seeded"][1], out["host"][1]):
        assert np.array_equal(a, b)
    assert np.array_equal(out["seeded"][2], out["host"][2])
