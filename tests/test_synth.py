"""Seeded input generators: Philox known answers and field properties."""
import os
import numpy as np

from synth import (Lattice, philox4x32_10, uniform53, gauge_exp_iA, momenta, chi_noise,
                   gauge_transform, metropolis_uniform)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(w, 16) for w in r]
        out = philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_uniform53_range():
    assert uniform53(0, 0) == 0.0
    assert uniform53(0xFFFFFFFF, 0xFFFFFFFF) < 1.0
    assert uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53


def test_links_are_su3_and_deterministic():
    lat = Lattice((2, 2, 2, 4))
    U = gauge_exp_iA(lat, 0.3, 7)
    I = np.eye(3)
    assert np.max(np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - I)) < 1e-13
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-13
    assert np.array_equal(U, gauge_exp_iA(lat, 0.3, 7))
    assert not np.array_equal(U, gauge_exp_iA(lat, 0.3, 8))
    Ur = gauge_exp_iA(lat, 0.3, 7, reunitarise=True)
    assert np.max(np.abs(Ur - U)) < 1e-13
    g = gauge_transform(lat, 3)
    assert np.max(np.abs(np.linalg.det(g) - 1.0)) < 1e-13


def test_noise_moments():
    lat = Lattice((8, 8, 8, 8))
    p = momenta(lat, 1, traj=2)
    assert abs(p.mean()) < 0.01 and abs(p.var() - 1.0) < 0.01
    c = chi_noise(lat, 1, traj=2)
    assert abs(np.mean(np.abs(c) ** 2) - 1.0) < 0.02       # E|chi|^2 = 1 for exp(-|chi|^2)
    assert not np.array_equal(momenta(lat, 1, 2), momenta(lat, 1, 3))
    u = metropolis_uniform(5, 3)
    assert 0.0 <= u < 1.0 and u == metropolis_uniform(5, 3)
