"""Seeded input generators: Philox known answers and field properties."""
import os
import numpy as np
import pytest

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


def test_generator_log_within_ulps_of_numpy():
    """The series logarithm of the generator against numpy's log over 2e6 uniforms and the
    edge cases (1, the smallest 1 - u, the reduction threshold): within 4 units in the last
    place, and exactly 0 at 1."""
    from synth.philox import log_unit
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.random(2_000_000), [1.0, 2.0 ** -53, 0.5, np.nextafter(1.0, 0.0),
                                                 0.7071067811865476, 0.7071067811865475, 1e-300, 3.0]])
    v = v[v > 0]
    a, b = log_unit(v), np.log(v)
    assert np.max(np.abs(a - b) / np.spacing(np.abs(b) + (b == 0))) <= 4.0
    assert log_unit(np.array([1.0]))[0] == 0.0


def test_generator_sincos_against_exact_values():
    """sin and cos of 2 pi u: exact at the quarter points, within 2e-16 of values computed
    with 120-bit arithmetic, and within 1e-15 of numpy (whose own 2 pi u carries a
    rounding error); sin^2 + cos^2 = 1 to rounding."""
    from synth.philox import sincos_2pi
    s, c = sincos_2pi(np.array([0.0, 0.25, 0.5, 0.75]))
    assert list(s) == [0.0, 1.0, 0.0, -1.0] and list(c) == [1.0, 0.0, -1.0, 0.0]
    rng = np.random.default_rng(2)
    u = rng.random(1_000_000)
    s, c = sincos_2pi(u)
    assert np.max(np.abs(s - np.sin(2 * np.pi * u))) < 1e-15
    assert np.max(np.abs(c - np.cos(2 * np.pi * u))) < 1e-15
    assert np.max(np.abs(s * s + c * c - 1.0)) < 1e-15
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    for x in rng.random(500):
        sx, cx = sincos_2pi(np.array([x]))
        a = 2 * mpmath.pi * mpmath.mpf(float(x))
        assert abs(float(mpmath.sin(a)) - sx[0]) <= 2.3e-16
        assert abs(float(mpmath.cos(a)) - cx[0]) <= 2.3e-16


def test_box_muller_matches_textbook_formula():
    """The generator's Gaussians equal sqrt(-2 log(1 - u1)) (cos, sin)(2 pi u2) evaluated with
    numpy's functions to a few units in the last place."""
    from synth.philox import box_muller
    rng = np.random.default_rng(3)
    u1, u2 = rng.random(500_000), rng.random(500_000)
    z0, z1 = box_muller(u1, u2)
    r = np.sqrt(-2.0 * np.log1p(-u1))
    assert np.max(np.abs(z0 - r * np.cos(2 * np.pi * u2)) / (1 + np.abs(z0))) < 4e-15
    assert np.max(np.abs(z1 - r * np.sin(2 * np.pi * u2)) / (1 + np.abs(z1))) < 4e-15
