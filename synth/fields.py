"""Seeded synthetic lattice fields in the canonical host layout.

Canonical layout (shared by every consumer):
  site index   s = x + Lx*(y + Ly*(z + Lz*t)),  direction mu = 0..3 = x, y, z, t
  gauge field  complex128 [V][4][3][3]   U_mu(s), row-major colour matrix
  spinor       complex128 [V][4][3]      psi(s), spin-major, colour fastest
  momentum     float64    [V][4][8]      coefficients p_a of p = sum_a p_a t_a

Random streams of the counter-based generator (key = (seed, stream)):
  0 links (site, mu, call)     1 momenta (site, mu + 4*traj, call)
  2 chi (site, traj, call)     3 Metropolis uniform (traj)
  4 gauge transforms (site, 0, call)   5 sources (site, index, call)
"""
from dataclasses import dataclass, field
import numpy as np

from .philox import gaussians, philox4x32_10, uniform53

STREAM_LINKS, STREAM_MOMENTA, STREAM_CHI, STREAM_METROPOLIS = 0, 1, 2, 3
STREAM_GAUGE_TRANSFORM, STREAM_SOURCE = 4, 5


@dataclass(frozen=True)
class Lattice:
    """A 4-d lattice Lx x Ly x Lz x Lt (x fastest)."""
    dims: tuple

    @property
    def V(self):
        return int(np.prod(self.dims))

    def coords(self):
        """(V, 4) integer coordinates (x, y, z, t) of every site in canonical order."""
        Lx, Ly, Lz, Lt = self.dims
        s = np.arange(self.V)
        return np.stack([s % Lx, (s // Lx) % Ly, (s // (Lx * Ly)) % Lz, s // (Lx * Ly * Lz)], axis=1)


def _hermitian_from_gaussians(g, sigma):
    """3x3 Hermitian traceless matrices from 9 standard normals per item."""
    n = g.shape[:-1]
    A = np.zeros(n + (3, 3), dtype=np.complex128)
    A[..., 0, 0], A[..., 1, 1], A[..., 2, 2] = g[..., 0], g[..., 1], g[..., 2]
    for (i, j), k in (((0, 1), 3), ((0, 2), 5), ((1, 2), 7)):
        A[..., i, j] = g[..., k] + 1j * g[..., k + 1]
        A[..., j, i] = g[..., k] - 1j * g[..., k + 1]
    A *= sigma
    tr = np.trace(A, axis1=-2, axis2=-1).real / 3.0
    for i in range(3):
        A[..., i, i] -= tr
    return A


def _expi_hermitian(A):
    """exp(iA) for Hermitian A through its eigen-decomposition."""
    w, v = np.linalg.eigh(A)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), v.conj())


def _project_su3(U):
    """Nearest unitary matrix (polar factor from the SVD), determinant phase removed."""
    W, _, Vh = np.linalg.svd(U)
    P = W @ Vh
    d = np.linalg.det(P)
    return P / (d ** (1.0 / 3.0))[..., None, None]


def gauge_exp_iA(lat, sigma, seed, reunitarise=False, chunk=1 << 19):
    """Links U = exp(iA), A traceless Hermitian with N(0, sigma^2) entries.

    The three real diagonal entries and the real and imaginary parts of the
    three upper off-diagonal entries are independent N(0, sigma^2); the
    trace is then removed.
    """
    V = lat.V
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    links = np.arange(V * 4, dtype=np.uint64)
    for lo in range(0, V * 4, chunk):
        idx = links[lo:lo + chunk]
        g = gaussians(5, idx >> np.uint64(2), idx & np.uint64(3), seed, STREAM_LINKS)
        blk = _expi_hermitian(_hermitian_from_gaussians(g, sigma))
        if reunitarise:
            blk = _project_su3(blk)
        U.reshape(V * 4, 3, 3)[lo:lo + chunk] = blk
    return U


def identity_gauge(lat):
    U = np.zeros((lat.V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gauge_transform(lat, seed, sigma=1.0):
    """One random SU(3) matrix per site (for covariance checks)."""
    s = np.arange(lat.V, dtype=np.uint64)
    g = gaussians(5, s, np.uint64(0), seed, STREAM_GAUGE_TRANSFORM)
    return _expi_hermitian(_hermitian_from_gaussians(g, sigma))


def momenta(lat, seed, traj=0):
    """su(3) momentum coefficients p_a ~ N(0, 1), shape (V, 4, 8)."""
    V = lat.V
    link = np.arange(V * 4, dtype=np.uint64)
    g = gaussians(4, link >> np.uint64(2), (link & np.uint64(3)) + np.uint64(4 * traj), seed, STREAM_MOMENTA)
    return g.reshape(V, 4, 8)


def chi_noise(lat, seed, traj=0):
    """Complex Gaussian spinor with density proportional to exp(-chi^dag chi)."""
    s = np.arange(lat.V, dtype=np.uint64)
    g = gaussians(12, s, np.uint64(traj), seed, STREAM_CHI) * np.sqrt(0.5)
    return (g[:, 0::2] + 1j * g[:, 1::2]).reshape(lat.V, 4, 3)


def source(lat, seed, index=0):
    """Random complex Gaussian source, re and im each N(0, 1/2)."""
    s = np.arange(lat.V, dtype=np.uint64)
    g = gaussians(12, s, np.uint64(index), seed, STREAM_SOURCE) * np.sqrt(0.5)
    return (g[:, 0::2] + 1j * g[:, 1::2]).reshape(lat.V, 4, 3)


def metropolis_uniform(seed, traj=0):
    w = philox4x32_10(traj, 0, 0, 0, seed, STREAM_METROPOLIS)
    return float(uniform53(w[0], w[1]))


def plane_wave(lat, n, u, t_antiperiodic=True):
    """psi(x) = exp(i p.x) u with p_mu = 2 pi n_mu / L_mu (+ pi / L_t in time if antiperiodic)."""
    c = lat.coords()
    p = np.array([2.0 * np.pi * n[m] / lat.dims[m] for m in range(4)])
    if t_antiperiodic:
        p[3] += np.pi / lat.dims[3]
    phase = np.exp(1j * (c @ p))
    return phase[:, None, None] * np.asarray(u, dtype=np.complex128)[None, :, :], p


@dataclass(frozen=True)
class Preset:
    """A named workload: lattice, start configuration and method parameters."""
    name: str
    dims: tuple
    sigma: float
    seed: int
    kappa: float
    beta: float = 5.6
    n_steps: int = 10
    tau: float = 1.0
    tol: float = 1e-10
    reunitarise: bool = False
    extra: dict = field(default_factory=dict)


PRESETS = {
    # one plain FP64 trajectory on a small lattice
    "hmc_4x4x4x4": Preset("hmc_4x4x4x4", (4, 4, 4, 4), 0.3, 0, 0.15, beta=5.6, n_steps=10),
    # operator, solve and trajectories at 16^4
    "wilson_16x16x16x16": Preset("wilson_16x16x16x16", (16, 16, 16, 16), 0.3, 1, 0.155,
                                 beta=5.6, n_steps=20, reunitarise=True),
    # mixed-precision solve at 32^3 x 64
    "cg_32x32x32x64": Preset("cg_32x32x32x64", (32, 32, 32, 64), 0.25, 2, 0.156,
                             extra={"reliable_every": 50}),
    # many right-hand sides sharing one gauge field
    "multirhs_24x24x24x24": Preset("multirhs_24x24x24x24", (24, 24, 24, 24), 0.3, 3, 0.155,
                                   extra={"nrhs": 12}),
    # differentiable fermion action
    "autograd_16x16x16x16": Preset("autograd_16x16x16x16", (16, 16, 16, 16), 0.3, 8, 0.15),
}
