"""Seeded scattered-node unit-disk fixtures (inputs only).

The paper solves Poisson's equation with Dirichlet data on the 2D unit disk,
discretised by scattered nodes (Sec. IV, Eqs. 2-3), with the manufactured
solution u = sin(pi x) sin(pi y) (Sec. IV).  Its own node generator lives in an
external library, so this module supplies a seeded stand-in with the same
structure: a jittered grid of spacing h inside the disk and equispaced nodes
on the boundary circle.

Recipe (all arithmetic in float64, numpy, vectorised):

* RNG: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014).  The k-th output (k = 1, 2, ...) of a generator
  seeded with s is mix(s + k * 0x9E3779B97F4A7C15) mod 2**64; a uniform double
  in [0, 1) is (z >> 11) * 2**-53.
* Grid points (i h, j h) for i, j in [-K, K], K = ceil(1/h), visited with j
  in the outer loop and i in the inner loop.  Every grid point consumes two
  draws, jx then jy, whether or not it is kept, so the stream position of a
  point never depends on earlier rejections.
* Jitter (2u - 1) * 0.25 h on each coordinate; keep the point if
  x^2 + y^2 < (1 - h/2)^2 after jitter.
* Boundary: N_b = round(2 pi / h) nodes at angle 2 pi k / N_b on r = 1.
* Node order: interior nodes in generation order, then boundary nodes.

Nothing here computes stencils, weights, matrices or solutions.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start+1 .. start+count of SplitMix64 seeded with `seed` (uint64)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(z: np.ndarray) -> np.ndarray:
    """Map uint64 draws to doubles in [0, 1) using the top 53 bits."""
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class DiskNodes:
    """A node set: xy is (N, 2) float64 C-contiguous, is_dirichlet (N,) uint8."""

    xy: np.ndarray
    is_dirichlet: np.ndarray
    h: float
    seed: int
    n_interior: int
    n_boundary: int

    @property
    def N(self) -> int:
        return int(self.xy.shape[0])


def disk_nodes(h: float, seed: int = 2107, jitter: float = 0.25) -> DiskNodes:
    """Jittered-grid unit disk with equispaced boundary nodes (recipe above).

    `jitter=0` gives the unjittered grid (heavy distance ties), used by tests.
    """
    K = int(math.ceil(1.0 / h))
    side = 2 * K + 1
    z = splitmix64(seed, 2 * side * side)
    u = uniform01(z).reshape(side * side, 2)
    jj, ii = np.meshgrid(np.arange(-K, K + 1), np.arange(-K, K + 1), indexing="ij")
    x = ii.reshape(-1).astype(np.float64) * h + (2.0 * u[:, 0] - 1.0) * (jitter * h)
    y = jj.reshape(-1).astype(np.float64) * h + (2.0 * u[:, 1] - 1.0) * (jitter * h)
    keep = x * x + y * y < (1.0 - 0.5 * h) ** 2
    xi, yi = x[keep], y[keep]
    nb = int(round(2.0 * math.pi / h))
    th = 2.0 * math.pi * np.arange(nb, dtype=np.float64) / nb
    xy = np.empty((xi.size + nb, 2), dtype=np.float64)
    xy[: xi.size, 0], xy[: xi.size, 1] = xi, yi
    xy[xi.size :, 0], xy[xi.size :, 1] = np.cos(th), np.sin(th)
    mask = np.zeros(xy.shape[0], dtype=np.uint8)
    mask[xi.size :] = 1
    return DiskNodes(np.ascontiguousarray(xy), mask, float(h), int(seed), int(xi.size), nb)


def h_for_nodes(n_target: float) -> float:
    """Grid spacing giving about n_target nodes in the unit disk (pi / h^2)."""
    return math.sqrt(math.pi / float(n_target))


def manufactured(xy: np.ndarray):
    """u = sin(pi x) sin(pi y), f = -lap u = 2 pi^2 u, g = u (Sec. IV, Eqs. 2-3)."""
    u = np.sin(math.pi * xy[:, 0]) * np.sin(math.pi * xy[:, 1])
    return u, 2.0 * math.pi * math.pi * u, u.copy()


def fourier_params(n_rhs: int, seed: int, n_waves: int = 8):
    """Wave numbers and amplitudes of the random Fourier sources, each (n_rhs, n_waves).

    kx_k, ky_k are integers uniform in [1, 8] (top three bits of a draw, + 1) and
    a_k ~ N(0, 1) by Box-Muller (u1 in (0, 1], u2 in [0, 1)).  Four draws per
    wave, in the order kx, ky, u1, u2, waves of one right-hand side contiguous.
    """
    z = splitmix64(seed, 4 * n_waves * n_rhs).reshape(n_rhs, n_waves, 4)
    kx = (z[..., 0] >> np.uint64(61)).astype(np.float64) + 1.0
    ky = (z[..., 1] >> np.uint64(61)).astype(np.float64) + 1.0
    u1 = 1.0 - uniform01(z[..., 2])
    u2 = uniform01(z[..., 3])
    a = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return kx, ky, a


def fourier_sources(xy: np.ndarray, n_rhs: int, seed: int, n_waves: int = 8) -> np.ndarray:
    """Random Fourier sources f = sum_k a_k sin(kx_k x + ky_k y), shape (n_rhs, N);
    the draws are those of fourier_params."""
    kx, ky, a = fourier_params(n_rhs, seed, n_waves)
    out = np.zeros((n_rhs, xy.shape[0]), dtype=np.float64)
    for r in range(n_rhs):
        for k in range(n_waves):
            out[r] += a[r, k] * np.sin(kx[r, k] * xy[:, 0] + ky[r, k] * xy[:, 1])
    return out


def sample_indices(N: int, count: int, seed: int) -> np.ndarray:
    """Up to `count` distinct indices in [0, N): the first distinct draws of
    SplitMix64 (top 53 bits scaled to [0, N)), sorted.  Picks the sampled
    nodes of the full-size parity checks."""
    z = splitmix64(seed, 4 * count)
    draws = ((z >> np.uint64(11)).astype(np.float64) * (N / 9007199254740992.0)).astype(np.int64)
    _, first = np.unique(draws, return_index=True)
    return np.sort(draws[np.sort(first)[:count]])


def batched_instances(seed: int = 2107, count: int = 256, n_lo: float = 1e4, n_hi: float = 2e5):
    """Per-instance (seed_i, h_i, m_i) for the batched uneven workload.

    N_i is log-uniform in [n_lo, n_hi], h_i = sqrt(pi / N_i), m_i uniform in
    {2, 4, 6}; seed_i is the first SplitMix64 output for state seed ^ i.
    """
    master = uniform01(splitmix64(seed, 2 * count)).reshape(count, 2)
    out = []
    for i in range(count):
        n_i = math.exp(math.log(n_lo) + master[i, 0] * (math.log(n_hi) - math.log(n_lo)))
        m_i = (2, 4, 6)[min(int(master[i, 1] * 3.0), 2)]
        s_i = int(splitmix64(seed ^ i, 1)[0])
        out.append((s_i, h_for_nodes(n_i), m_i))
    return out


# Problem configurations (grid spacing is fixed so N is reproducible).
#   m: highest monomial degree; n: stencil size (2 * (m+1)(m+2)/2).
CONFIGS = {
    "disk_h0.04_m2_n12": dict(h=0.04, m=2, n=12, seed=2107),
    "disk_1M_m4_n30": dict(h=1.7725e-3, m=4, n=30, seed=2107),
    "disk_4M_m6_n56": dict(h=8.862e-4, m=6, n=56, seed=2107),
}
