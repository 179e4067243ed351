"""Seeded synthetic inputs for the MAGPIE sweep (object, probe, scan raster,
Poisson noise, per-sweep permutations).

This module draws and shapes random numbers only.  It holds none of the
solver's arithmetic: the diffraction intensities themselves are produced by
each implementation's own forward model (Section 2.1, data model
d_k = |F(Q . P_k z*)|^2), and this module only adds the photon-counting
noise of Section 5 ("Noise level": d = eta * Poisson(d~ / eta)) to them.

Recipe (seeds are fixed per quantity so every consumer sees the same data):
  * object  (seed 1): amplitude i.i.d. U[0.8, 1]; phase = white N(0,1)
    field blurred by a periodic Gaussian of sigma 4 px, min-max scaled to
    [-pi/2, pi/2].
  * probe (deterministic): disk of radius 10*m/32 px with a Gaussian edge of
    sigma 2*m/32 px, times a quadratic defocus phase exp(i*pi*(r/R)^2),
    normalised to max |Q| = 1.
  * raster  (seed 3): g x g grid, step s, integer jitter in [-j, j], centred
    in the object and clamped to [0, n-m]; rows are (row, col) of the
    top-left corner of each m x m scan window.
  * noise   (seed 4): one eta per data set, eta = mean_k sum(d~_k) / photons.
  * order   (seed 100 + sweep): a uniform random permutation of 0..N-1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic ptychography problem, named by what it is."""

    name: str
    n: int              # object side (n x n pixels)
    m: int              # probe / patch side (power of two)
    grid: int           # g: the raster is g x g positions
    step: int           # raster step in pixels
    jitter: int         # integer jitter amplitude in pixels
    levels: int         # number of grids including the finest (1 = rPIE)
    minibatch: int      # positions per minibatch step
    alpha: float        # rPIE regularisation constant
    photons: float | None  # photons per pattern, None = noise-free
    iterations: int     # sweeps of the fixed-iteration runs

    @property
    def n_pos(self) -> int:
        return self.grid * self.grid


# Workloads of the evaluation.  alpha = 0.1 throughout: with this disk probe
# the sequential iteration diverges for alpha <= 0.03 even on noise-free data
# (the values 0.008-0.06 of Section 5 were tuned for the paper's zone-plate
# probe), while 0.1 converges for every level count and minibatch tried.
WORKLOADS = {
    "tiny": Workload("n128-m32-N64-L2-B16", 128, 32, 8, 8, 1, 2, 16, 0.1, None, 50),
    "mid": Workload("n512-m128-N900-L3-B64", 512, 128, 30, 12, 2, 3, 64, 0.1, 1e6, 200),
    # a 50 x 50 raster at step 16 spans 49*16+256 = 1040 > 1024 px; step 15
    # keeps the 2500 positions inside the object.
    "precision": Workload("n1024-m256-N2500-L4-B64", 1024, 256, 50, 15, 2, 4, 64, 0.1, 1e7, 50),
}


def make_batch(count: int = 48, seed: int = 5, levels: int = 3, minibatch: int = 64,
               sides=(256, 384, 512, 768, 1024), probes=(64, 128, 256)) -> list:
    """Independent problems of uneven sizes (the batched workload): object side
    from `sides`, probe side from `probes` with m <= n/2, a g x g raster with
    g uniform in [10, 40] (100 to 1600 windows), step s = (n - m - 2j)/(g - 1)
    and jitter j = max(1, s/8) (integer parts), photons 10^U[5, 7]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sides))
        m = int(rng.choice([p for p in probes if p <= n // 2]))
        g = int(rng.integers(10, 41))
        s = (n - m - 2) // (g - 1)
        j = max(1, s // 8)
        s = (n - m - 2 * j) // (g - 1)
        photons = float(10.0 ** rng.uniform(5.0, 7.0))
        out.append(Workload(f"batch{i}-n{n}-m{m}-N{g * g}", n, m, g, s, j, min(levels, int(math.log2(m)) + 1),
                            min(minibatch, g * g), 0.1, photons, 1))
    return out


def make_object(n: int, seed: int = 1) -> np.ndarray:
    """Complex128 n x n test object."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.8, 1.0, size=(n, n))
    white = rng.standard_normal(size=(n, n))
    smooth = ndimage.gaussian_filter(white, sigma=4.0, mode="wrap")
    lo, hi = smooth.min(), smooth.max()
    phase = (smooth - lo) / (hi - lo) * math.pi - math.pi / 2.0
    return amp * np.exp(1j * phase)


def make_probe(m: int) -> np.ndarray:
    """Complex128 m x m apodised, defocused disk probe with max |Q| = 1."""
    radius = 10.0 * m / 32.0
    sigma = 2.0 * m / 32.0
    c = (m - 1) / 2.0
    yy, xx = np.meshgrid(np.arange(m) - c, np.arange(m) - c, indexing="ij")
    r = np.sqrt(xx * xx + yy * yy)
    amp = np.where(r <= radius, 1.0, np.exp(-((r - radius) ** 2) / (2.0 * sigma * sigma)))
    q = amp * np.exp(1j * math.pi * (r / radius) ** 2)
    return q / np.abs(q).max()


def make_raster(n: int, m: int, grid: int, step: int, jitter: int, seed: int = 3) -> np.ndarray:
    """int32 [grid*grid, 2] top-left (row, col) of each scan window."""
    rng = np.random.default_rng(seed)
    span = (grid - 1) * step
    off = (n - m - span) // 2
    base = off + step * np.arange(grid)
    rows, cols = np.meshgrid(base, base, indexing="ij")
    pos = np.stack([rows.ravel(), cols.ravel()], axis=1)
    if jitter > 0:
        pos = pos + rng.integers(-jitter, jitter + 1, size=pos.shape)
    return np.clip(pos, 0, n - m).astype(np.int32)


def poisson_noise(clean: np.ndarray, photons: float | None, seed: int = 4) -> np.ndarray:
    """eta * Poisson(clean / eta), eta = mean per-pattern total / photons.

    `clean` is [N, m, m] noise-free intensities; returns float64 of the same
    shape.  photons=None returns the input unchanged (noise-free data).
    """
    if photons is None:
        return np.asarray(clean, dtype=np.float64)
    clean = np.asarray(clean, dtype=np.float64)
    eta = float(clean.reshape(clean.shape[0], -1).sum(axis=1).mean() / photons)
    rng = np.random.default_rng(seed)
    return eta * rng.poisson(clean / eta).astype(np.float64)


def make_order(n_pos: int, sweep: int) -> np.ndarray:
    """int32 uniform random permutation of 0..n_pos-1 for one sweep."""
    rng = np.random.default_rng(100 + sweep)
    return rng.permutation(n_pos).astype(np.int32)


def make_problem(w: Workload):
    """(object z*, probe Q, positions) of a workload, complex128/int32."""
    return make_problem_seeded(w, 1)


def make_problem_seeded(w: Workload, seed: int):
    """make_problem with the object drawn from `seed` and the raster jitter
    from `seed + 2` (seed 1 gives make_problem's data)."""
    z_true = make_object(w.n, seed=seed)
    probe = make_probe(w.m)
    pos = make_raster(w.n, w.m, w.grid, w.step, w.jitter, seed=seed + 2)
    return z_true, probe, pos


def make_cnn_params(layers, seed: int = 7, zero_last: bool = True) -> np.ndarray:
    """float32 initial parameters of a stack of 3x3 convolutions given as
    (c_in, c_out) pairs: per layer, weights [c_out][3][3][c_in] drawn
    N(0, 2 / (9 c_in)) (He initialisation) then c_out zero biases.  With
    `zero_last` the last layer's weights are zero too."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (ci, co) in enumerate(layers):
        w = rng.normal(0.0, math.sqrt(2.0 / (9 * ci)), co * 9 * ci)
        if zero_last and i == len(layers) - 1:
            w[:] = 0.0
        parts += [w, np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)
