"""The seeded synthetic inputs follow their stated recipe (CPU): object
amplitude and phase ranges, the normalised disk probe, rasters inside the
object, the Poisson scaling, permutations, and the batched workload's ranges."""
import math

import numpy as np
import pytest

from paper_2504_10118_gb300 import synth


def test_object_amplitude_and_phase_ranges():
    z = synth.make_object(128, seed=3)
    a, ph = np.abs(z), np.angle(z)
    assert a.min() >= 0.8 - 1e-12 and a.max() <= 1.0 + 1e-12
    # the smoothed field is scaled onto [-pi/2, pi/2] exactly
    assert ph.min() == pytest.approx(-math.pi / 2, abs=1e-12)
    assert ph.max() == pytest.approx(math.pi / 2, abs=1e-12)
    # smooth (sigma = 4 px): neighbouring phases differ far less than the range
    assert np.abs(np.diff(ph, axis=0)).mean() < 0.05 * math.pi
    assert np.array_equal(synth.make_object(128, seed=3), z)  # seeded


def test_probe_is_a_normalised_defocused_disk():
    for m in (32, 128, 256):
        Q = synth.make_probe(m)
        assert np.abs(Q).max() == pytest.approx(1.0, abs=1e-15)
        c = (m - 1) / 2.0
        radius = 10.0 * m / 32.0
        yy, xx = np.meshgrid(np.arange(m) - c, np.arange(m) - c, indexing="ij")
        r = np.hypot(xx, yy)
        inside = r <= radius
        # flat amplitude inside the disk, Gaussian edge outside it
        assert np.ptp(np.abs(Q[inside])) < 1e-12
        assert np.all(np.abs(Q[~inside]) < np.abs(Q[inside]).min() + 1e-12)
        # quadratic defocus phase: pi at the rim
        k = np.unravel_index(np.argmin(np.abs(r - radius)), r.shape)
        assert abs(np.angle(Q[k] / Q[int(c), int(c)]) - ((math.pi * (r[k] / radius) ** 2 - math.pi * (
            r[int(c), int(c)] / radius) ** 2 + math.pi) % (2 * math.pi) - math.pi)) < 1e-9


@pytest.mark.parametrize("name", sorted(synth.WORKLOADS))
def test_workload_rasters_fit_without_clamping(name):
    w = synth.WORKLOADS[name]
    pos = synth.make_raster(w.n, w.m, w.grid, w.step, w.jitter)
    assert pos.shape == (w.grid * w.grid, 2) and pos.dtype == np.int32
    assert pos.min() >= 0 and pos.max() <= w.n - w.m
    # the unjittered raster plus the jitter lies inside [0, n - m]: no clamp acted
    span = (w.grid - 1) * w.step
    off = (w.n - w.m - span) // 2
    assert off - w.jitter >= 0 and off + span + w.jitter <= w.n - w.m
    base = off + w.step * np.arange(w.grid)
    rows = pos[:, 0].reshape(w.grid, w.grid)
    assert np.all(np.abs(rows - base[:, None]) <= w.jitter)


def test_poisson_noise_scaling():
    rng = np.random.default_rng(0)
    clean = rng.random((200, 8, 8)) * 50.0
    photons = 1e4
    noisy = synth.poisson_noise(clean, photons, seed=1)
    eta = clean.reshape(200, -1).sum(axis=1).mean() / photons
    # every value is an integer multiple of eta, never negative, unbiased on average
    q = noisy / eta
    assert np.all(noisy >= 0) and np.allclose(q, np.round(q), atol=1e-9)
    assert noisy.sum() / clean.sum() == pytest.approx(1.0, rel=0.02)
    assert np.array_equal(synth.poisson_noise(clean, None), clean)  # noise-free: the input unchanged


def test_orders_are_seeded_permutations():
    o = synth.make_order(900, 7)
    assert o.dtype == np.int32 and np.array_equal(np.sort(o), np.arange(900))
    assert np.array_equal(o, synth.make_order(900, 7)) and not np.array_equal(o, synth.make_order(900, 8))


def test_batched_workload_ranges():
    ws = synth.make_batch()
    assert len(ws) == 48
    for w in ws:
        assert w.n in (256, 384, 512, 768, 1024) and w.m in (64, 128, 256) and w.m <= w.n // 2
        assert 10 <= w.grid <= 40 and 1e5 <= w.photons <= 1e7
        assert w.levels == min(3, int(math.log2(w.m)) + 1) and w.minibatch == min(64, w.grid * w.grid)
        pos = synth.make_raster(w.n, w.m, w.grid, w.step, w.jitter)
        assert pos.min() >= 0 and pos.max() <= w.n - w.m
    total = sum(w.n_pos for w in ws)
    assert 48 * 100 <= total <= 48 * 1600
