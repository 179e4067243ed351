"""Context groups (several reconstructions in batched launches) on the GPU.

A group sweep must give every member exactly what a separate sweep of that
member gives (same kernels, same order of arithmetic: bitwise), and so the
oracle's result within the per-sweep tolerance."""
import numpy as np
import pytest
import torch

from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import magpie, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    magpie.build()
    magpie.lib()


def f32(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


# (n, m, grid, step, jitter, levels, minibatch): different sizes, window
# sides, counts, minibatches and level counts; two share m = 32
SPECS = [(64, 16, 6, 8, 1, 3, 8), (128, 32, 5, 20, 2, 2, 7), (96, 32, 4, 20, 2, 4, 16),
         (192, 64, 4, 40, 3, 1, 5), (256, 128, 3, 60, 2, 3, 4)]


class Member:
    def __init__(self, spec, seed):
        n, m, g, s, j, L, B = spec
        self.n, self.m, self.L, self.B = n, m, L, B
        self.z_true = f32(synth.make_object(n, seed=seed))
        self.Q = f32(synth.make_probe(m))
        self.pos = synth.make_raster(n, m, g, s, j, seed=seed)
        self.N = len(self.pos)
        self.d = synth.poisson_noise(O.forward_intensities(self.z_true, self.Q, self.pos), 1e6,
                                     seed=seed).astype(np.float32).astype(np.float64)
        rng = np.random.default_rng(seed)
        self.z0 = f32(self.z_true + 0.2 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))))

    def ctx(self):
        dev = torch.device("cuda")
        self.zt = torch.from_numpy(self.z0.astype(np.complex64)).to(dev)
        p = magpie.magpie_params_of(self.n, self.n, self.m, self.N, self.L, self.B, 0.1)
        return magpie.magpie_create(p, self.zt, torch.from_numpy(self.Q.astype(np.complex64)).to(dev),
                                    torch.from_numpy(self.pos).to(dev),
                                    torch.from_numpy(self.d.astype(np.float32)).to(dev))


def orders(members, sweep):
    return [torch.from_numpy(synth.make_order(mb.N, 10 * sweep + i)).cuda() for i, mb in enumerate(members)]


def test_group_sweeps_equal_separate_sweeps_and_the_oracle():
    members = [Member(s, 11 + i) for i, s in enumerate(SPECS)]
    grouped = [mb.ctx() for mb in members]
    z_grouped = [mb.zt for mb in members]
    group = magpie.magpie_group_create(grouped)
    separate = [mb.ctx() for mb in members]
    z_separate = [mb.zt for mb in members]
    for sweep in range(2):
        ords = orders(members, sweep)
        magpie.magpie_group_sweep(group, ords)
        for c, o in zip(separate, ords):
            magpie.magpie_sweep(c, o)
    torch.cuda.synchronize()
    for i, mb in enumerate(members):
        assert torch.equal(z_grouped[i], z_separate[i]), i
        a = magpie.magpie_window_values(grouped[i])
        b = magpie.magpie_window_values(separate[i])
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    # against the oracle, two sweeps from the true object plus noise
    u = None
    for i, mb in enumerate(members):
        z = mb.z0
        uu = O.rpie_regulariser(mb.Q, 0.1)
        for sweep in range(2):
            z = O.sweep(z, mb.Q, mb.pos, mb.d, uu, mb.L, synth.make_order(mb.N, 10 * sweep + i), mb.B)
        got = z_grouped[i].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - z) / np.linalg.norm(z) < 1e-5, i
    group.close()
    for c in grouped + separate:
        c.close()


def test_group_arguments():
    members = [Member(SPECS[0], 3), Member(SPECS[1], 4)]
    a, b = members[0].ctx(), members[1].ctx()
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_group_create([a, b, a])
    assert ei.value.code == magpie.EINVAL
    mb = members[0]
    dev = torch.device("cuda")
    p = magpie.magpie_params_of(mb.n, mb.n, mb.m, mb.N, mb.L, mb.B, 0.1, 1, 0.1)
    zp = torch.from_numpy(mb.z0.astype(np.complex64)).to(dev)
    c = magpie.magpie_create(p, zp, torch.from_numpy(mb.Q.astype(np.complex64)).to(dev),
                             torch.from_numpy(mb.pos).to(dev), torch.from_numpy(mb.d.astype(np.float32)).to(dev))
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_group_create([a, c])
    assert ei.value.code == magpie.EINVAL
    for x in (a, b, c):
        x.close()


def test_autotuner_choices_give_identical_results():
    """The autotuner measured the three register bounds for every window side
    whose candidates differ, and its choice does not change results: groups
    forced to each candidate give bitwise equal objects."""
    members = [Member(spec, seed=40 + i) for i, spec in enumerate(SPECS)]
    outs = []
    for force in (0, 1, 2):
        ctxs = [mb.ctx() for mb in members]
        g = magpie.magpie_group_create(ctxs)
        tuning = magpie.magpie_group_tuning(g)
        print("autotuner:", tuning)
        assert 128 in tuning and all(all(x > 0 for x in ms) for _, ms in tuning.values())
        for m in (8, 16, 32, 64, 128, 256):
            minb = {8: (1, 2, 4), 16: (1, 2, 4), 32: (1, 2, 4), 64: (2, 1, 3), 128: (2, 1, 3),
                    256: (1, 1, 1)}[m][force]
            magpie.magpie_group_set_minb(g, m, minb)
        for s in range(2):
            magpie.magpie_group_sweep(g, orders(members, s))
        outs.append([mb.zt.cpu().numpy() for mb in members])
        g.close()
        for c in ctxs:
            c.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)
    with pytest.raises(magpie.MagpieError):
        magpie.magpie_group_set_minb(magpie.magpie_group_create([members[0].ctx()]), 128, 4)


def test_update_tile_shapes_give_identical_results():
    """The autotuner timed the update kernel's three tile shapes (16 x 16,
    32 x 8, 32 x 32) without touching the members' objects, and every shape
    sums each pixel's windows in minibatch order: groups forced to each shape
    give bitwise equal objects."""
    members = [Member(spec, seed=60 + i) for i, spec in enumerate(SPECS)]
    outs = []
    for shape in (0, 1, 2):
        ctxs = [mb.ctx() for mb in members]
        before = [mb.zt.clone() for mb in members]
        g = magpie.magpie_group_create(ctxs)
        torch.cuda.synchronize()
        assert all(torch.equal(a, mb.zt) for a, mb in zip(before, members))
        chosen, shapes = magpie.magpie_group_apply_tuning(g)
        print("update tile shapes:", chosen, shapes)
        assert chosen in (0, 1, 2) and [s[:2] for s in shapes] == [(16, 16), (32, 8), (32, 32)]
        assert all(ms > 0 for _, _, ms in shapes)
        magpie.magpie_group_set_apply_shape(g, shape)
        for s in range(2):
            magpie.magpie_group_sweep(g, orders(members, s))
        outs.append([mb.zt.cpu().numpy() for mb in members])
        g.close()
        for c in ctxs:
            c.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)


# the group specs plus window sides 8 (32-thread blocks) and 256 (512-thread
# blocks in clusters of 8), so that every update tile of the persistent form
# (16 x 16 and 32 x 32 over 32 .. 512 threads) runs
FORM_SPECS = SPECS + [(48, 8, 5, 8, 1, 2, 6), (320, 256, 2, 48, 2, 3, 3)]


def _group_run(members, persistent, sweeps=2):
    ctxs = [mb.ctx() for mb in members]
    before = [mb.zt.clone() for mb in members]
    g = magpie.magpie_group_create(ctxs)
    torch.cuda.synchronize()
    assert all(torch.equal(a, mb.zt) for a, mb in zip(before, members))  # the autotuner wrote scratch only
    chosen, ms = magpie.magpie_group_form_tuning(g)
    print("step form:", chosen, ms)
    assert chosen in (0, 1) and ms[0] > 0 and ms[1] > 0
    magpie.magpie_group_set_persistent(g, persistent)
    for s in range(sweeps):
        magpie.magpie_group_sweep(g, orders(members, s))
    assert magpie.magpie_group_status(g) == magpie.OK
    out = [mb.zt.cpu().numpy() for mb in members]
    g.close()
    for c in ctxs:
        c.close()
    return out


def test_persistent_form_equals_separate_launches_and_sweeps():
    """The persistent form (windows and update tiles of each window side from
    one launch's work queue, sides concurrent) gives bitwise the objects of
    the separate-launch form and of each member swept alone."""
    members = [Member(spec, seed=80 + i) for i, spec in enumerate(FORM_SPECS)]
    pers = _group_run(members, 1)
    sep = _group_run(members, 0)
    alone = []
    for i, mb in enumerate(members):
        c = mb.ctx()
        for s in range(2):
            magpie.magpie_sweep(c, orders(members, s)[i])
        alone.append(mb.zt.cpu().numpy())
        c.close()
    for i, (a, b, c) in enumerate(zip(pers, sep, alone)):
        assert np.array_equal(a, b), i
        assert np.array_equal(a, c), i


def test_bounded_waits_run_out_and_the_group_stays_usable():
    """Every dependency wait of a persistent step whose targets nothing meets
    runs out after its limit: the call returns MAGPIE_ETIMEOUT, skips every
    update (the objects are unchanged), ends promptly, and the next sweeps
    still give the objects of members swept alone."""
    import time
    members = [Member(spec, seed=90 + i) for i, spec in enumerate(SPECS)]
    ctxs = [mb.ctx() for mb in members]
    g = magpie.magpie_group_create(ctxs)
    magpie.magpie_group_set_persistent(g, 1)
    torch.cuda.synchronize()
    before = [mb.zt.clone() for mb in members]
    t0 = time.perf_counter()
    rc = magpie.magpie_group_check_waits(g, 2e-3)
    took = time.perf_counter() - t0
    assert rc == magpie.ETIMEOUT
    assert took < 5.0
    assert all(torch.equal(a, mb.zt) for a, mb in zip(before, members))
    assert magpie.magpie_group_status(g) == magpie.OK  # the flag was cleared
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_group_set_wait_limit(g, 0.0)
    assert ei.value.code == magpie.EINVAL
    magpie.magpie_group_set_wait_limit(g, 0.5)
    for s in range(2):
        magpie.magpie_group_sweep(g, orders(members, s))
    assert magpie.magpie_group_status(g) == magpie.OK
    got = [mb.zt.cpu().numpy() for mb in members]
    g.close()
    for c in ctxs:
        c.close()
    for i, mb in enumerate(members):
        mb.z0 = before[i].cpu().numpy().astype(np.complex128)
        c = mb.ctx()
        for s in range(2):
            magpie.magpie_sweep(c, orders(members, s)[i])
        assert np.array_equal(mb.zt.cpu().numpy(), got[i]), i
        c.close()
