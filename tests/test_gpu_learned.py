"""GPU parity of the learned coarse correction against the FP64 oracle
(network forward and backward, Adam step, coarse state, learned minibatch
step), plus training and what the trained network gains."""
import numpy as np
import pytest
import torch

from oracle import learned_oracle as L
from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import learned, magpie, synth
from tests.learned_pins import random_theta

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def _built():
    magpie.build()
    magpie.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def net_with(theta, h, B):
    net = magpie.magpie_cnn_create(h, B)
    magpie.magpie_cnn_set_params(net, torch.from_numpy(theta.astype(np.float32)).to(DEV))
    return net


def test_param_count():
    assert magpie.magpie_cnn_param_count() == L.param_count() == 980002


@pytest.mark.parametrize("path", [1, 0], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("h,B,check", [(8, 3, 3), (16, 5, 5), (32, 64, 4)])
def test_forward_matches_oracle(h, B, check, path):
    """BF16 tensor-core forward vs the oracle's BF16-rounded FP64 forward,
    with the 5th-generation tensor cores (tcgen05, TMEM accumulators) for the
    layers with 64-multiple channel counts and with register-fragment mma.sync
    everywhere; at h = 32 a full 64-window batch runs and four windows are
    checked."""
    theta = random_theta(L, 21).astype(np.float32).astype(np.float64)
    x = np.random.default_rng(22).normal(size=(B, h, h, 4)).astype(np.float32)
    net = net_with(theta, h, B)
    magpie.magpie_cnn_set_tensor_path(net, path)
    y = torch.empty((B, h, h, 2), dtype=torch.float32, device=DEV)
    magpie.magpie_cnn_forward(net, torch.from_numpy(x).to(DEV), y)
    magpie.magpie_cnn_status(net)
    yg = y.cpu().numpy().astype(np.float64)
    sel = np.linspace(0, B - 1, check).astype(int)
    yo, _ = L.forward(theta, x[sel].astype(np.float64))
    assert rel(yg[sel], yo) < 2e-3
    assert np.abs(yg[sel] - yo).max() < 2e-2 * np.abs(yo).max()


@pytest.mark.parametrize("h,B,seed,scale,tol", [(8, 1, 5, 1.0, 2e-6), (8, 2, 6, 0.5, 2e-6), (16, 2, 7, 2.0, 2e-6),
                                                  (16, 3, 23, 1.0, 2e-2)])
def test_backward_matches_oracle(h, B, seed, scale, tol):
    """Per-layer weight and bias gradients.  The BF16 roundings of the
    activations are decisions the GPU takes on FP32 sums; where none of them
    falls differently from the oracle's (the forward outputs then agree to
    1e-6), the gradients agree to FP32 accumulation error.  The last case has
    such a difference (forward 1e-3 apart) and shows how far it carries."""
    theta = random_theta(L, seed, scale=scale).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(24)
    x = rng.normal(size=(B, h, h, 4)).astype(np.float32)
    dy = rng.normal(size=(B, h, h, 2)).astype(np.float32)
    net = net_with(theta, h, B)
    # the cases were chosen where the register-fragment forward takes every
    # BF16 rounding decision as the oracle does; this test is about the FP32
    # backward pass, so it keeps that forward
    magpie.magpie_cnn_set_tensor_path(net, 0)
    y = torch.empty((B, h, h, 2), dtype=torch.float32, device=DEV)
    magpie.magpie_cnn_forward(net, torch.from_numpy(x).to(DEV), y)
    g = torch.empty(L.param_count(), dtype=torch.float32, device=DEV)
    magpie.magpie_cnn_backward(net, torch.from_numpy(dy).to(DEV), g)
    gg = g.cpu().numpy().astype(np.float64)
    yo, acts = L.forward(theta, x.astype(np.float64))
    go = L.backward(theta, acts, dy.astype(np.float64))
    if tol < 1e-4:
        assert rel(y.cpu().numpy(), yo) < 1e-6
    o = 0
    for ci, co, _, _, _ in L.LAYERS:
        n = co * 9 * ci
        assert rel(gg[o:o + n], go[o:o + n]) < tol, ("weights", ci, co)
        assert rel(gg[o + n:o + n + co], go[o + n:o + n + co]) < tol, ("biases", ci, co)
        o += n + co


@pytest.mark.parametrize("h,B", [(32, 64), (32, 16), (16, 7), (64, 4)])
def test_tensor_paths_agree(h, B):
    """The tcgen05 convolutions (TMEM accumulators, split-K over 64-element
    steps) and the mma.sync ones compute the same BF16 products with FP32
    accumulation in another order: outputs agree to the BF16 rounding of the
    activations, and no bounded wait ran out."""
    theta = random_theta(L, 31).astype(np.float32)
    x = torch.from_numpy(np.random.default_rng(32).normal(size=(B, h, h, 4)).astype(np.float32)).to(DEV)
    out = []
    for path in (1, 0):
        net = net_with(theta, h, B)
        magpie.magpie_cnn_set_tensor_path(net, path)
        y = torch.empty((B, h, h, 2), dtype=torch.float32, device=DEV)
        magpie.magpie_cnn_forward(net, x, y)
        magpie.magpie_cnn_status(net)
        out.append(y.cpu().numpy().astype(np.float64))
        net.close()
    assert rel(out[0], out[1]) < 2e-3, rel(out[0], out[1])


def test_train_step_matches_oracle():
    """Loss, gradient and one Adam step: the loss to 1e-4; the step moves each
    weight by -lr sign(g) (first Adam step) wherever |g| is not tiny."""
    h, B, lr = 8, 4, 1e-3
    theta = random_theta(L, 25).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(26)
    x0 = rng.normal(size=(B, h, h, 4)).astype(np.float32)
    zh = rng.normal(size=(B, h, h, 2)).astype(np.float32)
    s = rng.uniform(0.5, 2.0, B).astype(np.float32)
    net = net_with(theta, h, B)
    loss = torch.zeros(1, dtype=torch.float64, device=DEV)
    magpie.magpie_cnn_train_step(net, torch.from_numpy(x0).to(DEV), torch.from_numpy(zh).to(DEV),
                                 torch.from_numpy(s).to(DEV), lr, loss)
    th = torch.empty(L.param_count(), dtype=torch.float32, device=DEV)
    magpie.magpie_cnn_get_params(net, th)
    t = L.targets(x0.astype(np.float64), zh.astype(np.float64), s.astype(np.float64))
    y, acts = L.forward(theta, x0.astype(np.float64))
    lo, dy = L.loss_and_grad(y, t)
    g = L.backward(theta, acts, dy)
    th_o, _, _ = L.adam(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    assert abs(loss.item() - lo) < 1e-4 * lo
    d_gpu = th.cpu().numpy().astype(np.float64) - theta
    d_orc = th_o - theta
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    assert np.abs(d_gpu[big] - d_orc[big]).max() < 1e-2 * lr
    assert np.abs(d_gpu).max() <= 1.0001 * lr


def tiny_problem(levels=2, m=32):
    w = synth.WORKLOADS["tiny"]
    z_true, Q, pos = synth.make_problem(w)
    d = O.forward_intensities(z_true, Q, pos)
    rng = np.random.default_rng(27)
    z0 = (np.ones((w.n, w.n)) + 0.1 * rng.normal(size=(w.n, w.n)) * np.exp(1j * rng.normal(size=(w.n, w.n))))
    z0 = z0.astype(np.complex64).astype(np.complex128)
    return w, z_true, Q, pos, d, z0


def make_ctx(w, z0, Q, pos, d, levels, minibatch):
    zt = torch.from_numpy(z0.astype(np.complex64)).to(DEV)
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(DEV)
    pt = torch.from_numpy(pos.astype(np.int32)).to(DEV)
    dt = torch.from_numpy(d.astype(np.float32)).to(DEV)
    p = magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, levels, minibatch, w.alpha)
    return magpie.magpie_create(p, zt, Qt, pt, dt), zt


@pytest.mark.parametrize("levels", [2, 3])
def test_coarse_state_matches_oracle(levels):
    w, _, Q, pos, d, z0 = tiny_problem()
    ctx, _ = make_ctx(w, z0, Q, pos, d, levels, 16)
    idx = np.array([0, 5, 17, 63, 30], dtype=np.int32)
    h = w.m >> (levels - 1)
    x = torch.empty((len(idx), h, h, 4), dtype=torch.float32, device=DEV)
    s = torch.empty(len(idx), dtype=torch.float32, device=DEV)
    magpie.magpie_coarse_state(ctx, torch.from_numpy(idx).to(DEV), x, s)
    u = O.rpie_regulariser(Q, w.alpha)
    for i, k in enumerate(idx):
        zk = O.extract(z0, pos[k], w.m)
        xo, so, _ = L.coarse_state(zk, Q, O.revised_exit_wave(zk, Q, d[k]), u, levels)
        xg = x[i].cpu().numpy()
        print(k, "z_H", rel(xg[..., 0:2], xo[..., 0:2]), "e/s", rel(xg[..., 2:4], xo[..., 2:4]),
              "s", abs(s[i].item() - so) / so)
        assert rel(xg[..., 0:2], xo[..., 0:2]) < 1e-6
        assert rel(xg[..., 2:4], xo[..., 2:4]) < 1e-4
        assert abs(s[i].item() - so) < 1e-4 * so


@pytest.mark.parametrize("levels,seed,scale", [(2, 31, 0.3), (3, 32, 0.3), (2, 33, 3.0)])
def test_learned_step_matches_oracle(levels, seed, scale):
    """One learned minibatch step: the keep/reject decision of every window
    whose surrogate margin is not within rounding of zero, the margins, and
    the updated object."""
    w, _, Q, pos, d, z0 = tiny_problem()
    h = w.m >> (levels - 1)
    if h < 8:
        pytest.skip("network needs h >= 8")
    theta = random_theta(L, seed, scale=scale).astype(np.float32).astype(np.float64)
    ctx, zt = make_ctx(w, z0, Q, pos, d, levels, 16)
    net = net_with(theta, h, 16)
    magpie.magpie_attach_cnn(ctx, net)
    batch = np.arange(3, 19, dtype=np.int32)
    magpie.magpie_step(ctx, torch.from_numpy(batch).to(DEV))
    acc, margin = magpie.magpie_learned_window_values(ctx, len(batch))
    u = O.rpie_regulariser(Q, w.alpha)
    zo, acc_o, marg_o = L.learned_minibatch_step(z0, Q, pos, d, u, levels, list(batch), theta)
    scale_m = np.abs(marg_o).max()
    clear = np.abs(marg_o) > 1e-3 * scale_m
    assert np.array_equal(np.array(acc)[clear], acc_o[clear])
    assert rel(np.array(margin)[clear], marg_o[clear]) < 1e-2
    assert rel(zt.cpu().numpy(), zo) < 2e-5
    prop, kept = magpie.magpie_learned_stats(ctx)
    assert prop == len(batch) and kept == int(np.sum(acc))


@pytest.mark.parametrize("levels", [2, 3])
def test_learned_step_on_precision_form_matches_oracle(levels):
    """The learned correction on top of the precision form (tensor-core
    DFTs, m = 64): one 8-window step against the FP64 oracle's learned step;
    the keep/reject decisions of the clearly decided windows, the margins and
    the object, within the transforms' own error."""
    import dataclasses
    w = dataclasses.replace(synth.WORKLOADS["tiny"], name="n160-m64", n=160, m=64, grid=5, step=20, jitter=1)
    z_true, Q, pos = synth.make_problem(w)
    d = O.forward_intensities(z_true, Q, pos)
    rng = np.random.default_rng(35)
    z0 = (np.ones((w.n, w.n)) + 0.1 * rng.normal(size=(w.n, w.n)) * np.exp(1j * rng.normal(size=(w.n, w.n))))
    z0 = z0.astype(np.complex64).astype(np.complex128)
    h = w.m >> (levels - 1)
    theta = random_theta(L, 36 + levels, scale=0.3).astype(np.float32).astype(np.float64)
    ctx, zt = make_ctx(w, z0, Q, pos, d, levels, 8)
    magpie.magpie_set_precision(ctx, 1)
    magpie.magpie_attach_cnn(ctx, net_with(theta, h, 8))
    batch = np.array([0, 3, 6, 9, 12, 16, 20, 24], dtype=np.int32)
    magpie.magpie_step(ctx, torch.from_numpy(batch).to(DEV))
    acc, margin = magpie.magpie_learned_window_values(ctx, len(batch))
    u = O.rpie_regulariser(Q, w.alpha)
    zo, acc_o, marg_o = L.learned_minibatch_step(z0, Q, pos, d, u, levels, list(batch), theta)
    clear = np.abs(marg_o) > 1e-3 * np.abs(marg_o).max()
    e = rel(zt.cpu().numpy(), zo)
    print(f"levels={levels}: object {e:.2e}, kept {int(np.sum(acc))} of {len(batch)}, "
          f"margins {rel(np.array(margin)[clear], marg_o[clear]):.2e}")
    assert np.array_equal(np.array(acc)[clear], acc_o[clear])
    assert rel(np.array(margin)[clear], marg_o[clear]) < 2e-2
    assert e < 1e-4


def test_zero_last_layer_is_plain_step():
    """A network whose last layer is zero proposes the plain coarse step: every
    window keeps it and the step equals the plain step."""
    w, _, Q, pos, d, z0 = tiny_problem()
    theta = random_theta(L, 34)
    theta[-(64 * 9 * 2 + 2):] = 0.0
    ctx1, z1 = make_ctx(w, z0, Q, pos, d, 2, 16)
    ctx2, z2 = make_ctx(w, z0, Q, pos, d, 2, 16)
    magpie.magpie_attach_cnn(ctx1, net_with(theta, 16, 16))
    order = torch.from_numpy(synth.make_order(w.n_pos, 0)).to(DEV)
    magpie.magpie_sweep(ctx1, order)
    magpie.magpie_sweep(ctx2, order)
    assert rel(z1.cpu().numpy(), z2.cpu().numpy()) < 1e-6
    prop, kept = magpie.magpie_learned_stats(ctx1)
    assert prop == kept == w.n_pos


def test_attach_validation():
    w, _, Q, pos, d, z0 = tiny_problem()
    ctx, _ = make_ctx(w, z0, Q, pos, d, 2, 16)
    with pytest.raises(magpie.MagpieError):
        magpie.magpie_attach_cnn(ctx, magpie.magpie_cnn_create(8, 16))   # wrong h
    with pytest.raises(magpie.MagpieError):
        magpie.magpie_attach_cnn(ctx, magpie.magpie_cnn_create(16, 8))   # max_batch < minibatch
    ctx1, _ = make_ctx(w, z0, Q, pos, d, 1, 16)
    with pytest.raises(magpie.MagpieError):
        magpie.magpie_attach_cnn(ctx1, magpie.magpie_cnn_create(32, 16))  # one level
    magpie.magpie_attach_cnn(ctx, None)


def test_trajectories_follow_local_vcycles():
    """A trajectory's end state is T one-window MAGPS cycles (oracle) from its
    start."""
    w, _, Q, pos, d, z0 = tiny_problem()
    ctx, _ = make_ctx(w, z0, Q, pos, d, 2, 16)
    idx = np.array([4, 40], dtype=np.int32)
    T = 3
    tr = learned.window_trajectories(ctx, torch.from_numpy(Q.astype(np.complex64)).to(DEV),
                                     torch.from_numpy(d.astype(np.float32)).to(DEV),
                                     torch.from_numpy(idx).to(DEV), T)
    u = O.rpie_regulariser(Q, w.alpha)
    for i, k in enumerate(idx):
        zk = O.extract(z0, pos[k], w.m)
        for _ in range(T):
            zk = O.magps(zk, Q, O.revised_exit_wave(zk, Q, d[k]), u, 2)
        xT, _, _ = L.coarse_state(zk, Q, O.revised_exit_wave(zk, Q, d[k]), u, 2)
        assert rel(tr.zh[i].cpu().numpy(), xT[..., 0:2]) < 1e-4


def test_training_lowers_the_loss():
    w = synth.WORKLOADS["tiny"]
    data = learned.generate(w, seeds=[41, 42], stages=[0, 2, 5], per_stage=32, dev=DEV, final_sweeps=20)
    assert len(data) == 192
    net = magpie.magpie_cnn_create(16, 64)
    magpie.magpie_cnn_set_params(net, learned.initial_params(dev=DEV))
    losses = learned.train(net, data, epochs=30, batch=64, lr=1e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.7 * losses[0]


def test_trained_network_effect():
    """What the trained network changes against the method without it, on the
    mid workload's sizes (n = 512, m = 128, 900 windows, 3 levels, 10^6
    photons): trained on the plain solver's trajectories of three other seeded
    objects, then 40 sweeps of the held-out problem with and without it from
    z = 1.  Reported: proposals kept, objective and NRMSE against the ground
    truth.  No gain has been measured: about 2% of the proposals pass the
    surrogate test and the two runs end within a few percent of each other
    (the design notes record the runs).  Checked: the acceptance mechanics
    (every window proposes, some proposals are kept) and that the learned run,
    which keeps a proposal only where the window's surrogate is no worse than
    the plain V-cycle's, ends within 5% of the plain one."""
    w = synth.WORKLOADS["mid"]
    h = learned.coarse_side(w.m, w.levels)
    data = learned.generate(w, seeds=[11, 12, 13], stages=[0, 1, 2, 3, 4, 6, 8, 12, 16, 24], per_stage=100,
                            dev=DEV, final_sweeps=60)
    net = magpie.magpie_cnn_create(h, 64)
    magpie.magpie_cnn_set_params(net, learned.initial_params(dev=DEV))
    losses = learned.train(net, data, epochs=40, batch=64, lr=3e-4)
    z_true, Q, pos, d = learned.problem(w, 1, DEV)
    zt = z_true.cpu().numpy().astype(np.complex128)
    mask = O.illuminated_mask(Q.cpu().numpy().astype(np.complex128), pos.cpu().numpy(), zt.shape)
    out = {}
    for mode in ("plain", "learned"):
        z = torch.ones((w.n, w.n), dtype=torch.complex64, device=DEV)
        p = magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha)
        ctx = magpie.magpie_create(p, z, Q, pos, d)
        if mode == "learned":
            magpie.magpie_attach_cnn(ctx, net)
        for s in range(40):
            magpie.magpie_sweep(ctx, torch.from_numpy(synth.make_order(w.n_pos, s)).to(DEV))
        out[mode] = (magpie.magpie_objective(ctx), O.nrmse(z.cpu().numpy(), zt, mask),
                     magpie.magpie_learned_stats(ctx) if mode == "learned" else (0, 0))
    (phi_p, e_p, _), (phi_l, e_l, (prop, kept)) = out["plain"], out["learned"]
    print(f"training loss {losses[0]:.3e} -> {losses[-1]:.3e}; proposals kept {kept}/{prop}; "
          f"after 40 sweeps: objective {phi_l:.5e} vs {phi_p:.5e} plain, NRMSE {e_l:.4e} vs {e_p:.4e} plain")
    assert prop == 40 * w.n_pos and kept > 0
    assert e_l <= 1.05 * e_p and phi_l <= 1.05 * phi_p
