"""Training the learned coarse-level correction on trajectories of the plain
solver, through the library's C ABI (every arithmetic step runs in its CUDA
kernels; this module only schedules the calls and moves tensors).

The plain solver runs from z = 1 on seeded problems; the network input of a
window at an intermediate sweep and the window's coarse object in the
solver's final state give one training pair (the network learns where the
method's own iteration takes a window's coarse state).  The alternative
"local" target follows one window for T V-cycles on its own: windows of the
current object are tiled without overlap into a tall object, and a context
over that object with all of them in one minibatch advances each exactly as
the plain method advances a single window (Algorithm MAGPS with its revised
exit wave refreshed every cycle).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import magpie, synth

# (c_in, c_out) of the six convolutions (the architecture the library declares)
LAYERS = ((4, 32), (32, 64), (64, 128), (128, 512), (512, 64), (64, 2))


def coarse_side(m: int, levels: int) -> int:
    return m >> (levels - 1)


@dataclasses.dataclass
class Trajectories:
    x0: torch.Tensor     # [n][h][h][4] network input at the start
    zh: torch.Tensor     # [n][h][h][2] coarse object T cycles later
    scale: torch.Tensor  # [n] RMS of the plain coarse step at the start

    def __len__(self) -> int:
        return self.x0.shape[0]


def problem(w: synth.Workload, seed: int, dev: torch.device):
    """(ground truth, probe, positions, intensities) of workload `w` with the
    object drawn from `seed`; intensities by the library's forward model plus
    the workload's photon noise."""
    z_true, Q, pos = synth.make_problem_seeded(w, seed)
    zt = torch.from_numpy(z_true.astype(np.complex64)).to(dev)
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(dev)
    post = torch.from_numpy(pos).to(dev)
    clean = magpie.magpie_forward_intensities(zt, Qt, post, w.m)
    if w.photons is not None:
        clean = torch.from_numpy(synth.poisson_noise(clean.cpu().numpy(), w.photons, seed=seed + 3)
                                 .astype(np.float32)).to(dev)
    return zt, Qt, post, clean


def window_trajectories(ctx: magpie.Context, Q: torch.Tensor, d: torch.Tensor, idx: torch.Tensor,
                        T: int) -> Trajectories:
    """Trajectories of windows `idx` of ctx's current object."""
    p = ctx.params
    m, K = p.m, idx.numel()
    dev = Q.device
    h = coarse_side(m, p.levels)
    patches = torch.empty((K, m, m), dtype=torch.complex64, device=dev)
    magpie.magpie_gather_windows(ctx, idx, patches)
    stack = patches.reshape(K * m, m).contiguous()
    spos = torch.stack([torch.arange(K, dtype=torch.int32, device=dev) * m,
                        torch.zeros(K, dtype=torch.int32, device=dev)], dim=1).contiguous()
    sd = d.index_select(0, idx.long()).contiguous()
    sp = magpie.magpie_params_of(K * m, m, m, K, p.levels, K, p.alpha)
    sctx = magpie.magpie_create(sp, stack, Q, spos, sd)
    every = torch.arange(K, dtype=torch.int32, device=dev)
    x0 = torch.empty((K, h, h, 4), dtype=torch.float32, device=dev)
    s0 = torch.empty(K, dtype=torch.float32, device=dev)
    magpie.magpie_coarse_state(sctx, every, x0, s0)
    for _ in range(T):
        magpie.magpie_sweep(sctx, every)
    xT = torch.empty_like(x0)
    sT = torch.empty_like(s0)
    magpie.magpie_coarse_state(sctx, every, xT, sT)
    magpie.magpie_destroy(sctx)
    return Trajectories(x0, xT[..., 0:2].contiguous(), s0)


def generate(w: synth.Workload, seeds, stages, per_stage: int, dev: torch.device, final_sweeps: int = 60,
             target: str = "final", T: int = 4, rng_seed: int = 11) -> Trajectories:
    """Training pairs from problems drawn with `seeds`.  The plain solver runs
    from z = 1 for `final_sweeps` sweeps; after each number of sweeps in
    `stages`, `per_stage` random windows give a network input.  Their target
    is the coarse object of the same windows in the solver's final state
    (target "final"), or after T further cycles of each window on its own
    (target "local", `window_trajectories`)."""
    rng = np.random.default_rng(rng_seed)
    h = coarse_side(w.m, w.levels)
    X, Z, S = [], [], []
    for seed in seeds:
        _, Q, pos, d = problem(w, seed, dev)
        z = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
        p = magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha)
        ctx = magpie.magpie_create(p, z, Q, pos, d)
        saved = {}
        last = final_sweeps if target == "final" else max(stages)
        for s in range(last + 1):
            if s in stages:
                saved[s] = z.clone()
            if s < last:
                magpie.magpie_sweep(ctx, torch.from_numpy(synth.make_order(w.n_pos, s)).to(dev))
        z_final = z.clone()
        for s in sorted(stages):
            idx = torch.from_numpy(rng.choice(w.n_pos, per_stage, replace=False).astype(np.int32)).to(dev)
            z.copy_(saved[s])
            if target == "local":
                t = window_trajectories(ctx, Q, d, idx, T)
                X.append(t.x0)
                Z.append(t.zh)
                S.append(t.scale)
                continue
            for i0 in range(0, per_stage, w.minibatch):
                sel = idx[i0:i0 + w.minibatch]
                x0 = torch.empty((sel.numel(), h, h, 4), dtype=torch.float32, device=dev)
                s0 = torch.empty(sel.numel(), dtype=torch.float32, device=dev)
                xf = torch.empty_like(x0)
                sf = torch.empty_like(s0)
                z.copy_(saved[s])
                magpie.magpie_coarse_state(ctx, sel, x0, s0)
                z.copy_(z_final)
                magpie.magpie_coarse_state(ctx, sel, xf, sf)
                X.append(x0)
                Z.append(xf[..., 0:2].contiguous())
                S.append(s0)
        magpie.magpie_destroy(ctx)
    return Trajectories(torch.cat(X), torch.cat(Z), torch.cat(S))


def train(net: magpie.Cnn, data: Trajectories, epochs: int, batch: int = 64, lr: float = 3e-4,
          seed: int = 13):
    """Adam on shuffled minibatches; returns the mean loss of every epoch."""
    g = torch.Generator(device=data.x0.device)
    g.manual_seed(seed)
    n = len(data)
    losses = torch.zeros((epochs, (n + batch - 1) // batch), dtype=torch.float64, device=data.x0.device)
    for e in range(epochs):
        perm = torch.randperm(n, generator=g, device=data.x0.device)
        for i, s in enumerate(range(0, n, batch)):
            sel = perm[s:s + batch]
            magpie.magpie_cnn_train_step(net, data.x0.index_select(0, sel).contiguous(),
                                         data.zh.index_select(0, sel).contiguous(),
                                         data.scale.index_select(0, sel).contiguous(), lr, losses[e, i:i + 1])
    return losses.mean(dim=1).cpu().numpy()


def initial_params(seed: int = 7, dev: torch.device | None = None) -> torch.Tensor:
    """He-initialised parameters with a zero last layer (the first proposals
    are the plain coarse step)."""
    return torch.from_numpy(synth.make_cnn_params(LAYERS, seed=seed)).to(dev)
