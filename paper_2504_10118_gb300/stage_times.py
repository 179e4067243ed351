"""Per-stage timeline of the FP32 window kernel on the n=512, m=128,
900-window, 3-level, minibatch-64 workload.

Builds (and loads) the library variant with the window kernel's %globaltimer
stamps compiled in, runs warm minibatch steps, and prints, per stage, the
mean over all blocks of the time since each block's start, the mean length
of the stage, and the latest block's time, in microseconds:

    MAGPIE_STAGE_TIMES=1 python -m paper_2504_10118_gb300.stage_times [--update atomic|ordered]

(the module sets the variable itself when it is run this way).
"""
from __future__ import annotations

import argparse
import os
import sys

os.environ["MAGPIE_STAGE_TIMES"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402

from . import magpie, synth  # noqa: E402

STAGES = ["start", "exit wave gathered", "column FFTs sent", "row data received",
          "row pass (FFT, projection, inverse FFT) sent", "column data received", "inverse column FFTs",
          "g0", "block sums", "V-cycle and increments"]


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--update", choices=["atomic", "ordered"], default="atomic")
    ap.add_argument("--steps", type=int, default=3, help="timed steps (after three warm ones)")
    args = ap.parse_args(argv)
    magpie.build()
    magpie.lib()
    dev = torch.device("cuda")
    w = synth.WORKLOADS["mid"]
    z_true, Q, pos = synth.make_problem(w)
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(dev)
    post = torch.from_numpy(pos).to(dev)
    d = magpie.magpie_forward_intensities(torch.from_numpy(z_true.astype(np.complex64)).to(dev), Qt, post, w.m)
    z = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
    det = 1 if args.update == "ordered" else 0
    ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha,
                                                       deterministic=det), z, Qt, post, d)
    cl = magpie.blocks_per_window(w.m)
    order = synth.make_order(w.n_pos, 0)
    rows = []
    for s in range(3 + args.steps):
        idx = torch.from_numpy(order[s * w.minibatch:(s + 1) * w.minibatch].copy()).to(dev)
        st = magpie.magpie_stage_times(ctx, idx, cl).numpy().astype(np.float64)
        if s >= 3:
            rows.append(st.reshape(-1, len(STAGES)))
    ctx.close()
    t = np.concatenate(rows)
    rel = (t - t[:, :1]) * 1e-3  # us since each block's start
    starts = t[:, 0] * 1e-3
    print(f"window kernel, m={w.m}, {args.update} update: {t.shape[0]} blocks over {args.steps} steps; "
          f"block starts spread {starts.max() - starts.min():.2f} us within a step at most "
          f"{max((r[:, 0].max() - r[:, 0].min()) * 1e-3 for r in rows):.2f} us")
    print("| stage | mean since block start (us) | mean stage length (us) | max (us) |")
    print("|---|---|---|---|")
    prev = np.zeros(t.shape[0])
    for i, name in enumerate(STAGES):
        if i == 0:
            continue
        col = rel[:, i]
        ok = t[:, i] > 0
        print(f"| {name} | {col[ok].mean():.2f} | {(col[ok] - prev[ok]).mean():.2f} | {col[ok].max():.2f} |")
        prev = np.where(ok, col, prev)
    return 0


if __name__ == "__main__":
    sys.exit(main())
