#!/usr/bin/env python
"""Throughput of the MAGPIE sweep on GB300: patterns/s per sweep.

One step = one sweep (one iteration of Algorithm MAGPIE) over all windows of
the n=512, m=128, 900-window, 3-level, minibatch-64 Poisson workload, with
its inputs resident in HBM.  L2 is flushed (a 256 MiB write) before every
timed sweep, outside the timed interval; each sweep is timed with CUDA
events on the library's stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Several GPUs run independent replicas (the sweep itself runs on one GPU):
rank r uses cuda:LOCAL_RANK, the value is all ranks' patterns over the
slowest rank's time.  `--impl reference` times the FP64 CPU oracle on this
host's cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_10118_gb300 import synth  # noqa: E402

FP32_LANES_PER_SM = 128
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# ncu DRAM traffic of the window kernel per update (1: ordered, 0: atomic)
TRAFFIC_FILES = {1: os.path.join(ROOT, "profiles", "window_kernel_m128_mid.txt"),
                 0: os.path.join(ROOT, "profiles", "window_kernel_atomic_m128_mid.txt")}
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2504_10118_gb300", "csrc", f)
                  for f in ("fft_lines.cuh", "window_kernel.cuh", "window_body.inc")]


def flops_per_window(m: int) -> float:
    """Algorithmic flops of one window: two 2-D FFTs at the nominal 5 M log2 M
    each, plus 60 M for the element-wise work (exit wave, projection,
    residual, gradient, V-cycle and the weighted scatter), M = m^2."""
    M = m * m
    return 10.0 * M * math.log2(M) + 60.0 * M


_FP32_PEAK = {}


def fp32_peak(dev, magpie):
    """(TFLOP/s, source) of the FP32 FMA peak of this GPU: the library's FMA
    rate measurement (8 blocks of 256 threads per SM, 8 independent FMA chains
    per thread, best of three launches), with the nominal figure from the SM
    count and the maximum SM clock beside it.  Measured once per process."""
    import torch
    key = str(dev)
    if key not in _FP32_PEAK:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        pk, src = peaks()
        nominal = sms * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        tf, ms = magpie.magpie_fp32_fma_rate(8192)
        _FP32_PEAK[key] = (tf, f"FP32 FMA rate measured on this GPU ({tf:.1f} TFLOP/s, {ms:.3f} ms launch); "
                               f"nominal {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                               f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz = {nominal:.1f} TFLOP/s")
    return _FP32_PEAK[key]


def tc_flops_per_window(m: int) -> float:
    """Tensor-core flops of one window in the precision form: a forward and an
    inverse 2-D DFT, each 2 m lines x 2 stages of real block GEMMs
    (stage 1: 32 x 32 by 32 x m/16; stage 2: m rows x K x 2 m/16 with K the
    stage's padded depth), three FP16 products each for the hi+lo split."""
    qr = m // 16
    k2 = 16 * ((2 * qr + 15) // 16)
    per_line = 2 * 32 * 32 * qr + 2 * 16 * k2 * 2 * qr
    return 2 * 2 * m * per_line * 3.0


def cnn_flops_per_window(h: int) -> float:
    """Tensor-core flops of the learned correction's network on one window
    (side h on the coarsest grid): 2 x weights x output pixels per layer."""
    layers = ((4, 32, h), (32, 64, h // 2), (64, 128, h // 4), (128, 512, h // 8), (512, 64, h // 4), (64, 2, h))
    return float(sum(2 * 9 * ci * co * s * s for ci, co, s in layers))


def hbm_bytes_per_window(m: int) -> float:
    """Compulsory HBM bytes of one window: its float32 amplitudes."""
    return 4.0 * m * m


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, pg, device) -> float:
    """The largest x over all ranks of the process group (x itself alone)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, steps: int, n_pos: int, slowest_ms: float) -> float:
    """patterns/s of all replicas together: every rank ran `steps` sweeps of
    `n_pos` windows; the job took as long as its slowest rank."""
    return world * steps * n_pos / (slowest_ms * 1e-3)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash() -> str:
    """sha256 over the window kernel's source files (the ncu figures go stale
    when it changes)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def measured_traffic(deterministic: int = 1):
    """DRAM bytes per launch of the window kernel (of the given update) from
    the committed ncu summary, or None when the kernel source changed since it
    was taken."""
    try:
        lines = open(TRAFFIC_FILES[deterministic]).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ":" in ln:
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    src = kernel_source_hash()
    if kv.get("source_sha256") != src or "dram_bytes_per_launch" not in kv:
        return None
    return float(kv["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi samples of one GPU while the benchmark runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", device_id, "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power),
                "window": "warm-up and timed sweeps"}


def gpu_uuid(dev) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x for x in vis.split(",") if x]
        return ids[dev.index] if dev.index < len(ids) else str(dev.index)


def make_data(w, dev, magpie):
    """Object, probe, positions and noisy intensities of workload w on dev.
    Noise-free intensities come from the library's forward model."""
    import torch
    z_true, Q, pos = synth.make_problem(w)
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(dev)
    post = torch.from_numpy(pos).to(dev)
    clean = magpie.magpie_forward_intensities(torch.from_numpy(z_true.astype(np.complex64)).to(dev), Qt, post, w.m)
    d = synth.poisson_noise(clean.cpu().numpy(), w.photons).astype(np.float32)
    return z_true, Qt, post, torch.from_numpy(d).to(dev), d


def oracle_windows_per_second(w, budget_s: float, min_s: float = 10.0):
    """FP64 oracle on this host: minibatch steps of workload w until at least
    min_s seconds have passed (bounded by budget_s); returns (windows/s,
    windows, seconds)."""
    from oracle import magpie_oracle as O
    z_true, Q, pos = synth.make_problem(w)
    clean = O.forward_intensities(z_true, Q, pos)
    d = synth.poisson_noise(clean, w.photons)
    u = O.rpie_regulariser(Q, w.alpha)
    z = np.ones((w.n, w.n), dtype=np.complex128)
    order = synth.make_order(w.n_pos, 0)
    done, t0 = 0, time.perf_counter()
    s = 0
    while True:
        batch = order[s:s + w.minibatch]
        if len(batch) == 0:
            s = 0
            continue
        z = O.minibatch_step(z, Q, pos, d, u, w.levels, batch)
        done += len(batch)
        s += w.minibatch
        el = time.perf_counter() - t0
        if el >= min_s or el >= budget_s:
            return done / el, done, el


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_worker(w, first, warm, timed, per_step, barrier, out):
    """One process of the all-cores oracle timing.  It draws its own slice of
    the workload's windows (four minibatches of the sweep order, starting at
    minibatch `first`, data generated here, untimed), runs `warm` untimed
    steps, meets the others at `barrier`, then runs `timed` steps of
    `per_step` FP64 oracle minibatch steps each, cycling over its four
    minibatches, and puts (windows, seconds) on `out`."""
    from oracle import magpie_oracle as O
    z_true, Q, pos = synth.make_problem(w)
    B = w.minibatch
    order = synth.make_order(w.n_pos, 0)
    sub = pos[order[(first * B + np.arange(4 * B)) % w.n_pos]]
    d = synth.poisson_noise(O.forward_intensities(z_true, Q, sub), w.photons)
    u = O.rpie_regulariser(Q, w.alpha)
    z = np.ones((w.n, w.n), dtype=np.complex128)
    batches = [list(range(b * B, (b + 1) * B)) for b in range(4)]
    done = 0

    def step():
        nonlocal z, done
        for _ in range(per_step):
            z = O.minibatch_step(z, Q, sub, d, u, w.levels, batches[done % 4])
            done += 1

    for _ in range(warm):
        step()
    barrier.wait(timeout=900)
    t0 = time.perf_counter()
    for _ in range(timed):
        step()
    out.put((timed * per_step * B, time.perf_counter() - t0))


def oracle_all_cores(w, warm: int, timed: int, per_step: int):
    """The FP64 oracle on every host core at once: one spawned process per
    core, each timing its own minibatch steps of workload w (see
    _oracle_worker).  Returns (windows/s, windows, seconds, processes), the
    rate being all windows over the slowest process's timed span."""
    import multiprocessing as mp
    import queue

    n = host_cores()
    ctx = mp.get_context("spawn")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    barrier, out = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(w, 4 * i, warm, timed, per_step, barrier, out))
             for i in range(n)]
    for p in procs:
        p.start()
    try:
        res = [out.get(timeout=1200) for _ in procs]
    except queue.Empty:
        raise RuntimeError("an oracle timing process did not report")
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    windows = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return windows / el, windows, el, n


def run_reference(args, w):
    """The reference arm: the FP64 oracle on all host cores, every process
    running two minibatch steps of the workload per step (a bounded sample),
    W untimed steps, then K timed ones; rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    per_step = 2
    value, windows, el, n = oracle_all_cores(w, args.warmup, args.steps, per_step)
    line = {
        "impl": "reference", "metric": "patterns/s per sweep", "value": value, "unit": "patterns/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w),
        "cpu_baseline": {"value": value, "unit": "patterns/s", "cores": n, "kind": "oracle",
                         "sample": f"{n} processes, one per host core, each {per_step} minibatches "
                                   f"({per_step * w.minibatch} windows) of the workload per step; "
                                   f"{windows} windows timed in {el:.1f} s, FP64 NumPy oracle"},
        "e2e": {"value": value, "unit": "patterns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batched_measure(dev, magpie, warmup: int, steps: int, pg=None, clocks=None):
    """The batched workload: 48 independent reconstructions of uneven sizes
    advanced together by one context group; returns (record, total_ms,
    launches, windows).  Photon noise is drawn on the device (3 GB of
    intensities would take tens of seconds on the host)."""
    import torch
    ws = synth.make_batch()
    gen = torch.Generator(device=dev)
    gen.manual_seed(4)
    ctxs, keep = [], []
    for i, w in enumerate(ws):
        z_true, Q, pos = synth.make_problem_seeded(w, 1 + i)
        Qt = torch.from_numpy(Q.astype(np.complex64)).to(dev)
        post = torch.from_numpy(pos).to(dev)
        clean = magpie.magpie_forward_intensities(torch.from_numpy(z_true.astype(np.complex64)).to(dev), Qt, post,
                                                  w.m)
        eta = float(clean.sum(dim=(1, 2)).mean().item() / w.photons)
        d = torch.poisson(clean / eta, generator=gen) * eta
        z = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
        ctxs.append(magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch,
                                                                 w.alpha), z, Qt, post, d))
        keep.append((z, Qt, post, d))
        del clean
    group = magpie.magpie_group_create(ctxs)
    n_total = sum(w.n_pos for w in ws)
    orders = [[torch.from_numpy(synth.make_order(w.n_pos, s)).to(dev) for w in ws] for s in range(warmup + steps)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed():
        for s in range(warmup):
            magpie.magpie_group_sweep(group, orders[s])
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        hold_gpu(min(100.0, 5.0 + 0.25 * steps))
        for s in range(steps):
            flush.zero_()
            ev0[s].record(stream)
            magpie.magpie_group_sweep(group, orders[warmup + s])
            ev1[s].record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        return sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))

    persistent, form_ms = magpie.magpie_group_form_tuning(group)
    total_ms = timed()
    status = magpie.magpie_group_status(group)
    # the other form of a batched step, timed the same way (members' objects
    # continue from where the timed sweeps left them)
    magpie.magpie_group_set_persistent(group, 1 - persistent)
    other_ms = timed()
    status = status or magpie.magpie_group_status(group)
    magpie.magpie_group_set_persistent(group, persistent)
    steps_max = max(math.ceil(w.n_pos / w.minibatch) for w in ws)
    sides = [len({w.m for w in ws if math.ceil(w.n_pos / w.minibatch) > t}) for t in range(steps_max)]
    launches = sum(sides) if persistent else sum(n + 1 for n in sides)
    tuning = magpie.magpie_group_tuning(group)
    shape, shapes = magpie.magpie_group_apply_tuning(group)
    group.close()
    for c in ctxs:
        c.close()
    rec = {"value": steps * n_total / (total_ms * 1e-3), "unit": "patterns/s", "ms_per_step": total_ms / steps,
           "steps": steps, "warmup": warmup,
           "config": {"workload": "batch48", "problems": len(ws), "windows": n_total,
                      "window_sides": sorted({w.m for w in ws}), "object_sides": sorted({w.n for w in ws}),
                      "levels": 3, "minibatch": 64, "update": "ordered (context groups)",
                      "data": "photon noise drawn on the device"},
           "gpu_launches_per_step": launches,
           "form": {"used": "persistent" if persistent else "separate launches",
                    "ms_per_sweep": {"persistent" if persistent else "separate launches": total_ms / steps,
                                     "separate launches" if persistent else "persistent": other_ms / steps},
                    "bounded_waits": "none ran out" if status == magpie.OK else "a wait ran out"},
           "autotuner": {"window_register_bound": {str(m): {"blocks_per_sm": v[0], "ms_per_launch": list(v[1])}
                                                   for m, v in tuning.items()},
                         "update_tile": {"choice": f"{shapes[shape][0]}x{shapes[shape][1]}",
                                         "ms_per_launch": {f"{w}x{h}": ms for w, h, ms in shapes}},
                         "step_form": {"choice": "persistent" if persistent else "separate launches",
                                       "ms_batched_step0": {"separate launches": form_ms[0],
                                                            "persistent": form_ms[1]}}}}
    flops = sum(w.n_pos * flops_per_window(w.m) for w in ws) * steps
    return rec, total_ms, launches, flops


def run_batched(args):
    """The batched workload as its own bench line."""
    import torch
    from paper_2504_10118_gb300 import magpie

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    if rank == 0:
        magpie.build()
    if pg:
        pg.barrier()
    magpie.lib()
    clocks = ClockSampler(gpu_uuid(dev))
    rec, local_ms, launches, flops = batched_measure(dev, magpie, args.warmup, args.steps, pg)
    clk = clocks.stop()
    total_ms = max_over_ranks(local_ms, pg, dev)
    peak, peak_src = fp32_peak(dev, magpie)
    achieved = flops / (total_ms * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": "patterns/s per sweep",
            "value": whole_job_value(world, args.steps, rec["config"]["windows"], total_ms),
            "unit": "patterns/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (48 seeded problems; photon noise drawn on the device)",
            "config": dict(rec["config"], parallelism="replicas",
                           l2="flushed (256 MiB write) before every timed sweep"),
            "gpu_launches": launches * args.steps, "clocks": clk,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "whole group sweep (window and update work of every member)",
                         "peak_source": peak_src},
            "autotuner": rec["autotuner"],
            "form": rec["form"],
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def config_of(w):
    return {"workload": w.name, "n": w.n, "m": w.m, "n_pos": w.n_pos, "levels": w.levels,
            "minibatch": w.minibatch, "alpha": w.alpha, "photons_per_pattern": w.photons,
            "parallelism": "replicas", "l2": "flushed (256 MiB write) before every timed sweep"}


def nrmse_lit(z, z_true, q2, pos, rel: float = 1e-3) -> float:
    """Reconstruction error modulo a global phase, min_phi ||e^{i phi} z - z*|| / ||z*||,
    over the pixels whose summed illumination sum_k P_k^T |Q|^2 reaches
    `rel` of its maximum (unlit pixels carry no data)."""
    m = q2.shape[0]
    cov = np.zeros(z_true.shape)
    for r, c in pos:
        cov[r:r + m, c:c + m] += q2
    lit = cov >= rel * cov.max()
    a, b = np.asarray(z, dtype=np.complex128)[lit], np.asarray(z_true, dtype=np.complex128)[lit]
    ip = np.vdot(a, b)
    ph = ip / abs(ip) if abs(ip) > 0 else 1.0
    return float(np.linalg.norm(ph * a - b) / np.linalg.norm(b))


def sweeps_to_nrmse(w, dev, magpie, target: float, max_sweeps: int, every: int = 10, deterministic: int = 1,
                    precision: int = 0, net=None) -> dict:
    """Sweeps of workload w from z = 1 until the object's NRMSE against the
    truth (global phase removed, lit pixels, as nrmse_lit) is at most
    `target`, checked every `every` sweeps, or `max_sweeps` have run.  Reports
    the device time of the sweeps (CUDA events around each chunk) and the wall
    time from the first sweep to the last check, checks included.  The form:
    the update (`deterministic`), tensor-core DFTs (`precision`) and a
    learned coarse correction (`net`, attached to the context)."""
    import torch
    z_true, Qt, post, dt, _ = make_data(w, dev, magpie)
    q2 = np.abs(Qt.cpu().numpy().astype(np.complex128)) ** 2
    pos = post.cpu().numpy()
    cov = np.zeros(z_true.shape)
    for r, c in pos:
        cov[r:r + w.m, c:c + w.m] += q2
    lit = torch.from_numpy(cov >= 1e-3 * cov.max()).to(dev)
    zt = torch.from_numpy(z_true.astype(np.complex64)).to(dev)[lit].to(torch.complex128)
    z = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
    ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha,
                                                       deterministic=deterministic), z, Qt, post, dt)
    if precision:
        magpie.magpie_set_precision(ctx, precision)
    if net is not None:
        magpie.magpie_attach_cnn(ctx, net)
    orders = torch.from_numpy(np.stack([synth.make_order(w.n_pos, i) for i in range(max_sweeps)])).to(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweeps, ms, err, best = 0, 0.0, 1.0, 1.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while sweeps < max_sweeps and err > target:
        ev0.record()
        for i in range(every):
            magpie.magpie_sweep(ctx, orders[sweeps + i])
        ev1.record()
        a = z[lit].to(torch.complex128)
        ip = torch.vdot(a, zt)
        ph = ip / ip.abs() if ip.abs() > 0 else 1.0
        err = float(torch.linalg.vector_norm(ph * a - zt) / torch.linalg.vector_norm(zt))
        ms += ev0.elapsed_time(ev1)
        sweeps += every
        best = min(best, err)
    wall = time.perf_counter() - t0
    out = {"levels": w.levels, "minibatch": w.minibatch, "alpha": w.alpha, "reached": err <= target,
           "sweeps": sweeps, "seconds": ms * 1e-3, "wall_seconds": wall, "nrmse": err, "best_nrmse": best,
           "update": "ordered" if deterministic else "atomic",
           "dft": {1: "tensor-core FP16 hi+lo (mma.sync)", 2: "tensor-core FP16 hi+lo (tcgen05)"}.get(precision,
                                                                                              "FP32 FFT"),
           "learned": net is not None}
    if net is not None:
        out["proposals_kept"], out["proposals"] = magpie.magpie_learned_stats(ctx)[::-1]
    ctx.close()
    return out


def time_to_nrmse(w, dev, magpie) -> dict:
    """Time to NRMSE <= 1e-3 on the noise-free version of workload w, every
    form at one setting (three levels, minibatch 16, alpha 0.5; with 1e6
    photons per pattern the NRMSE of every form levels off near 0.09, and at
    the workload's minibatch of 64 the iteration stalls near 0.06; at alpha
    0.3 whether a run leaves a plateau at 0.052 turns on rounding, while at
    0.5 every run tried reached the target): the plain FP32 form with either update,
    the precision form (tensor-core DFTs), and the combined form (tensor-core
    DFTs plus the learned coarse correction, its network trained first on
    trajectories of the plain solver at the same setting, untimed).  For
    context, the workload's own setting and the fastest one-level setting."""
    import dataclasses
    import torch
    from paper_2504_10118_gb300 import learned
    clean = dataclasses.replace(w, photons=None)
    setting = dataclasses.replace(clean, levels=3, minibatch=16, alpha=0.5)
    # every form first runs ten untimed sweeps on a context of its own, so
    # that no timed arm pays the process's one-time loading of its kernels
    # (each timed arm still captures its own sweep graph)
    for det, prec in ((1, 0), (0, 0), (1, 1)):
        sweeps_to_nrmse(setting, dev, magpie, 0.0, 10, deterministic=det, precision=prec)
    out = {"target": 1e-3, "data": f"noise-free intensities of {w.name}",
           "setting": {"levels": 3, "minibatch": 16, "alpha": 0.5},
           "warm_up": "10 untimed sweeps of every form on a context of its own first",
           "fp32": sweeps_to_nrmse(setting, dev, magpie, 1e-3, 3000, deterministic=1),
           "fp32_atomic": sweeps_to_nrmse(setting, dev, magpie, 1e-3, 3000, deterministic=0),
           "precision": sweeps_to_nrmse(setting, dev, magpie, 1e-3, 3000, precision=1)}
    t0 = time.perf_counter()
    data = learned.generate(setting, seeds=[11, 12, 13], stages=[0, 1, 2, 3, 4, 6, 8, 12, 16, 24], per_stage=96,
                            dev=dev, final_sweeps=200)
    net = magpie.magpie_cnn_create(learned.coarse_side(setting.m, setting.levels), 64)  # training batch 64
    magpie.magpie_cnn_set_params(net, learned.initial_params(dev=dev))
    losses = learned.train(net, data, epochs=30, batch=64, lr=3e-4)
    torch.cuda.synchronize()
    training = {"pairs": len(data), "epochs": 30, "loss_first_epoch": float(losses[0]),
                "loss_last_epoch": float(losses[-1]), "seconds": time.perf_counter() - t0,
                "targets": "coarse state of the same windows after 200 plain sweeps"}
    sweeps_to_nrmse(setting, dev, magpie, 0.0, 10, precision=1, net=net)
    out["combined"] = sweeps_to_nrmse(setting, dev, magpie, 1e-3, 2500, precision=1, net=net)
    out["combined"]["training"] = training
    net.close()
    sweeps_to_nrmse(clean, dev, magpie, 0.0, 10)
    out["context"] = {
        "workload_setting": sweeps_to_nrmse(clean, dev, magpie, 1e-3, 3000),
        "rpie": sweeps_to_nrmse(dataclasses.replace(clean, levels=1, minibatch=16), dev, magpie, 1e-3, 3000)}
    return out


def precision_record(dev, magpie, warmup: int = 2, steps: int = 3) -> dict:
    """patterns/s of the n=1024, m=256, 2500-window, 4-level workload with
    tensor-core DFTs and with the FP32 FFT window kernel (one context, the
    form switched between the two runs; photon noise drawn on the device)."""
    import torch
    w = synth.WORKLOADS["precision"]
    z_true, Q, pos = synth.make_problem(w)
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(dev)
    post = torch.from_numpy(pos).to(dev)
    clean = magpie.magpie_forward_intensities(torch.from_numpy(z_true.astype(np.complex64)).to(dev), Qt, post, w.m)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4)
    eta = float(clean.sum(dim=(1, 2)).mean().item() / w.photons)
    d = torch.poisson(clean / eta, generator=gen) * eta
    del clean
    z = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
    ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha),
                               z, Qt, post, d)
    del d
    orders = torch.from_numpy(np.stack([synth.make_order(w.n_pos, s) for s in range(warmup + steps)])).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rec = {"config": config_of(w), "data": "photon noise drawn on the device"}
    for name, mode in (("tensor_core_dft", 1), ("tensor_core_dft_tcgen05", 2), ("fp32_fft", 0)):
        magpie.magpie_set_precision(ctx, mode)
        ms = time_sweeps(magpie, ctx, orders, warmup, steps, flush, torch.cuda.current_stream())
        rec[name] = {"value": steps * w.n_pos / (ms * 1e-3), "unit": "patterns/s", "ms_per_step": ms / steps}
    rec["tensor_core_dft"]["mma"] = "mma.sync m16n8k16 (register fragments)"
    rec["tensor_core_dft_tcgen05"]["mma"] = "tcgen05.mma M = 128 (operands in shared memory, accumulators in TMEM)"
    magpie.magpie_stop_metric(ctx)  # reads the context's error flags (a bounded wait that ran out raises)
    ctx.close()
    return rec


def learned_record(dev, magpie, warmup: int = 3, steps: int = 5) -> dict:
    """patterns/s of the learned form on the mid workload (its network
    generated and trained first, untimed, as `--workload learned` does),
    beside the plain FP32 form with the ordered update on the same data."""
    import torch
    from paper_2504_10118_gb300 import learned
    w = synth.WORKLOADS["mid"]
    z_true, Qt, post, dt, _ = make_data(w, dev, magpie)
    t0 = time.perf_counter()
    data = learned.generate(w, seeds=[11, 12, 13], stages=[0, 1, 2, 3, 4, 6, 8, 12, 16, 24], per_stage=100,
                            dev=dev, final_sweeps=60)
    net = magpie.magpie_cnn_create(learned.coarse_side(w.m, w.levels), w.minibatch)
    magpie.magpie_cnn_set_params(net, learned.initial_params(dev=dev))
    losses = learned.train(net, data, epochs=40, batch=64, lr=3e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    orders = torch.from_numpy(np.stack([synth.make_order(w.n_pos, s) for s in range(warmup + steps)])).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    rec = {"config": dict(config_of(w), workload="learned correction on " + w.name),
           "training": {"pairs": len(data), "epochs": 40, "loss_first_epoch": float(losses[0]),
                        "loss_last_epoch": float(losses[-1]), "seconds": train_s,
                        "untimed": "generation and training run before the timed sweeps"}}
    for name, attach in (("learned", True), ("plain_ordered", False)):
        z = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
        ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha),
                                   z, Qt, post, dt)
        if attach:
            magpie.magpie_attach_cnn(ctx, net)
        ms = time_sweeps(magpie, ctx, orders, warmup, steps, flush, torch.cuda.current_stream())
        rec[name] = {"value": steps * w.n_pos / (ms * 1e-3), "unit": "patterns/s", "ms_per_step": ms / steps}
        if attach:
            kept, total = magpie.magpie_learned_stats(ctx)[::-1]
            rec[name]["proposals_kept"], rec[name]["proposals"] = kept, total
        ctx.close()
    net.close()
    return rec


def hold_gpu(ms: float = 20.0) -> None:
    """A bounded spin kernel (about `ms` of GPU time) on the current stream,
    so that the host queues the timed work behind it instead of racing the
    GPU: a timed interval then never includes the GPU waiting for the host's
    next submission (host jitter on a shared machine once inflated a sweep's
    event-timed interval by a third)."""
    import torch
    torch.cuda._sleep(int(ms * 1e-3 * 2.07e9))


def time_sweeps(magpie, ctx, orders, warmup: int, steps: int, flush, stream, pg=None) -> float:
    """Milliseconds of `steps` sweeps after `warmup` untimed ones, each timed
    with CUDA events on `stream` after an L2 flush (outside the events), the
    timed sweeps queued behind a short GPU hold (hold_gpu)."""
    import torch
    for s in range(warmup):
        magpie.magpie_sweep(ctx, orders[s])
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    hold_gpu(min(100.0, 5.0 + 0.25 * steps))
    for s in range(steps):
        flush.zero_()
        ev0[s].record(stream)
        magpie.magpie_sweep(ctx, orders[warmup + s])
        ev1[s].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))


def launches_per_step(args, w) -> int:
    """Kernel launches of one minibatch step of the configured form."""
    if args.learned:
        return 1 + 1 + 1 + 6 + 4 + 1 + 1  # window, coarse state, cast, 6 convolutions, split-K sums, V-cycle, update
    if args.dft in ("tc", "tcgen05"):
        # exit wave + column DFTs, row DFTs + projection, inverse column DFTs + g^0
        # (+ g^1, g^2), the coarse levels (three levels or more), the update
        # (which also forms the finest level)
        return 3 + (1 if w.levels >= 3 else 0) + 1
    return 2


def tensor_roofline(args, w, windows, wk_ms, ap_ms, prof_sweeps, launches, pk, src):
    """Roofline of the tensor-core work of the precision or learned form over
    its window phase (every kernel between the window's exit wave and the
    update kernel), against the measured BF16 dense peak."""
    if args.learned:
        fl = cnn_flops_per_window(w.m >> (w.levels - 1))
        what = "learned form: window phase (window kernel, coarse state, 6 BF16 convolutions, V-cycle)"
    else:
        fl = tc_flops_per_window(w.m)
        what = ("precision form: window phase (3 tensor-core DFT launches with the exit wave, projection and "
                "g0 fused in, V-cycle)")
    ach = windows * fl / (wk_ms * 1e-3) / 1e12
    peak = pk.get("bf16_tflops", 1900.0)
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel": what, "avg_launch_ms": wk_ms / max(launches, 1),
            "peak_source": (f"bf16 dense, {src} (the precision form's FP16 products: the same nominal dense "
                            f"rate as BF16, ratio 1)" if not args.learned else f"bf16 dense, {src}"),
            "tensor_flops_per_window": fl,
            "apply_kernel_ms_per_sweep": ap_ms / prof_sweeps, "window_phase_ms_per_sweep": wk_ms / prof_sweeps}


def run_ours(args, w):
    import torch
    from paper_2504_10118_gb300 import magpie

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    if rank == 0:
        magpie.build()
    if pg:
        pg.barrier()
    magpie.lib()

    fp32_form = args.dft == "fft" and not args.learned
    det = 0 if (fp32_form and args.update == "atomic") else 1
    z_true, Qt, post, dt, d_host = make_data(w, dev, magpie)
    z = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
    ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha,
                                                       deterministic=det), z, Qt, post, dt)
    if args.dft in ("tc", "tcgen05"):
        magpie.magpie_set_precision(ctx, 2 if args.dft == "tcgen05" else 1)
    net = None
    train_info = None
    if args.learned:
        from paper_2504_10118_gb300 import learned
        t0 = time.perf_counter()
        data = learned.generate(w, seeds=[11, 12, 13], stages=[0, 1, 2, 3, 4, 6, 8, 12, 16, 24], per_stage=100,
                                dev=dev, final_sweeps=60)
        net = magpie.magpie_cnn_create(learned.coarse_side(w.m, w.levels), w.minibatch)
        magpie.magpie_cnn_set_params(net, learned.initial_params(dev=dev))
        losses = learned.train(net, data, epochs=40, batch=64, lr=3e-4)
        torch.cuda.synchronize()
        train_info = {"trajectories": len(data), "epochs": 40, "loss_first_epoch": float(losses[0]),
                      "loss_last_epoch": float(losses[-1]), "seconds": time.perf_counter() - t0,
                      "untimed": "generation and training run before the timed region"}
        magpie.magpie_attach_cnn(ctx, net)
    orders = torch.from_numpy(np.stack([synth.make_order(w.n_pos, s)
                                        for s in range(args.warmup + args.steps)])).to(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(gpu_uuid(dev))
    local_ms = time_sweeps(magpie, ctx, orders, args.warmup, args.steps, flush, stream, pg)
    clk = clocks.stop()
    total_ms = max_over_ranks(local_ms, pg, dev)

    # reconstruction quality after warm-up + timed sweeps (host arithmetic on
    # the downloaded object, outside every timed region)
    quality = {"sweeps": args.warmup + args.steps,
               "nrmse_vs_truth": nrmse_lit(z.cpu().numpy(), z_true, np.abs(Qt.cpu().numpy()) ** 2, post.cpu().numpy()),
               "objective": magpie.magpie_objective(ctx)}
    if args.learned:
        quality["proposals_kept"], quality["proposals"] = magpie.magpie_learned_stats(ctx)[::-1]

    # dominant kernel: the per-window kernel, timed with events around each
    # launch of the same kind of sweeps on the library's stream
    prof_sweeps = min(args.steps, 20)
    wk_ms, ap_ms, launches = 0.0, 0.0, 0
    for s in range(prof_sweeps):
        flush.zero_()
        a, b, n = magpie.magpie_profile_sweep(ctx, orders[args.warmup + s])
        wk_ms += a
        ap_ms += b
        launches += n
    windows = prof_sweeps * w.n_pos
    pk, src = peaks()
    alu_peak, alu_src = fp32_peak(dev, magpie)
    achieved_tf = windows * flops_per_window(w.m) / (wk_ms * 1e-3) / 1e12
    achieved_gbs = windows * hbm_bytes_per_window(w.m) / (wk_ms * 1e-3) / 1e9
    traffic = measured_traffic(det) if fp32_form else None

    # the other update of the FP32 form on the same data, timed the same way
    update_ab = None
    if fp32_form and rank == 0 and world == 1:
        z2 = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
        ctx2 = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha,
                                                            deterministic=1 - det), z2, Qt, post, dt)
        ms2 = time_sweeps(magpie, ctx2, orders, args.warmup, args.steps, flush, stream)
        wk2, ap2 = 0.0, 0.0
        for s in range(prof_sweeps):
            flush.zero_()
            a, b, n = magpie.magpie_profile_sweep(ctx2, orders[args.warmup + s])
            wk2 += a
            ap2 += b
        ctx2.close()
        del z2
        rec = {"atomic" if det == 0 else "ordered": {"ms_per_step": total_ms / args.steps,
                                                     "window_kernel_ms_per_sweep": wk_ms / prof_sweeps,
                                                     "update_kernel_ms_per_sweep": ap_ms / prof_sweeps},
               "ordered" if det == 0 else "atomic": {"ms_per_step": ms2 / args.steps,
                                                     "window_kernel_ms_per_sweep": wk2 / prof_sweeps,
                                                     "update_kernel_ms_per_sweep": ap2 / prof_sweeps}}
        update_ab = dict(rec, headline=args.update,
                         note="same data and sweep orders; per-kernel times from event-bracketed launches")

    # end to end through the host-buffer call: order + intensities in, object out
    order_h = [torch.from_numpy(synth.make_order(w.n_pos, 1000 + s)).pin_memory() for s in range(max(2, args.steps))]
    d_pin = torch.from_numpy(d_host).pin_memory()
    z_out = torch.empty((w.n, w.n), dtype=torch.complex64).pin_memory()
    for s in range(2):  # both data buffers allocated and their sweep graphs captured, untimed
        magpie.magpie_sweep_host_async(ctx, order_h[s], d_pin, z_out)
    magpie.magpie_sync(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(args.steps):
        magpie.magpie_sweep_host_async(ctx, order_h[s], d_pin, z_out)
    magpie.magpie_sync(ctx)
    e2e_s = max_over_ranks(time.perf_counter() - t0, pg, dev)
    ctx.close()
    del dt, d_pin

    extras = (w.name == synth.WORKLOADS["mid"].name and fp32_form and rank == 0 and world == 1
              and not args.no_extras)
    ttn = time_to_nrmse(w, dev, magpie) if extras else None
    prec = precision_record(dev, magpie) if extras else None
    batched = None
    if extras:
        batched, _, _, _ = batched_measure(dev, magpie, 3, 5)
    learned_rec = learned_record(dev, magpie) if extras else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v1, nwin1, el1 = oracle_windows_per_second(w, budget_s=30.0)
        timed = max(2, math.ceil(10.0 * v1 / w.minibatch))
        v, nwin, el, n = oracle_all_cores(w, 1, timed, 1)
        cpu = {"value": v, "unit": "patterns/s", "cores": n, "kind": "oracle",
               "sample": f"{n} processes, one per host core, each {timed} minibatch steps of the same "
                         f"workload: {nwin} windows in {el:.1f} s, FP64 NumPy oracle",
               "single_core": {"value": v1, "unit": "patterns/s", "cores": 1,
                               "sample": f"{nwin1} windows in minibatch steps, {el1:.1f} s"}}
    if rank == 0:
        value = whole_job_value(world, args.steps, w.n_pos, total_ms)
        line = {
            "metric": "patterns/s per sweep", "value": value, "unit": "patterns/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp16x3 (hi+lo) DFTs, f32" if args.dft in ("tc", "tcgen05")
                     else ("f32 + bf16 network" if args.learned else "f32"),
            "data": "synthetic (seeded object, probe, raster and Poisson noise)",
            "config": dict(config_of(w), workload=("learned correction on " + w.name) if args.learned else w.name,
                           dft={"tc": "tensor-core FP16 hi+lo (mma.sync)",
                                "tcgen05": "tensor-core FP16 hi+lo (tcgen05, TMEM accumulators)"}.get(args.dft,
                                                                                                  "FP32 FFT"),
                           update="ordered" if det else "atomic"),
            "quality": quality,
            "update_ab": update_ab,
            "time_to_nrmse": ttn,
            "precision": prec,
            "batched": batched,
            "training": train_info,
            "learned": learned_rec,
            "roofline": ({"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved_tf / alu_peak, "traffic": traffic,
                         "kernel": f"window_kernel<{w.m}, {'step' if det else 'step_atomic'}>",
                         "avg_launch_ms": wk_ms / max(launches, 1),
                         "flops_per_window": flops_per_window(w.m),
                         "peak_source": alu_src,
                         "hbm_view": {"achieved": achieved_gbs, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                                      "frac": achieved_gbs / pk.get("hbm_gbs", 6800.0),
                                      "peak_source": f"hbm_gbs, {src}"},
                         "apply_kernel_ms_per_sweep": ap_ms / prof_sweeps,
                         "window_kernel_ms_per_sweep": wk_ms / prof_sweeps}
                         if fp32_form else
                         tensor_roofline(args, w, windows, wk_ms, ap_ms, prof_sweeps, launches, pk, src)),
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_value(world, args.steps, w.n_pos, 1e3 * e2e_s), "unit": "patterns/s",
                    "h2d_bytes_per_step": 4 * w.n_pos + 4 * w.n_pos * w.m * w.m,
                    "d2h_bytes_per_step": 8 * w.n * w.n,
                    "call": "magpie_sweep_host_async x steps, then magpie_sync: every sweep copies its order "
                            "and the whole intensity set in (pinned host buffers, on a copy stream while the "
                            "previous sweep computes) and the object out"},
            "gpu_launches": launches_per_step(args, w) * math.ceil(w.n_pos / w.minibatch) * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(synth.WORKLOADS) + ["batched", "learned"], default="mid")
    ap.add_argument("--dft", choices=["fft", "tc", "tcgen05"], default=None,
                    help="fft: FP32 FFT path; tc: tensor-core FP16 hi+lo DFTs on mma.sync (default for the "
                         "precision workload); tcgen05: the same DFTs on tcgen05 with TMEM accumulators")
    ap.add_argument("--update", choices=["atomic", "ordered"], default="atomic",
                    help="update of the FP32 form: float-atomic accumulation (default) or the ordered, bitwise "
                         "reproducible reduction; the other one is timed too (update_ab)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the time-to-NRMSE, precision and batched records of the default workload")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.workload == "batched":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU reference arm"}))
            return 0
        return run_batched(args)
    if args.dft is None:
        args.dft = "tc" if args.workload == "precision" else "fft"
    args.learned = args.workload == "learned"
    w = synth.WORKLOADS["mid" if args.learned else args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
