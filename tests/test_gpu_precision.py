"""GPU parity of the precision form (tensor-core FP16 hi+lo DFTs) against the
FP64 oracle: the transforms themselves, single minibatch steps at small and
full window size, and a run of sweeps, each on both tensor-core paths
(path 1: register-fragment mma.sync; path 2: tcgen05 with TMEM
accumulators).  Every check prints its error."""
import numpy as np
import pytest
import torch

from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import magpie, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")
PATHS = [1, 2]


@pytest.fixture(scope="module", autouse=True)
def _built():
    magpie.build()
    magpie.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("m", [64, 128, 256])
def test_dft2_matches_library_fft(m, path):
    """Forward and conjugate 2-D DFTs of random windows against numpy's FFT in
    float64: relative error per window within the hi+lo FP16 bound (operands
    to 2^-22, FP32 accumulation over two stages: measured 4.5e-7 to 7.3e-7
    for m = 64 to 256); windows scaled by 2^20 and 2^-30, which the block's
    power-of-two scaling brings into FP16's range, with the same error; and
    an all-zero window, transformed to zeros."""
    rng = np.random.default_rng(m)
    x = (rng.normal(size=(4, m, m)) + 1j * rng.normal(size=(4, m, m))).astype(np.complex64)
    xd = torch.from_numpy(x).to(DEV)
    X = magpie.magpie_dft2_tc(xd, path=path).cpu().numpy()
    Xi = magpie.magpie_dft2_tc(xd, inverse=True, path=path).cpu().numpy()
    for c in range(4):
        ref = O.fft2(x[c].astype(np.complex128))
        refi = O.ifft2(x[c].astype(np.complex128)) * m * m
        e, ei = rel(X[c], ref), rel(Xi[c], refi)
        print(f"path {path} m={m} window {c}: forward {e:.2e} inverse {ei:.2e}")
        assert e < 3e-6 and ei < 3e-6
    for k in (20, -30):  # far above FP16's range, and far below its normal range
        sc = (x[:1] * np.float32(2.0 ** k)).astype(np.complex64)
        Xs = magpie.magpie_dft2_tc(torch.from_numpy(sc).to(DEV), path=path).cpu().numpy()
        es = rel(Xs[0], O.fft2(sc[0].astype(np.complex128)))
        print(f"path {path} m={m} window scaled by 2^{k}: forward {es:.2e}")
        assert es < 3e-6
    zero = torch.zeros((1, m, m), dtype=torch.complex64, device=DEV)
    assert torch.count_nonzero(magpie.magpie_dft2_tc(zero, path=path)) == 0


def small_problem(levels):
    """n = 160, m = 64, 5 x 5 raster at step 20 +-1, noise-free."""
    n, m = 160, 64
    z_true = synth.make_object(n, seed=1)
    Q = synth.make_probe(m)
    pos = synth.make_raster(n, m, 5, 20, 1, seed=3)
    d = O.forward_intensities(z_true, Q, pos)
    rng = np.random.default_rng(8)
    z0 = np.ones((n, n)) + 0.05 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    z0 = z0.astype(np.complex64).astype(np.complex128)
    return n, m, Q, pos, d, z0


def make_ctx(n, m, Q, pos, d, z0, levels, minibatch, alpha=0.1, path=1):
    zt = torch.from_numpy(z0.astype(np.complex64)).to(DEV)
    p = magpie.magpie_params_of(n, n, m, len(pos), levels, minibatch, alpha)
    ctx = magpie.magpie_create(p, zt, torch.from_numpy(Q.astype(np.complex64)).to(DEV),
                               torch.from_numpy(pos.astype(np.int32)).to(DEV),
                               torch.from_numpy(d.astype(np.float32)).to(DEV))
    magpie.magpie_set_precision(ctx, path)
    return ctx, zt


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("levels", [1, 2, 3, 4])
def test_precision_step_matches_oracle(levels, path):
    n, m, Q, pos, d, z0 = small_problem(levels)
    ctx, zt = make_ctx(n, m, Q, pos, d, z0, levels, 8, path=path)
    batch = np.array([3, 7, 11, 12, 13, 17, 21, 24], dtype=np.int32)
    magpie.magpie_step(ctx, torch.from_numpy(batch).to(DEV))
    u = O.rpie_regulariser(Q, 0.1)
    zo = O.minibatch_step(z0, Q, pos, d, u, levels, list(batch))
    zg = zt.cpu().numpy()
    e, de = rel(zg, zo), rel(zg - z0, zo - z0)
    print(f"path {path} levels={levels}: object {e:.2e}, increment {de:.2e}")
    assert e < 1e-5 and de < 1e-4
    phi, gn = magpie.magpie_window_values(ctx)
    for k in batch:
        zk = O.extract(z0, pos[k], m)
        assert abs(phi[k].item() - O.objective_k(zk, Q, d[k])) < 1e-4 * O.objective_k(zk, Q, d[k])


@pytest.mark.parametrize("path", PATHS)
def test_precision_step_m128_matches_oracle(path):
    """The fused transform kernels at m = 128 (eight 16-line blocks per
    window): one 8-window step with three levels, noise-free, from a state
    near the object, against the oracle; and each window's Phi_k."""
    n, m = 320, 128
    z_true = synth.make_object(n, seed=2)
    Q = synth.make_probe(m)
    pos = synth.make_raster(n, m, 4, 60, 2, seed=4)
    d = O.forward_intensities(z_true, Q, pos)
    rng = np.random.default_rng(10)
    z0 = z_true * (1 + 0.05 * (rng.normal(size=z_true.shape) + 1j * rng.normal(size=z_true.shape)))
    z0 = z0.astype(np.complex64).astype(np.complex128)
    ctx, zt = make_ctx(n, m, Q, pos, d, z0, 3, 8, path=path)
    batch = np.array([0, 2, 5, 7, 8, 11, 13, 15], dtype=np.int32)
    magpie.magpie_step(ctx, torch.from_numpy(batch).to(DEV))
    zo = O.minibatch_step(z0, Q, pos, d, O.rpie_regulariser(Q, 0.1), 3, list(batch))
    zg = zt.cpu().numpy()
    e, de = rel(zg, zo), rel(zg - z0, zo - z0)
    print(f"path {path} m=128 L=3 B=8: object {e:.2e}, increment {de:.2e}")
    assert e < 1e-5 and de < 1e-3
    phi, _ = magpie.magpie_window_values(ctx)
    for k in batch:
        ref = O.objective_k(O.extract(z0, pos[k], m), Q, d[k])
        assert abs(phi[k].item() - ref) < 1e-4 * ref


def fp32_ctx(n, m, Q, pos, d, z0, levels, minibatch, alpha=0.1):
    zt = torch.from_numpy(z0.astype(np.complex64)).to(DEV)
    p = magpie.magpie_params_of(n, n, m, len(pos), levels, minibatch, alpha)
    ctx = magpie.magpie_create(p, zt, torch.from_numpy(Q.astype(np.complex64)).to(DEV),
                               torch.from_numpy(pos.astype(np.int32)).to(DEV),
                               torch.from_numpy(d.astype(np.float32)).to(DEV))
    return ctx, zt


def transform_error_ratio(z_true, Q, pos, path=1):
    """Relative error of the windows' intensities |F(Q z_k)|^2 by the
    tensor-core transform over that of the FP32 FFT path (the library's
    forward model), both against the oracle, on the same windows."""
    m = Q.shape[0]
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(DEV)
    zt = torch.from_numpy(z_true.astype(np.complex64)).to(DEV)
    pt = torch.from_numpy(pos.astype(np.int32)).to(DEV)
    i32 = magpie.magpie_forward_intensities(zt, Qt, pt, m).cpu().numpy()
    psi = np.stack([Q * O.extract(z_true, p, m) for p in pos]).astype(np.complex64)
    itc = np.abs(magpie.magpie_dft2_tc(torch.from_numpy(psi).to(DEV), path=path).cpu().numpy()) ** 2
    ref = O.forward_intensities(z_true, Q, pos)
    return rel(itc, ref) / rel(i32, ref)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("start", ["near", "flat"])
def test_precision_full_size_step(start, path):
    """The precision workload's sizes (n = 1024, m = 256, 4 levels): one 64-window
    minibatch step against the oracle (the context holds just those windows),
    from a state near the object and from the flat start z = 1."""
    w = synth.WORKLOADS["precision"]
    z_true, Q, pos = synth.make_problem(w)
    batch = synth.make_order(w.n_pos, 0)[:w.minibatch]
    sub = pos[batch]
    d = O.forward_intensities(z_true, Q, sub)
    if start == "flat":
        z0 = np.ones((w.n, w.n), dtype=np.complex128)
    else:
        rng = np.random.default_rng(9)
        z0 = z_true * (1 + 0.02 * (rng.normal(size=z_true.shape) + 1j * rng.normal(size=z_true.shape)))
        z0 = z0.astype(np.complex64).astype(np.complex128)
    ctx, zt = make_ctx(w.n, w.m, Q, sub, d, z0, w.levels, w.minibatch, path=path)
    ctx32, z32 = fp32_ctx(w.n, w.m, Q, sub, d, z0, w.levels, w.minibatch)
    idx = torch.arange(w.minibatch, dtype=torch.int32, device=DEV)
    magpie.magpie_step(ctx, idx)
    magpie.magpie_step(ctx32, idx)
    u = O.rpie_regulariser(Q, w.alpha)
    zo = O.minibatch_step(z0, Q, sub, d, u, w.levels, list(range(w.minibatch)))
    e_tc, e_32 = rel(zt.cpu().numpy(), zo), rel(z32.cpu().numpy(), zo)
    ratio = transform_error_ratio(z_true, Q, sub[:8], path)
    print(f"path {path} n=1024 m=256 L=4 B=64, {start} start: object error tensor-core {e_tc:.2e}, FP32 FFT {e_32:.2e}; "
          f"transform error ratio {ratio:.1f}")
    # Where the projection amplifies rounding (|Psi| tiny against sqrt(d), as
    # at a flat start) both paths' errors grow by the same conditioning
    # factor: the precision form is held to twice the ratio of the two
    # transforms' own errors times the FP32 path's error, or to 1e-5.
    assert e_tc < max(1e-5, 2 * ratio * e_32)


@pytest.mark.parametrize("path", PATHS)
def test_precision_sweeps_track_oracle(path):
    """Twenty sweeps from the same start: NRMSE between the GPU and the oracle
    iterates, against that of the FP32 FFT path."""
    n, m, Q, pos, d, z0 = small_problem(3)
    ctx, zt = make_ctx(n, m, Q, pos, d, z0, 3, 8, path=path)
    ctx32, z32 = fp32_ctx(n, m, Q, pos, d, z0, 3, 8)
    u = O.rpie_regulariser(Q, 0.1)
    zo = z0.copy()
    for s in range(20):
        order = synth.make_order(len(pos), s)
        magpie.magpie_sweep(ctx, torch.from_numpy(order).to(DEV))
        magpie.magpie_sweep(ctx32, torch.from_numpy(order).to(DEV))
        zo = O.sweep(zo, Q, pos, d, u, 3, order, 8)
    mask = O.illuminated_mask(Q, pos, zo.shape)
    e_tc = O.nrmse(zt.cpu().numpy(), zo, mask)
    e_32 = O.nrmse(z32.cpu().numpy(), zo, mask)
    ratio = transform_error_ratio(O.extract(zo, (0, 0), n), Q, pos[:8], path)
    print(f"path {path} 20 sweeps: NRMSE vs oracle tensor-core {e_tc:.2e}, FP32 FFT {e_32:.2e}; transform error ratio {ratio:.1f}")
    assert e_tc < max(1e-4, 2 * ratio * e_32)


@pytest.mark.parametrize("path", PATHS)
def test_precision_sweeps_bitwise_reproducible(path):
    """Each transform kernel of a step hands its windows to the next one
    window by window (counted tiles, bounded waits) so that their waves
    overlap; the arithmetic does not depend on that timing.  Two contexts
    on the precision workload's sizes (n = 1024, m = 256, 4 levels, five
    64-window minibatches, 1024 blocks per transform launch) end two sweeps
    bit for bit equal, and no wait runs out."""
    w = synth.WORKLOADS["precision"]
    z_true, Q, pos = synth.make_problem(w)
    pos = np.ascontiguousarray(pos[:5 * w.minibatch])
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(DEV)
    pt = torch.from_numpy(pos.astype(np.int32)).to(DEV)
    d = magpie.magpie_forward_intensities(torch.from_numpy(z_true.astype(np.complex64)).to(DEV), Qt, pt, w.m)
    outs = []
    for _ in range(2):
        zt = torch.ones((w.n, w.n), dtype=torch.complex64, device=DEV)
        p = magpie.magpie_params_of(w.n, w.n, w.m, len(pos), w.levels, w.minibatch, w.alpha)
        ctx = magpie.magpie_create(p, zt, Qt, pt, d)
        magpie.magpie_set_precision(ctx, path)
        for s in range(2):
            magpie.magpie_sweep(ctx, torch.from_numpy(synth.make_order(len(pos), s)).to(DEV))
        magpie.magpie_stop_metric(ctx)  # raises on a wait that ran out
        torch.cuda.synchronize()
        outs.append(zt.clone())
        ctx.close()
    assert torch.equal(outs[0], outs[1])
    assert float((outs[0] - 1).abs().max()) > 0  # the sweeps moved the object


@pytest.mark.parametrize("path", PATHS)
def test_handoff_waits_run_out_and_report(path):
    """The self-test of the hand-off waits: every wait asks for one tile more
    than its window has, runs out under a 1 ms limit and skips its tile; the
    call returns MAGPIE_ETIMEOUT, the object is untouched, and the context's
    next step still matches the oracle (the counts were cleared)."""
    n, m, Q, pos, d, z0 = small_problem(3)
    ctx, zt = make_ctx(n, m, Q, pos, d, z0, 3, 8, path=path)
    before = zt.clone()
    assert magpie.magpie_precision_check_waits(ctx, 1e-3) == magpie.ETIMEOUT
    torch.cuda.synchronize()
    assert torch.equal(zt, before)
    batch = np.array([3, 7, 11, 12, 13, 17, 21, 24], dtype=np.int32)
    magpie.magpie_step(ctx, torch.from_numpy(batch).to(DEV))
    zo = O.minibatch_step(z0, Q, pos, d, O.rpie_regulariser(Q, 0.1), 3, list(batch))
    assert rel(zt.cpu().numpy(), zo) < 1e-5
    magpie.magpie_stop_metric(ctx)  # no wait ran out in the real step
    ctx.close()
    ctx32, _ = fp32_ctx(n, m, Q, pos, d, z0, 3, 8)
    assert magpie.magpie_precision_check_waits(ctx32, 1e-3) == magpie.EINVAL
    ctx32.close()
