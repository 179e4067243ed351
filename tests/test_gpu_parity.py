"""CUDA path (FP32) against the FP64 oracle, through the C ABI (GPU).

Both sides start from the same FP32-representable inputs.  Tolerances: a
minibatch step must agree with the oracle to 1e-5 relative, both over the
whole object and over the step's increment z_after - z_before; the
objective/stopping values to 1e-5 relative; the forward intensities to 1e-5
norm-wise; after the 50-sweep run of the small workload the two objects must
agree to NRMSE 1e-4 (global phase removed).  At full size every step's
increment is also compared pixel by pixel (bars derived in the test).
"""
import numpy as np
import pytest
import torch

from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import magpie, synth

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
INC_TOL = 1e-5  # the same bar on the increment of a step, ||dz_gpu - dz_orc|| / ||dz_orc||


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    magpie.build()
    magpie.lib()


def f32(a):
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


class Problem:
    """A synthetic problem with FP32-representable data for both sides."""

    def __init__(self, n, m, grid, step, jitter, levels, B, alpha=0.1, photons=None, perturb=0.2, seed=0):
        self.n, self.m, self.levels, self.B, self.alpha = n, m, levels, B, alpha
        self.z_true = f32(synth.make_object(n))
        self.Q = f32(synth.make_probe(m))
        self.pos = synth.make_raster(n, m, grid, step, jitter)
        self.N = len(self.pos)
        clean = O.forward_intensities(self.z_true, self.Q, self.pos)
        self.d = synth.poisson_noise(clean, photons).astype(np.float32).astype(np.float64)
        rng = np.random.default_rng(seed)
        z0 = self.z_true + perturb * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        self.z0 = f32(z0)
        self.u = O.rpie_regulariser(self.Q, alpha)

    def ctx(self, z=None, update_probe=0, beta=0.0, probe=None, deterministic=1):
        dev = torch.device("cuda")
        self.zt = torch.from_numpy((self.z0 if z is None else z).astype(np.complex64)).to(dev)
        p = magpie.magpie_params_of(self.n, self.n, self.m, self.N, self.levels, self.B, self.alpha,
                                    update_probe, beta, deterministic)
        Q = self.Q if probe is None else probe
        return magpie.magpie_create(p, self.zt, torch.from_numpy(Q.astype(np.complex64)).to(dev),
                                    torch.from_numpy(self.pos).to(dev),
                                    torch.from_numpy(self.d.astype(np.float32)).to(dev))

    def z_gpu(self):
        torch.cuda.synchronize()
        return self.zt.cpu().numpy().astype(np.complex128)


def dev_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


# ------------------------------------------------------------- forward model
@pytest.mark.parametrize("m", [8, 16, 32, 64, 128, 256])
def test_forward_intensities(m):
    n = 3 * m
    z = f32(synth.make_object(n))
    Q = f32(synth.make_probe(m))
    pos = synth.make_raster(n, m, 3, m // 2, 1)
    ref = O.forward_intensities(z, Q, pos)
    got = magpie.magpie_forward_intensities(torch.from_numpy(z.astype(np.complex64)).cuda(),
                                            torch.from_numpy(Q.astype(np.complex64)).cuda(),
                                            dev_i32(pos), m).cpu().numpy()
    assert rel(got, ref) < STEP_TOL
    big = ref > 1e-3 * ref.max()
    assert np.max(np.abs(got[big] - ref[big]) / ref[big]) < 1e-3


# ------------------------------------------------------------ one minibatch
STEP_CASES = [
    # n, m, grid, step, jitter, levels, B, batch size
    (48, 8, 6, 7, 1, 1, 5, 5), (48, 8, 6, 7, 1, 2, 5, 3), (48, 8, 6, 7, 1, 3, 36, 36),
    (48, 8, 6, 7, 1, 4, 4, 4),
    (64, 16, 6, 8, 1, 1, 8, 8), (64, 16, 6, 8, 1, 3, 8, 7), (64, 16, 6, 8, 1, 5, 8, 8),
    (128, 32, 8, 8, 1, 1, 16, 16), (128, 32, 8, 8, 1, 2, 16, 16), (128, 32, 8, 8, 1, 3, 16, 13),
    (128, 32, 8, 8, 1, 4, 1, 1), (128, 32, 8, 8, 1, 6, 64, 64),
    (192, 64, 6, 24, 2, 1, 9, 9), (192, 64, 6, 24, 2, 3, 9, 9), (192, 64, 6, 24, 2, 7, 9, 5),
    (256, 128, 5, 30, 2, 1, 6, 6), (256, 128, 5, 30, 2, 3, 6, 6), (256, 128, 5, 30, 2, 4, 6, 4),
    (256, 128, 5, 30, 2, 8, 25, 25),
    (512, 256, 3, 100, 2, 1, 4, 4), (512, 256, 3, 100, 2, 4, 9, 9), (512, 256, 3, 100, 2, 6, 3, 3),
    (512, 256, 3, 100, 2, 9, 9, 9),
]


@pytest.mark.parametrize("n,m,grid,step,jit,L,B,cnt", STEP_CASES)
def test_minibatch_step(n, m, grid, step, jit, L, B, cnt):
    P = Problem(n, m, grid, step, jit, L, B, seed=m + L)
    ctx = P.ctx()
    batch = synth.make_order(P.N, L)[:cnt]
    magpie.magpie_step(ctx, dev_i32(batch))
    got = P.z_gpu()
    ref = O.minibatch_step(P.z0, P.Q, P.pos, P.d, P.u, L, batch)
    assert rel(got, ref) < STEP_TOL
    # the increments themselves
    inc_rel = rel(got - P.z0, ref - P.z0)
    assert inc_rel < INC_TOL, inc_rel
    ctx.close()


def test_largest_minibatch():
    """The largest minibatch the library takes (4096 windows, the update
    kernel's corner list filling 48 KiB of shared memory): one step of
    4096 windows of 8 x 8 on a 64 x 64 raster against the oracle."""
    P = Problem(136, 8, 64, 2, 0, 2, 4096, seed=41)
    assert P.N == 4096
    ctx = P.ctx()
    batch = synth.make_order(P.N, 3)
    magpie.magpie_step(ctx, dev_i32(batch))
    got = P.z_gpu()
    ref = O.minibatch_step(P.z0, P.Q, P.pos, P.d, P.u, 2, batch)
    assert rel(got, ref) < STEP_TOL
    assert rel(got - P.z0, ref - P.z0) < INC_TOL
    ctx.close()


def test_duplicate_and_border_windows():
    n, m = 64, 16
    P = Problem(n, m, 4, 12, 0, 3, 6)
    P.pos = np.array([[0, 0], [0, n - m], [n - m, 0], [n - m, n - m], [20, 20], [20, 21]], dtype=np.int32)
    P.N = len(P.pos)
    P.d = O.forward_intensities(P.z_true, P.Q, P.pos).astype(np.float32).astype(np.float64)
    ctx = P.ctx()
    batch = np.array([0, 1, 2, 3, 4, 4], dtype=np.int32)
    magpie.magpie_step(ctx, dev_i32(batch))
    ref = O.minibatch_step(P.z0, P.Q, P.pos, P.d, P.u, 3, batch)
    assert rel(P.z_gpu(), ref) < STEP_TOL
    ctx.close()


# ---------------------------------------------------- objective and metrics
@pytest.mark.parametrize("m,L", [(32, 2), (128, 3)])
def test_objective_and_stop_metric(m, L):
    n = 4 * m
    P = Problem(n, m, 5, m // 2, 1, L, 4, photons=1e6)
    ctx = P.ctx()
    phi = magpie.magpie_objective(ctx)
    stop = magpie.magpie_stop_metric(ctx)
    assert abs(phi - O.objective(P.z0, P.Q, P.pos, P.d)) < STEP_TOL * O.objective(P.z0, P.Q, P.pos, P.d)
    ref_stop = O.stop_metric(P.z0, P.Q, P.pos, P.d)
    assert abs(stop - ref_stop) < STEP_TOL * ref_stop
    phis, gns = magpie.magpie_window_values(ctx)
    for k in (0, P.N // 2, P.N - 1):
        zk = O.extract(P.z0, P.pos[k], m)
        assert abs(phis[k] - O.objective_k(zk, P.Q, P.d[k])) < 1e-4 * O.objective_k(zk, P.Q, P.d[k])
        gk = np.linalg.norm(O.gradient_k(zk, P.Q, P.d[k]))
        assert abs(gns[k] - gk) < 1e-4 * gk
    ctx.close()


# ------------------------------------------------------------------ sweeps
def tiny_problem():
    w = synth.WORKLOADS["tiny"]
    P = Problem(w.n, w.m, w.grid, w.step, w.jitter, w.levels, w.minibatch, alpha=w.alpha, perturb=0.0)
    P.z0 = np.ones((w.n, w.n), dtype=np.complex128)
    return P, w


def test_sweep_matches_oracle():
    P, w = tiny_problem()
    ctx = P.ctx()
    order = synth.make_order(P.N, 0)
    magpie.magpie_sweep(ctx, dev_i32(order))
    ref = O.sweep(P.z0, P.Q, P.pos, P.d, P.u, w.levels, order, w.minibatch)
    assert rel(P.z_gpu(), ref) < STEP_TOL
    ctx.close()


def test_ragged_last_minibatch():
    # 64 windows in minibatches of 24: 24, 24, 16
    P, w = tiny_problem()
    P.B = 24
    ctx = P.ctx()
    order = synth.make_order(P.N, 3)
    magpie.magpie_sweep(ctx, dev_i32(order))
    ref = O.sweep(P.z0, P.Q, P.pos, P.d, P.u, w.levels, order, 24)
    assert rel(P.z_gpu(), ref) < STEP_TOL
    ctx.close()


def test_fixed_iteration_run_small_workload():
    """50 sweeps of the n=128, m=32, 2-level, B=16 workload: final objects
    agree to NRMSE 1e-4 (global phase removed, illuminated pixels)."""
    P, w = tiny_problem()
    ctx = P.ctx()
    z = P.z0.copy()
    for it in range(w.iterations):
        order = synth.make_order(P.N, it)
        magpie.magpie_sweep(ctx, dev_i32(order))
        z = O.sweep(z, P.Q, P.pos, P.d, P.u, w.levels, order, w.minibatch)
    mask = O.illuminated_mask(P.Q, P.pos, z.shape)
    err = O.nrmse(P.z_gpu(), z, mask)
    assert err < 1e-4, err
    # both are reconstructions: the objective went down
    assert magpie.magpie_objective(ctx) < 0.1 * O.objective(P.z0, P.Q, P.pos, P.d)
    ctx.close()


def test_sweeps_are_bitwise_reproducible():
    P, w = tiny_problem()
    outs = []
    for rep in range(2):
        ctx = P.ctx()
        for it in range(3):
            magpie.magpie_sweep(ctx, dev_i32(synth.make_order(P.N, it)))
        outs.append(P.z_gpu())
        ctx.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_and_resume_is_bitwise(precision):
    """Checkpoint/resume: the reconstruction state is the caller's object
    (the probe is fixed), so six sweeps, a host copy of the object, a fresh
    context built from that copy and six more sweeps give bit for bit the
    object of twelve uninterrupted sweeps, for the FP32 and the precision
    form alike."""
    P = Problem(160, 64, 5, 20, 1, 3, 8)
    orders = [dev_i32(synth.make_order(P.N, it)) for it in range(12)]

    def run(z, sweeps):
        ctx = P.ctx(z=z)
        if precision:
            magpie.magpie_set_precision(ctx, 1)
        for o in sweeps:
            magpie.magpie_sweep(ctx, o)
        out = P.z_gpu()
        ctx.close()
        return out

    straight = run(None, orders)
    saved = run(None, orders[:6]).astype(np.complex64)  # the checkpoint: a host copy of the object
    resumed = run(saved.astype(np.complex128), orders[6:])
    assert np.array_equal(straight, resumed)


def oracle_with_float32_ffts():
    """A private copy of the oracle whose 2-D DFTs run in float32 (SciPy),
    used only to measure how much float32 rounding alone moves a result."""
    import importlib.util
    import os

    import scipy.fft as sf
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "magpie_oracle.py")
    spec = importlib.util.spec_from_file_location("oracle_f32_ffts", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.fft2 = lambda x: sf.fft2(np.asarray(x, dtype=np.complex64)).astype(np.complex128)
    mod.ifft2 = lambda x: sf.ifft2(np.asarray(x, dtype=np.complex64)).astype(np.complex128)
    return mod


def increment_errors(before, got, ref):
    """Errors of one step's increment dz = z_after - z_before against the
    oracle's: norm-wise relative, and the largest element-wise relative error
    on the pixels whose oracle increment exceeds 1e-3 and 1e-2 of its
    largest modulus."""
    dg, do = got - before, ref - before
    a = np.abs(do)
    out = [rel(dg, do)]
    for t in (1e-3, 1e-2):
        big = a > t * a.max()
        out.append(float(np.max(np.abs(dg[big] - do[big]) / a[big])))
    return out


# Element-wise bars on a step's increment at full size.  Every pixel's
# increment carries an absolute float32 error of a few 1e-6 of the largest
# increment (the transforms' and the V-cycle's rounding, relative to the
# spectrum and the object, not to the pixel's own increment), so the relative
# error of a pixel grows as its increment shrinks: measured at most 1.8e-3 to
# 3.2e-3 where |dz| > 1e-3 max|dz| (depending on how the kernels' sums of two
# products are rounded) and 4.5e-4 to 6.7e-4 where |dz| > 1e-2 max|dz| over
# the 15 steps of a sweep; the bars leave a factor of 1.5 to 4.
EW_TOL = {1e-3: 5e-3, 1e-2: 2e-3}


# The atomic update sums each pixel's contributions (about seven per step
# here) in an order that varies from run to run.  Where the contributions
# nearly cancel, their float32 rounding is large against the net increment, so
# its errors scatter from run to run around the ordered update's fixed ones:
# over three runs the worst step's increment error measured 0.8e-5, 1.06e-5
# and 1.53e-5 (ordered: 7.5e-6, deterministic), and the element-wise errors
# 3.0e-3 / 6.2e-3 where |dz| > 1e-3 max|dz| and 0.63e-3 / 0.89e-3 where
# |dz| > 1e-2 max|dz|.  Its bars are about twice the worst measured value.
INC_TOL_ATOMIC = 3e-5
EW_TOL_ATOMIC = {1e-3: 1.2e-2, 1e-2: 2e-3}


def check_mid_steps(deterministic):
    """Every step of one sweep of the mid workload from the GPU's own state
    before the step: object to 1e-5, increment to 1e-5 (3e-5 with the atomic
    update), increment element-wise (EW_TOL, EW_TOL_ATOMIC)."""
    w = synth.WORKLOADS["mid"]
    P = Problem(w.n, w.m, w.grid, w.step, w.jitter, w.levels, w.minibatch, alpha=w.alpha,
                photons=w.photons, perturb=0.2)
    order = synth.make_order(P.N, 0)
    ctx = P.ctx(deterministic=deterministic)
    worst = np.zeros(4)
    for s in range(0, P.N, w.minibatch):
        before = P.z_gpu()
        batch = order[s:s + w.minibatch]
        magpie.magpie_step(ctx, dev_i32(batch))
        got = P.z_gpu()
        ref = O.minibatch_step(before, P.Q, P.pos, P.d, P.u, w.levels, batch)
        worst = np.maximum(worst, [rel(got, ref)] + increment_errors(before, got, ref))
    ctx.close()
    assert worst[0] < STEP_TOL, worst
    ew = EW_TOL if deterministic else EW_TOL_ATOMIC
    assert worst[1] < (INC_TOL if deterministic else INC_TOL_ATOMIC), worst
    assert worst[2] < ew[1e-3], worst
    assert worst[3] < ew[1e-2], worst
    return P, order


def test_mid_workload_full_size():
    """The n=512, m=128, 900-window, 3-level, B=64 Poisson workload at full
    size, in the launch configuration the benchmark times.

    Every one of the 15 minibatch steps of a sweep meets the 1e-5 bar, on the
    object and on the step's increment, when the oracle starts from the state
    the GPU reached before that step, and its increment matches pixel by
    pixel (EW_TOL).  Whole sweeps are compared with a bar set by the
    conditioning of the iteration (a reading recorded in the design notes):
    a step's rounding-level differences are carried into every later window
    that overlaps it, so the oracle's own arithmetic with float32 FFTs ends a
    sweep 4.3e-5 from its FP64 result from the true object plus noise, and
    2.5e-3 from the flat start z = 1, whose window spectra are F(Q) itself,
    with exact zeros where the phase is decided by rounding (theta(0) = 0 in
    FP64, a rounding-noise phase in FP32).  The CUDA path (2.4e-5 and 2.6e-3
    measured) must stay within twice the distance measured that way."""
    w = synth.WORKLOADS["mid"]
    P, order = check_mid_steps(1)

    f32_oracle = oracle_with_float32_ffts()
    for start in (P.z0, np.ones((w.n, w.n), dtype=np.complex128)):
        ctx = P.ctx(start)
        magpie.magpie_sweep(ctx, dev_i32(order))
        ref = O.sweep(start, P.Q, P.pos, P.d, P.u, w.levels, order, w.minibatch)
        drift = rel(f32_oracle.sweep(start, P.Q, P.pos, P.d, P.u, w.levels, order, w.minibatch), ref)
        got = rel(P.z_gpu(), ref)
        assert got < max(STEP_TOL, 2.0 * drift), (got, drift)
        ctx.close()


# ------------------------------------------------------------ API behaviour
def test_invalid_window_index_is_reported():
    P, w = tiny_problem()
    ctx = P.ctx()
    batch = np.array([0, 1, P.N, 2], dtype=np.int32)
    magpie.magpie_step(ctx, dev_i32(batch))
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_objective(ctx)
    assert ei.value.code == magpie.EINDEX
    # the valid windows were applied as a minibatch of three
    ref = O.minibatch_step(P.z0, P.Q, P.pos, P.d, P.u, w.levels, [0, 1, 2])
    assert rel(P.z_gpu(), ref) < STEP_TOL
    # the flag was cleared
    magpie.magpie_objective(ctx)
    ctx.close()


def test_set_probe():
    P, w = tiny_problem()
    ctx = P.ctx()
    Q2 = f32(P.Q * np.exp(0.3j) * 0.9)
    magpie.magpie_set_probe(ctx, torch.from_numpy(Q2.astype(np.complex64)).cuda())
    batch = synth.make_order(P.N, 5)[: w.minibatch]
    magpie.magpie_step(ctx, dev_i32(batch))
    ref = O.minibatch_step(P.z0, Q2, P.pos, P.d, O.rpie_regulariser(Q2, w.alpha), w.levels, batch)
    assert rel(P.z_gpu(), ref) < STEP_TOL
    ctx.close()


def probe_problem(L):
    """The small workload with a probe that is 10% off the true one."""
    P, w = tiny_problem()
    P.levels = L
    rng = np.random.default_rng(7)
    Q0 = f32(P.Q * (1 + 0.1 * (rng.standard_normal(P.Q.shape) + 1j * rng.standard_normal(P.Q.shape))))
    return P, w, Q0


@pytest.mark.parametrize("L", [1, 2, 4])
def test_probe_step(L):
    P, w, Q0 = probe_problem(L)
    beta = 0.2
    ctx = P.ctx(update_probe=1, beta=beta, probe=Q0)
    batch = synth.make_order(P.N, 1)[: w.minibatch]
    magpie.magpie_step(ctx, dev_i32(batch))
    z_ref, Q_ref = O.minibatch_step_with_probe(P.z0, Q0, P.pos, P.d, w.alpha, L, batch, beta)
    assert rel(P.z_gpu(), z_ref) < STEP_TOL
    Q_gpu = magpie.magpie_get_probe(ctx).cpu().numpy().astype(np.complex128)
    assert rel(Q_gpu, Q_ref) < STEP_TOL
    ctx.close()


def test_probe_sweep():
    P, w, Q0 = probe_problem(2)
    beta = 0.2
    ctx = P.ctx(update_probe=1, beta=beta, probe=Q0)
    order = synth.make_order(P.N, 2)
    magpie.magpie_sweep(ctx, dev_i32(order))
    z_ref, Q_ref = O.sweep_with_probe(P.z0, Q0, P.pos, P.d, w.alpha, 2, order, w.minibatch, beta)
    assert rel(P.z_gpu(), z_ref) < STEP_TOL
    assert rel(magpie.magpie_get_probe(ctx).cpu().numpy().astype(np.complex128), Q_ref) < STEP_TOL
    # the objective evaluation uses the moved probe
    phi = magpie.magpie_objective(ctx)
    assert abs(phi - O.objective(z_ref, Q_ref, P.pos, P.d)) < 1e-4 * phi
    ctx.close()


def test_probe_fixed_by_default():
    P, w = tiny_problem()
    ctx = P.ctx()
    magpie.magpie_sweep(ctx, dev_i32(synth.make_order(P.N, 0)))
    assert np.array_equal(magpie.magpie_get_probe(ctx).cpu().numpy(), P.Q.astype(np.complex64))
    ctx.close()


def test_sweep_from_host_buffers():
    P, w = tiny_problem()
    ctx = P.ctx()
    order = torch.from_numpy(synth.make_order(P.N, 0)).pin_memory()
    d = torch.from_numpy(P.d.astype(np.float32)).pin_memory()
    out = torch.empty((w.n, w.n), dtype=torch.complex64).pin_memory()
    magpie.magpie_sweep_host(ctx, order, d, out)
    ref = O.sweep(P.z0, P.Q, P.pos, P.d, P.u, w.levels, order.numpy(), w.minibatch)
    assert rel(out.numpy().astype(np.complex128), ref) < STEP_TOL
    ctx.close()


def test_pipelined_host_sweeps():
    """Three pipelined host sweeps (two data buffers in turn, the data of a
    sweep copied while the previous one computes) give exactly the results of
    three magpie_sweep_host calls; the context's own data is untouched."""
    P, w = tiny_problem()
    orders = [torch.from_numpy(synth.make_order(P.N, s)).pin_memory() for s in range(3)]
    d = torch.from_numpy(P.d.astype(np.float32)).pin_memory()
    d2 = (d * 1.25).pin_memory()  # a second data set for the middle sweep
    outs = [torch.empty((w.n, w.n), dtype=torch.complex64).pin_memory() for _ in range(3)]
    ctx = P.ctx()
    for s, dd in enumerate((d, d2, d)):
        magpie.magpie_sweep_host_async(ctx, orders[s], dd, outs[s])
    magpie.magpie_sync(ctx)
    ref_out = torch.empty((w.n, w.n), dtype=torch.complex64).pin_memory()
    ctx2 = P.ctx()
    for s, dd in enumerate((d, d2, d)):
        magpie.magpie_sweep_host(ctx2, orders[s], dd, ref_out)
        assert np.array_equal(outs[s].numpy(), ref_out.numpy())
    ref = O.sweep(P.z0, P.Q, P.pos, P.d, P.u, w.levels, orders[0].numpy(), w.minibatch)
    ctx3 = P.ctx()
    magpie.magpie_sweep_host_async(ctx3, orders[0], d, outs[0])
    magpie.magpie_sync(ctx3)
    assert rel(outs[0].numpy().astype(np.complex128), ref) < STEP_TOL
    ctx.close()
    ctx2.close()
    ctx3.close()


def test_bad_positions_rejected():
    P, w = tiny_problem()
    P.pos = P.pos.copy()
    P.pos[3] = [w.n - w.m + 1, 0]
    with pytest.raises(magpie.MagpieError) as ei:
        P.ctx()
    assert ei.value.code == magpie.EINVAL


@pytest.mark.parametrize("deterministic", [1, 0])
@pytest.mark.parametrize("levels,alpha", [(1, 0.1), (3, 0.1), (3, 0.0), (1, 0.0)])
def test_hard_edged_probe(levels, alpha, deterministic):
    """A probe that is exactly zero outside its disk and on a 4 x 4 block
    inside it: the division rule (a quotient with a zero denominator is 0)
    acts on dead 2 x 2 bins at every level, and with alpha = 0 (u = 0) the
    weight w = |Q|^2 vanishes there, so pixels that only zero parts of the
    probe reach keep their value (the update's positive-denominator rule)."""
    n, m, grid, step = 96, 32, 5, 14
    P = Problem(n, m, grid, step, 1, levels, 8, alpha=alpha, seed=5)
    c = (m - 1) / 2.0
    yy, xx = np.meshgrid(np.arange(m) - c, np.arange(m) - c, indexing="ij")
    Q = P.Q * (np.sqrt(xx ** 2 + yy ** 2) <= 10.0 * m / 32.0)
    Q[12:16, 12:16] = 0.0
    P.Q = f32(Q)
    P.d = O.forward_intensities(P.z_true, P.Q, P.pos).astype(np.float32).astype(np.float64)
    P.u = O.rpie_regulariser(P.Q, alpha)
    assert np.sum(np.abs(P.Q) == 0) > 100
    ctx = P.ctx(deterministic=deterministic)
    batch = synth.make_order(P.N, 2)[:8]
    magpie.magpie_step(ctx, dev_i32(batch))
    got = P.z_gpu()
    ref = O.minibatch_step(P.z0, P.Q, P.pos, P.d, P.u, levels, batch)
    assert rel(got, ref) < STEP_TOL
    assert rel(got - P.z0, ref - P.z0) < INC_TOL
    # pixels no window of the batch reaches with a nonzero weight are unchanged, bit for bit
    w = P.u + np.abs(P.Q) ** 2
    den = np.zeros((n, n))
    for k in batch:
        r, cc = P.pos[k]
        den[r:r + m, cc:cc + m] += w
    assert np.array_equal(got[den == 0], P.z0[den == 0])
    ctx.close()
