"""The float-atomic update (deterministic = 0) against the FP64 oracle and
against the ordered update (GPU).

The atomic update computes the same minibatch combination
z <- z + sum_k P_k^T (w . Delta_k) / sum_k P_k^T w as the ordered one; only the
order of the float32 sums differs, so every parity bar of the ordered update
applies unchanged.
"""
import numpy as np
import pytest
import torch

from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import magpie, synth
from tests.test_gpu_parity import (INC_TOL, STEP_CASES, STEP_TOL, Problem, check_mid_steps, dev_i32, rel,
                                   tiny_problem)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    magpie.build()
    magpie.lib()


@pytest.mark.parametrize("n,m,grid,step,jit,L,B,cnt", STEP_CASES)
def test_atomic_minibatch_step(n, m, grid, step, jit, L, B, cnt):
    P = Problem(n, m, grid, step, jit, L, B, seed=m + L)
    ctx = P.ctx(deterministic=0)
    batch = synth.make_order(P.N, L)[:cnt]
    magpie.magpie_step(ctx, dev_i32(batch))
    got = P.z_gpu()
    ref = O.minibatch_step(P.z0, P.Q, P.pos, P.d, P.u, L, batch)
    assert rel(got, ref) < STEP_TOL
    assert rel(got - P.z0, ref - P.z0) < INC_TOL
    ctx.close()


def test_atomic_sweeps_match_oracle_and_ordered_update():
    """Three sweeps of the small workload: the atomic update ends within the
    parity bar of the oracle and within rounding of the ordered update; the
    accumulators are cleared between steps (a second context run gives the
    same object to rounding)."""
    P, w = tiny_problem()
    orders = [synth.make_order(P.N, it) for it in range(3)]
    ref = P.z0
    for o in orders:
        ref = O.sweep(ref, P.Q, P.pos, P.d, P.u, w.levels, o, w.minibatch)
    outs = {}
    for det in (1, 0):
        ctx = P.ctx(deterministic=det)
        for o in orders:
            magpie.magpie_sweep(ctx, dev_i32(o))
        outs[det] = P.z_gpu()
        ctx.close()
    assert rel(outs[0], ref) < STEP_TOL
    assert rel(outs[0], outs[1]) < 1e-6


def test_atomic_probe_step():
    """The probe step reads its own per-window terms; with the atomic object
    update the probe and object still match the oracle."""
    P, w = tiny_problem()
    rng = np.random.default_rng(7)
    Q0 = (P.Q * (1 + 0.1 * (rng.standard_normal(P.Q.shape) + 1j * rng.standard_normal(P.Q.shape))))
    Q0 = Q0.astype(np.complex64).astype(np.complex128)
    beta = 0.2
    ctx = P.ctx(update_probe=1, beta=beta, probe=Q0, deterministic=0)
    batch = synth.make_order(P.N, 1)[: w.minibatch]
    magpie.magpie_step(ctx, dev_i32(batch))
    z_ref, Q_ref = O.minibatch_step_with_probe(P.z0, Q0, P.pos, P.d, w.alpha, w.levels, batch, beta)
    assert rel(P.z_gpu(), z_ref) < STEP_TOL
    assert rel(magpie.magpie_get_probe(ctx).cpu().numpy().astype(np.complex128), Q_ref) < STEP_TOL
    ctx.close()


def test_atomic_window_values_and_skipped_index():
    """Per-window Phi_k and ||grad Phi_k|| come out of the atomic update kernel
    too, and a window index out of range is skipped and reported."""
    P, w = tiny_problem()
    ctx = P.ctx(deterministic=0)
    batch = np.array([0, 1, P.N + 3, 2], dtype=np.int32)
    magpie.magpie_step(ctx, dev_i32(batch))
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_objective(ctx)
    assert ei.value.code == magpie.EINDEX
    ref = O.minibatch_step(P.z0, P.Q, P.pos, P.d, P.u, w.levels, [0, 1, 2])
    assert rel(P.z_gpu(), ref) < STEP_TOL
    ctx.close()
    ctx = P.ctx(deterministic=0)
    batch = synth.make_order(P.N, 4)[: w.minibatch]
    magpie.magpie_step(ctx, dev_i32(batch))
    phis, gns = magpie.magpie_window_values(ctx)
    for k in batch[:4]:
        zk = O.extract(P.z0, P.pos[k], w.m)
        assert abs(phis[k] - O.objective_k(zk, P.Q, P.d[k])) < 1e-4 * O.objective_k(zk, P.Q, P.d[k])
        gk = np.linalg.norm(O.gradient_k(zk, P.Q, P.d[k]))
        assert abs(gns[k] - gk) < 1e-4 * gk
    ctx.close()


def test_atomic_mid_workload_full_size():
    """Every step of a sweep of the n=512, m=128, B=64 workload with the atomic
    update, against the oracle from the GPU's state before the step: the same
    object, increment and element-wise bars as the ordered update."""
    check_mid_steps(0)
