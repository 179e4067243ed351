"""Ragged and non-square objects (GPU): object sides that are multiples of
neither the update kernels' tiles (16 and 32 pixels) nor of each other, and
windows whose corners sit on the last admissible row and column, so that
every update form writes partial tiles at the object's bottom and right
edges.  Each form is compared with the FP64 oracle at the bars of the square
cases (1e-5 relative on the object and on the step's increment)."""
import numpy as np
import pytest
import torch

from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import magpie, synth
from tests.test_gpu_parity import INC_TOL, STEP_TOL, dev_i32, f32, rel

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    magpie.build()
    magpie.lib()


def ragged_problem(n_rows, n_cols, m, n_pos, seed):
    """A crop of the square generator's object, corners drawn uniformly over
    [0, n_rows - m] x [0, n_cols - m] with the four extreme corners always
    present, noise-free data, a start 10 % off the object."""
    big = synth.make_object(max(n_rows, n_cols), seed=seed)
    z_true = f32(big[:n_rows, :n_cols])
    Q = f32(synth.make_probe(m))
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.integers(0, n_rows - m + 1, n_pos), rng.integers(0, n_cols - m + 1, n_pos)], 1)
    pos[:4] = [[0, 0], [0, n_cols - m], [n_rows - m, 0], [n_rows - m, n_cols - m]]
    pos = pos.astype(np.int32)
    d = O.forward_intensities(z_true, Q, pos).astype(np.float32).astype(np.float64)
    z0 = f32(z_true * (1 + 0.1 * (rng.standard_normal(z_true.shape) + 1j * rng.standard_normal(z_true.shape))))
    return z_true, Q, pos, d, z0


def make_ctx(z0, Q, pos, d, levels, B, alpha=0.1, deterministic=1):
    n_rows, n_cols = z0.shape
    zt = torch.from_numpy(z0.astype(np.complex64)).to(DEV)
    p = magpie.magpie_params_of(n_rows, n_cols, Q.shape[0], len(pos), levels, B, alpha, 0, 0.0, deterministic)
    ctx = magpie.magpie_create(p, zt, torch.from_numpy(Q.astype(np.complex64)).to(DEV), torch.from_numpy(pos).to(DEV),
                               torch.from_numpy(d.astype(np.float32)).to(DEV))
    return ctx, zt


# object rows x columns, window side, windows, levels
RAGGED = [(150, 203, 32, 12, 3), (203, 150, 64, 10, 4), (131, 97, 16, 24, 2), (300, 277, 128, 6, 3)]
FORMS = ["ordered", "atomic", "precision"]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("nr,nc,m,N,L", RAGGED)
def test_ragged_step(nr, nc, m, N, L, form):
    if form == "precision" and m not in (64, 128, 256):
        pytest.skip("tensor-core DFTs need m = 64, 128 or 256")
    z_true, Q, pos, d, z0 = ragged_problem(nr, nc, m, N, seed=nr + m)
    ctx, zt = make_ctx(z0, Q, pos, d, L, N, deterministic=0 if form == "atomic" else 1)
    if form == "precision":
        magpie.magpie_set_precision(ctx, 1)
    batch = synth.make_order(N, 3)  # every window, the four corner windows among them
    magpie.magpie_step(ctx, dev_i32(batch))
    torch.cuda.synchronize()
    got = zt.cpu().numpy().astype(np.complex128)
    ref = O.minibatch_step(z0, Q, pos, d, O.rpie_regulariser(Q, 0.1), L, list(batch))
    e, de = rel(got, ref), rel(got - z0, ref - z0)
    print(f"{form} {nr}x{nc} m={m} L={L}: object {e:.2e}, increment {de:.2e}")
    assert e < STEP_TOL
    # the tensor-core transforms carry about ten times the FP32 FFT's rounding
    assert de < (10 * INC_TOL if form == "precision" else INC_TOL)
    # pixels no window covers are untouched, bit for bit
    cover = np.zeros(z0.shape, dtype=bool)
    for r, c in pos:
        cover[r:r + m, c:c + m] = True
    assert np.array_equal(got[~cover], z0[~cover])
    ctx.close()


@pytest.mark.parametrize("deterministic", [1, 0])
def test_ragged_sweeps(deterministic):
    """Three sweeps over a 150 x 203 object in minibatches of 5 (the last
    one short): the GPU stays within the step bar of the oracle."""
    z_true, Q, pos, d, z0 = ragged_problem(150, 203, 32, 23, seed=5)
    ctx, zt = make_ctx(z0, Q, pos, d, 3, 5, deterministic=deterministic)
    ref = z0
    for s in range(3):
        order = synth.make_order(len(pos), 10 + s)
        magpie.magpie_sweep(ctx, dev_i32(order))
        ref = O.sweep(ref, Q, pos, d, O.rpie_regulariser(Q, 0.1), 3, order, 5)
    torch.cuda.synchronize()
    got = zt.cpu().numpy().astype(np.complex128)
    e = rel(got, ref)
    print(f"deterministic={deterministic}: three sweeps, object {e:.2e}")
    assert e < STEP_TOL
    ctx.close()


def test_ragged_group():
    """Non-square ragged members in one context group: two group sweeps give
    each member exactly the object of two separate sweeps (the group's
    update tiles, up to 32 x 32, also end in partial tiles) and stay within
    the step bar of the oracle."""
    specs = [(150, 203, 32, 12, 3, 5), (203, 150, 64, 10, 4, 4), (131, 97, 16, 24, 2, 7)]
    probs = [ragged_problem(nr, nc, m, N, seed=40 + i) for i, (nr, nc, m, N, L, B) in enumerate(specs)]
    grouped = [make_ctx(p[4], p[1], p[2], p[3], s[4], s[5]) for p, s in zip(probs, specs)]
    separate = [make_ctx(p[4], p[1], p[2], p[3], s[4], s[5]) for p, s in zip(probs, specs)]
    group = magpie.magpie_group_create([c for c, _ in grouped])
    refs = [p[4] for p in probs]
    for sweep in range(2):
        ords = [synth.make_order(s[3], 20 * sweep + i) for i, s in enumerate(specs)]
        magpie.magpie_group_sweep(group, [dev_i32(o) for o in ords])
        for (c, _), o in zip(separate, ords):
            magpie.magpie_sweep(c, dev_i32(o))
        refs = [O.sweep(r, p[1], p[2], p[3], O.rpie_regulariser(p[1], 0.1), s[4], o, s[5])
                for r, p, s, o in zip(refs, probs, specs, ords)]
    torch.cuda.synchronize()
    for (_, zg), (_, zs), ref in zip(grouped, separate, refs):
        assert torch.equal(zg, zs)
        e = rel(zg.cpu().numpy().astype(np.complex128), ref)
        print(f"group member {tuple(zg.shape)}: object {e:.2e}")
        assert e < STEP_TOL
    magpie.magpie_group_destroy(group)
    for c, _ in grouped + separate:
        c.close()
