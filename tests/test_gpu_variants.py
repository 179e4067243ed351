"""GPU parity of the paper's variants (the MG/OPT correction term and the
phase rule of Eq. (specification)) against the FP64 oracle, on the FP32 FFT
path and the tensor-core precision path."""
import numpy as np
import pytest
import torch

from oracle import magpie_oracle as O
from paper_2504_10118_gb300 import magpie, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def _built():
    magpie.build()
    magpie.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def problem(m):
    """m = 32: the small workload (n = 128, 8 x 8 raster); m = 64: n = 160,
    5 x 5 raster at step 20.  Noise-free; start = 1 + 5% complex noise."""
    if m == 32:
        w = synth.WORKLOADS["tiny"]
        z_true, Q, pos = synth.make_problem(w)
        n = w.n
    else:
        n = 160
        z_true, Q = synth.make_object(n, seed=1), synth.make_probe(m)
        pos = synth.make_raster(n, m, 5, 20, 1, seed=3)
    d = O.forward_intensities(z_true, Q, pos)
    rng = np.random.default_rng(40)
    z0 = np.ones((n, n)) + 0.05 * (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    return n, Q, pos, d, z0.astype(np.complex64).astype(np.complex128)


def make_ctx(n, Q, pos, d, z0, levels, minibatch, precision):
    m = Q.shape[0]
    zt = torch.from_numpy(z0.astype(np.complex64)).to(DEV)
    p = magpie.magpie_params_of(n, n, m, len(pos), levels, minibatch, 0.1)
    ctx = magpie.magpie_create(p, zt, torch.from_numpy(Q.astype(np.complex64)).to(DEV),
                               torch.from_numpy(pos.astype(np.int32)).to(DEV),
                               torch.from_numpy(d.astype(np.float32)).to(DEV))
    if precision:
        magpie.magpie_set_precision(ctx, 1)
    return ctx, zt


@pytest.mark.parametrize("m,levels,precision", [(32, 2, 0), (32, 3, 0), (64, 3, 0), (64, 4, 1)])
def test_mgopt_step_matches_oracle(m, levels, precision):
    n, Q, pos, d, z0 = problem(m)
    ctx, zt = make_ctx(n, Q, pos, d, z0, levels, 8, precision)
    magpie.magpie_set_variant(ctx, magpie.MGOPT)
    batch = np.array([1, 4, 6, 9, 12, 15, 19, 22], dtype=np.int32)
    magpie.magpie_step(ctx, torch.from_numpy(batch).to(DEV))
    u = O.rpie_regulariser(Q, 0.1)
    zo = O.minibatch_step_variant(z0, Q, pos, d, u, levels, list(batch), mgopt=True)
    zp = O.minibatch_step(z0, Q, pos, d, u, levels, list(batch))
    e = rel(zt.cpu().numpy(), zo)
    print(f"m={m} L={levels} precision={precision}: MG/OPT step error {e:.2e}; "
          f"MG/OPT vs plain step {rel(zo, zp):.2e}")
    assert e < (1e-5 if not precision else 2e-5)
    assert rel(zo, zp) > 10 * e  # the variant is visible above the rounding


@pytest.mark.parametrize("m,precision", [(32, 0), (64, 1)])
def test_phase_rule_matches_oracle(m, precision):
    """Window k is visited with its patch intact, then with its patch set to
    exactly zero (its spectrum is then exactly 0): the second visit must use
    the phases of the first.  Without the rule the second visit uses 0."""
    n, Q, pos, d, z0 = problem(m)
    k = 5
    ctx, zt = make_ctx(n, Q, pos, d, z0, 2, 4, precision)
    magpie.magpie_set_variant(ctx, magpie.PHASE_RULE)
    u = O.rpie_regulariser(Q, 0.1)
    first = [k, 0, 20, 11]
    magpie.magpie_step(ctx, torch.from_numpy(np.array(first, dtype=np.int32)).to(DEV))
    phases = {}
    zo = O.minibatch_step_variant(z0, Q, pos, d, u, 2, first, phases=phases)
    r, c = pos[k]
    zt[r:r + m, c:c + m] = 0
    zo[r:r + m, c:c + m] = 0
    zero_start = zo.copy()
    magpie.magpie_step(ctx, torch.from_numpy(np.array([k], dtype=np.int32)).to(DEV))
    zo = O.minibatch_step_variant(zo, Q, pos, d, u, 2, [k], phases=phases)
    z_default = O.minibatch_step(zero_start, Q, pos, d, u, 2, [k])
    e = rel(zt.cpu().numpy(), zo)
    print(f"m={m} precision={precision}: phase-rule step error {e:.2e}; rule vs theta(0)=0 {rel(zo, z_default):.2e}")
    assert e < (1e-5 if not precision else 2e-5)
    assert rel(zo, z_default) > 1e-2


def test_variant_flags_are_checked():
    n, Q, pos, d, z0 = problem(32)
    ctx, _ = make_ctx(n, Q, pos, d, z0, 2, 8, 0)
    with pytest.raises(magpie.MagpieError):
        magpie.magpie_set_variant(ctx, 4)
    magpie.magpie_set_variant(ctx, magpie.MGOPT | magpie.PHASE_RULE)
    magpie.magpie_set_variant(ctx, 0)
