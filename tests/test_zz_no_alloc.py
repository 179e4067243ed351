"""The minibatch step that allocates no GPU memory, against the context step (GPU).

Some callers cannot allocate device memory: code running inside a host
framework that hands out a fixed memory budget, plug-ins whose host owns all
device allocations, or acquisition loops that cannot afford cudaMalloc's
implicit synchronisation.  magpie_step_noalloc serves them from one fixed
workspace compiled into the library.  Two consecutive calls (the second
reuses the workspace the first one left behind) must give the same object and
per-window values as magpie_step on a context built from the same inputs.
"""
import numpy as np
import pytest
import torch

from paper_2504_10118_gb300 import magpie, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the per-step tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    magpie.build()
    magpie.lib()


def test_noalloc_step_matches_context_step_on_two_calls():
    w = synth.WORKLOADS["mid"]  # 64 windows of 128 x 128: the workspace's full size
    z_true, Q, pos = synth.make_problem(w)
    dev = torch.device("cuda")
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(dev)
    post = torch.from_numpy(pos).to(dev)
    d = magpie.magpie_forward_intensities(torch.from_numpy(z_true.astype(np.complex64)).to(dev), Qt, post, w.m)
    amp = torch.sqrt(d)
    z_ctx = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
    z_na = z_ctx.clone()
    ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, w.n_pos, w.levels, w.minibatch, w.alpha),
                               z_ctx, Qt, post, d)
    phi = torch.zeros(w.n_pos, dtype=torch.float64, device=dev)
    gn = torch.zeros(w.n_pos, dtype=torch.float64, device=dev)
    for call in range(2):
        batch = torch.from_numpy(synth.make_order(w.n_pos, call)[: w.minibatch]).to(dev)
        magpie.magpie_step(ctx, batch)
        magpie.magpie_step_noalloc(z_na, Qt, post, amp, batch, w.levels, w.alpha, phi, gn)
        torch.cuda.synchronize()
        rel = (torch.linalg.vector_norm(z_na - z_ctx) / torch.linalg.vector_norm(z_ctx)).item()
        assert rel < TOL, (call, rel)
        phi_ctx, gn_ctx = magpie.magpie_window_values(ctx)
        b = batch.cpu().numpy()
        np.testing.assert_allclose(phi.cpu().numpy()[b], phi_ctx.numpy()[b], rtol=TOL)
        np.testing.assert_allclose(gn.cpu().numpy()[b], gn_ctx.numpy()[b], rtol=TOL)
    ctx.close()


def test_noalloc_step_rejects_sizes_beyond_its_workspace():
    dev = torch.device("cuda")
    m, N = 128, 65
    obj = torch.ones((256, 256), dtype=torch.complex64, device=dev)
    probe = torch.ones((m, m), dtype=torch.complex64, device=dev)
    pos = torch.zeros((N, 2), dtype=torch.int32, device=dev)
    amp = torch.ones((N, m, m), dtype=torch.float32, device=dev)
    idx = torch.arange(N, dtype=torch.int32, device=dev)  # 65 * 128^2 > 2^20
    phi = torch.zeros(N, dtype=torch.float64, device=dev)
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_step_noalloc(obj, probe, pos, amp, idx, 3, 0.1, phi, phi.clone())
    assert ei.value.code == magpie.EINVAL


def _small_inputs(m, n, step, seed):
    """A raster problem of window side m on an n x n object (data from the
    library's forward model)."""
    dev = torch.device("cuda")
    w = synth.Workload(name=f"n{n}-m{m}", n=n, m=m, grid=(n - m) // step + 1, step=step, jitter=1, levels=1,
                       minibatch=8, alpha=0.1, photons=None, iterations=1)
    z_true, Q, pos = synth.make_problem_seeded(w, seed)
    Qt = torch.from_numpy(Q.astype(np.complex64)).to(dev)
    post = torch.from_numpy(pos).to(dev)
    d = magpie.magpie_forward_intensities(torch.from_numpy(z_true.astype(np.complex64)).to(dev), Qt, post, m)
    return w, Qt, post, d


def test_noalloc_one_level_m64_matches_context_step():
    dev = torch.device("cuda")
    w, Qt, post, d = _small_inputs(64, 160, 12, 7)
    n_pos = post.shape[0]
    z_ctx = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
    z_na = z_ctx.clone()
    ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, n_pos, 1, 8, w.alpha), z_ctx, Qt, post, d)
    phi = torch.zeros(n_pos, dtype=torch.float64, device=dev)
    gn = torch.zeros(n_pos, dtype=torch.float64, device=dev)
    for call in range(2):
        batch = torch.from_numpy(synth.make_order(n_pos, 10 + call)[:8]).to(dev)
        magpie.magpie_step(ctx, batch)
        magpie.magpie_step_noalloc(z_na, Qt, post, torch.sqrt(d), batch, 1, w.alpha, phi, gn)
        torch.cuda.synchronize()
        rel = (torch.linalg.vector_norm(z_na - z_ctx) / torch.linalg.vector_norm(z_ctx)).item()
        assert rel < TOL, (call, rel)
    ctx.close()


def test_noalloc_skips_an_out_of_range_window_and_reports_it():
    """One index beyond n_pos: the call returns MAGPIE_EINDEX and the object is
    what a context step over the remaining windows gives."""
    dev = torch.device("cuda")
    w, Qt, post, d = _small_inputs(64, 160, 12, 8)
    n_pos = post.shape[0]
    z_ctx = torch.ones((w.n, w.n), dtype=torch.complex64, device=dev)
    z_na = z_ctx.clone()
    ctx = magpie.magpie_create(magpie.magpie_params_of(w.n, w.n, w.m, n_pos, 2, 8, w.alpha), z_ctx, Qt, post, d)
    good = synth.make_order(n_pos, 3)[:7]
    bad = np.concatenate([good[:3], [n_pos + 5], good[3:]]).astype(np.int32)
    phi = torch.zeros(n_pos, dtype=torch.float64, device=dev)
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_step_noalloc(z_na, Qt, post, torch.sqrt(d), torch.from_numpy(bad).to(dev), 2, w.alpha, phi,
                                   phi.clone())
    assert ei.value.code == magpie.EINDEX
    magpie.magpie_step(ctx, torch.from_numpy(good.astype(np.int32)).to(dev))
    torch.cuda.synchronize()
    rel = (torch.linalg.vector_norm(z_na - z_ctx) / torch.linalg.vector_norm(z_ctx)).item()
    assert rel < TOL, rel
    assert (z_na - 1).abs().max().item() > 1e-3  # the valid windows did move the object
    ctx.close()


def test_noalloc_rejects_m256():
    dev = torch.device("cuda")
    m, N = 256, 2
    obj = torch.ones((512, 512), dtype=torch.complex64, device=dev)
    probe = torch.ones((m, m), dtype=torch.complex64, device=dev)
    pos = torch.zeros((N, 2), dtype=torch.int32, device=dev)
    amp = torch.ones((N, m, m), dtype=torch.float32, device=dev)
    idx = torch.arange(N, dtype=torch.int32, device=dev)
    phi = torch.zeros(N, dtype=torch.float64, device=dev)
    with pytest.raises(magpie.MagpieError) as ei:
        magpie.magpie_step_noalloc(obj, probe, pos, amp, idx, 2, 0.1, phi, phi.clone())
    assert ei.value.code == magpie.EUNSUPPORTED
