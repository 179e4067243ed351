"""The C ABI library builds, loads and exports every declared symbol; its
argument checks run without a GPU (CPU)."""
import ctypes
import os
import re
import shutil

import pytest

from paper_2504_10118_gb300 import magpie

needs_nvcc = pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available")


@pytest.fixture(scope="module")
def L():
    if shutil.which("nvcc") is not None:
        magpie.build()
    if not os.path.exists(magpie.LIB_PATH):
        pytest.skip("library not built and nvcc not available")
    return magpie.lib()


def declared_functions():
    text = open(magpie.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(magpie_\w+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["magpie_create", "magpie_destroy", "magpie_step", "magpie_sweep", "magpie_objective",
              "magpie_stop_metric", "magpie_set_probe", "magpie_get_probe", "magpie_forward_intensities",
              "magpie_sweep_host", "magpie_group_create", "magpie_group_sweep", "magpie_group_destroy"]:
        assert n in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_error_strings_and_version(L):
    assert L.magpie_version() == 10300
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.magpie_strerror(code)
    assert L.magpie_strerror(-99) == b"unknown error"


def _create(L, **kw):
    p = dict(n_rows=128, n_cols=128, m=32, n_pos=64, levels=2, minibatch=16, alpha=0.1, update_probe=0, beta=0.0,
             deterministic=1)
    p.update(kw)
    h = ctypes.c_void_p()
    params = magpie.magpie_params(p["n_rows"], p["n_cols"], p["m"], p["n_pos"], p["levels"],
                                  p["minibatch"], p["alpha"], p["update_probe"], p["beta"], p["deterministic"])
    # dummy non-NULL pointers: argument checks fail before any of them is used
    dummy = ctypes.c_void_p(0x1000)
    rc = L.magpie_create(ctypes.byref(h), ctypes.byref(params), dummy, dummy, dummy, dummy, None)
    return rc, h


@pytest.mark.parametrize("kw,code", [
    (dict(m=12), magpie.EINVAL),
    (dict(m=512, n_rows=1024, n_cols=1024), magpie.EUNSUPPORTED),
    (dict(m=4), magpie.EUNSUPPORTED),
    (dict(levels=0), magpie.EINVAL),
    (dict(levels=7), magpie.EINVAL),
    (dict(minibatch=0), magpie.EINVAL),
    (dict(minibatch=65), magpie.EINVAL),
    (dict(n_pos=0, minibatch=1), magpie.EINVAL),
    (dict(n_rows=16), magpie.EINVAL),
    (dict(alpha=-1.0), magpie.EINVAL),
    (dict(alpha=float("nan")), magpie.EINVAL),
    (dict(alpha=float("inf")), magpie.EINVAL),
    (dict(update_probe=2), magpie.EINVAL),
    (dict(update_probe=1, beta=-0.5), magpie.EINVAL),
    (dict(update_probe=1, beta=float("nan")), magpie.EINVAL),
    (dict(deterministic=2), magpie.EINVAL),
    (dict(deterministic=-1), magpie.EINVAL),
])
def test_create_rejects_bad_arguments_without_a_gpu(L, kw, code):
    rc, h = _create(L, **kw)
    assert rc == code
    assert not h.value
    assert L.magpie_last_error()


def test_params_layout_matches_the_header():
    text = open(magpie.HEADER).read()
    body = text[text.index("typedef struct {"):text.index("} magpie_params;")]
    fields = [f for f in re_fields(body)]
    assert fields == [name for name, _ in magpie.magpie_params._fields_]
    assert ctypes.sizeof(magpie.magpie_params) == 4 * len(fields)


def re_fields(body):
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl or decl.startswith("typedef"):
            decl = decl.replace("typedef struct {", "").strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1]
        out += [n.strip() for n in names.split(",")]
    return out


def test_null_arguments(L):
    assert L.magpie_step(None, None, 1) == magpie.EINVAL
    assert L.magpie_sweep(None, None) == magpie.EINVAL
    v = ctypes.c_double()
    assert L.magpie_objective(None, ctypes.byref(v)) == magpie.EINVAL
    assert L.magpie_stop_metric(None, ctypes.byref(v)) == magpie.EINVAL
    rc = L.magpie_create(None, None, None, None, None, None, None)
    assert rc == magpie.EINVAL
    assert L.magpie_group_create(None, None, 0, None) == magpie.EINVAL
    assert L.magpie_group_sweep(None, None) == magpie.EINVAL
    on, ms = ctypes.c_int32(), (ctypes.c_float * 2)()
    assert L.magpie_group_form_tuning(None, ctypes.byref(on), ms) == magpie.EINVAL
    assert L.magpie_group_set_persistent(None, 1) == magpie.EINVAL
    assert L.magpie_group_set_wait_limit(None, ctypes.c_double(1.0)) == magpie.EINVAL
    assert L.magpie_group_status(None) == magpie.EINVAL
    assert L.magpie_group_check_waits(None, ctypes.c_double(1e-3)) == magpie.EINVAL
    L.magpie_group_destroy(None)
    L.magpie_destroy(None)


def test_learned_and_precision_entry_points_without_a_gpu(L):
    """Argument checks that run before any device work."""
    assert L.magpie_cnn_param_count() == 980002
    h = ctypes.c_void_p()
    assert L.magpie_cnn_create(None, 16, 8, None) == magpie.EINVAL
    assert L.magpie_cnn_create(ctypes.byref(h), 12, 8, None) == magpie.EINVAL   # h not 8/16/32/64
    assert L.magpie_cnn_create(ctypes.byref(h), 16, 0, None) == magpie.EINVAL   # empty batch
    assert L.magpie_cnn_set_params(None, None) == magpie.EINVAL
    assert L.magpie_cnn_forward(None, None, 1, None) == magpie.EINVAL
    assert L.magpie_cnn_backward(None, None, None) == magpie.EINVAL
    assert L.magpie_cnn_train_step(None, None, None, None, 1, 1e-3, None) == magpie.EINVAL
    assert L.magpie_coarse_state(None, None, 1, None, None) == magpie.EINVAL
    assert L.magpie_gather_windows(None, None, 1, None) == magpie.EINVAL
    assert L.magpie_attach_cnn(None, None) == magpie.EINVAL
    a, b = ctypes.c_int64(), ctypes.c_int64()
    assert L.magpie_learned_stats(None, ctypes.byref(a), ctypes.byref(b)) == magpie.EINVAL
    assert L.magpie_learned_window_values(None, 1, None, None) == magpie.EINVAL
    assert L.magpie_set_precision(None, 1) == magpie.EINVAL
    assert L.magpie_dft2_tc(None, None, 64, 1, 0, None) == magpie.EINVAL
    x = ctypes.c_void_p(16)
    assert L.magpie_dft2_tc(x, x, 32, 1, 0, None) == magpie.EUNSUPPORTED      # m not 64/128/256
    assert L.magpie_dft2_tc(x, x, 64, 0, 0, None) == magpie.EINVAL            # no windows
    assert L.magpie_dft2_tcgen05(None, None, 64, 1, 0, None) == magpie.EINVAL
    assert L.magpie_dft2_tcgen05(x, x, 32, 1, 0, None) == magpie.EUNSUPPORTED
    assert L.magpie_dft2_tcgen05(x, x, 64, 1, 2, None) == magpie.EINVAL        # inverse not 0/1
    assert L.magpie_set_precision(None, 2) == magpie.EINVAL
    assert L.magpie_precision_check_waits(None, ctypes.c_double(1e-3)) == magpie.EINVAL
    L.magpie_cnn_destroy(None)


def test_binding_marshals_only_matching_tensors():
    """The binding passes raw pointers only for tensors of the declared kind,
    dtype, layout and size; anything else raises before any library call."""
    import torch
    cpu = torch.zeros(16, dtype=torch.int32)
    with pytest.raises(TypeError):
        magpie._dev(cpu, torch.int32, 16, "order")              # a host tensor where a device one is due
    assert magpie._host(cpu, torch.int32, 16, "order") == cpu.data_ptr()
    with pytest.raises(ValueError):
        magpie._host(cpu, torch.int64 if cpu.dtype == torch.int32 else torch.int32, 16, "order")
    with pytest.raises(ValueError):
        magpie._host(cpu, torch.int32, 15, "order")             # wrong element count
    with pytest.raises(ValueError):
        magpie._host(torch.zeros(4, 8, dtype=torch.int32).t(), torch.int32, 32, "order")  # not contiguous
    with pytest.raises(TypeError):
        magpie._host([0] * 16, torch.int32, 16, "order")        # not a tensor
