"""ctypes binding of the MAGPIE sweep library (include/magpie.h).

Argument marshalling only: every function forwards to the C function of the
same name in the in-tree shared library, passing raw device pointers of
torch tensors and the current CUDA stream.  There is no Python or CPU
implementation behind these calls; when the library has not been built the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libmagpie.so")
# the same library with the window kernel's per-stage timestamps compiled in
# (MAGPIE_STAGE_TIMES); build() and lib() use it when the environment variable
# MAGPIE_STAGE_TIMES is 1
STAGES_LIB_PATH = os.path.join(BUILD_DIR, "libmagpie_stages.so")


def _stages() -> bool:
    return os.environ.get("MAGPIE_STAGE_TIMES") == "1"
# translation units, compiled in parallel: the host side and the other
# kernels, and the window kernels of each window side
SOURCES = [os.path.join(HERE, "csrc", f) for f in ("magpie.cu", "window_small.cu", "window_64.cu", "window_128.cu",
                                                   "window_256.cu")]
DEPENDS = [os.path.join(HERE, "csrc", f) for f in ("core.cuh", "fft_lines.cuh", "window_kernel.cuh", "window_body.inc",
                                                   "window_launch.cuh", "learned.cuh", "precision.cuh", "umma.cuh",
                                                   "update.cuh")]
HEADER = os.path.join(ROOT, "include", "magpie.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]

OK, EINVAL, ECUDA, ENOMEM, EUNSUPPORTED, EINDEX, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6


class MagpieError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{message} (code {code})")
        self.code = code


class magpie_params(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("m", ctypes.c_int32),
                ("n_pos", ctypes.c_int32), ("levels", ctypes.c_int32), ("minibatch", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("update_probe", ctypes.c_int32), ("beta", ctypes.c_float),
                ("deterministic", ctypes.c_int32)]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library for sm_103a into the package's _build/ folder
    (the per-stage timestamp variant when MAGPIE_STAGE_TIMES=1)."""
    path = STAGES_LIB_PATH if _stages() else LIB_PATH
    newest = max(os.path.getmtime(p) for p in SOURCES + DEPENDS + [HEADER])
    if not force and os.path.exists(path) and os.path.getmtime(path) >= newest:
        return path
    os.makedirs(BUILD_DIR, exist_ok=True)
    tag = "stages_" if _stages() else ""
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD_DIR, tag + os.path.basename(src) + ".o")
        cmd = ["nvcc", *NVCC_FLAGS, *(["-DMAGPIE_STAGE_TIMES"] if _stages() else []), "-I",
               os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd))
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd)))
    failed = [cmd for cmd, p in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    tmp = path + ".tmp"
    cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = STAGES_LIB_PATH if _stages() else LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"MAGPIE CUDA library not built ({path} missing); "
                               "run paper_2504_10118_gb300.magpie.build()")
        L = ctypes.CDLL(path)
        vp, i32, f32p = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "magpie_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(magpie_params), vp, vp, vp, vp, vp]),
            "magpie_destroy": (None, [vp]),
            "magpie_step": (ctypes.c_int, [vp, vp, i32]),
            "magpie_sweep": (ctypes.c_int, [vp, vp]),
            "magpie_objective": (ctypes.c_int, [vp, dp]),
            "magpie_profile_sweep": (ctypes.c_int, [vp, vp, dp, dp, ctypes.POINTER(i32)]),
            "magpie_stop_metric": (ctypes.c_int, [vp, dp]),
            "magpie_precision_check_waits": (ctypes.c_int, [vp, ctypes.c_double]),
            "magpie_set_probe": (ctypes.c_int, [vp, vp]),
            "magpie_get_probe": (ctypes.c_int, [vp, vp]),
            "magpie_window_values": (ctypes.c_int, [vp, vp, vp]),
            "magpie_sweep_host": (ctypes.c_int, [vp, vp, vp, vp]),
            "magpie_sweep_host_async": (ctypes.c_int, [vp, vp, vp, vp]),
            "magpie_sync": (ctypes.c_int, [vp]),
            "magpie_forward_intensities": (ctypes.c_int, [vp, i32, i32, vp, i32, vp, i32, vp, vp]),
            "magpie_step_noalloc": (ctypes.c_int, [vp, i32, i32, vp, i32, vp, i32, vp, vp, i32, i32,
                                                    ctypes.c_float, vp, vp, vp]),
            "magpie_group_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(vp), i32, vp]),
            "magpie_group_sweep": (ctypes.c_int, [vp, ctypes.POINTER(vp)]),
            "magpie_group_destroy": (None, [vp]),
            "magpie_group_tuning": (ctypes.c_int, [vp, vp, vp]),
            "magpie_group_set_minb": (ctypes.c_int, [vp, i32, i32]),
            "magpie_group_apply_tuning": (ctypes.c_int, [vp, vp, vp, vp, vp]),
            "magpie_group_set_apply_shape": (ctypes.c_int, [vp, i32]),
            "magpie_group_form_tuning": (ctypes.c_int, [vp, vp, vp]),
            "magpie_group_set_persistent": (ctypes.c_int, [vp, i32]),
            "magpie_group_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_double]),
            "magpie_group_status": (ctypes.c_int, [vp]),
            "magpie_group_check_waits": (ctypes.c_int, [vp, ctypes.c_double]),
            "magpie_cnn_param_count": (i32, []),
            "magpie_cnn_create": (ctypes.c_int, [ctypes.POINTER(vp), i32, i32, vp]),
            "magpie_cnn_destroy": (None, [vp]),
            "magpie_cnn_set_tensor_path": (ctypes.c_int, [vp, i32]),
            "magpie_cnn_status": (ctypes.c_int, [vp]),
            "magpie_cnn_set_params": (ctypes.c_int, [vp, vp]),
            "magpie_cnn_get_params": (ctypes.c_int, [vp, vp]),
            "magpie_cnn_forward": (ctypes.c_int, [vp, vp, i32, vp]),
            "magpie_cnn_backward": (ctypes.c_int, [vp, vp, vp]),
            "magpie_cnn_train_step": (ctypes.c_int, [vp, vp, vp, vp, i32, ctypes.c_float, vp]),
            "magpie_coarse_state": (ctypes.c_int, [vp, vp, i32, vp, vp]),
            "magpie_gather_windows": (ctypes.c_int, [vp, vp, i32, vp]),
            "magpie_attach_cnn": (ctypes.c_int, [vp, vp]),
            "magpie_learned_stats": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
            "magpie_learned_window_values": (ctypes.c_int, [vp, i32, vp, vp]),
            "magpie_set_precision": (ctypes.c_int, [vp, i32]),
            "magpie_set_variant": (ctypes.c_int, [vp, i32]),
            "magpie_dft2_tc": (ctypes.c_int, [vp, vp, i32, i32, i32, vp]),
            "magpie_dft2_tcgen05": (ctypes.c_int, [vp, vp, i32, i32, i32, vp]),
            "magpie_fp32_fma_rate": (ctypes.c_int, [i32, dp, dp, vp]),
            "magpie_stage_times": (ctypes.c_int, [vp, vp, i32, vp, ctypes.c_int64]),
            "magpie_window_blocks": (i32, [i32]),
            "magpie_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "magpie_last_error": (ctypes.c_char_p, []),
            "magpie_version": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != OK:
        L = lib()
        raise MagpieError(rc, f"{L.magpie_strerror(rc).decode()}: {L.magpie_last_error().decode()}")


def _dev(t: torch.Tensor, dtype: torch.dtype, numel: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of {numel} elements")
    return t.data_ptr()


def _host(t: torch.Tensor, dtype: torch.dtype, numel: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of {numel} elements")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def magpie_params_of(n_rows, n_cols, m, n_pos, levels, minibatch, alpha, update_probe=0, beta=0.0,
                     deterministic=1) -> magpie_params:
    return magpie_params(int(n_rows), int(n_cols), int(m), int(n_pos), int(levels), int(minibatch), float(alpha),
                         int(update_probe), float(beta), int(deterministic))


class Context:
    """Owns a magpie_ctx and keeps the caller's tensors alive with it."""

    def __init__(self, params: magpie_params, obj, probe, positions, intensities):
        self.params = params
        n, m, N = params.n_rows * params.n_cols, params.m, params.n_pos
        self._keep = (obj, probe, positions, intensities)
        h = ctypes.c_void_p()
        _check(lib().magpie_create(ctypes.byref(h), ctypes.byref(params),
                                   _dev(obj, torch.complex64, n, "object"),
                                   _dev(probe, torch.complex64, m * m, "probe"),
                                   _dev(positions, torch.int32, 2 * N, "positions"),
                                   _dev(intensities, torch.float32, N * m * m, "intensities"),
                                   _stream()))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().magpie_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def magpie_create(params: magpie_params, obj, probe, positions, intensities) -> Context:
    return Context(params, obj, probe, positions, intensities)


def magpie_destroy(ctx: Context) -> None:
    ctx.close()


def magpie_step(ctx: Context, idx: torch.Tensor) -> None:
    _check(lib().magpie_step(ctx.handle, _dev(idx, torch.int32, idx.numel(), "idx"), idx.numel()))


def magpie_sweep(ctx: Context, order: torch.Tensor) -> None:
    _check(lib().magpie_sweep(ctx.handle, _dev(order, torch.int32, ctx.params.n_pos, "order")))


def magpie_profile_sweep(ctx: Context, order: torch.Tensor):
    """(window-kernel ms, apply-kernel ms, steps) of one sweep timed with events."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().magpie_profile_sweep(ctx.handle, _dev(order, torch.int32, ctx.params.n_pos, "order"),
                                      ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
    return a.value, b.value, n.value


def magpie_objective(ctx: Context) -> float:
    v = ctypes.c_double()
    _check(lib().magpie_objective(ctx.handle, ctypes.byref(v)))
    return v.value


def magpie_stop_metric(ctx: Context) -> float:
    v = ctypes.c_double()
    _check(lib().magpie_stop_metric(ctx.handle, ctypes.byref(v)))
    return v.value


def magpie_set_probe(ctx: Context, probe: torch.Tensor) -> None:
    _check(lib().magpie_set_probe(ctx.handle, _dev(probe, torch.complex64, ctx.params.m ** 2, "probe")))


def magpie_get_probe(ctx: Context) -> torch.Tensor:
    m = ctx.params.m
    out = torch.empty((m, m), dtype=torch.complex64, device=ctx._keep[0].device)
    _check(lib().magpie_get_probe(ctx.handle, out.data_ptr()))
    return out


def magpie_window_values(ctx: Context):
    N = ctx.params.n_pos
    phi = torch.empty(N, dtype=torch.float64)
    gn = torch.empty(N, dtype=torch.float64)
    _check(lib().magpie_window_values(ctx.handle, phi.data_ptr(), gn.data_ptr()))
    return phi, gn


def magpie_sweep_host(ctx: Context, order: torch.Tensor, intensities=None, object_out=None) -> None:
    p = ctx.params
    o = _host(order, torch.int32, p.n_pos, "order")
    d = None if intensities is None else _host(intensities, torch.float32, p.n_pos * p.m * p.m, "intensities")
    z = None if object_out is None else _host(object_out, torch.complex64, p.n_rows * p.n_cols, "object_out")
    _check(lib().magpie_sweep_host(ctx.handle, o, d, z))


def magpie_sweep_host_async(ctx: Context, order: torch.Tensor, intensities: torch.Tensor, object_out=None) -> None:
    """Enqueue one pipelined host sweep (see the C header); the tensors are
    kept alive until magpie_sync."""
    p = ctx.params
    o = _host(order, torch.int32, p.n_pos, "order")
    d = _host(intensities, torch.float32, p.n_pos * p.m * p.m, "intensities")
    z = None if object_out is None else _host(object_out, torch.complex64, p.n_rows * p.n_cols, "object_out")
    ctx._pending = getattr(ctx, "_pending", []) + [(order, intensities, object_out)]
    _check(lib().magpie_sweep_host_async(ctx.handle, o, d, z))


def magpie_sync(ctx: Context) -> None:
    _check(lib().magpie_sync(ctx.handle))
    ctx._pending = []


def magpie_forward_intensities(obj, probe, positions, m: int) -> torch.Tensor:
    n_rows, n_cols = obj.shape
    N = positions.shape[0]
    out = torch.empty((N, m, m), dtype=torch.float32, device=obj.device)
    _check(lib().magpie_forward_intensities(_dev(obj, torch.complex64, n_rows * n_cols, "object"),
                                            n_rows, n_cols, _dev(probe, torch.complex64, m * m, "probe"), m,
                                            _dev(positions, torch.int32, 2 * N, "positions"), N,
                                            out.data_ptr(), _stream()))
    return out


def magpie_step_noalloc(obj, probe, positions, amplitudes, idx, levels: int, alpha: float, phi, gnorm) -> None:
    """One minibatch step that allocates no GPU memory (see the C header)."""
    n_rows, n_cols = obj.shape
    m = probe.shape[0]
    N = positions.shape[0]
    _check(lib().magpie_step_noalloc(_dev(obj, torch.complex64, n_rows * n_cols, "object"), n_rows, n_cols,
                                     _dev(probe, torch.complex64, m * m, "probe"), m,
                                     _dev(positions, torch.int32, 2 * N, "positions"), N,
                                     _dev(amplitudes, torch.float32, N * m * m, "amplitudes"),
                                     _dev(idx, torch.int32, idx.numel(), "idx"), idx.numel(), int(levels),
                                     float(alpha), _dev(phi, torch.float64, N, "phi"),
                                     _dev(gnorm, torch.float64, N, "gnorm"), _stream()))


class Group:
    """Owns a magpie_group; keeps its member contexts alive."""

    def __init__(self, ctxs):
        self.members = list(ctxs)
        arr = (ctypes.c_void_p * len(self.members))(*[c.handle for c in self.members])
        h = ctypes.c_void_p()
        _check(lib().magpie_group_create(ctypes.byref(h), arr, len(self.members), _stream()))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().magpie_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def magpie_group_create(ctxs) -> Group:
    return Group(ctxs)


def magpie_group_sweep(group: Group, orders) -> None:
    ptrs = []
    for c, o in zip(group.members, orders):
        ptrs.append(_dev(o, torch.int32, c.params.n_pos, "order"))
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    group._orders = list(orders)  # alive until the next call
    _check(lib().magpie_group_sweep(group.handle, arr))


def magpie_group_destroy(group: Group) -> None:
    group.close()


def magpie_group_tuning(group: Group):
    """{m: (register bound in use, ms per launch of the three candidates, 0
    for one equal to an earlier candidate)} for the window sides the
    autotuner measured."""
    minb = (ctypes.c_int32 * 6)()
    ms = (ctypes.c_float * 18)()
    _check(lib().magpie_group_tuning(group.handle, minb, ms))
    return {8 << i: (minb[i], tuple(ms[3 * i + v] for v in range(3))) for i in range(6) if ms[3 * i] > 0}


def magpie_group_apply_tuning(group: Group):
    """(shape in use, [(tile_w, tile_h, ms per launch)] for the three update tile shapes)."""
    shape = ctypes.c_int32()
    tw, th = (ctypes.c_int32 * 3)(), (ctypes.c_int32 * 3)()
    ms = (ctypes.c_float * 3)()
    _check(lib().magpie_group_apply_tuning(group.handle, ctypes.byref(shape), tw, th, ms))
    return shape.value, [(tw[i], th[i], ms[i]) for i in range(3)]


def magpie_group_set_apply_shape(group: Group, shape: int) -> None:
    _check(lib().magpie_group_set_apply_shape(group.handle, int(shape)))


def magpie_group_set_minb(group: Group, m: int, minb: int) -> None:
    _check(lib().magpie_group_set_minb(group.handle, int(m), int(minb)))


def magpie_group_form_tuning(group: Group):
    """(1 if sweeps use the persistent form else 0, (ms per batched step 0 as
    separate launches, ms in the persistent form))."""
    on = ctypes.c_int32()
    ms = (ctypes.c_float * 2)()
    _check(lib().magpie_group_form_tuning(group.handle, ctypes.byref(on), ms))
    return on.value, (ms[0], ms[1])


def magpie_group_set_persistent(group: Group, persistent: int) -> None:
    _check(lib().magpie_group_set_persistent(group.handle, int(persistent)))


def magpie_group_set_wait_limit(group: Group, seconds: float) -> None:
    _check(lib().magpie_group_set_wait_limit(group.handle, float(seconds)))


def magpie_group_status(group: Group) -> int:
    """OK, or ETIMEOUT if a dependency wait of the persistent form ran out
    since the last call (returned, not raised)."""
    return lib().magpie_group_status(group.handle)


def magpie_group_check_waits(group: Group, seconds: float) -> int:
    """Self-test of the persistent form's bounded waits: ETIMEOUT expected
    (returned, not raised)."""
    return lib().magpie_group_check_waits(group.handle, float(seconds))


# ----------------------------------------------------------- paper variants
MGOPT, PHASE_RULE = 1, 2


def magpie_set_variant(ctx: Context, flags: int) -> None:
    _check(lib().magpie_set_variant(ctx.handle, int(flags)))


# ----------------------------------------------------------- precision form
def magpie_set_precision(ctx: Context, mode: int) -> None:
    """0: FP32 FFTs; 1: tensor-core DFTs with mma.sync; 2: with tcgen05."""
    _check(lib().magpie_set_precision(ctx.handle, int(mode)))


def magpie_precision_check_waits(ctx: Context, seconds: float) -> int:
    """Return code of the hand-off wait self-test (MAGPIE_ETIMEOUT when every
    bounded wait ran out, as it should)."""
    return int(lib().magpie_precision_check_waits(ctx.handle, float(seconds)))


def magpie_dft2_tc(x: torch.Tensor, inverse: bool = False, path: int = 1) -> torch.Tensor:
    """2-D DFTs of x [count][m][m] (complex64, CUDA) by the tensor-core path
    (path 1: mma.sync, 2: tcgen05; the numbering of magpie_set_precision)."""
    count, m, _ = x.shape
    out = torch.empty_like(x)
    fn = lib().magpie_dft2_tcgen05 if path == 2 else lib().magpie_dft2_tc
    _check(fn(_dev(x, torch.complex64, count * m * m, "x"), out.data_ptr(), m, count, int(bool(inverse)), _stream()))
    return out


# ------------------------------------------------- learned coarse correction
def magpie_cnn_param_count() -> int:
    return lib().magpie_cnn_param_count()


class Cnn:
    """Owns a magpie_cnn (the network of the learned coarse correction)."""

    def __init__(self, h: int, max_batch: int):
        self.h, self.max_batch = h, max_batch
        self.P = magpie_cnn_param_count()
        hd = ctypes.c_void_p()
        _check(lib().magpie_cnn_create(ctypes.byref(hd), h, max_batch, _stream()))
        self.handle = hd

    def close(self):
        if getattr(self, "handle", None):
            lib().magpie_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def magpie_cnn_create(h: int, max_batch: int) -> Cnn:
    return Cnn(h, max_batch)


def magpie_cnn_destroy(cnn: Cnn) -> None:
    cnn.close()


def magpie_cnn_set_tensor_path(cnn: Cnn, path: int) -> None:
    """1: tcgen05 convolutions where the layer fits, 0: mma.sync everywhere."""
    _check(lib().magpie_cnn_set_tensor_path(cnn.handle, int(path)))


def magpie_cnn_status(cnn: Cnn) -> None:
    """Raises MagpieError(ETIMEOUT) if a convolution's bounded wait ran out."""
    _check(lib().magpie_cnn_status(cnn.handle))


def magpie_cnn_set_params(cnn: Cnn, theta: torch.Tensor) -> None:
    _check(lib().magpie_cnn_set_params(cnn.handle, _dev(theta, torch.float32, cnn.P, "theta")))


def magpie_cnn_get_params(cnn: Cnn, theta: torch.Tensor) -> None:
    _check(lib().magpie_cnn_get_params(cnn.handle, _dev(theta, torch.float32, cnn.P, "theta")))


def magpie_cnn_forward(cnn: Cnn, x: torch.Tensor, y: torch.Tensor) -> None:
    b = x.shape[0]
    hh = cnn.h * cnn.h
    _check(lib().magpie_cnn_forward(cnn.handle, _dev(x, torch.float32, b * hh * 4, "x"), b,
                                    _dev(y, torch.float32, b * hh * 2, "y")))


def magpie_cnn_backward(cnn: Cnn, dy: torch.Tensor, grad: torch.Tensor) -> None:
    _check(lib().magpie_cnn_backward(cnn.handle, _dev(dy, torch.float32, dy.numel(), "dy"),
                                     _dev(grad, torch.float32, cnn.P, "grad")))


def magpie_cnn_train_step(cnn: Cnn, x0: torch.Tensor, zh: torch.Tensor, scale: torch.Tensor, lr: float,
                          loss: torch.Tensor) -> None:
    b = x0.shape[0]
    hh = cnn.h * cnn.h
    _check(lib().magpie_cnn_train_step(cnn.handle, _dev(x0, torch.float32, b * hh * 4, "x0"),
                                       _dev(zh, torch.float32, b * hh * 2, "zh"),
                                       _dev(scale, torch.float32, b, "scale"), b, float(lr),
                                       _dev(loss, torch.float64, 1, "loss")))


def magpie_coarse_state(ctx: Context, idx: torch.Tensor, x: torch.Tensor, scale: torch.Tensor) -> None:
    n = idx.numel()
    h = ctx.params.m >> (ctx.params.levels - 1)
    _check(lib().magpie_coarse_state(ctx.handle, _dev(idx, torch.int32, n, "idx"), n,
                                     _dev(x, torch.float32, n * h * h * 4, "x"), _dev(scale, torch.float32, n, "scale")))


def magpie_gather_windows(ctx: Context, idx: torch.Tensor, patches: torch.Tensor) -> None:
    n = idx.numel()
    m = ctx.params.m
    _check(lib().magpie_gather_windows(ctx.handle, _dev(idx, torch.int32, n, "idx"), n,
                                       _dev(patches, torch.complex64, n * m * m, "patches")))


def magpie_attach_cnn(ctx: Context, cnn) -> None:
    _check(lib().magpie_attach_cnn(ctx.handle, cnn.handle if cnn is not None else None))
    ctx._cnn = cnn  # alive while attached


def magpie_learned_stats(ctx: Context):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().magpie_learned_stats(ctx.handle, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def magpie_learned_window_values(ctx: Context, count: int):
    acc = (ctypes.c_int32 * count)()
    mg = (ctypes.c_double * count)()
    _check(lib().magpie_learned_window_values(ctx.handle, count, acc, mg))
    return list(acc), list(mg)


def magpie_fp32_fma_rate(iters: int = 4096):
    """(TFLOP/s, ms) of the FP32 FMA rate measurement (see the C header)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().magpie_fp32_fma_rate(int(iters), ctypes.byref(tf), ctypes.byref(ms), _stream()))
    return tf.value, ms.value


def blocks_per_window(m: int) -> int:
    """Thread blocks per window of the window kernel for window side m."""
    return int(lib().magpie_window_blocks(int(m)))


def magpie_stage_times(ctx: Context, idx: torch.Tensor, blocks_per_window: int) -> torch.Tensor:
    """Per-stage %globaltimer stamps of one step (see the C header): uint64
    [count][blocks_per_window][10] on the host."""
    count = idx.numel()
    out = torch.zeros((count, blocks_per_window, 10), dtype=torch.int64)
    _check(lib().magpie_stage_times(ctx.handle, _dev(idx, torch.int32, count, "idx"), count, out.data_ptr(),
                                    out.numel()))
    return out


def magpie_strerror(code: int) -> str:
    return lib().magpie_strerror(code).decode()


def magpie_last_error() -> str:
    return lib().magpie_last_error().decode()


def magpie_version() -> int:
    return lib().magpie_version()
