"""Thin ctypes binding of the C ABI in include/jacpcg.h.

Names mirror the C entry points (jacpcg_create, jacpcg_precode, ...).  This
module only marshals arguments: every step of the precoder runs in the CUDA
kernels of libjacpcg.so.  There is no CPU fallback: if the library is not
built, or the GPU is missing, the calls raise.

``Precoder`` is a convenience wrapper for torch tensors (PyTorch supplies
device memory and streams only).
"""
from __future__ import annotations

import ctypes
import pathlib
import threading

PKG = pathlib.Path(__file__).resolve().parent
LIB_PATH = PKG / "_build" / "libjacpcg.so"

JACPCG_OK, JACPCG_EINVAL, JACPCG_ENOMEM, JACPCG_ECUDA = 0, 1, 2, 3
JACPCG_ENOTCONV, JACPCG_ENOTHPD, JACPCG_ENONFINITE, JACPCG_ETIMEOUT, JACPCG_EBUSY = 4, 5, 6, 7, 8
JACPCG_STANDARD, JACPCG_ALG1, JACPCG_CG, JACPCG_JOR, JACPCG_DIRECT = 0, 1, 2, 3, 4
JACPCG_FP32, JACPCG_TF32X3 = 0, 1
JACPCG_FLAG_PROFILE = 1
JACPCG_FLAG_SIMT_ITERATION = 2
JACPCG_FLAG_REFINE_SELECTIVE = 4
JACPCG_H_C64, JACPCG_H_BF16 = 0, 1
JACPCG_RESID_DOT2, JACPCG_RESID_FP64, JACPCG_RESID_SLICED = 0, 1, 2
RESIDUALS = {"dot2": JACPCG_RESID_DOT2, "fp64": JACPCG_RESID_FP64, "sliced": JACPCG_RESID_SLICED}
VARIANTS = {"standard": JACPCG_STANDARD, "alg1": JACPCG_ALG1, "cg": JACPCG_CG, "jor": JACPCG_JOR,
            "direct": JACPCG_DIRECT}
PRECISIONS = {"fp32": JACPCG_FP32, "tf32x3": JACPCG_TF32X3}

EXPORTS = ("jacpcg_create", "jacpcg_precode", "jacpcg_plan_create", "jacpcg_plan_execute",
           "jacpcg_plan_destroy", "jacpcg_plan_bytes", "jacpcg_arena_free_bytes",
           "jacpcg_profile_read", "jacpcg_launch_count", "jacpcg_destroy", "jacpcg_strerror",
           "jacpcg_version", "jacpcg_precode_noalloc", "jacpcg_precode_plain",
           "jacpcg_server_create", "jacpcg_submit", "jacpcg_poll", "jacpcg_server_replay",
           "jacpcg_server_stats", "jacpcg_server_destroy", "jacpcg_autotune", "jacpcg_set_shape",
           "jacpcg_get_shape", "jacpcg_last_cuda_error", "jacpcg_blocks", "jacpcg_probe_fp32_fma")


class jacpcg_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_instances", ctypes.c_int), ("max_M", ctypes.c_int),
                ("max_K", ctypes.c_int), ("arena_bytes", ctypes.c_size_t),
                ("precision", ctypes.c_int), ("variant", ctypes.c_int), ("flags", ctypes.c_int),
                ("refine_sweeps", ctypes.c_int), ("refine_residual", ctypes.c_int),
                ("refine_tol", ctypes.c_float), ("refine_solve_tol", ctypes.c_float)]


class jacpcg_instance(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("K", ctypes.c_int), ("ldh", ctypes.c_int),
                ("H", ctypes.c_void_p), ("xi", ctypes.c_double), ("power", ctypes.c_double),
                ("W", ctypes.c_void_p), ("ldw", ctypes.c_int), ("X", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("max_iter", ctypes.c_int), ("tol", ctypes.c_float),
                ("h_dtype", ctypes.c_int), ("resid_hist", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int), ("n_rhs", ctypes.c_int),
                ("X0", ctypes.c_void_p), ("omega", ctypes.c_float), ("sinr", ctypes.c_void_p),
                ("noise", ctypes.c_float)]


class jacpcg_block(ctypes.Structure):
    _fields_ = [("row0", ctypes.c_int), ("rows", ctypes.c_int), ("col0", ctypes.c_int),
                ("cols", ctypes.c_int)]


class jacpcg_server_config(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("plain", ctypes.c_int), ("plain_variant", ctypes.c_int),
                ("batch_policy", ctypes.c_int)]


class JacpcgError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {strerror(status)} (status {status})")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: pathlib.Path | str | None = None):
    """Load libjacpcg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = pathlib.Path(path) if path else LIB_PATH
        if not p.exists():
            raise RuntimeError(f"libjacpcg.so not built ({p}); run paper_2305_13925_gb300.build.build()")
        L = ctypes.CDLL(str(p))
        P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.jacpcg_create.argtypes = [ctypes.POINTER(jacpcg_config), ctypes.POINTER(P)]
        L.jacpcg_precode.argtypes = [P, ctypes.POINTER(jacpcg_instance), I, P, P, P, P, P]
        L.jacpcg_plan_create.argtypes = [P, ctypes.POINTER(jacpcg_instance), I, P, P, P, P, I,
                                         ctypes.POINTER(P)]
        L.jacpcg_plan_execute.argtypes = [P, P]
        L.jacpcg_plan_destroy.argtypes = [P]
        L.jacpcg_plan_bytes.argtypes = [P, ctypes.POINTER(jacpcg_instance), I, ctypes.POINTER(S)]
        L.jacpcg_arena_free_bytes.argtypes = [P, ctypes.POINTER(S)]
        L.jacpcg_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(I),
                                          ctypes.POINTER(I)]
        L.jacpcg_launch_count.argtypes = [P]
        L.jacpcg_launch_count.restype = ctypes.c_int64
        L.jacpcg_destroy.argtypes = [P]
        L.jacpcg_precode_noalloc.argtypes = [ctypes.POINTER(jacpcg_instance), I, I, P, P, P, P, P]
        L.jacpcg_precode_plain.argtypes = [ctypes.POINTER(jacpcg_instance), I, I, P, S, P, P, P, P, P]
        U64, D = ctypes.c_uint64, ctypes.c_double
        L.jacpcg_server_create.argtypes = [P, ctypes.POINTER(jacpcg_server_config), ctypes.POINTER(P)]
        L.jacpcg_submit.argtypes = [P, ctypes.POINTER(jacpcg_instance), ctypes.POINTER(U64)]
        L.jacpcg_poll.argtypes = [P, U64, ctypes.POINTER(I), ctypes.POINTER(D), I]
        L.jacpcg_server_replay.argtypes = [P, ctypes.POINTER(jacpcg_instance), I, P, P, I, P, P]
        L.jacpcg_server_stats.argtypes = [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(D)]
        L.jacpcg_server_destroy.argtypes = [P]
        L.jacpcg_autotune.argtypes = [P, ctypes.POINTER(jacpcg_instance), I, P, ctypes.c_char_p, S]
        L.jacpcg_set_shape.argtypes = [P, I, I]
        L.jacpcg_last_cuda_error.argtypes = [P]
        L.jacpcg_last_cuda_error.restype = ctypes.c_char_p
        L.jacpcg_get_shape.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                       ctypes.POINTER(I)]
        L.jacpcg_blocks.argtypes = [ctypes.POINTER(jacpcg_instance), ctypes.POINTER(jacpcg_block), I,
                                    ctypes.POINTER(jacpcg_instance)]
        L.jacpcg_strerror.argtypes = [I]
        L.jacpcg_probe_fp32_fma.argtypes = [I, I, P, P, ctypes.POINTER(ctypes.c_double)]
        L.jacpcg_strerror.restype = ctypes.c_char_p
        L.jacpcg_version.restype = ctypes.c_char_p
        for n in ("jacpcg_create", "jacpcg_precode", "jacpcg_plan_create", "jacpcg_plan_execute",
                  "jacpcg_plan_destroy", "jacpcg_plan_bytes", "jacpcg_arena_free_bytes",
                  "jacpcg_profile_read", "jacpcg_destroy", "jacpcg_precode_noalloc",
                  "jacpcg_precode_plain", "jacpcg_server_create", "jacpcg_submit", "jacpcg_poll",
                  "jacpcg_server_replay", "jacpcg_server_stats", "jacpcg_server_destroy",
                  "jacpcg_autotune", "jacpcg_set_shape", "jacpcg_get_shape", "jacpcg_blocks"):
            getattr(L, n).restype = I
        _lib = L
        return L


def strerror(status: int) -> str:
    try:
        return load().jacpcg_strerror(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def _check(st: int, what: str):
    if st != JACPCG_OK:
        raise JacpcgError(st, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


# --- C entry points, same names ------------------------------------------------

def jacpcg_version() -> str:
    return load().jacpcg_version().decode()


def jacpcg_blocks(full: jacpcg_instance, blocks) -> list:
    """Sub-instances of the per-subarray block precoder (Eq. 7): ``blocks``
    is a sequence of (row0, rows, col0, cols); host only."""
    bl = (jacpcg_block * len(blocks))(*[jacpcg_block(*b) for b in blocks])
    out = (jacpcg_instance * len(blocks))()
    _check(load().jacpcg_blocks(ctypes.byref(full), bl, len(blocks), out), "jacpcg_blocks")
    return list(out)


def jacpcg_strerror(status: int) -> str:
    return strerror(status)


def jacpcg_create(cfg: jacpcg_config) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(load().jacpcg_create(ctypes.byref(cfg), ctypes.byref(ctx)), "jacpcg_create")
    return ctx


def jacpcg_destroy(ctx) -> None:
    _check(load().jacpcg_destroy(ctx), "jacpcg_destroy")


def _array(insts):
    if isinstance(insts, ctypes.Array):
        return insts
    return (jacpcg_instance * len(insts))(*insts)


def jacpcg_precode(ctx, insts, status=None, iters=None, resid=None, beta=None, stream=0) -> None:
    arr = _array(insts)
    _check(load().jacpcg_precode(ctx, arr, len(insts), _ptr(status), _ptr(iters), _ptr(resid),
                                 _ptr(beta), ctypes.c_void_p(stream)), "jacpcg_precode")


def jacpcg_precode_noalloc(insts, variant=JACPCG_STANDARD, status=None, iters=None, resid=None,
                           beta=None, stream=0) -> None:
    """Precode with no allocation at all (static device scratch; see the header)."""
    arr = _array(insts)
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _check(load().jacpcg_precode_noalloc(arr, len(arr), v, _ptr(status), _ptr(iters), _ptr(resid),
                                         _ptr(beta), ctypes.c_void_p(stream)),
           "jacpcg_precode_noalloc")


def plain_workspace_bytes(max_K: int) -> int:
    return 5 * max_K * max_K * 8 + 16 * max_K + 256


def jacpcg_precode_plain(insts, workspace, variant=JACPCG_STANDARD, status=None, iters=None,
                         resid=None, beta=None, stream=0) -> None:
    """The plain FP32 per-instance comparator (see the header)."""
    arr = _array(insts)
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _check(load().jacpcg_precode_plain(arr, len(arr), v, ctypes.c_void_p(workspace.data_ptr()),
                                       workspace.numel() * workspace.element_size(), _ptr(status),
                                       _ptr(iters), _ptr(resid), _ptr(beta), ctypes.c_void_p(stream)),
           "jacpcg_precode_plain")


def jacpcg_plan_create(ctx, insts, status=None, iters=None, resid=None, beta=None,
                       use_graph: bool = False) -> ctypes.c_void_p:
    arr = _array(insts)
    plan = ctypes.c_void_p()
    _check(load().jacpcg_plan_create(ctx, arr, len(insts), _ptr(status), _ptr(iters), _ptr(resid),
                                     _ptr(beta), int(use_graph), ctypes.byref(plan)),
           "jacpcg_plan_create")
    return plan


def jacpcg_plan_execute(plan, stream=0) -> None:
    _check(load().jacpcg_plan_execute(plan, ctypes.c_void_p(stream)), "jacpcg_plan_execute")


def jacpcg_plan_destroy(plan) -> None:
    _check(load().jacpcg_plan_destroy(plan), "jacpcg_plan_destroy")


def jacpcg_plan_bytes(ctx, insts) -> int:
    arr = _array(insts)
    b = ctypes.c_size_t()
    _check(load().jacpcg_plan_bytes(ctx, arr, len(insts), ctypes.byref(b)), "jacpcg_plan_bytes")
    return b.value


def jacpcg_arena_free_bytes(ctx) -> int:
    b = ctypes.c_size_t()
    _check(load().jacpcg_arena_free_bytes(ctx, ctypes.byref(b)), "jacpcg_arena_free_bytes")
    return b.value


def jacpcg_profile_read(ctx):
    """(ms per phase summed over executes, executes covered, launches per execute)."""
    ms = (ctypes.c_float * 4)()
    n = ctypes.c_int()
    per = ctypes.c_int()
    _check(load().jacpcg_profile_read(ctx, ms, ctypes.byref(n), ctypes.byref(per)),
           "jacpcg_profile_read")
    return list(ms), n.value, per.value


def jacpcg_probe_fp32_fma(blocks: int, iters: int, scratch, stream) -> float:
    """Enqueue the FP32 FMA measurement kernel; returns the launch's flops."""
    f = ctypes.c_double()
    _check(load().jacpcg_probe_fp32_fma(int(blocks), int(iters), scratch.data_ptr(), stream,
                                        ctypes.byref(f)), "jacpcg_probe_fp32_fma")
    return f.value


def jacpcg_last_cuda_error(ctx) -> str:
    return load().jacpcg_last_cuda_error(ctx).decode()


def jacpcg_launch_count(ctx) -> int:
    return int(load().jacpcg_launch_count(ctx))


def jacpcg_autotune(ctx, insts, stream=0) -> dict:
    """Tune the iteration launch shape per K class on these instances; returns the table."""
    import json
    arr = _array(insts)
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().jacpcg_autotune(ctx, arr, len(arr), ctypes.c_void_p(stream), buf, len(buf)),
           "jacpcg_autotune")
    return json.loads(buf.value.decode())


def jacpcg_set_shape(ctx, k_class: int, shape: int) -> None:
    _check(load().jacpcg_set_shape(ctx, int(k_class), int(shape)), "jacpcg_set_shape")


def jacpcg_get_shape(ctx, k_class: int):
    """(shape, number of candidates, columns per warp, warps per CTA)."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(load().jacpcg_get_shape(ctx, int(k_class), *[ctypes.byref(x) for x in v]), "jacpcg_get_shape")
    return tuple(x.value for x in v)


def save_tuning(ctx, path) -> None:
    """Persist the context's chosen shapes as JSON {k_class: shape}."""
    import json
    table = {str(k): jacpcg_get_shape(ctx, k)[0] for k in (8, 16, 32, 64, 128, 256)}
    with open(path, "w") as f:
        json.dump(table, f)


def load_tuning(ctx, path) -> None:
    import json
    with open(path) as f:
        for k, v in json.load(f).items():
            jacpcg_set_shape(ctx, int(k), int(v["shape"] if isinstance(v, dict) else v))


JACPCG_BATCH_COST_CLASS, JACPCG_BATCH_FIFO = 0, 1


def jacpcg_server_create(ctx, max_batch=256, max_inflight=4, max_queue=0, plain=False,
                         plain_variant=JACPCG_STANDARD, batch_policy=JACPCG_BATCH_COST_CLASS):
    cfg = jacpcg_server_config(max_batch=max_batch, max_inflight=max_inflight, max_queue=max_queue,
                               plain=int(plain), plain_variant=int(plain_variant),
                               batch_policy=int(batch_policy))
    srv = ctypes.c_void_p()
    _check(load().jacpcg_server_create(ctx, ctypes.byref(cfg), ctypes.byref(srv)), "jacpcg_server_create")
    return srv


def jacpcg_submit(srv, inst: jacpcg_instance) -> int:
    t = ctypes.c_uint64()
    _check(load().jacpcg_submit(srv, ctypes.byref(inst), ctypes.byref(t)), "jacpcg_submit")
    return t.value


def jacpcg_poll(srv, ticket: int, blocking: bool = True):
    """(request status, latency in microseconds); raises on EBUSY / ETIMEOUT."""
    r = ctypes.c_int()
    lat = ctypes.c_double()
    _check(load().jacpcg_poll(srv, ctypes.c_uint64(ticket), ctypes.byref(r), ctypes.byref(lat),
                              int(blocking)), "jacpcg_poll")
    return r.value, lat.value


def jacpcg_server_replay(srv, pool, which, arrival_us):
    """Open-loop replay; returns (latency_us array, status array) as numpy."""
    import numpy as np
    arr = _array(pool)
    which = np.ascontiguousarray(which, dtype=np.int32)
    arrival = np.ascontiguousarray(arrival_us, dtype=np.float64)
    n = len(which)
    lat = np.zeros(n, dtype=np.float64)
    st = np.zeros(n, dtype=np.int32)
    _check(load().jacpcg_server_replay(srv, arr, len(arr), which.ctypes.data_as(ctypes.c_void_p),
                                       arrival.ctypes.data_as(ctypes.c_void_p), n,
                                       lat.ctypes.data_as(ctypes.c_void_p),
                                       st.ctypes.data_as(ctypes.c_void_p)), "jacpcg_server_replay")
    return lat, st


def jacpcg_server_stats(srv):
    a, b, m = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_double()
    _check(load().jacpcg_server_stats(srv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(m)),
           "jacpcg_server_stats")
    return a.value, b.value, m.value


def jacpcg_server_destroy(srv) -> None:
    _check(load().jacpcg_server_destroy(srv), "jacpcg_server_destroy")


# --- torch convenience ---------------------------------------------------------

def instance(H, W, xi: float, max_iter: int, tol: float = 0.0, power: float = 1.0, X=None,
             A=None, resid_hist=None, B=None, X0=None, omega: float = 0.0, sinr=None,
             noise: float = 0.0) -> jacpcg_instance:
    """Describe one channel held in torch tensors of device storage layout:
    H (complex64, or bfloat16 with a trailing (re, im) axis) and W
    (complex64) have shape (K, M) (column k of the matrix is row k of the
    tensor, i.e. column-major storage of the M x K matrix).  B: optional
    (n_rhs, K) complex64 symbol vectors (Eq. 16; W then has shape (n_rhs, M)
    and X (n_rhs, K)); X0: optional initial point, contiguous (n, K); omega:
    the JOR relaxation factor (variant "jor"; 0 means 1); sinr: optional float32
    (K,) device tensor for the per-user SINR of Eq. 9 (noise: sigma^2, 0 means 1)."""
    import torch
    bf16 = H.dtype == torch.bfloat16
    if bf16:
        assert H.shape[-1] == 2 and H.stride(-1) == 1
        K, M, ldh = H.shape[-3], H.shape[-2], H.stride(-3) // 2
    else:
        K, M, ldh = H.shape[-2], H.shape[-1], H.stride(-2)
    if B is not None:
        assert B.dtype == torch.complex64 and B.shape[-1] == K and B.stride(-1) == 1
    if X0 is not None:
        assert X0.dtype == torch.complex64 and X0.shape[-1] == K and X0.is_contiguous()
    return jacpcg_instance(M=M, K=K, ldh=ldh, H=H.data_ptr(), xi=float(xi),
                           power=float(power), W=W.data_ptr(), ldw=W.stride(-2),
                           X=None if X is None else X.data_ptr(),
                           A=None if A is None else A.data_ptr(), max_iter=int(max_iter),
                           tol=float(tol), h_dtype=JACPCG_H_BF16 if bf16 else JACPCG_H_C64,
                           resid_hist=None if resid_hist is None else resid_hist.data_ptr(),
                           B=None if B is None else B.data_ptr(),
                           ldb=0 if B is None else B.stride(-2),
                           n_rhs=0 if B is None else B.shape[-2],
                           X0=None if X0 is None else X0.data_ptr(), omega=float(omega),
                           sinr=None if sinr is None else sinr.data_ptr(), noise=float(noise))


class Precoder:
    """Owns a context; precodes batches of torch tensors on the current stream."""

    def __init__(self, max_instances: int, max_M: int, max_K: int, variant="standard",
                 precision="fp32", device: int = 0, arena_bytes: int = 0, profile: bool = False,
                 refine_sweeps: int = 0, refine_fp64: bool = False, simt_iteration: bool = False,
                 refine_tol: float = 0.0, refine_solve_tol: float = 0.0, refine_selective: bool = False,
                 refine_residual: str | None = None):
        self.cfg = jacpcg_config(device=device, max_instances=max_instances, max_M=max_M,
                                 max_K=max_K, arena_bytes=arena_bytes,
                                 precision=PRECISIONS[precision] if isinstance(precision, str) else precision,
                                 variant=VARIANTS[variant] if isinstance(variant, str) else variant,
                                 flags=(JACPCG_FLAG_PROFILE if profile else 0)
                                 | (JACPCG_FLAG_SIMT_ITERATION if simt_iteration else 0)
                                 | (JACPCG_FLAG_REFINE_SELECTIVE if refine_selective else 0),
                                 refine_sweeps=int(refine_sweeps),
                                 refine_residual=(RESIDUALS[refine_residual] if refine_residual is not None
                                                  else JACPCG_RESID_FP64 if refine_fp64 else JACPCG_RESID_DOT2),
                                 refine_tol=float(refine_tol), refine_solve_tol=float(refine_solve_tol))
        self.ctx = jacpcg_create(self.cfg)

    def close(self):
        if self.ctx:
            jacpcg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def precode(self, insts, status=None, iters=None, resid=None, beta=None, stream=None):
        import torch
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        try:
            jacpcg_precode(self.ctx, insts, status, iters, resid, beta, s)
        except JacpcgError as e:
            if e.status == JACPCG_ECUDA:
                raise JacpcgError(e.status, f"jacpcg_precode ({jacpcg_last_cuda_error(self.ctx)})") from None
            raise

    def plan(self, insts, status=None, iters=None, resid=None, beta=None, use_graph=False):
        return jacpcg_plan_create(self.ctx, insts, status, iters, resid, beta, use_graph)
