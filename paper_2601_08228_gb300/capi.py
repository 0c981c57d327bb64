"""ctypes binding of libwprod.so (include/wprod.h), one wrapper per entry point.

Argument marshalling only: each wrapper checks that its tensors are CUDA
float32 and contiguous, allocates outputs and the workspace with PyTorch's
allocator, passes raw device pointers plus the current CUDA stream to the C
function, and raises WPError on a non-zero status.  Every step of the
computation runs in the library's kernels; there is no fallback path, and a
missing library raises at the first call.
"""

import ctypes
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libwprod.so")
_lib = None

PREC = {"fp32": 0, "bf16": 1, "bf16x3": 2, "fp8": 3}

STATUS_NAMES = {
    0: "WP_OK", 1: "WP_ERR_NULL", 2: "WP_ERR_SHAPE", 3: "WP_ERR_LEVELS", 4: "WP_ERR_RANK",
    5: "WP_ERR_PREC", 6: "WP_ERR_ALIGN", 7: "WP_ERR_WORKSPACE", 8: "WP_ERR_NOT_CONVERGED",
    9: "WP_ERR_TIMEOUT", 10: "WP_ERR_CUDA", 11: "WP_ERR_ALIAS", 12: "WP_ERR_UNSUPPORTED",
}


# Named status codes (include/wprod.h wp_status).
globals().update({name: code for code, name in STATUS_NAMES.items()})


class WPError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {lib().wp_status_string(status).decode()}")


class WPBatchItem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("C_r", ctypes.c_void_p), ("n1", ctypes.c_int32), ("n2", ctypes.c_int32),
                ("n4", ctypes.c_int32), ("p", ctypes.c_int32), ("L", ctypes.c_int32),
                ("r", ctypes.c_int32)]


class WPBatchPlan(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("n_lift_fwd", ctypes.c_int32), ("n_lift_inv", ctypes.c_int32),
                ("gemm_threads", ctypes.c_int32), ("svd_threads", ctypes.c_int32),
                ("svd_vec_floats", ctypes.c_int32), ("n_units", ctypes.c_int64), ("n_units_narrow", ctypes.c_int64), ("n_units_mid", ctypes.c_int64),
                ("lift_fwd_blocks", ctypes.c_int64), ("lift_inv_blocks", ctypes.c_int64),
                ("items_off", ctypes.c_uint64), ("lift_fwd_off", ctypes.c_uint64), ("lift_inv_off", ctypes.c_uint64),
                ("units_off", ctypes.c_uint64), ("svd_group", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class WPLiftOps(ctypes.Structure):
    _fields_ = [("predict_offset", ctypes.c_int32), ("predict_taps", ctypes.c_int32),
                ("predict", ctypes.c_float * 4), ("update_offset", ctypes.c_int32),
                ("update_taps", ctypes.c_int32), ("update", ctypes.c_float * 4)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_SZ = ctypes.c_size_t

_SIGNATURES = {
    "wp_status_string": ([_I], ctypes.c_char_p),
    "wp_version": ([], _I),
    "wp_launch_count": ([], ctypes.c_uint64),
    "wp_get_device_error": ([_P], _I),
    "wp_jacobi_stats": ([ctypes.POINTER(_I64), ctypes.POINTER(_I)], _I),
    "wp_set_jacobi_max_sweeps": ([_I], _I),
    "wp_set_jacobi_precondition": ([_I], _I),
    "wp_set_jacobi_column_split": ([_I], _I),
    "wp_set_jacobi_cluster_size": ([_I], _I),
    "wp_jacobi_cluster_capacity": ([_I, ctypes.POINTER(_I)], _I),
    "wp_selftest_bounded_wait": ([_I, _I64, _P], _I),
    "wp_wprod_tune": ([_P, _P, _P, _I64, _I64, _I64, _I64, _I, _I, _P, _SZ, _P, ctypes.POINTER(_I),
                       ctypes.POINTER(ctypes.c_double)], _I),
    "wp_glift": ([_P, _P, _I64, _I64, _I64, _I, ctypes.POINTER(WPLiftOps), _I, _P], _I),
    "wp_gwprod_workspace": ([_I64, _I64, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "wp_gwprod": ([_P, _P, _P, _I64, _I64, _I64, _I64, _I, ctypes.POINTER(WPLiftOps), _I, _P, _SZ, _P], _I),
    "wp_gwprod_backward_workspace": ([_I64, _I64, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "wp_gwprod_backward": ([_P, _P, _P, _P, _P, _I64, _I64, _I64, _I64, _I, ctypes.POINTER(WPLiftOps), _I, _P,
                            _SZ, _P], _I),
    "wp_plan_set": ([_I64, _I64, _I64, _I64, _I, _I, _I], _I),
    "wp_plan_get": ([_I64, _I64, _I64, _I64, _I, _I, ctypes.POINTER(_I)], _I),
    "wp_plan_clear": ([], _I),
    "wp_plan_save": ([ctypes.c_char_p], _I),
    "wp_plan_load": ([ctypes.c_char_p, ctypes.POINTER(_I)], _I),
    "wp_deblur_pinv_workspace": ([_I64, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "wp_deblur_pinv": ([_P, _P, _P, _P, _I64, _I64, _I64, _I, ctypes.c_double, _I, _I, _P, _SZ, _P], _I),
    "wp_profile_begin": ([], _I),
    "wp_profile_only": ([ctypes.c_char_p], _I),
    "wp_profile_end": ([], _I),
    "wp_profile_count": ([], _I),
    "wp_profile_get": ([_I, ctypes.c_char_p, _I, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double)], _I),
    "wp_lift_forward": ([_P, _P, _I64, _I64, _I64, _I, _P], _I),
    "wp_lift_inverse": ([_P, _P, _I64, _I64, _I64, _I, _P], _I),
    "wp_lift_adjoint": ([_P, _P, _I64, _I64, _I64, _I, _I, _P], _I),
    "wp_facewise_workspace": ([_I64, _I64, _I64, _I64, _I, ctypes.POINTER(_SZ)], _I),
    "wp_facewise": ([_P, _P, _P, _I64, _I64, _I64, _I64, _I, _I, _I, _P, _SZ, _P], _I),
    "wp_wprod_workspace": ([_I64, _I64, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "wp_wprod": ([_P, _P, _P, _I64, _I64, _I64, _I64, _I, _I, _I, _I, _P, _SZ, _P], _I),
    "wp_wprod_noalloc": ([_P, _P, _P, _I64, _I64, _I64, _I64, _I, _I, _I, _I, _P], _I),
    "wp_wprod_host_workspace": ([_I64, _I64, _I64, _I64, _I, _I, _I64, ctypes.POINTER(_SZ)], _I),
    "wp_wprod_host": ([_P, _P, _P, _I64, _I64, _I64, _I64, _I, _I, _I64, _P, _SZ, _P], _I),
    "wp_wprod_backward_workspace": ([_I64, _I64, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "wp_wprod_backward": ([_P, _P, _P, _P, _P, _I64, _I64, _I64, _I64, _I, _I, _P, _SZ, _P], _I),
    "wp_deblur_workspace": ([_I64, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "wp_deblur_step": ([_P, _P, _P, _I64, _I64, _I64, _I, ctypes.c_float, ctypes.c_float, _I, _P, _P, _SZ, _P], _I),
    "wp_wsvd_workspace": ([_I64, _I64, _I64, _I, _I, ctypes.POINTER(_SZ)], _I),
    "wp_wsvd": ([_P, _P, _P, _P, _P, _I64, _I64, _I64, _I, _I, _I, _I, _P, _SZ, _P], _I),
    "wp_wpinv_workspace": ([_I64, _I64, _I64, _I, ctypes.POINTER(_SZ)], _I),
    "wp_wpinv": ([_P, _P, _I64, _I64, _I64, _I, ctypes.c_double, _I, _P, _SZ, _P], _I),
    "wp_batched_workspace": ([ctypes.POINTER(WPBatchItem), _I, ctypes.POINTER(_SZ)], _I),
    "wp_batched_plan": ([ctypes.POINTER(WPBatchItem), _I, _I, _P, _SZ, ctypes.POINTER(WPBatchPlan), _P], _I),
    "wp_batched_run": ([ctypes.POINTER(WPBatchPlan), _P, _P], _I),
}


def lib():
    """Load libwprod.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2601_08228_gb300.build.build()")
        handle = ctypes.CDLL(_LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def _check(status, where):
    if status != 0:
        raise WPError(status, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _req(t, name, ndim=3):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != ndim:
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor with {ndim} dims")
    return t


def _prec(prec):
    if isinstance(prec, int):
        return prec
    return PREC[prec]


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ---- lifting ------------------------------------------------------------------

def wp_lift_forward(x, L, out=None):
    _req(x, "x")
    p, n1, n2 = x.shape
    y = torch.empty_like(x) if out is None else _req(out, "out")
    _check(lib().wp_lift_forward(_ptr(x), _ptr(y), n1, n2, p, L, _stream()), "wp_lift_forward")
    return y


def wp_lift_inverse(y, L, out=None):
    _req(y, "y")
    p, n1, n2 = y.shape
    x = torch.empty_like(y) if out is None else _req(out, "out")
    _check(lib().wp_lift_inverse(_ptr(y), _ptr(x), n1, n2, p, L, _stream()), "wp_lift_inverse")
    return x


def wp_lift_adjoint(g, L, of_inverse=False, out=None):
    _req(g, "g")
    p, n1, n2 = g.shape
    h = torch.empty_like(g) if out is None else _req(out, "out")
    _check(lib().wp_lift_adjoint(_ptr(g), _ptr(h), n1, n2, p, L, int(bool(of_inverse)), _stream()),
           "wp_lift_adjoint")
    return h


# ---- face-product and w-product --------------------------------------------------

def _prod_dims(A, B, transA, transB):
    p = A.shape[0]
    n1, n2 = (A.shape[2], A.shape[1]) if transA else (A.shape[1], A.shape[2])
    n2b, n4 = (B.shape[2], B.shape[1]) if transB else (B.shape[1], B.shape[2])
    if B.shape[0] != p or n2b != n2:
        raise ValueError(f"shape mismatch: op(A) {n1}x{n2}, op(B) {n2b}x{n4}")
    return p, n1, n2, n4


def wp_facewise(Ah, Bh, transA=False, transB=False, prec="fp32", out=None):
    _req(Ah, "Ah"), _req(Bh, "Bh")
    p, n1, n2, n4 = _prod_dims(Ah, Bh, transA, transB)
    pr = _prec(prec)
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_facewise_workspace(n1, n2, n4, p, pr, ctypes.byref(nbytes)), "wp_facewise_workspace")
    ws = _workspace(nbytes.value, Ah.device)
    C = torch.empty((p, n1, n4), dtype=torch.float32, device=Ah.device) if out is None else _req(out, "out")
    _check(lib().wp_facewise(_ptr(Ah), _ptr(Bh), _ptr(C), n1, n2, n4, p, int(transA), int(transB), pr,
                             _ptr(ws), ws.numel(), _stream()), "wp_facewise")
    return C


def wp_wprod_workspace(n1, n2, n4, p, L, prec="fp32"):
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_wprod_workspace(n1, n2, n4, p, L, _prec(prec), ctypes.byref(nbytes)), "wp_wprod_workspace")
    return nbytes.value


def wp_wprod(A, B, L, transA=False, transB=False, prec="fp32", out=None, ws=None):
    """C = op(A) *w op(B) (Def. 2.1) on the GPU."""
    _req(A, "A"), _req(B, "B")
    p, n1, n2, n4 = _prod_dims(A, B, transA, transB)
    pr = _prec(prec)
    need = wp_wprod_workspace(n1, n2, n4, p, L, pr)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, A.device)
    C = torch.empty((p, n1, n4), dtype=torch.float32, device=A.device) if out is None else _req(out, "out")
    _check(lib().wp_wprod(_ptr(A), _ptr(B), _ptr(C), n1, n2, n4, p, L, int(transA), int(transB), pr,
                          _ptr(ws), ws.numel(), _stream()), "wp_wprod")
    return C


GLIFT_OPS = {"forward": 0, "inverse": 1, "adjoint": 2, "inverse_adjoint": 3}


def lift_ops(levels):
    """ctypes array of wp_lift_ops from [((p_off, p_taps), (u_off, u_taps)), ...]."""
    arr = (WPLiftOps * max(1, len(levels)))()
    for j, ((po, pt), (uo, ut)) in enumerate(levels):
        if len(pt) > 4 or len(ut) > 4:
            raise ValueError("at most 4 taps per operator")
        arr[j].predict_offset, arr[j].predict_taps = int(po), len(pt)
        arr[j].update_offset, arr[j].update_taps = int(uo), len(ut)
        for t, c in enumerate(pt):
            arr[j].predict[t] = float(c)
        for t, c in enumerate(ut):
            arr[j].update[t] = float(c)
    return arr


def wp_glift(x, L, levels, op="forward", out=None):
    """General-operator lifting of every mode-3 tube (see include/wprod.h)."""
    _req(x, "x")
    p, n1, n2 = x.shape
    y = torch.empty_like(x) if out is None else _req(out, "out")
    _check(lib().wp_glift(_ptr(x), _ptr(y), n1, n2, p, L, lift_ops(levels), GLIFT_OPS[op], _stream()), "wp_glift")
    return y


def wp_gwprod(A, B, L, levels, prec="fp32", out=None):
    _req(A, "A"), _req(B, "B")
    p, n1, n2, n4 = _prod_dims(A, B, False, False)
    pr = _prec(prec)
    n = _SZ(0)
    _check(lib().wp_gwprod_workspace(n1, n2, n4, p, L, pr, ctypes.byref(n)), "wp_gwprod_workspace")
    ws = _workspace(n.value, A.device)
    C = torch.empty((p, n1, n4), dtype=torch.float32, device=A.device) if out is None else _req(out, "out")
    _check(lib().wp_gwprod(_ptr(A), _ptr(B), _ptr(C), n1, n2, n4, p, L, lift_ops(levels), pr, _ptr(ws), ws.numel(),
                           _stream()), "wp_gwprod")
    return C


def wp_gwprod_backward(A, B, G, L, levels, prec="fp32", need_dA=True, need_dB=True):
    _req(A, "A"), _req(B, "B"), _req(G, "G")
    p, n1, n2, n4 = _prod_dims(A, B, False, False)
    pr = _prec(prec)
    n = _SZ(0)
    _check(lib().wp_gwprod_backward_workspace(n1, n2, n4, p, L, pr, ctypes.byref(n)), "wp_gwprod_backward_workspace")
    ws = _workspace(n.value, A.device)
    dA = torch.empty_like(A) if need_dA else None
    dB = torch.empty_like(B) if need_dB else None
    _check(lib().wp_gwprod_backward(_ptr(A), _ptr(B), _ptr(G), _ptr(dA) if dA is not None else None,
                                    _ptr(dB) if dB is not None else None, n1, n2, n4, p, L, lift_ops(levels), pr,
                                    _ptr(ws), ws.numel(), _stream()), "wp_gwprod_backward")
    return dA, dB


WPROD_VARIANTS = {"fused": 1, "persistent": 2, "lifted": 3}


def wp_wprod_tune(A, B, L, prec="bf16x3", out=None, ws=None):
    """Time the tensor-core w-product kernels on these tensors and cache the
    fastest; returns (variant, best_ms): 1 fused inverse-lift epilogue, 2
    persistent GEMM + inverse lift, 3 lift in the producer warps + inverse-lift
    epilogue; (0, 0.0) when there is only one kernel."""
    _req(A, "A"), _req(B, "B")
    p, n1, n2, n4 = _prod_dims(A, B, False, False)
    pr = _prec(prec)
    need = wp_wprod_workspace(n1, n2, n4, p, L, pr)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, A.device)
    C = torch.empty((p, n1, n4), dtype=torch.float32, device=A.device) if out is None else _req(out, "out")
    cg, ms = _I(0), ctypes.c_double(0.0)
    _check(lib().wp_wprod_tune(_ptr(A), _ptr(B), _ptr(C), n1, n2, n4, p, L, pr, _ptr(ws), ws.numel(), _stream(),
                               ctypes.byref(cg), ctypes.byref(ms)), "wp_wprod_tune")
    return int(cg.value), float(ms.value)


def wp_plan_set(n1, n2, n4, p, L, prec, variant):
    v = WPROD_VARIANTS.get(variant, variant) if isinstance(variant, str) else variant
    _check(lib().wp_plan_set(n1, n2, n4, p, L, _prec(prec), int(v)), "wp_plan_set")


def wp_plan_get(n1, n2, n4, p, L, prec):
    v = _I(0)
    _check(lib().wp_plan_get(n1, n2, n4, p, L, _prec(prec), ctypes.byref(v)), "wp_plan_get")
    return int(v.value)


def wp_plan_clear():
    _check(lib().wp_plan_clear(), "wp_plan_clear")


def wp_plan_save(path):
    _check(lib().wp_plan_save(os.fsencode(path)), "wp_plan_save")


def wp_plan_load(path):
    n = _I(0)
    _check(lib().wp_plan_load(os.fsencode(path), ctypes.byref(n)), "wp_plan_load")
    return int(n.value)


def _req_host(t, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.dim() != 3:
        raise ValueError(f"{name} must be a contiguous host float32 tensor with 3 dims")
    return t


def wp_wprod_host_workspace(n1, n2, n4, p, L, prec, chunk_slices=0):
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_wprod_host_workspace(n1, n2, n4, p, L, _prec(prec), chunk_slices, ctypes.byref(nbytes)),
           "wp_wprod_host_workspace")
    return nbytes.value


def wp_wprod_host(A, B, L, prec="fp32", out=None, ws=None, chunk_slices=0):
    """C = A *w B for HOST tensors (pin them for overlap): chunks of whole
    tube groups are copied in, multiplied and copied back on overlapping
    streams.  Ordered on the current CUDA stream: C is complete once that
    stream has been synchronised."""
    _req_host(A, "A"), _req_host(B, "B")
    p, n1, n2 = A.shape
    if B.shape[0] != p or B.shape[1] != n2:
        raise ValueError("shape mismatch in wp_wprod_host")
    n4 = B.shape[2]
    pr = _prec(prec)
    need = wp_wprod_host_workspace(n1, n2, n4, p, L, pr, chunk_slices)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, torch.device("cuda", torch.cuda.current_device()))
    C = torch.empty((p, n1, n4), dtype=torch.float32, pin_memory=A.is_pinned()) if out is None else _req_host(out, "out")
    _check(lib().wp_wprod_host(_ptr(A), _ptr(B), _ptr(C), n1, n2, n4, p, L, pr, chunk_slices, _ptr(ws), ws.numel(),
                               _stream()), "wp_wprod_host")
    return C


def wp_wprod_noalloc(A, B, L, transA=False, transB=False, prec="fp32", out=None):
    """C = op(A) *w op(B) using the library's own fixed scratch array instead
    of a workspace (for callers that cannot allocate device memory)."""
    _req(A, "A"), _req(B, "B")
    p, n1, n2, n4 = _prod_dims(A, B, transA, transB)
    C = torch.empty((p, n1, n4), dtype=torch.float32, device=A.device) if out is None else _req(out, "out")
    _check(lib().wp_wprod_noalloc(_ptr(A), _ptr(B), _ptr(C), n1, n2, n4, p, L, int(transA), int(transB),
                                  _prec(prec), _stream()), "wp_wprod_noalloc")
    return C


def wp_wprod_backward(A, B, G, L, need_dA=True, need_dB=True, prec="fp32", ws=None):
    """(dA, dB) of <G, A *w B> by the adjoint route."""
    _req(A, "A"), _req(B, "B"), _req(G, "G")
    p, n1, n2 = A.shape
    n4 = B.shape[2]
    if B.shape[:2] != (p, n2) or tuple(G.shape) != (p, n1, n4):
        raise ValueError("shape mismatch in wp_wprod_backward")
    pr = _prec(prec)
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_wprod_backward_workspace(n1, n2, n4, p, L, pr, ctypes.byref(nbytes)),
           "wp_wprod_backward_workspace")
    if ws is None or ws.numel() < nbytes.value:
        ws = _workspace(nbytes.value, A.device)
    dA = torch.empty_like(A) if need_dA else None
    dB = torch.empty_like(B) if need_dB else None
    _check(lib().wp_wprod_backward(_ptr(A), _ptr(B), _ptr(G), _ptr(dA), _ptr(dB), n1, n2, n4, p, L, pr,
                                   _ptr(ws), ws.numel(), _stream()), "wp_wprod_backward")
    return dA, dB


# ---- deblurring ------------------------------------------------------------------

def wp_deblur_workspace(n1, n2, p, L, prec="fp32"):
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_deblur_workspace(n1, n2, p, L, _prec(prec), ctypes.byref(nbytes)), "wp_deblur_workspace")
    return nbytes.value


def wp_deblur_pinv_workspace(n1, n2, p, L, prec="fp32"):
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_deblur_pinv_workspace(n1, n2, p, L, _prec(prec), ctypes.byref(nbytes)),
           "wp_deblur_pinv_workspace")
    return nbytes.value


def wp_deblur_pinv(AV, AH, B, L, rtol=-1.0, refine_iters=2, prec="fp32", out=None, ws=None):
    """X = A_V^+ *w B *w (A_H^T)^+ (two-sided deblurring, Sec. IV-C) on the GPU."""
    _req(AV, "AV"), _req(AH, "AH"), _req(B, "B")
    p, n1, n2 = B.shape
    need = wp_deblur_pinv_workspace(n1, n2, p, L, prec)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, B.device)
    X = torch.empty_like(B) if out is None else _req(out, "out")
    _check(lib().wp_deblur_pinv(_ptr(AV), _ptr(AH), _ptr(B), _ptr(X), n1, n2, p, L, float(rtol), int(refine_iters),
                                _prec(prec), _ptr(ws), ws.numel(), _stream()), "wp_deblur_pinv")
    return X


def wp_deblur_step(K, Y, X, L, lam, eta, prec="fp32", loss=None, ws=None):
    """In-place gradient step X <- X - eta grad f(X), f = |K *w X - Y|^2 + lam |X|^2.
    `loss`: optional CUDA float64 tensor of one element; f(X) is added to it."""
    _req(K, "K"), _req(Y, "Y"), _req(X, "X")
    p, n1, n2 = X.shape
    if tuple(K.shape) != (p, n1, n1) or tuple(Y.shape) != (p, n1, n2):
        raise ValueError("shape mismatch in wp_deblur_step")
    if loss is not None and (not loss.is_cuda or loss.dtype != torch.float64 or loss.numel() != 1):
        raise ValueError("loss must be a one-element CUDA float64 tensor")
    need = wp_deblur_workspace(n1, n2, p, L, prec)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, X.device)
    _check(lib().wp_deblur_step(_ptr(K), _ptr(Y), _ptr(X), n1, n2, p, L, float(lam), float(eta), _prec(prec),
                                _ptr(loss), _ptr(ws), ws.numel(), _stream()), "wp_deblur_step")
    return X


# ---- w-svd / sp-w-svd ------------------------------------------------------------

def wp_wsvd(A, L, r, sparse=False, factors=False, factors_in_wavelet_domain=True, ws=None):
    """Rank-r w-svd (sparse=False) or sp-w-svd (sparse=True) of A (p, n1, n2).

    Returns C_r, or (C_r, U, S, V) with factors=True."""
    _req(A, "A")
    p, n1, n2 = A.shape
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_wsvd_workspace(n1, n2, p, L, r, ctypes.byref(nbytes)), "wp_wsvd_workspace")
    if ws is None or ws.numel() < nbytes.value:
        ws = _workspace(nbytes.value, A.device)
    C = torch.empty_like(A)
    U = S = V = None
    if factors:
        U = torch.empty((p, n1, r), dtype=torch.float32, device=A.device)
        S = torch.empty((p, r), dtype=torch.float32, device=A.device)
        V = torch.empty((p, n2, r), dtype=torch.float32, device=A.device)
    _check(lib().wp_wsvd(_ptr(A), _ptr(C), _ptr(U), _ptr(S), _ptr(V), n1, n2, p, L, r, int(bool(sparse)),
                         int(bool(factors_in_wavelet_domain)), _ptr(ws), ws.numel(), _stream()), "wp_wsvd")
    return (C, U, S, V) if factors else C


# ---- Moore-Penrose inverse ----------------------------------------------------------

def wp_wpinv_workspace(m, n, p, L):
    """Workspace bytes of wp_wpinv for A (p, m, n)."""
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_wpinv_workspace(m, n, p, L, ctypes.byref(nbytes)), "wp_wpinv_workspace")
    return nbytes.value


def wp_wpinv(A, L, rtol=-1.0, refine_iters=0, ws=None):
    _req(A, "A")
    p, m, n = A.shape
    nbytes = ctypes.c_size_t(0)
    _check(lib().wp_wpinv_workspace(m, n, p, L, ctypes.byref(nbytes)), "wp_wpinv_workspace")
    if ws is None or ws.numel() < nbytes.value:
        ws = _workspace(nbytes.value, A.device)
    X = torch.empty((p, n, m), dtype=torch.float32, device=A.device)
    _check(lib().wp_wpinv(_ptr(A), _ptr(X), m, n, p, L, float(rtol), int(refine_iters), _ptr(ws), ws.numel(),
                          _stream()), "wp_wpinv")
    return X


# ---- batched launch -----------------------------------------------------------------

class BatchedLaunch:
    """w-product + rank-r w-svd over many uneven items (wp_batched_plan /
    wp_batched_run).  `items`: list of dicts with CUDA tensors A, B, C, C_r
    and ints L, r.  run() only launches, so it may be captured in a CUDA graph."""

    def __init__(self, items, tune=False):
        arr = (WPBatchItem * len(items))()
        for i, it in enumerate(items):
            A, B, C, Cr = it["A"], it["B"], it["C"], it["C_r"]
            for t, nm in ((A, "A"), (B, "B"), (C, "C"), (Cr, "C_r")):
                _req(t, nm)
            p, n1, n2 = A.shape
            arr[i] = WPBatchItem(A.data_ptr(), B.data_ptr(), C.data_ptr(), Cr.data_ptr(), n1, n2, B.shape[2], p,
                                 int(it["L"]), int(it["r"]))
        self._arr = arr
        self._keep = items
        nbytes = ctypes.c_size_t(0)
        _check(lib().wp_batched_workspace(arr, len(items), ctypes.byref(nbytes)), "wp_batched_workspace")
        self.ws = _workspace(nbytes.value, items[0]["A"].device)
        self.plan = WPBatchPlan()
        _check(lib().wp_batched_plan(arr, len(items), int(bool(tune)), _ptr(self.ws), self.ws.numel(),
                                     ctypes.byref(self.plan), _stream()), "wp_batched_plan")

    def run(self):
        _check(lib().wp_batched_run(ctypes.byref(self.plan), _ptr(self.ws), _stream()), "wp_batched_run")


def wp_profile_only(name=None):
    """Limit per-kernel timing to launches named `name` (None: all launches)."""
    _check(lib().wp_profile_only(name.encode() if name else None), "wp_profile_only")


def wp_profile_begin():
    _check(lib().wp_profile_begin(), "wp_profile_begin")


def wp_profile_end():
    """Stop per-kernel timing; return {kernel name: (launches, total ms)}."""
    _check(lib().wp_profile_end(), "wp_profile_end")
    out = {}
    buf = ctypes.create_string_buffer(128)
    n, ms = _I64(0), ctypes.c_double(0.0)
    for i in range(lib().wp_profile_count()):
        _check(lib().wp_profile_get(i, buf, 128, ctypes.byref(n), ctypes.byref(ms)), "wp_profile_get")
        out[buf.value.decode()] = (int(n.value), float(ms.value))
    return out


def wp_jacobi_stats():
    """(total slice-sweeps, max sweeps of one slice) since the last call."""
    t, m = _I64(0), _I(0)
    _check(lib().wp_jacobi_stats(ctypes.byref(t), ctypes.byref(m)), "wp_jacobi_stats")
    return int(t.value), int(m.value)


def wp_set_jacobi_max_sweeps(n):
    """Set the Jacobi sweep limit of later launches (default 40)."""
    _check(lib().wp_set_jacobi_max_sweeps(int(n)), "wp_set_jacobi_max_sweeps")


def wp_set_jacobi_precondition(on):
    """QR preconditioning of the Jacobi SVD on (True, default) or off."""
    _check(lib().wp_set_jacobi_precondition(int(bool(on))), "wp_set_jacobi_precondition")


def wp_set_jacobi_column_split(on):
    """Column-split Jacobi kernel for the shapes it takes on (True, default) or
    off (row-split block kernel)."""
    _check(lib().wp_set_jacobi_column_split(int(bool(on))), "wp_set_jacobi_column_split")


def wp_set_jacobi_cluster_size(cl):
    """Cluster size of the column-split Jacobi kernel: 0 automatic, 2, 3 or 4."""
    _check(lib().wp_set_jacobi_cluster_size(int(cl)), "wp_set_jacobi_cluster_size")


def wp_jacobi_cluster_capacity(cl):
    """Resident clusters of `cl` CTAs of the column-split Jacobi kernel."""
    n = _I(0)
    _check(lib().wp_jacobi_cluster_capacity(int(cl), ctypes.byref(n)), "wp_jacobi_cluster_capacity")
    return int(n.value)


def wp_selftest_bounded_wait(which, limit_ns):
    """Launch a wait that must expire after limit_ns (see include/wprod.h)."""
    _check(lib().wp_selftest_bounded_wait(int(which), int(limit_ns), _stream()), "wp_selftest_bounded_wait")


def wp_launch_count():
    return int(lib().wp_launch_count())


def wp_get_device_error():
    return lib().wp_get_device_error(_stream())
