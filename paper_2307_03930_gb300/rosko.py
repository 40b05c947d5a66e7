"""Thin ctypes binding of the C-ABI in include/rosko.h.

Names match the C entry points; every function only marshals arguments
(tensor -> device pointer, sizes, dtype codes, stream) and checks the returned
status.  All compute happens in the CUDA library; if that library is missing
this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libroskogb300.so")

F32, BF16, I8, F64, I32 = 0, 1, 2, 3, 4
SCHED_ANALYTIC, SCHED_AUTOTUNE, SCHED_LEARNED, SCHED_FORCED = 0, 1, 2, 3
ORDER_COLUMN, ORDER_ROWSLOT = 1, 2
STATUS_NAMES = ["ROSKO_OK", "ROSKO_ERR_INVALID_ARG", "ROSKO_ERR_UNSUPPORTED", "ROSKO_ERR_OOM",
                "ROSKO_ERR_CUDA", "ROSKO_ERR_TIMEOUT", "ROSKO_ERR_BAD_HANDLE", "ROSKO_ERR_DEVICE"]
TORCH_TO_CODE = {torch.float32: F32, torch.bfloat16: BF16, torch.int8: I8,
                 torch.float64: F64, torch.int32: I32}
CODE_TO_TORCH = {v: k for k, v in TORCH_TO_CODE.items()}
ELEM_SIZE = {F32: 4, BF16: 2, I8: 1, F64: 8, I32: 4}


class RoskoError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else f"status {status}"
        super().__init__(f"{what} failed: {name}")


class rosko_tile(ctypes.Structure):
    _fields_ = [("m_r", ctypes.c_int32), ("n_r", ctypes.c_int32), ("k_c", ctypes.c_int32),
                ("m_c", ctypes.c_int32), ("split_k", ctypes.c_int32),
                ("dense_split_pm", ctypes.c_int32), ("dense_n_r", ctypes.c_int32),
                ("dense_split_k", ctypes.c_int32), ("order", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("dense_m_c", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rosko_plan(ctypes.Structure):
    _fields_ = [("dense_tiles", ctypes.c_int64), ("sparse_panels", ctypes.c_int64),
                ("order", ctypes.c_int32), ("zero_fill", ctypes.c_int32), ("tile", rosko_tile)]

    def as_dict(self):
        return {"dense_tiles": self.dense_tiles, "sparse_panels": self.sparse_panels,
                "order": self.order, "zero_fill": self.zero_fill, "tile": self.tile.as_dict()}


def make_tile(**kw) -> rosko_tile:
    t = rosko_tile()
    for f, _ in rosko_tile._fields_:
        setattr(t, f, int(kw.get(f, 0)))
    return t


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run `python -m paper_2307_03930_gb300.build`)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    P_tile = ctypes.POINTER(rosko_tile)
    sig = {
        "rosko_status_string": (ctypes.c_char_p, [ci]),
        "rosko_pack": (ci, [vp, ci, i64, i64, i64, ci, vp, P_tile, vp, ctypes.POINTER(vp)]),
        "rosko_spmm": (ci, [vp, vp, ci, i64, i64, vp, vp, ci, i64, ci, P_tile, vp]),
        "rosko_pack_transposed": (ci, [vp, ci, i64, i64, i64, ci, vp, P_tile, vp,
                                       ctypes.POINTER(vp)]),
        "rosko_spmm_plan": (ci, [vp, vp, ci, i64, i64, vp, vp, ci, i64, ci, P_tile,
                                 ctypes.POINTER(rosko_plan), vp]),
        "rosko_free": (None, [vp]),
        "rosko_unpack": (ci, [vp, vp, i64, vp]),
        "rosko_packed_info": (ci, [vp] + [ctypes.POINTER(i64)] * 4 +
                              [ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]),
        "rosko_packed_export": (ci, [vp, vp, vp, vp, vp, vp]),
        "rosko_schedule_analytic": (ci, [i64, i64, i64, i64, i32, ci, P_tile]),
        "rosko_device_status": (ci, [ctypes.POINTER(i32), ci]),
        "rosko_kernel_launches": (i64, []),
        "rosko_set_wait_limit": (ci, [i64]),
        "rosko_pack_save": (ci, [vp, vp, i64, ctypes.POINTER(i64)]),
        "rosko_packed_shape": (ci, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                    ctypes.POINTER(i64)]),
        "rosko_pack_load": (ci, [vp, i64, vp, ctypes.POINTER(vp)]),
        "rosko_probe_bounded_wait": (ci, [vp]),
        "rosko_num_candidates": (i32, []),
        "rosko_candidate": (ci, [vp, i64, i32, P_tile]),
        "rosko_autotune": (ci, [vp, vp, ci, i64, i64, vp, vp, ci, i64, i32, P_tile,
                                ctypes.POINTER(ctypes.c_float), vp]),
        "rosko_time_tile": (ci, [vp, vp, ci, i64, i64, vp, vp, ci, i64, P_tile, i32,
                                 ctypes.POINTER(ctypes.c_float), vp]),
        "rosko_features": (ci, [vp, i64, ctypes.POINTER(ctypes.c_double), vp]),
        "rosko_candidate_index": (i32, [P_tile, ci]),
        "rosko_features_static": (ci, [vp, i64, vp, vp]),
        "rosko_mlp_param_count": (i64, [i32, i32]),
        "rosko_mlp_workspace_floats": (i64, [i64, i32]),
        "rosko_mlp_forward": (ci, [vp, vp, i64, i32, i32, vp, vp, vp]),
        "rosko_mlp_loss_grad": (ci, [vp, vp, vp, i64, i32, i32, vp, vp, vp, vp]),
        "rosko_mlp_adam": (ci, [vp, vp, vp, vp, i64, i32, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, ctypes.c_float, vp]),
        "rosko_selector_set": (ci, [ctypes.POINTER(ctypes.c_float), i64] +
                               [ctypes.POINTER(ctypes.c_double)] * 4),
        "rosko_spmm_batched": (ci, [i32, vp, vp, vp, vp, vp, vp, ci, ci, ci, P_tile, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, what: str):
    if status != 0:
        raise RoskoError(status, what)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected (the library works on device pointers)")
    return ctypes.c_void_p(t.data_ptr())


def _ld(t: torch.Tensor) -> int:
    """Leading dimension of a row-major 2-D tensor (the stride of a size-1
    dimension carries no layout and is ignored)."""
    if t.dim() != 2 or (t.size(1) > 1 and t.stride(1) != 1):
        raise ValueError("row-major 2-D tensor with unit column stride expected")
    if t.size(0) <= 1:
        return max(int(t.stride(0)), int(t.size(1)), 1)
    return int(t.stride(0))


class PackedA:
    """Owner of a rosko_packed_t handle; frees it when collected."""

    def __init__(self, handle: int, M: int, K: int):
        self.handle = ctypes.c_void_p(handle)
        self.M, self.K = M, K

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.rosko_free(h)
            self.handle = None

    def free(self):
        rosko_free(self)

    def info(self) -> dict:
        return rosko_packed_info(self)


def rosko_status_string(status: int) -> str:
    return lib().rosko_status_string(int(status)).decode()


def rosko_pack(A: torch.Tensor, packed_dtype: int, m_r: int = 0,
               row_scale: Optional[torch.Tensor] = None, stream=None,
               dense_min_pm: int = 0) -> PackedA:
    """Alg. 1 on the device: pack the dense row-major A (F32, BF16 or I8)."""
    L = lib()
    M, K = A.shape
    lda = _ld(A) if A.numel() else max(K, 1)
    tile = make_tile(m_r=m_r, dense_split_pm=dense_min_pm)
    out = ctypes.c_void_p()
    st = L.rosko_pack(_ptr(A) if A.numel() else None, TORCH_TO_CODE[A.dtype], M, K, lda,
                      int(packed_dtype), _ptr(row_scale), ctypes.byref(tile),
                      ctypes.c_void_p(_stream(stream)), ctypes.byref(out))
    _check(st, "rosko_pack")
    return PackedA(out.value, M, K)


def rosko_pack_transposed(A: torch.Tensor, packed_dtype: int, m_r: int = 0,
                          row_scale: Optional[torch.Tensor] = None, stream=None,
                          dense_min_pm: int = 0) -> PackedA:
    """Alg. 1 on the device applied to the transpose of the dense row-major A
    (the handle is K x M)."""
    L = lib()
    M, K = A.shape
    lda = _ld(A) if A.numel() else max(K, 1)
    tile = make_tile(m_r=m_r, dense_split_pm=dense_min_pm)
    out = ctypes.c_void_p()
    st = L.rosko_pack_transposed(_ptr(A) if A.numel() else None, TORCH_TO_CODE[A.dtype], M, K,
                                 lda, int(packed_dtype), _ptr(row_scale), ctypes.byref(tile),
                                 ctypes.c_void_p(_stream(stream)), ctypes.byref(out))
    _check(st, "rosko_pack_transposed")
    return PackedA(out.value, K, M)


def rosko_spmm(A: PackedA, B: torch.Tensor, C: torch.Tensor,
               col_scale: Optional[torch.Tensor] = None, accumulate: bool = False,
               tile: Optional[rosko_tile] = None, stream=None) -> torch.Tensor:
    """C = A.B (or C += A.B); returns C."""
    L = lib()
    K, N = B.shape
    st = L.rosko_spmm(A.handle, _ptr(B) if B.numel() else None, TORCH_TO_CODE[B.dtype], N,
                      _ld(B) if B.numel() else max(N, 1), _ptr(col_scale),
                      _ptr(C) if C.numel() else None, TORCH_TO_CODE[C.dtype],
                      _ld(C) if C.numel() else max(N, 1), int(bool(accumulate)),
                      ctypes.byref(tile) if tile is not None else None,
                      ctypes.c_void_p(_stream(stream)))
    _check(st, "rosko_spmm")
    return C


def rosko_spmm_plan(A: PackedA, B: torch.Tensor, C: torch.Tensor,
                    col_scale: Optional[torch.Tensor] = None, accumulate: bool = False,
                    tile: Optional[rosko_tile] = None, stream=None) -> dict:
    """What rosko_spmm would run for these arguments (nothing is launched
    for the product itself): dense tiles, sparse panels, traversal, tile."""
    L = lib()
    K, N = B.shape
    out = rosko_plan()
    st = L.rosko_spmm_plan(A.handle, _ptr(B) if B.numel() else None, TORCH_TO_CODE[B.dtype], N,
                           _ld(B) if B.numel() else max(N, 1), _ptr(col_scale),
                           _ptr(C) if C.numel() else None, TORCH_TO_CODE[C.dtype],
                           _ld(C) if C.numel() else max(N, 1), int(bool(accumulate)),
                           ctypes.byref(tile) if tile is not None else None,
                           ctypes.byref(out), ctypes.c_void_p(_stream(stream)))
    _check(st, "rosko_spmm_plan")
    return out.as_dict()


def rosko_free(A: PackedA) -> None:
    if A.handle is not None and A.handle.value:
        lib().rosko_free(A.handle)
    A.handle = None


def rosko_unpack(A: PackedA, out: torch.Tensor, stream=None) -> torch.Tensor:
    st = lib().rosko_unpack(A.handle, _ptr(out), _ld(out), ctypes.c_void_p(_stream(stream)))
    _check(st, "rosko_unpack")
    return out


def rosko_packed_info(A: PackedA) -> dict:
    i64 = [ctypes.c_int64() for _ in range(5)]
    m_r, dt = ctypes.c_int32(), ctypes.c_int32()
    st = lib().rosko_packed_info(A.handle, ctypes.byref(i64[0]), ctypes.byref(i64[1]),
                                 ctypes.byref(i64[2]), ctypes.byref(i64[3]),
                                 ctypes.byref(m_r), ctypes.byref(dt), ctypes.byref(i64[4]))
    _check(st, "rosko_packed_info")
    M, K, dev_bytes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().rosko_packed_shape(A.handle, ctypes.byref(M), ctypes.byref(K),
                                    ctypes.byref(dev_bytes)), "rosko_packed_shape")
    return {"nnz": i64[0].value, "bytes": i64[1].value, "touched_k": i64[2].value,
            "n_panels": i64[3].value, "m_r": m_r.value, "dtype": dt.value,
            "n_cols": i64[4].value, "M": M.value, "K": K.value,
            "device_bytes": dev_bytes.value}


def rosko_packed_export(A: PackedA) -> dict:
    """Canonical Alg. 1 arrays (numpy), concatenated over panels."""
    import numpy as np
    info = rosko_packed_info(A)
    np_dt = {F32: np.float32, BF16: np.uint16, I8: np.int8, F64: np.float64}[info["dtype"]]
    A_p = np.zeros(info["nnz"], dtype=np_dt)
    loc_m = np.zeros(info["nnz"], dtype=np.uint8)
    col_ind = np.zeros(info["n_cols"], dtype=np.int32)
    nnz = np.zeros(info["n_cols"], dtype=np.int32)
    panel_cols = np.zeros(info["n_panels"] + 1, dtype=np.int64)
    c = lambda a: ctypes.c_void_p(a.ctypes.data) if a.size else None
    st = lib().rosko_packed_export(A.handle, c(A_p), c(loc_m), c(col_ind), c(nnz), c(panel_cols))
    _check(st, "rosko_packed_export")
    return {"A_p": A_p, "loc_m": loc_m, "col_ind": col_ind, "nnz": nnz, "panel_cols": panel_cols}


def rosko_schedule_analytic(M: int, K: int, N: int, nnz: int, m_r: int = 0,
                            packed_dtype: int = F32) -> dict:
    t = rosko_tile()
    _check(lib().rosko_schedule_analytic(M, K, N, nnz, m_r, packed_dtype, ctypes.byref(t)),
           "rosko_schedule_analytic")
    return t.as_dict()


def rosko_candidate_index(tile, packed_dtype: int) -> int:
    """Candidate index of a tile (rosko_tile or its dict), -1 if none."""
    if isinstance(tile, dict):
        tile = make_tile(**tile)
    return int(lib().rosko_candidate_index(ctypes.byref(tile), int(packed_dtype)))


def analytic_candidates(features, packed_dtype: int = BF16, m_r: int = 16):
    """Per feature row (log2 M, log2 K, log2 N, density, ...): the index of
    the candidate matching the analytic rule's schedule, -1 if none."""
    import numpy as np
    out = np.full(len(features), -1, dtype=np.int64)
    for i, f in enumerate(np.asarray(features, dtype=np.float64)):
        M, K, N = (int(round(2.0 ** f[j])) for j in range(3))
        nnz = int(round(f[3] * M * K))
        t = rosko_schedule_analytic(M, K, N, nnz, m_r, packed_dtype)
        out[i] = rosko_candidate_index(t, packed_dtype)
    return out


def rosko_device_status(clear: bool = False) -> int:
    v = ctypes.c_int32()
    _check(lib().rosko_device_status(ctypes.byref(v), int(bool(clear))), "rosko_device_status")
    return v.value


def rosko_kernel_launches() -> int:
    return int(lib().rosko_kernel_launches())


def rosko_pack_save(A: PackedA) -> bytes:
    """Byte image of a packed handle (rosko_pack_load restores it)."""
    L = lib()
    n = ctypes.c_int64()
    _check(L.rosko_pack_save(A.handle, None, 0, ctypes.byref(n)), "rosko_pack_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(L.rosko_pack_save(A.handle, buf, n.value, ctypes.byref(n)), "rosko_pack_save")
    return buf.raw[: n.value]


def rosko_pack_load(image: bytes, stream=None) -> PackedA:
    """A new handle on the current device from a rosko_pack_save image."""
    L = lib()
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(bytes(image), len(image))
    _check(L.rosko_pack_load(buf, len(image), ctypes.c_void_p(_stream(stream)), ctypes.byref(out)),
           "rosko_pack_load")
    h = PackedA(out.value, 0, 0)
    i = rosko_packed_info(h)
    h.M, h.K = i["M"], i["K"]
    return h


def rosko_set_wait_limit(ns: int) -> None:
    """Bounded-wait limit of the current device in ns (0: the 2 s default)."""
    _check(lib().rosko_set_wait_limit(int(ns)), "rosko_set_wait_limit")


def rosko_probe_bounded_wait(stream=None) -> None:
    """Launch the failure-detection probe (a wait that runs out)."""
    _check(lib().rosko_probe_bounded_wait(ctypes.c_void_p(_stream(stream))),
           "rosko_probe_bounded_wait")


def rosko_num_candidates() -> int:
    return int(lib().rosko_num_candidates())


def rosko_candidate(A: PackedA, N: int, index: int):
    """Candidate schedule `index` as a forced tile, or None if it does not apply."""
    t = rosko_tile()
    st = lib().rosko_candidate(A.handle, N, index, ctypes.byref(t))
    if st == 2:
        return None
    _check(st, "rosko_candidate")
    return t


def rosko_autotune(A: PackedA, B: torch.Tensor, C: torch.Tensor,
                   col_scale: Optional[torch.Tensor] = None, reps: int = 3, stream=None):
    """Time every candidate; returns (best tile, list of per-candidate ms or None)."""
    K, N = B.shape
    nc = rosko_num_candidates()
    times = (ctypes.c_float * nc)()
    best = rosko_tile()
    st = lib().rosko_autotune(A.handle, _ptr(B), TORCH_TO_CODE[B.dtype], N, _ld(B),
                              _ptr(col_scale), _ptr(C), TORCH_TO_CODE[C.dtype], _ld(C), reps,
                              ctypes.byref(best), times, ctypes.c_void_p(_stream(stream)))
    _check(st, "rosko_autotune")
    return best, [None if t < 0 else float(t) for t in times]


def rosko_time_tile(A: PackedA, B: torch.Tensor, C: torch.Tensor, tile: Optional[rosko_tile] = None,
                    col_scale: Optional[torch.Tensor] = None, reps: int = 3, stream=None) -> float:
    """Mean device ms of one SpMM with `tile` (L2 flushed before each launch)."""
    K, N = B.shape
    ms = ctypes.c_float()
    st = lib().rosko_time_tile(A.handle, _ptr(B), TORCH_TO_CODE[B.dtype], N, _ld(B),
                               _ptr(col_scale), _ptr(C), TORCH_TO_CODE[C.dtype], _ld(C),
                               ctypes.byref(tile) if tile is not None else None, reps,
                               ctypes.byref(ms), ctypes.c_void_p(_stream(stream)))
    _check(st, "rosko_time_tile")
    return float(ms.value)


def rosko_features(A: PackedA, N: int, stream=None):
    import numpy as np
    f = (ctypes.c_double * 16)()
    _check(lib().rosko_features(A.handle, N, f, ctypes.c_void_p(_stream(stream))),
           "rosko_features")
    return np.array(f[:], dtype=np.float64)


def rosko_features_static(A: PackedA, N: int, out=None, stream=None):
    """FP32 features into a 16-float CUDA tensor (allocation-free library
    path; `out` is allocated here by torch when not given)."""
    import torch
    if out is None:
        out = torch.empty(16, dtype=torch.float32, device="cuda")
    if out.dtype != torch.float32 or not out.is_cuda or out.numel() < 16 or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA float32 tensor of >= 16 elements")
    _check(lib().rosko_features_static(A.handle, N, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(_stream(stream))),
           "rosko_features_static")
    return out


def rosko_mlp_param_count(n_in: int, n_out: int) -> int:
    return int(lib().rosko_mlp_param_count(n_in, n_out))


def rosko_mlp_workspace_floats(batch: int, n_out: int) -> int:
    return int(lib().rosko_mlp_workspace_floats(batch, n_out))


def rosko_mlp_forward(params: torch.Tensor, X: torch.Tensor, n_out: int, stream=None):
    batch, n_in = X.shape
    acts = torch.empty((3, batch, 64), dtype=torch.float32, device=X.device)
    logits = torch.empty((batch, n_out), dtype=torch.float32, device=X.device)
    _check(lib().rosko_mlp_forward(_ptr(params), _ptr(X), batch, n_in, n_out, _ptr(acts),
                                   _ptr(logits), ctypes.c_void_p(_stream(stream))),
           "rosko_mlp_forward")
    return logits


def rosko_mlp_loss_grad(params: torch.Tensor, X: torch.Tensor, Y: torch.Tensor,
                        workspace: Optional[torch.Tensor] = None, stream=None):
    """Returns (loss tensor[1], grads tensor like params)."""
    batch, n_in = X.shape
    n_out = Y.shape[1]
    if workspace is None:
        workspace = torch.empty(rosko_mlp_workspace_floats(batch, n_out), dtype=torch.float32,
                                device=X.device)
    grads = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(lib().rosko_mlp_loss_grad(_ptr(params), _ptr(X), _ptr(Y), batch, n_in, n_out,
                                     _ptr(grads), _ptr(loss), _ptr(workspace),
                                     ctypes.c_void_p(_stream(stream))), "rosko_mlp_loss_grad")
    return loss, grads


def rosko_mlp_adam(params, grads, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   weight_decay=0.0, stream=None):
    _check(lib().rosko_mlp_adam(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.numel(),
                                step, lr, beta1, beta2, eps, weight_decay,
                                ctypes.c_void_p(_stream(stream))),
           "rosko_mlp_adam")


def rosko_selector_set(params_host, mean, std, lo, hi) -> None:
    import numpy as np
    p = np.ascontiguousarray(params_host, dtype=np.float32)
    arr = [np.ascontiguousarray(a, dtype=np.float64) for a in (mean, std, lo, hi)]
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().rosko_selector_set(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size,
                                    *[a.ctypes.data_as(dp) for a in arr]), "rosko_selector_set")


def rosko_spmm_batched(As, Bs, Cs, accumulate: bool = False, tiles=None, stream=None):
    """C_i = A_i . B_i for up to 64 problems in one dense-panel launch plus one
    sparse launch per problem that needs it."""
    n = len(As)
    h = (ctypes.c_void_p * n)(*[a.handle.value for a in As])
    b = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Bs])
    c = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Cs])
    N = (ctypes.c_int64 * n)(*[x.shape[1] for x in Bs])
    ldb = (ctypes.c_int64 * n)(*[_ld(x) for x in Bs])
    ldc = (ctypes.c_int64 * n)(*[_ld(x) for x in Cs])
    tl = None
    if tiles is not None:
        tl = (rosko_tile * n)(*tiles)
    st = lib().rosko_spmm_batched(n, h, b, N, ldb, c, ldc, TORCH_TO_CODE[Bs[0].dtype],
                                  TORCH_TO_CODE[Cs[0].dtype], int(bool(accumulate)),
                                  ctypes.cast(tl, ctypes.POINTER(rosko_tile)) if tl is not None else None,
                                  ctypes.c_void_p(_stream(stream)))
    _check(st, "rosko_spmm_batched")
    return Cs
