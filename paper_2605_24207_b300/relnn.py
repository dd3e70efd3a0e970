"""Thin Python binding of librelnn.so (argument marshalling only; every step runs in the library's
CUDA kernels). PyTorch supplies device memory and the current stream.

The library is built in-tree by ``build_lib.build()``; importing this module never compiles and
never falls back to another implementation: if the shared library is missing the import of
``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import itertools
import os
from typing import Sequence

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# RELNN_LIB=checked selects the checked build (device-side bounds checks, librelnn_checked.so)
LIB_PATH = os.path.join(HERE, "librelnn_checked.so" if os.environ.get("RELNN_LIB") == "checked" else "librelnn.so")

I32, I64 = 0, 1
F32, BF16 = 0, 1
ACT_NONE, ACT_RELU = 0, 1
FLAG_BF16 = 0x1
FLAG_KAHAN = 0x2
FLAG_IDENTITY = 0x4
FLAG_NO_JOIN_DST = 0x8
FLAG_NO_CONCAT_DST = 0x10
FLAG_RELU_MASK = 0x20
FLAG_TILE128 = 0x40
FLAG_PUSHDOWN = 0x80
FLAG_MEAN = 0x100
FLAG_MAX = 0x200
FLAG_PER_TUPLE = 0x400

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOSPC", 4: "EAGAIN", 5: "ETIMEDOUT", 6: "ECUDA",
          7: "EDEVICE", 8: "ENOTSUP"}


class RelnnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Filter(C.Structure):
    _fields_ = [("lhs", C.c_int32), ("op", C.c_int32), ("rhs", C.c_int32), ("reserved", C.c_int32),
                ("lhs_const", C.c_int64), ("rhs_const", C.c_int64)]


class BranchDesc(C.Structure):
    _fields_ = [("d_src", C.c_void_p), ("d_dst", C.c_void_p), ("n_tuples", C.c_int64), ("d_r", C.c_int32),
                ("n_filters", C.c_int32), ("filters", C.POINTER(Filter))]


TERM_SRC, TERM_DST, TERM_CONST = 0, 1, 2
_CMP = {"==": 0, "!=": 1, "<": 2, "<=": 3, ">": 4, ">=": 5}
MAX_FILTERS = 4


def _filters(preds):
    """A relnn_filter array from (lhs, op, rhs) triples: lhs / rhs are "src", "dst" or an int."""
    if not preds:
        return None, 0
    assert len(preds) <= MAX_FILTERS, "at most 4 predicates per branch"
    arr = (Filter * len(preds))()
    for i, (lhs, op, rhs) in enumerate(preds):
        def term(x):
            if isinstance(x, str):
                return {"src": TERM_SRC, "dst": TERM_DST}[x], 0
            return TERM_CONST, int(x)
        (lt, lc), (rt, rc) = term(lhs), term(rhs)
        arr[i] = Filter(lt, _CMP[op], rt, 0, lc, rc)
    return arr, len(preds)


class RuleDesc(C.Structure):
    _fields_ = [("key_type", C.c_int), ("d_h_ids", C.c_void_p), ("n_h", C.c_int64), ("d", C.c_int32),
                ("d_out", C.c_int32), ("n_branches", C.c_int32), ("branches", C.POINTER(BranchDesc)),
                ("act", C.c_int), ("flags", C.c_uint32)]


ATTN_SOFTMAX, ATTN_PRODUCT = 0, 1


class AttnParams(C.Structure):
    _fields_ = [("d_q", C.c_void_p), ("d_k", C.c_void_p), ("d_v", C.c_void_p), ("dtype", C.c_int), ("d", C.c_int32),
                ("d_val", C.c_int32), ("n_heads", C.c_int32), ("scale", C.c_float), ("mode", C.c_int32)]


class TriDesc(C.Structure):
    _fields_ = [("key_type", C.c_int), ("d_h_ids", C.c_void_p), ("n_h", C.c_int64), ("d_src", C.c_void_p),
                ("d_dst", C.c_void_p), ("n_edges", C.c_int64)]


class StreamDesc(C.Structure):
    _fields_ = [("key_type", C.c_int), ("d_h_ids", C.c_void_p), ("n_h", C.c_int64), ("d", C.c_int32),
                ("d_out", C.c_int32), ("act", C.c_int), ("flags", C.c_uint32), ("h_src", C.c_void_p),
                ("h_dst", C.c_void_p), ("n_tuples", C.c_int64), ("d_r", C.c_int32), ("n_filters", C.c_int32),
                ("filters", C.POINTER(Filter)), ("chunk_tuples", C.c_int64), ("mem_budget_bytes", C.c_int64)]


class RuleParams(C.Structure):
    _fields_ = [("d_z", C.c_void_p), ("z_dtype", C.c_int), ("d_r", C.POINTER(C.c_void_p)), ("r_dtype", C.c_int),
                ("d_W", C.POINTER(C.c_void_p)), ("w_dtype", C.c_int), ("d_b", C.POINTER(C.c_void_p))]


_LIB = None

EXPORTS = [
    "relnn_version", "relnn_status_string", "relnn_last_error", "relnn_last_device_error",
    "relnn_join_build", "relnn_join_probe", "relnn_join_destroy",
    "relnn_rule_plan", "relnn_plan_info", "relnn_plan_out_keys", "relnn_plan_check", "relnn_plan_set_z_version",
    "relnn_rule_forward", "relnn_rule_backward", "relnn_plan_destroy",
    "relnn_profile_enable", "relnn_profile_read", "relnn_profile_reset", "relnn_launch_count",
]
(PROF_FWD_TC, PROF_FWD_FP32, PROF_FIXUP, PROF_BWD_TC, PROF_BWD_FP32, PROF_PLAN, PROF_AGG_FWD, PROF_AGG_BWD,
 PROF_AGG_SUM) = range(9)


def lib():
    """Load librelnn.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{os.path.basename(LIB_PATH)} not built at {LIB_PATH}; run paper_2605_24207_b300/build_lib.py")
    L = C.CDLL(LIB_PATH)
    L.relnn_version.restype = C.c_int32
    L.relnn_status_string.restype = C.c_char_p
    L.relnn_last_error.restype = C.c_char_p
    L.relnn_last_device_error.restype = C.c_int32
    vp, i64 = C.c_void_p, C.c_int64
    L.relnn_join_build.argtypes = [vp, i64, C.c_int, vp, C.POINTER(vp)]
    L.relnn_join_probe.argtypes = [vp, vp, i64, vp, vp, i64, vp, vp]
    L.relnn_join_destroy.argtypes = [vp]
    L.relnn_rule_plan.argtypes = [C.POINTER(RuleDesc), vp, C.POINTER(vp)]
    L.relnn_plan_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.relnn_plan_out_keys.argtypes = [vp, vp, vp]
    L.relnn_plan_check.argtypes = [vp, vp]
    L.relnn_plan_set_z_version.argtypes = [vp, C.c_uint64]
    L.relnn_rule_forward.argtypes = [vp, C.POINTER(RuleParams), vp, vp, vp, vp]
    L.relnn_rule_backward.argtypes = [vp, C.POINTER(RuleParams), vp, vp, vp, vp, vp, vp]
    L.relnn_plan_destroy.argtypes = [vp]
    L.relnn_plan_release.argtypes = [vp, vp]
    L.relnn_plan_release.restype = C.c_int
    L.relnn_rule_forward_noalloc.argtypes = [vp, C.c_int32, vp, vp, vp, i64, vp, vp, C.c_int32, C.c_int, vp, vp]
    L.relnn_rule_forward_noalloc.restype = C.c_int
    L.relnn_mse_loss.argtypes = [vp, vp, i64, vp, vp, i64, C.c_int32, C.c_int, vp, vp, vp]
    L.relnn_mse_loss.restype = C.c_int
    L.relnn_attention_forward.argtypes = [vp, C.POINTER(AttnParams), vp, vp, vp]
    L.relnn_attention_backward.argtypes = [vp, C.POINTER(AttnParams), vp, vp, vp, vp, vp, vp, vp]
    L.relnn_attention_forward.restype = C.c_int
    L.relnn_attention_backward.restype = C.c_int
    L.relnn_triangle_plan.argtypes = [C.POINTER(TriDesc), vp, C.POINTER(vp)]
    L.relnn_triangle_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.relnn_triangle_out_keys.argtypes = [vp, vp, vp]
    L.relnn_triangle_forward.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int32, vp, vp]
    L.relnn_triangle_backward.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int32, vp, vp, vp, vp, vp]
    L.relnn_triangle_destroy.argtypes = [vp]
    for name in ("relnn_triangle_plan", "relnn_triangle_info", "relnn_triangle_out_keys", "relnn_triangle_forward",
                 "relnn_triangle_backward", "relnn_triangle_destroy"):
        getattr(L, name).restype = C.c_int
    L.relnn_stream_create.argtypes = [C.POINTER(StreamDesc), vp, C.POINTER(vp)]
    L.relnn_stream_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.relnn_stream_forward.argtypes = [vp, C.POINTER(RuleParams), vp, vp, C.POINTER(i64), vp]
    L.relnn_stream_backward.argtypes = [vp, C.POINTER(RuleParams), vp, vp, vp, vp, vp, vp]
    L.relnn_stream_destroy.argtypes = [vp]
    for name in ("relnn_stream_create", "relnn_stream_info", "relnn_stream_forward", "relnn_stream_backward",
                 "relnn_stream_destroy"):
        getattr(L, name).restype = C.c_int
    L.relnn_profile_enable.argtypes = [C.c_int32]
    L.relnn_profile_read.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(i64)]
    for name in EXPORTS[4:-1]:
        getattr(L, name).restype = C.c_int
    L.relnn_launch_count.restype = C.c_uint64
    L.relnn_tune_set.argtypes = [C.c_int32, i64]
    L.relnn_tune_set.restype = C.c_int
    L.relnn_tune_get.argtypes = [C.c_int32, C.POINTER(i64)]
    L.relnn_tune_get.restype = C.c_int
    L.relnn_build_flags.restype = C.c_int32
    L.relnn_test_wait_timeout.argtypes = [C.c_int32, vp]
    L.relnn_test_wait_timeout.restype = C.c_int
    L.relnn_peak_fma_f32.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    L.relnn_peak_fma_f32.restype = C.c_int
    _LIB = L
    return L


def _check(status: int):
    if status != 0:
        msg = lib().relnn_last_error().decode(errors="replace")
        raise RelnnError(status, msg)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


def _key_type(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return I32
    if t.dtype == torch.int64:
        return I64
    raise TypeError(f"keys must be int32 or int64, got {t.dtype}")


def _float_type(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"embeddings must be float32 or bfloat16, got {t.dtype}")


def launch_count() -> int:
    """Kernels launched by librelnn since it was loaded."""
    return int(lib().relnn_launch_count())


def profile_enable(on: bool = True):
    _check(lib().relnn_profile_enable(1 if on else 0))


def profile_reset():
    _check(lib().relnn_profile_reset())


TUNE_SORT_BITS, TUNE_AGG_ROWS, TUNE_AGG_STAGES, TUNE_AGG_EPI, TUNE_KAHAN_MIN, TUNE_GROUP_SORT, TUNE_AGG_FUSE = 0, 1, 2, 3, 4, 5, 6


def tune_set(knob: int, value: int):
    """Sets a process-wide tuning knob (relnn_tune_set)."""
    _check(lib().relnn_tune_set(int(knob), int(value)))


def tune_get(knob: int) -> int:
    v = C.c_int64()
    _check(lib().relnn_tune_get(int(knob), C.byref(v)))
    return v.value


def peak_fma_f32(iters: int = 1 << 15, stream=None):
    """(TFLOP/s, ms) of the library's FP32 FMA throughput probe (relnn_peak_fma_f32)."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().relnn_peak_fma_f32(int(iters), C.byref(tf), C.byref(ms), _stream(stream)))
    return tf.value, ms.value


def profile_read(kernel_id: int):
    """(total device ms, launches) of a library kernel since the last reset (waits for events)."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib().relnn_profile_read(kernel_id, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def mse_loss(pred, pred_keys, target, target_keys, need_grad: bool = True, stream=None):
    """relnn_mse_loss: (loss [1] f32 device tensor, d loss / d pred or None)."""
    loss = torch.empty(1, dtype=torch.float32, device=pred.device)
    grad = torch.empty_like(pred) if need_grad else None
    _check(lib().relnn_mse_loss(_ptr(pred), _ptr(pred_keys), pred.shape[0], _ptr(target), _ptr(target_keys),
                                target.shape[0], pred.shape[1], _key_type(pred_keys), _ptr(loss), _ptr(grad),
                                _stream(stream)))
    return loss, grad


def rule_forward_noalloc(z, hs, hd, seg, W, b, out, act: int = ACT_NONE, stream=None):
    """relnn_rule_forward_noalloc: FP32-form forward over join output already grouped by output row,
    with no device allocation (the library's fixed scratch array is used). ``out`` must be a
    preallocated f32 [n_out, d_out] tensor; returns it."""
    _check(lib().relnn_rule_forward_noalloc(_ptr(z), z.shape[1], _ptr(hs), _ptr(hd), _ptr(seg), hs.numel(),
                                            _ptr(W), _ptr(b), W.shape[0], act, _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------------------------------------ join
class Join:
    """relnn_join_build / relnn_join_probe (bag-semantics equi-join of two key columns)."""

    def __init__(self, keys: torch.Tensor, stream=None):
        self._h = C.c_void_p()
        self.kt = _key_type(keys)
        self.dtype = keys.dtype
        _check(lib().relnn_join_build(_ptr(keys), keys.numel(), self.kt, _stream(stream), C.byref(self._h)))

    def probe(self, keys: torch.Tensor, capacity: int | None = None, stream=None):
        """All (probe row, build row) pairs, ordered by probe row then build row."""
        assert keys.dtype == self.dtype, "probe keys must have the build key type"
        dev = keys.device
        cap = keys.numel() if capacity is None else int(capacity)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        while True:
            pi = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            bi = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
            st = lib().relnn_join_probe(self._h, _ptr(keys), keys.numel(), _ptr(pi), _ptr(bi), cap, _ptr(cnt),
                                        _stream(stream))
            if st == 3 and capacity is None:  # ENOSPC: grow to the reported size
                cap = int(cnt.item())
                continue
            _check(st)
            n = int(cnt.item())
            return pi[:n], bi[:n]

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _LIB is not None:
            _LIB.relnn_join_destroy(self._h)
            self._h = C.c_void_p()


# ------------------------------------------------------------------------------------------ rules
class RulePlan:
    """relnn_rule_plan: the cached content track of
    H'(dst; SUM tau(Concat(z_src, z_dst[, r]))) :- E_i(src, dst[; r]), H(src; z_src), H(dst; z_dst)."""

    def __init__(self, h_ids: torch.Tensor, branches: Sequence, d: int, d_out: int, act: int = ACT_NONE,
                 flags: int = 0, d_r: int = 0, stream=None, filters=None):
        """``branches``: sequence of (src, dst) device key tensors. ``filters``: per branch, None or a
        list of up to 4 conjunctive predicates (lhs, op, rhs) with lhs / rhs "src", "dst" or an integer
        constant and op one of == != < <= > >= (the rule's selection on its content variables)."""
        self.kt = _key_type(h_ids)
        self.key_dtype = h_ids.dtype
        self.device = h_ids.device
        self.n_branches = len(branches)
        self.flags, self.act, self.d, self.d_r = flags, act, d, d_r
        self.n_tuples = [int(s.numel()) for s, _ in branches]
        arr = (BranchDesc * len(branches))()
        self._filters = []
        for i, (s, t) in enumerate(branches):
            assert s.dtype == self.key_dtype and t.dtype == self.key_dtype
            farr, nf = _filters(filters[i] if filters else None)
            self._filters.append(farr)
            arr[i] = BranchDesc(_ptr(s), _ptr(t), s.numel(), d_r, nf,
                                C.cast(farr, C.POINTER(Filter)) if farr is not None else None)
        desc = RuleDesc(self.kt, _ptr(h_ids), h_ids.numel(), d, d_out, len(branches), arr, act, flags)
        self._h = C.c_void_p()
        _check(lib().relnn_rule_plan(C.byref(desc), _stream(stream), C.byref(self._h)))
        n_out, n_tot = C.c_int64(), C.c_int64()
        per = (C.c_int64 * len(branches))()
        _check(lib().relnn_plan_info(self._h, C.byref(n_out), C.byref(n_tot), per))
        self.n_out = n_out.value
        self.n_matched = n_tot.value
        self.matched = list(per)
        concat = d * (1 if (flags & (FLAG_NO_JOIN_DST | FLAG_NO_CONCAT_DST)) else 2) + d_r
        self.d_in = concat
        self.d_out = concat if flags & FLAG_IDENTITY else d_out

    def out_keys(self, stream=None) -> torch.Tensor:
        k = torch.empty(max(self.n_out, 1), dtype=self.key_dtype, device=self.device)
        _check(lib().relnn_plan_out_keys(self._h, _ptr(k), _stream(stream)))
        return k[: self.n_out]

    def check(self, stream=None):
        _check(lib().relnn_plan_check(self._h, _stream(stream)))

    def _params(self, z, W, b, r):
        n = self.n_branches
        Ws = (C.c_void_p * n)(*[_ptr(w) for w in W]) if W is not None else None
        bs = (C.c_void_p * n)(*[_ptr(x) for x in b]) if b is not None else None
        rs = (C.c_void_p * n)(*[_ptr(x) for x in r]) if r is not None else None
        w_dt = _float_type(W[0]) if W is not None else F32
        r_dt = _float_type(r[0]) if r is not None else F32
        keep = (Ws, bs, rs)
        prm = RuleParams(_ptr(z), _float_type(z), rs, r_dt, Ws, w_dt, bs)
        return prm, keep

    @staticmethod
    def _attn(q, k, v, n_heads, scale, mode):
        return AttnParams(_ptr(q), _ptr(k), _ptr(v), _float_type(q), q.shape[1], v.shape[1], n_heads, float(scale),
                          {"softmax": ATTN_SOFTMAX, "product": ATTN_PRODUCT}[mode])

    def attention(self, q, k, v, n_heads: int = 1, scale: float = 1.0, mode: str = "softmax", stream=None):
        """relnn_attention_forward: (Out [n_out, d] f32, log-sum-exp [n_out, n_heads] or None). q is read at
        each tuple's dst H row, k and v at its src H row."""
        out = torch.empty((max(self.n_out, 1), v.shape[1]), dtype=torch.float32, device=self.device)
        lse = torch.empty((max(self.n_out, 1), n_heads), dtype=torch.float32, device=self.device) \
            if mode == "softmax" else None
        prm = self._attn(q, k, v, n_heads, scale, mode)
        _check(lib().relnn_attention_forward(self._h, C.byref(prm), _ptr(out), _ptr(lse), _stream(stream)))
        return out[: self.n_out], (lse[: self.n_out] if lse is not None else None)

    def attention_backward(self, dout, out, lse, q, k, v, n_heads: int = 1, scale: float = 1.0,
                           mode: str = "softmax", stream=None):
        """relnn_attention_backward: (dq, dk, dv) [n_h, d] f32."""
        dq, dk, dv = (torch.empty(x.shape, dtype=torch.float32, device=self.device) for x in (q, k, v))
        prm = self._attn(q, k, v, n_heads, scale, mode)
        dout = dout.contiguous()
        _check(lib().relnn_attention_backward(self._h, C.byref(prm), _ptr(out), _ptr(lse), _ptr(dout), _ptr(dq),
                                              _ptr(dk), _ptr(dv), _stream(stream)))
        return dq, dk, dv

    def _set_z_version(self, z, z_version):
        v = 0
        if z_version == "auto":
            v = _auto_z_version(z)
        elif z_version is not None:
            v = int(z_version)
        _check(lib().relnn_plan_set_z_version(self._h, v))

    def forward(self, z, W=None, b=None, r=None, out=None, stream=None, z_version=None) -> torch.Tensor:
        """Output embeddings [n_out, d_out] f32 (rows in out_keys() order). z_version: None (an f32 z
        is converted to bf16 on every call of the BF16 form), "auto" (the tensor object and its
        in-place version counter key the plan's bf16 copy) or a caller-managed nonzero int."""
        if out is None:
            out = torch.empty((max(self.n_out, 1), self.d_out), dtype=torch.float32, device=self.device)
        self._set_z_version(z, z_version)
        prm, keep = self._params(z, W, b, r)
        _check(lib().relnn_rule_forward(self._h, C.byref(prm), None, _ptr(out), None, _stream(stream)))
        return out[: self.n_out]

    def backward(self, dout, z, W=None, b=None, r=None, need_dz=True, stream=None, z_version=None):
        """Gradients (dW list, db list, dz, dr list) of the forward for output gradient ``dout``
        (z_version as for forward)."""
        dev, n = self.device, self.n_branches
        self._set_z_version(z, z_version)
        dW = [torch.empty((self.d_out, self.d_in), dtype=torch.float32, device=dev) for _ in range(n)] \
            if W is not None else None
        db = [torch.empty(self.d_out, dtype=torch.float32, device=dev) for _ in range(n)] if W is not None else None
        dz = torch.empty(z.shape, dtype=torch.float32, device=dev) if need_dz else None
        dr = [torch.empty((self.n_tuples[i], self.d_r), dtype=torch.float32, device=dev) for i in range(n)] \
            if (r is not None and self.d_r > 0) else None
        prm, keep = self._params(z, W, b, r)
        dWp = (C.c_void_p * n)(*[_ptr(x) for x in dW]) if dW else None
        dbp = (C.c_void_p * n)(*[_ptr(x) for x in db]) if db else None
        drp = (C.c_void_p * n)(*[_ptr(x) for x in dr]) if dr else None
        dout = dout.contiguous()
        _check(lib().relnn_rule_backward(self._h, C.byref(prm), _ptr(dout), dWp, dbp, _ptr(dz), drp,
                                         _stream(stream)))
        return dW, db, dz, dr

    def release(self, stream=None):
        """Frees the plan in the order of ``stream`` (no device-wide wait); every call that used
        the plan must have been issued on that stream."""
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().relnn_plan_release(self._h, _stream(stream)))
            self._h = C.c_void_p()

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _LIB is not None:
            _LIB.relnn_plan_destroy(self._h)
            self._h = C.c_void_p()


class TrianglePlan:
    """relnn_triangle_*: Out(n; sum(a_n * b_v * c_w)) :- E(n, v), E(v, w), E(w, n), H(n; a), H(v; b),
    H(w; c) (the cyclic self-join of a triangle homomorphism), with cached match records."""

    def __init__(self, h_ids: torch.Tensor, src: torch.Tensor, dst: torch.Tensor, stream=None):
        self.kt = _key_type(h_ids)
        self.key_dtype = h_ids.dtype
        self.device = h_ids.device
        assert src.dtype == self.key_dtype and dst.dtype == self.key_dtype
        desc = TriDesc(self.kt, _ptr(h_ids), h_ids.numel(), _ptr(src), _ptr(dst), src.numel())
        self._h = C.c_void_p()
        _check(lib().relnn_triangle_plan(C.byref(desc), _stream(stream), C.byref(self._h)))
        n_out, n_rec, n_kept = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().relnn_triangle_info(self._h, C.byref(n_out), C.byref(n_rec), C.byref(n_kept)))
        self.n_out, self.n_records, self.n_edges_kept = n_out.value, n_rec.value, n_kept.value

    def out_keys(self, stream=None) -> torch.Tensor:
        k = torch.empty(max(self.n_out, 1), dtype=self.key_dtype, device=self.device)
        _check(lib().relnn_triangle_out_keys(self._h, _ptr(k), _stream(stream)))
        return k[: self.n_out]

    def forward(self, a, b, c, stream=None) -> torch.Tensor:
        out = torch.empty((max(self.n_out, 1), a.shape[1]), dtype=torch.float32, device=self.device)
        _check(lib().relnn_triangle_forward(self._h, _ptr(a), _ptr(b), _ptr(c), _float_type(a), a.shape[1],
                                            _ptr(out), _stream(stream)))
        return out[: self.n_out]

    def backward(self, dout, a, b, c, stream=None):
        da, db, dc = (torch.empty(x.shape, dtype=torch.float32, device=self.device) for x in (a, b, c))
        dout = dout.contiguous()
        _check(lib().relnn_triangle_backward(self._h, _ptr(a), _ptr(b), _ptr(c), _float_type(a), a.shape[1],
                                             _ptr(dout), _ptr(da), _ptr(db), _ptr(dc), _stream(stream)))
        return da, db, dc

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _LIB is not None:
            _LIB.relnn_triangle_destroy(self._h)
            self._h = C.c_void_p()


class StreamRule:
    """relnn_stream_*: a single-branch rule whose E (src, dst and the optional per-tuple r) stays in
    host memory and is streamed to the device in chunks; H (ids, z) is on the device."""

    def __init__(self, h_ids: torch.Tensor, src: torch.Tensor, dst: torch.Tensor, d: int, d_out: int,
                 act: int = ACT_NONE, flags: int = 0, d_r: int = 0, chunk_tuples: int = 0, mem_budget: int = 0,
                 filters=None, stream=None):
        """``src`` / ``dst``: CPU key tensors (pinned memory lets the copies overlap the compute);
        they are kept referenced for the stream's lifetime."""
        assert not src.is_cuda and not dst.is_cuda, "E stays in host memory"
        self.kt = _key_type(h_ids)
        self.key_dtype = h_ids.dtype
        self.device = h_ids.device
        self.src, self.dst = src.contiguous(), dst.contiguous()
        assert self.src.dtype == self.key_dtype and self.dst.dtype == self.key_dtype
        self.flags, self.act, self.d, self.d_r = flags, act, d, d_r
        self.n_tuples = int(self.src.numel())
        self._farr, nf = _filters(filters)
        desc = StreamDesc(self.kt, _ptr(h_ids), h_ids.numel(), d, d_out, act, flags, self.src.data_ptr(),
                          self.dst.data_ptr(), self.n_tuples, d_r, nf,
                          C.cast(self._farr, C.POINTER(Filter)) if self._farr is not None else None,
                          chunk_tuples, mem_budget)
        self._h = C.c_void_p()
        _check(lib().relnn_stream_create(C.byref(desc), _stream(stream), C.byref(self._h)))
        u, ch, nc = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().relnn_stream_info(self._h, C.byref(u), C.byref(ch), C.byref(nc)))
        self.max_out, self.chunk_tuples, self.n_chunks = u.value, ch.value, nc.value
        concat = d * (1 if flags & FLAG_NO_CONCAT_DST else 2) + d_r
        self.d_in = concat
        self.d_out = concat if flags & FLAG_IDENTITY else d_out
        self.n_out = None

    def _params(self, z, W, b, r):
        Ws = (C.c_void_p * 1)(_ptr(W)) if W is not None else None
        bs = (C.c_void_p * 1)(_ptr(b)) if b is not None else None
        rs = None
        if r is not None:
            assert not r.is_cuda and r.is_contiguous(), "r is streamed from host memory"
            rs = (C.c_void_p * 1)(r.data_ptr())
        prm = RuleParams(_ptr(z), _float_type(z), rs, _float_type(r) if r is not None else F32, Ws,
                         _float_type(W) if W is not None else F32, bs)
        return prm, (Ws, bs, rs)

    def forward(self, z, W=None, b=None, r=None, stream=None):
        """(output keys [n_out], output embeddings [n_out, d_out] f32), keys ascending."""
        keys = torch.empty(max(self.max_out, 1), dtype=self.key_dtype, device=self.device)
        out = torch.empty((max(self.max_out, 1), self.d_out), dtype=torch.float32, device=self.device)
        prm, keep = self._params(z, W, b, r)
        n = C.c_int64()
        _check(lib().relnn_stream_forward(self._h, C.byref(prm), _ptr(keys), _ptr(out), C.byref(n), _stream(stream)))
        self.n_out = n.value
        return keys[: self.n_out], out[: self.n_out]

    def backward(self, dout, z, W=None, b=None, r=None, need_dz=True, stream=None):
        """(dW, db, dz, dr) for the output gradient of the last forward; dr is a CPU tensor."""
        dev = self.device
        dW = torch.empty((self.d_out, self.d_in), dtype=torch.float32, device=dev) if W is not None else None
        db = torch.empty(self.d_out, dtype=torch.float32, device=dev) if W is not None else None
        dz = torch.empty(z.shape, dtype=torch.float32, device=dev) if need_dz else None
        dr = torch.empty((self.n_tuples, self.d_r), dtype=torch.float32) if (r is not None and self.d_r > 0) else None
        prm, keep = self._params(z, W, b, r)
        dout = dout.contiguous()
        _check(lib().relnn_stream_backward(self._h, C.byref(prm), _ptr(dout), _ptr(dW), _ptr(db), _ptr(dz),
                                           dr.data_ptr() if dr is not None else None, _stream(stream)))
        return dW, db, dz, dr

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value and _LIB is not None:
            _LIB.relnn_stream_destroy(self._h)
            self._h = C.c_void_p()


_Z_SERIAL = itertools.count(1)


def _auto_z_version(z) -> int:
    """A nonzero version for tensor object ``z``: a serial number given to the object on first use
    (a new tensor at a reused address gets a new one) and its in-place version counter."""
    s = getattr(z, "_relnn_z_serial", None)
    if s is None:
        s = next(_Z_SERIAL)
        z._relnn_z_serial = s
    return ((s & 0xFFFFFFFFFF) << 24) | (z._version & 0xFFFFFF)


class RelnnRule(torch.autograd.Function):
    """Autograd wrapper: forward = relnn_rule_forward, backward = relnn_rule_backward (the gathered
    Concat is recomputed in the backward, not stored). Single-branch rules; for a union use the
    plan's forward/backward directly."""

    @staticmethod
    def forward(ctx, plan: RulePlan, z, W, b, r=None):
        ctx.plan = plan
        ctx.save_for_backward(z, W, b, r)
        return plan.forward(z, [W] if W is not None else None, [b] if b is not None else None,
                            [r] if r is not None else None, z_version="auto")

    @staticmethod
    def backward(ctx, dout):
        z, W, b, r = ctx.saved_tensors
        dW, db, dz, dr = ctx.plan.backward(dout, z, [W] if W is not None else None,
                                           [b] if b is not None else None, [r] if r is not None else None,
                                           need_dz=ctx.needs_input_grad[1], z_version="auto")
        return (None, dz, dW[0] if dW else None, db[0] if db else None, dr[0] if dr else None)


# ------------------------------------------------------------------------------------------ serving
class ServerCfg(C.Structure):
    _fields_ = [("d", C.c_int32), ("d_out", C.c_int32), ("d_W", C.c_void_p), ("w_dtype", C.c_int),
                ("d_b", C.c_void_p), ("act", C.c_int), ("flags", C.c_uint32), ("z_dtype", C.c_int),
                ("max_queue", C.c_int32), ("mem_budget_bytes", C.c_int64), ("max_batch_tuples", C.c_int64),
                ("max_batch_queries", C.c_int32), ("tile128_below", C.c_int64), ("n_workers", C.c_int32)]


class Query(C.Structure):
    _fields_ = [("d_h_ids", C.c_void_p), ("n_h", C.c_int64), ("d_z", C.c_void_p), ("d_src", C.c_void_p),
                ("d_dst", C.c_void_p), ("n_tuples", C.c_int64)]


class Result(C.Structure):
    _fields_ = [("n_out", C.c_int64), ("d_out_keys", C.c_void_p), ("d_out_z", C.c_void_p),
                ("latency_us", C.c_double), ("batch_queries", C.c_int32)]


def _server_lib():
    L = lib()
    if not getattr(L, "_server_types", False):
        vp = C.c_void_p
        L.relnn_server_create.argtypes = [C.POINTER(ServerCfg), C.POINTER(vp)]
        L.relnn_serve_submit.argtypes = [vp, C.POINTER(Query), C.POINTER(C.c_uint64)]
        L.relnn_serve_poll.argtypes = [vp, C.c_uint64, C.POINTER(Result), C.c_uint32]
        L.relnn_serve_release.argtypes = [vp, C.c_uint64]
        L.relnn_server_destroy.argtypes = [vp]
        for n in ("relnn_server_create", "relnn_serve_submit", "relnn_serve_poll", "relnn_serve_release",
                  "relnn_server_destroy"):
            getattr(L, n).restype = C.c_int
        L._server_types = True
    return L


class Server:
    """relnn_server_*: memory-admitted continuous batching of rule queries sharing one Linear.
    Query tensors (int32 keys, z) must stay alive until their ticket completes."""

    def __init__(self, W, b, d: int, act: int = ACT_NONE, flags: int = FLAG_BF16, z_dtype=torch.bfloat16,
                 max_queue: int = 256, mem_budget_bytes: int = 0, max_batch_tuples: int = 4_000_000,
                 max_batch_queries: int = 64, tile128_below: int = 0, n_workers: int = 4):
        self.L = _server_lib()
        self.W, self.b = W, b  # keep alive
        self.d_out = W.shape[0]
        cfg = ServerCfg(d, W.shape[0], _ptr(W), _float_type(W), _ptr(b), act, flags,
                        BF16 if z_dtype == torch.bfloat16 else F32, max_queue, mem_budget_bytes, max_batch_tuples,
                        max_batch_queries, tile128_below, n_workers)
        self._h = C.c_void_p()
        _check(self.L.relnn_server_create(C.byref(cfg), C.byref(self._h)))
        self._keep = {}

    def submit(self, h_ids, z, src, dst) -> int:
        """Ticket, or raises RelnnError (EAGAIN when the queue is full, ENOMEM if it can never fit)."""
        q = Query(_ptr(h_ids), h_ids.numel(), _ptr(z), _ptr(src), _ptr(dst), src.numel())
        t = C.c_uint64()
        _check(self.L.relnn_serve_submit(self._h, C.byref(q), C.byref(t)))
        self._keep[t.value] = (h_ids, z, src, dst)
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0):
        """None while pending; else (keys int32 [n], out f32 [n, d_out], latency_us, batch size) as
        views of the server's buffers (copy them before release)."""
        r = Result()
        st = self.L.relnn_serve_poll(self._h, ticket, C.byref(r), timeout_us)
        if st in (4, 5):  # EAGAIN / ETIMEDOUT
            return None
        _check(st)
        n = r.n_out
        if n == 0:
            keys = torch.zeros(0, dtype=torch.int32, device="cuda")
            out = torch.zeros((0, self.d_out), dtype=torch.float32, device="cuda")
        else:
            keys = _wrap_device(r.d_out_keys, (n,), torch.int32)
            out = _wrap_device(r.d_out_z, (n, self.d_out), torch.float32)
        return keys, out, r.latency_us, r.batch_queries

    def release(self, ticket: int):
        _check(self.L.relnn_serve_release(self._h, ticket))
        self._keep.pop(ticket, None)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.L.relnn_server_destroy(self._h)
            self._h = C.c_void_p()
            self._keep.clear()

    def __del__(self):
        self.close()


def _wrap_device(ptr: int, shape, dtype):
    """A torch view of library-owned device memory (no copy, no ownership)."""
    class _Cai:
        pass
    o = _Cai()
    typestr = {torch.int32: "<i4", torch.float32: "<f4"}[dtype]
    o.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                  "version": 3, "strides": None, "stream": None}
    return torch.as_tensor(o, device="cuda")
