"""Thin ctypes binding of libqsa (include/qsa.h).

Each function has the name of the C entry point it wraps and only marshals
arguments: numpy arrays become host pointers, integers stand for device
pointers and CUDA streams (for example ``tensor.data_ptr()`` and
``torch.cuda.current_stream().cuda_stream``).  All arithmetic runs in the
library's CUDA kernels; there is no fallback.  Importing this package raises
if libqsa.so has not been built (``paper_2608_16940_gb300.build.build()``).

Status codes other than QSA_OK raise :class:`QsaError` carrying the code and
``qsa_last_error()``.
"""
from __future__ import annotations

import ctypes
import itertools
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# QSA_LIB_VARIANT=debug loads the bounds-checked build (libqsa_debug.so, from
# build.py --debug-bounds) instead of the release library
LIB_PATH = os.path.join(_HERE, "libqsa_debug.so" if os.environ.get("QSA_LIB_VARIANT") == "debug" else "libqsa.so")

QSA_OK, QSA_E_ARG, QSA_E_RANGE, QSA_E_NOMEM, QSA_E_CUDA, QSA_E_TIMEOUT, QSA_E_UNSUPPORTED, QSA_E_STATE = range(8)
QSA_C64, QSA_C128 = 0, 1
QSA_LOWER_AUTO, QSA_LOWER_STRIDED, QSA_LOWER_PERMUTE = 0, 1, 2
QSA_PREC_FP32, QSA_PREC_TF32X3 = 0, 1
QSA_PLAN_PER_GATE, QSA_PLAN_GREEDY, QSA_PLAN_DP, QSA_PLAN_DP_MLP = 0, 1, 2, 3
QSA_OP_DIAG = 1
QSA_MAX_K, QSA_MAX_DIAG, QSA_MAX_PROD, QSA_MAX_LAYER = 6, 12, 11, 12
QSA_VICTIM_FIRST_FREE, QSA_VICTIM_FARTHEST = 0, 1
MLP_PARAMS = 6657
MLP_IN = 37


class QsaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qsa status {code}: {msg}")
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2608_16940_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)
_c = ctypes
_dp = _c.POINTER(_c.c_double)
_fp = _c.POINTER(_c.c_float)
_i32p = _c.POINTER(_c.c_int32)
_u64p = _c.POINTER(_c.c_uint64)
_szp = _c.POINTER(_c.c_size_t)


class qsa_op(_c.Structure):
    _fields_ = [("k", _c.c_int32), ("targets", _c.c_int32 * 6), ("matrix", _dp), ("flags", _c.c_uint32)]


class qsa_plan_opts(_c.Structure):
    _fields_ = [("planner", _c.c_int32), ("kmax", _c.c_int32), ("kmax_diag", _c.c_int32), ("window", _c.c_int32),
                ("rounds", _c.c_int32), ("precision", _c.c_int32), ("lowering", _c.c_int32),
                ("timing", _c.c_int32), ("victim", _c.c_int32), ("kmax_prod", _c.c_int32), ("layer", _c.c_int32),
                ("zero_init", _c.c_int32)]


class qsa_run_stats(_c.Structure):
    _fields_ = [("seconds", _c.c_double), ("apply_seconds", _c.c_double), ("permute_seconds", _c.c_double),
                ("hbm_bytes", _c.c_double), ("blocks", _c.c_uint64), ("passes", _c.c_uint64),
                ("permutes", _c.c_uint64), ("tc_blocks", _c.c_uint64), ("launches", _c.c_uint64),
                ("h2d_bytes", _c.c_double), ("tc_seconds", _c.c_double), ("diag_blocks", _c.c_uint64),
                ("diag_seconds", _c.c_double), ("prod_blocks", _c.c_uint64), ("prod_seconds", _c.c_double),
                ("layer_blocks", _c.c_uint64), ("layer_seconds", _c.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _sig(name, args, res=_c.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_vp = _c.c_void_p
_f = {
    "qsa_state_create": _sig("qsa_state_create", [_c.c_int, _c.c_int, _c.POINTER(_vp)]),
    "qsa_state_create_ex": _sig("qsa_state_create_ex", [_c.c_int, _c.c_int, _vp, _c.c_size_t, _vp, _c.c_int,
                                                        _c.POINTER(_vp)]),
    "qsa_state_destroy": _sig("qsa_state_destroy", [_vp]),
    "qsa_set_stream": _sig("qsa_set_stream", [_vp, _vp]),
    "qsa_state_reset": _sig("qsa_state_reset", [_vp]),
    "qsa_state_info": _sig("qsa_state_info", [_vp, _c.POINTER(_c.c_int), _c.POINTER(_vp)]),
    "qsa_set_layout": _sig("qsa_set_layout", [_vp, _i32p, _c.c_int]),
    "qsa_get_layout": _sig("qsa_get_layout", [_vp, _i32p]),
    "qsa_permute_bits": _sig("qsa_permute_bits", [_vp, _i32p, _i32p, _c.c_int]),
    "qsa_apply_fused": _sig("qsa_apply_fused", [_vp, _i32p, _c.c_int, _dp]),
    "qsa_apply_fused_ex": _sig("qsa_apply_fused_ex", [_vp, _i32p, _c.c_int, _dp, _c.c_int, _c.c_int]),
    "qsa_apply_diag": _sig("qsa_apply_diag", [_vp, _i32p, _c.c_int, _dp]),
    "qsa_apply_product": _sig("qsa_apply_product", [_vp, _i32p, _c.c_int, _dp]),
    "qsa_apply_layer": _sig("qsa_apply_layer", [_vp, _vp, _c.c_size_t, _i32p, _c.c_int, _dp]),
    "qsa_plan_order": _sig("qsa_plan_order", [_vp, _vp, _c.c_size_t]),
    "qsa_plan_execute_from_zero": _sig("qsa_plan_execute_from_zero", [_vp, _vp, _c.POINTER(qsa_run_stats)]),
    "qsa_plan_block_kinds": _sig("qsa_plan_block_kinds", [_vp, _i32p, _i32p, _c.c_size_t]),
    "qsa_plan_opts_default": _sig("qsa_plan_opts_default", [_c.POINTER(qsa_plan_opts)], None),
    "qsa_plan_circuit": _sig("qsa_plan_circuit", [_c.POINTER(qsa_op), _c.c_size_t, _c.c_int,
                                                  _c.POINTER(qsa_plan_opts), _szp, _szp]),
    "qsa_fuse_ops": _sig("qsa_fuse_ops", [_c.POINTER(qsa_op), _c.c_size_t, _i32p, _c.POINTER(_c.c_int), _dp]),
    "qsa_apply_circuit": _sig("qsa_apply_circuit", [_vp, _c.POINTER(qsa_op), _c.c_size_t,
                                                    _c.POINTER(qsa_plan_opts), _c.POINTER(qsa_run_stats)]),
    "qsa_plan_create": _sig("qsa_plan_create", [_c.POINTER(qsa_op), _c.c_size_t, _c.c_int,
                                                _c.POINTER(qsa_plan_opts), _i32p, _c.POINTER(_vp)]),
    "qsa_plan_info": _sig("qsa_plan_info", [_vp, _szp, _szp, _c.POINTER(_c.c_int), _szp]),
    "qsa_plan_blocks": _sig("qsa_plan_blocks", [_vp, _szp, _i32p, _c.c_size_t]),
    "qsa_plan_promotions": _sig("qsa_plan_promotions", [_vp, _i32p, _c.c_int, _c.POINTER(_c.c_uint64),
                                                         _c.POINTER(_c.c_uint64), _i32p]),
    "qsa_plan_execute": _sig("qsa_plan_execute", [_vp, _vp, _c.POINTER(qsa_run_stats)]),
    "qsa_plan_destroy": _sig("qsa_plan_destroy", [_vp]),
    "qsa_state_counters": _sig("qsa_state_counters", [_vp, _u64p]),
    "qsa_state_sync": _sig("qsa_state_sync", [_vp]),
    "qsa_probabilities": _sig("qsa_probabilities", [_vp, _dp, _dp]),
    "qsa_probabilities_device": _sig("qsa_probabilities_device", [_vp, _vp, _dp]),
    "qsa_expectation_z": _sig("qsa_expectation_z", [_vp, _c.c_uint64, _dp]),
    "qsa_expectation_z_batch": _sig("qsa_expectation_z_batch", [_vp, _u64p, _c.c_int, _dp]),
    "qsa_measure": _sig("qsa_measure", [_vp, _u64p, _c.c_int, _dp, _c.c_uint64, _c.c_uint64, _u64p, _u64p,
                                        _c.c_size_t, _c.POINTER(_c.c_size_t)]),
    "qsa_dm_apply_channel": _sig("qsa_dm_apply_channel", [_vp, _c.c_int, _i32p, _c.c_int, _dp, _c.c_int,
                                                           _c.c_int]),
    "qsa_dm_superoperator": _sig("qsa_dm_superoperator", [_c.c_int, _i32p, _c.c_int, _dp, _c.c_int, _i32p, _dp]),
    "qsa_dm_probabilities": _sig("qsa_dm_probabilities", [_vp, _c.c_int, _dp, _dp]),
    "qsa_dm_expectation_z": _sig("qsa_dm_expectation_z", [_vp, _c.c_int, _c.c_uint64, _dp]),
    "qsa_sample_counts": _sig("qsa_sample_counts", [_vp, _c.c_uint64, _c.c_uint64, _u64p, _u64p, _c.c_size_t,
                                                    _szp]),
    "qsa_last_error": _sig("qsa_last_error", [], _c.c_char_p),
    "qsa_costmodel_features": _sig("qsa_costmodel_features", [_c.c_int, _c.c_uint64, _c.c_int, _c.c_int, _fp]),
    "qsa_costmodel_set": _sig("qsa_costmodel_set", [_fp]),
    "qsa_costmodel_predict": _sig("qsa_costmodel_predict", [_fp, _c.c_size_t, _dp]),
}


def _optional(name, args, res=_c.c_int):
    if hasattr(_lib, name):
        _f[name] = _sig(name, args, res)


def qsa_last_error() -> str:
    v = _f["qsa_last_error"]()
    return v.decode() if v else ""


def _check(code: int) -> None:
    if code != QSA_OK:
        raise QsaError(code, qsa_last_error())


def _i32(seq) -> Tuple[object, object]:
    a = np.ascontiguousarray(np.asarray(seq, dtype=np.int32))
    return a, a.ctypes.data_as(_i32p)


def _cmat(m) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(m, dtype=np.complex128))


# ---- state ----------------------------------------------------------------

def qsa_state_create(n_qubits: int, dtype: int = QSA_C64) -> int:
    h = _vp()
    _check(_f["qsa_state_create"](n_qubits, dtype, _c.byref(h)))
    return h.value


def qsa_state_create_ex(n_qubits: int, dev_ptr: int, nbytes: int, stream: int = 0, init_zero: int = 1,
                        dtype: int = QSA_C64) -> int:
    h = _vp()
    _check(_f["qsa_state_create_ex"](n_qubits, dtype, _vp(dev_ptr), nbytes, _vp(stream), init_zero, _c.byref(h)))
    return h.value


def qsa_state_destroy(s: int) -> None:
    _check(_f["qsa_state_destroy"](_vp(s)))


def qsa_set_stream(s: int, stream: int) -> None:
    _check(_f["qsa_set_stream"](_vp(s), _vp(stream)))


def qsa_state_reset(s: int) -> None:
    _check(_f["qsa_state_reset"](_vp(s)))


def qsa_state_info(s: int) -> Tuple[int, int]:
    n = _c.c_int()
    p = _vp()
    _check(_f["qsa_state_info"](_vp(s), _c.byref(n), _c.byref(p)))
    return n.value, p.value


def qsa_set_layout(s: int, phys_of_logical: Sequence[int], materialise: int = 1) -> None:
    a, p = _i32(phys_of_logical)
    _check(_f["qsa_set_layout"](_vp(s), p, materialise))


def qsa_get_layout(s: int) -> List[int]:
    n, _ = qsa_state_info(s)
    a = np.zeros(n, dtype=np.int32)
    _check(_f["qsa_get_layout"](_vp(s), a.ctypes.data_as(_i32p)))
    return [int(v) for v in a]


def qsa_permute_bits(s: int, phys_a: Sequence[int], phys_b: Sequence[int]) -> None:
    a, pa = _i32(phys_a)
    b, pb = _i32(phys_b)
    _check(_f["qsa_permute_bits"](_vp(s), pa, pb, len(a)))


def qsa_apply_fused(s: int, targets: Sequence[int], matrix) -> None:
    t, pt = _i32(targets)
    m = _cmat(matrix)
    _check(_f["qsa_apply_fused"](_vp(s), pt, len(t), m.view(np.float64).ctypes.data_as(_dp)))


def qsa_apply_fused_ex(s: int, targets: Sequence[int], matrix, lowering: int, precision: int) -> None:
    t, pt = _i32(targets)
    m = _cmat(matrix)
    _check(_f["qsa_apply_fused_ex"](_vp(s), pt, len(t), m.view(np.float64).ctypes.data_as(_dp), lowering,
                                    precision))


def qsa_apply_product(s: int, targets: Sequence[int], factors) -> None:
    """Product of 2x2 factors, factor j on targets[j]."""
    t, pt = _i32(targets)
    f = np.ascontiguousarray(np.asarray(factors, dtype=np.complex128).reshape(len(t), 2, 2))
    _check(_f["qsa_apply_product"](_vp(s), pt, len(t), f.view(np.float64).ctypes.data_as(_dp)))


def qsa_apply_layer(s: int, diag_ops, targets: Sequence[int], factors) -> None:
    """Diagonal ops (objects with ``targets`` and a diagonal ``matrix``, k = 1
    or 2), then the 2x2 factor j on targets[j], in one layer block."""
    oa = diag_ops if isinstance(diag_ops, OpArray) else OpArray(list(diag_ops))
    t = np.ascontiguousarray(np.asarray(list(targets), dtype=np.int32))
    f = np.ascontiguousarray(np.asarray(factors, dtype=np.complex128).reshape(len(t), 2, 2)) if len(t) else \
        np.zeros((1, 2, 2), dtype=np.complex128)
    _check(_f["qsa_apply_layer"](_vp(s), _c.cast(oa.arr, _vp) if oa.n else None, oa.n,
                                 t.ctypes.data_as(_i32p) if len(t) else None, len(t),
                                 f.view(np.float64).ctypes.data_as(_dp)))


def qsa_apply_diag(s: int, targets: Sequence[int], diag) -> None:
    """Diagonal operator on ``targets``: ``diag`` holds 2^k complex entries,
    entry c for the target bits c (bit j = target j)."""
    t, pt = _i32(targets)
    d = np.ascontiguousarray(np.asarray(diag, dtype=np.complex128).reshape(-1))
    if d.size != (1 << len(t)):
        raise ValueError("diag must have 2^k entries")
    _check(_f["qsa_apply_diag"](_vp(s), pt, len(t), d.view(np.float64).ctypes.data_as(_dp)))


# ---- circuits ---------------------------------------------------------------

class OpArray:
    """A qsa_op[] built from objects with ``targets``, ``matrix`` (complex,
    2^k x 2^k) and optional ``diag``; the matrices are copied into one
    contiguous buffer that the array keeps alive.  The records are filled
    through a numpy view of the C layout (per-op ctypes calls cost several
    microseconds each)."""

    _dtype = np.dtype({"names": ["k", "targets", "matrix", "flags"],
                       "formats": ["<i4", ("<i4", 6), "<u8", "<u4"],
                       "offsets": [qsa_op.k.offset, qsa_op.targets.offset, qsa_op.matrix.offset,
                                   qsa_op.flags.offset],
                       "itemsize": _c.sizeof(qsa_op)})

    def __init__(self, ops: Iterable):
        ops = list(ops)
        n = len(ops)
        targets = [o.targets for o in ops]
        ks = np.fromiter(map(len, targets), dtype=np.int64, count=n)
        flat = [np.asarray(o.matrix, dtype=np.complex128).ravel() for o in ops]
        dims = np.left_shift(1, 2 * ks)
        if not np.array_equal(np.fromiter(map(len, flat), dtype=np.int64, count=n), dims):
            raise ValueError("every op's matrix must be 2^k x 2^k for its k targets")
        offs = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(dims, out=offs[1:])
        self.mats = np.concatenate(flat) if n else np.empty(1, dtype=np.complex128)
        tg = np.zeros((max(1, n), 6), dtype=np.int32)
        nt = int(offs.size and ks.sum())
        if nt:   # row i, columns 0..k_i - 1 from the flattened target lists
            rows = np.repeat(np.arange(n), ks)
            cols = np.arange(nt) - np.repeat(np.cumsum(ks) - ks, ks)
            tg[rows, cols] = np.fromiter(itertools.chain.from_iterable(targets), dtype=np.int32, count=nt)
        rec = np.zeros(max(1, n), dtype=self._dtype)
        rec["k"][:n] = ks
        rec["targets"] = tg
        rec["matrix"][:n] = self.mats.ctypes.data + 16 * offs[:n]
        rec["flags"][:n] = [QSA_OP_DIAG if getattr(o, "diag", False) else 0 for o in ops]
        self.rec = rec
        self.arr = (qsa_op * max(1, n)).from_buffer(rec)
        self.n = n


def qsa_plan_opts_default() -> qsa_plan_opts:
    o = qsa_plan_opts()
    _f["qsa_plan_opts_default"](_c.byref(o))
    return o


def make_opts(**kw) -> qsa_plan_opts:
    o = qsa_plan_opts_default()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def qsa_plan_circuit(ops, n_qubits: int, opts: Optional[qsa_plan_opts] = None) -> List[int]:
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    starts = (_c.c_size_t * max(1, oa.n))()
    nb = _c.c_size_t()
    _check(_f["qsa_plan_circuit"](oa.arr, oa.n, n_qubits, _c.byref(opts) if opts else None, starts, _c.byref(nb)))
    return [int(starts[i]) for i in range(nb.value)]


def qsa_fuse_ops(ops) -> Tuple[List[int], np.ndarray]:
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    t = (_c.c_int32 * 6)()
    w = _c.c_int()
    m = np.zeros(2 * 4096, dtype=np.float64)
    _check(_f["qsa_fuse_ops"](oa.arr, oa.n, t, _c.byref(w), m.ctypes.data_as(_dp)))
    u = w.value
    M = m[: 2 * 4 ** u].view(np.complex128).reshape(1 << u, 1 << u).copy()
    return [int(t[j]) for j in range(u)], M


def qsa_apply_circuit(s: int, ops, opts: Optional[qsa_plan_opts] = None) -> dict:
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    st = qsa_run_stats()
    _check(_f["qsa_apply_circuit"](_vp(s), oa.arr, oa.n, _c.byref(opts) if opts else None, _c.byref(st)))
    return st.as_dict()


def qsa_plan_create(ops, n_qubits: int, opts: Optional[qsa_plan_opts] = None, layout=None) -> int:
    oa = ops if isinstance(ops, OpArray) else OpArray(ops)
    h = _vp()
    lay = None
    if layout is not None:
        la, lay = _i32(layout)
    _check(_f["qsa_plan_create"](oa.arr, oa.n, n_qubits, _c.byref(opts) if opts else None, lay, _c.byref(h)))
    return h.value


def qsa_plan_info(p: int) -> dict:
    nb, no, mb = _c.c_size_t(), _c.c_size_t(), _c.c_size_t()
    mw = _c.c_int()
    _check(_f["qsa_plan_info"](_vp(p), _c.byref(nb), _c.byref(no), _c.byref(mw), _c.byref(mb)))
    return {"blocks": nb.value, "ops": no.value, "max_width": mw.value, "matrix_bytes": mb.value}


def qsa_plan_blocks(p: int) -> Tuple[List[int], List[int]]:
    nb = qsa_plan_info(p)["blocks"]
    fo = (_c.c_size_t * max(1, nb))()
    w = np.zeros(max(1, nb), dtype=np.int32)
    _check(_f["qsa_plan_blocks"](_vp(p), fo, w.ctypes.data_as(_i32p), nb))
    return [int(fo[i]) for i in range(nb)], [int(v) for v in w[:nb]]


def qsa_plan_order(p: int) -> List[int]:
    """Execution order of the input ops (moved by layer grouping)."""
    n = qsa_plan_info(p)["ops"]
    o = (_c.c_size_t * max(1, n))()
    _check(_f["qsa_plan_order"](_vp(p), _c.cast(o, _vp), n))
    return [int(o[i]) for i in range(n)]


def qsa_plan_block_kinds(p: int) -> Tuple[List[int], List[int]]:
    """Per block: kind (0 dense, 1 diagonal, 2 product, 3 layer) and the size
    of a layer block's diagonal part."""
    nb = qsa_plan_info(p)["blocks"]
    k = np.zeros(max(1, nb), dtype=np.int32)
    d = np.zeros(max(1, nb), dtype=np.int32)
    _check(_f["qsa_plan_block_kinds"](_vp(p), k.ctypes.data_as(_i32p), d.ctypes.data_as(_i32p), nb))
    return [int(v) for v in k[:nb]], [int(v) for v in d[:nb]]


def qsa_plan_promotions(p: int, n_qubits: int, victim: int, layout=None) -> Tuple[int, int, List[int]]:
    """Host replay of the plan's QSA_LOWER_PERMUTE promotions: (promoted
    position pairs, permutation passes, final layout)."""
    lay = None
    if layout is not None:
        la, lay = _i32(layout)
    pr, ps = _c.c_uint64(), _c.c_uint64()
    out = np.zeros(n_qubits, dtype=np.int32)
    _check(_f["qsa_plan_promotions"](_vp(p), lay, victim, _c.byref(pr), _c.byref(ps), out.ctypes.data_as(_i32p)))
    return int(pr.value), int(ps.value), [int(v) for v in out]


class qsa_exchange(_c.Structure):
    _fields_ = [("block", _c.c_uint64), ("rank_pos", _c.c_int32), ("local_pos", _c.c_int32)]


_f["qsa_plan_exchanges"] = _sig("qsa_plan_exchanges", [_vp, _c.c_int, _i32p, _c.c_int, _c.POINTER(qsa_exchange),
                                                       _c.c_size_t, _szp, _i32p])


def qsa_plan_exchanges(p: int, n_qubits: int, rank_bits: int, layout=None, victim: int = 0):
    """(list of (block, rank_pos, local_pos), final layout) of running plan p
    on 2^rank_bits ranks."""
    n = n_qubits
    lay = (_c.c_int32 * n)(*layout) if layout is not None else None
    cnt = _c.c_size_t()
    out_l = (_c.c_int32 * n)()
    rc = _f["qsa_plan_exchanges"](_vp(p), rank_bits, lay, victim, None, 0, _c.byref(cnt), out_l)
    if rc not in (QSA_OK, QSA_E_RANGE):
        _check(rc)
    buf = (qsa_exchange * max(1, cnt.value))()
    _check(_f["qsa_plan_exchanges"](_vp(p), rank_bits, lay, victim, buf, cnt.value, _c.byref(cnt), out_l))
    return [(int(buf[i].block), int(buf[i].rank_pos), int(buf[i].local_pos)) for i in range(cnt.value)], list(out_l)


def qsa_plan_execute(s: int, p: int) -> dict:
    st = qsa_run_stats()
    _check(_f["qsa_plan_execute"](_vp(s), _vp(p), _c.byref(st)))
    return st.as_dict()


def qsa_plan_execute_from_zero(s: int, p: int) -> dict:
    """Run the plan from |0...0> (in the plan's layout), discarding the state."""
    st = qsa_run_stats()
    _check(_f["qsa_plan_execute_from_zero"](_vp(s), _vp(p), _c.byref(st)))
    return st.as_dict()


def qsa_plan_destroy(p: int) -> None:
    _check(_f["qsa_plan_destroy"](_vp(p)))


def qsa_state_sync(s: int) -> None:
    _check(_f["qsa_state_sync"](_vp(s)))


def qsa_state_counters(s: int) -> int:
    v = _c.c_uint64()
    _check(_f["qsa_state_counters"](_vp(s), _c.byref(v)))
    return v.value


# ---- outputs ------------------------------------------------------------------

def qsa_probabilities(s: int, want_probs: bool = True) -> Tuple[Optional[np.ndarray], float]:
    n, _ = qsa_state_info(s)
    norm = _c.c_double()
    out = np.empty(1 << n, dtype=np.float64) if want_probs else None
    _check(_f["qsa_probabilities"](_vp(s), out.ctypes.data_as(_dp) if want_probs else None, _c.byref(norm)))
    return out, norm.value


def qsa_probabilities_device(s: int, out_dev_ptr: int) -> float:
    norm = _c.c_double()
    _check(_f["qsa_probabilities_device"](_vp(s), _vp(out_dev_ptr), _c.byref(norm)))
    return norm.value


def qsa_expectation_z(s: int, logical_mask: int) -> float:
    out = _c.c_double()
    _check(_f["qsa_expectation_z"](_vp(s), _c.c_uint64(logical_mask), _c.byref(out)))
    return out.value


# ---- density matrices ---------------------------------------------------------

def qsa_dm_apply_channel(s: int, n: int, targets: Sequence[int], kraus, precision: int = 0) -> None:
    """rho <- sum_i E_i rho E_i^dagger on the n-qubit density matrix held by
    the 2n-qubit state ``s``; ``kraus`` is one 2^k x 2^k matrix or a stack."""
    t, pt = _i32(targets)
    d = 1 << len(t)
    e = np.ascontiguousarray(np.asarray(kraus, dtype=np.complex128).reshape(-1, d, d))
    _check(_f["qsa_dm_apply_channel"](_vp(s), n, pt, len(t), e.view(np.float64).ctypes.data_as(_dp), e.shape[0],
                                      precision))


class DensityOp:
    """A channel lowered to one 2k-qubit operator of vec(rho) (the op shape the
    planner takes: ``targets``, ``matrix``)."""

    def __init__(self, targets, matrix):
        self.targets = tuple(int(t) for t in targets)
        self.matrix = matrix
        self.diag = False


def qsa_dm_superoperator(n: int, targets: Sequence[int], kraus) -> DensityOp:
    """sum_i conj(E_i) (x) E_i on (targets, targets + n), built by the library."""
    t, pt = _i32(targets)
    k = len(t)
    d = 1 << k
    e = np.ascontiguousarray(np.asarray(kraus, dtype=np.complex128).reshape(-1, d, d))
    to = np.zeros(2 * k, dtype=np.int32)
    m = np.zeros((d * d, d * d), dtype=np.complex128)
    _check(_f["qsa_dm_superoperator"](n, pt, k, e.view(np.float64).ctypes.data_as(_dp), e.shape[0],
                                      to.ctypes.data_as(_i32p), m.view(np.float64).ctypes.data_as(_dp)))
    return DensityOp(to, m)


def qsa_dm_probabilities(s: int, n: int, want_probs: bool = True) -> Tuple[Optional[np.ndarray], float]:
    """Diagonal of rho in logical order and its trace."""
    tr = _c.c_double()
    out = np.empty(1 << n, dtype=np.float64) if want_probs else None
    _check(_f["qsa_dm_probabilities"](_vp(s), n, out.ctypes.data_as(_dp) if want_probs else None, _c.byref(tr)))
    return out, tr.value


def qsa_dm_expectation_z(s: int, n: int, mask: int) -> float:
    out = _c.c_double()
    _check(_f["qsa_dm_expectation_z"](_vp(s), n, _c.c_uint64(mask), _c.byref(out)))
    return out.value


def qsa_expectation_z_batch(s: int, logical_masks) -> List[float]:
    m = np.ascontiguousarray(np.asarray(list(logical_masks), dtype=np.uint64))
    out = np.zeros(len(m), dtype=np.float64)
    _check(_f["qsa_expectation_z_batch"](_vp(s), m.ctypes.data_as(_u64p), len(m), out.ctypes.data_as(_dp)))
    return [float(v) for v in out]


def qsa_sample_counts(s: int, shots: int, seed: int, capacity: Optional[int] = None) -> Tuple[np.ndarray, np.ndarray]:
    cap = shots if capacity is None else capacity
    outc = np.zeros(max(1, cap), dtype=np.uint64)
    cnt = np.zeros(max(1, cap), dtype=np.uint64)
    nd = _c.c_size_t()
    _check(_f["qsa_sample_counts"](_vp(s), shots, _c.c_uint64(seed), outc.ctypes.data_as(_u64p),
                                   cnt.ctypes.data_as(_u64p), cap, _c.byref(nd)))
    return outc[: nd.value].copy(), cnt[: nd.value].copy()


def qsa_measure(s: int, z_masks, shots: int, seed: int, capacity: Optional[int] = None):
    """(<Z_mask> for each mask, outcomes, counts) from one pass over the state."""
    cap = shots if capacity is None else capacity
    m = np.ascontiguousarray(np.asarray(list(z_masks), dtype=np.uint64))
    z = np.zeros(max(1, len(m)), dtype=np.float64)
    outc = np.zeros(max(1, cap), dtype=np.uint64)
    cnt = np.zeros(max(1, cap), dtype=np.uint64)
    nd = _c.c_size_t()
    _check(_f["qsa_measure"](_vp(s), m.ctypes.data_as(_u64p) if len(m) else None, len(m),
                             z.ctypes.data_as(_dp) if len(m) else None, shots, _c.c_uint64(seed),
                             outc.ctypes.data_as(_u64p), cnt.ctypes.data_as(_u64p), cap, _c.byref(nd)))
    return [float(v) for v in z[: len(m)]], outc[: nd.value].copy(), cnt[: nd.value].copy()


# ---- cost model -------------------------------------------------------------

def qsa_costmodel_features(k: int, phys_mask: int, n_qubits: int, batch: int = 1) -> np.ndarray:
    x = np.zeros(MLP_IN, dtype=np.float32)
    _check(_f["qsa_costmodel_features"](k, _c.c_uint64(phys_mask), n_qubits, batch, x.ctypes.data_as(_fp)))
    return x


def qsa_costmodel_set(params: Optional[np.ndarray]) -> None:
    if params is None:
        _check(_f["qsa_costmodel_set"](None))
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == MLP_PARAMS
    _check(_f["qsa_costmodel_set"](p.ctypes.data_as(_fp)))


def qsa_costmodel_predict(features: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, MLP_IN)
    out = np.zeros(X.shape[0], dtype=np.float64)
    _check(_f["qsa_costmodel_predict"](X.ctypes.data_as(_fp), X.shape[0], out.ctypes.data_as(_dp)))
    return out


_f["qsa_costmodel_init"] = _sig("qsa_costmodel_init", [_c.c_uint64, _fp])
_f["qsa_mlp_workspace_bytes"] = _sig("qsa_mlp_workspace_bytes", [_c.c_size_t], _c.c_size_t)
_f["qsa_mlp_forward"] = _sig("qsa_mlp_forward", [_vp, _vp, _c.c_size_t, _vp, _vp, _vp])
_f["qsa_mlp_loss_grad"] = _sig("qsa_mlp_loss_grad", [_vp, _vp, _vp, _c.c_size_t, _vp, _vp, _vp, _vp])
_f["qsa_mlp_adam_step"] = _sig("qsa_mlp_adam_step", [_vp, _vp, _vp, _vp, _c.c_size_t, _c.c_int, _c.c_float,
                                                     _c.c_float, _c.c_float, _c.c_float, _vp])
_f["qsa_costmodel_collect"] = _sig("qsa_costmodel_collect", [_vp, _c.c_size_t, _c.c_int, _c.c_int, _c.c_uint64,
                                                             _fp, _fp])
_f["qsa_costmodel_train"] = _sig("qsa_costmodel_train", [_fp, _fp, _c.c_size_t, _c.c_int, _c.c_int, _c.c_float,
                                                         _c.c_float, _c.c_uint64, _fp, _fp])


_f["qsa_costmodel_save"] = _sig("qsa_costmodel_save", [_c.c_char_p])
_f["qsa_costmodel_load"] = _sig("qsa_costmodel_load", [_vp, _c.c_char_p])
_f["qsa_debug_fail_alloc"] = _sig("qsa_debug_fail_alloc", [_c.c_int64])
_f["qsa_debug_live_allocations"] = _sig("qsa_debug_live_allocations", [], _c.c_uint64)
_f["qsa_debug_bounds_status"] = _sig("qsa_debug_bounds_status", [], _c.c_uint64)
_f["qsa_debug_bounds_enabled"] = _sig("qsa_debug_bounds_enabled", [], _c.c_int)


def qsa_costmodel_save(path: str) -> None:
    _check(_f["qsa_costmodel_save"](os.fsencode(path)))


def qsa_costmodel_load(s: Optional[int], path: Optional[str]) -> None:
    """s = None: install process-wide; else attach to state s.  path = None removes."""
    _check(_f["qsa_costmodel_load"](_vp(s) if s else None, os.fsencode(path) if path is not None else None))


def qsa_debug_fail_alloc(nth: int) -> None:
    _check(_f["qsa_debug_fail_alloc"](nth))


def qsa_debug_live_allocations() -> int:
    return int(_f["qsa_debug_live_allocations"]())


def qsa_debug_bounds_status() -> Tuple[int, int]:
    """(check code, index) of the first failed bounds check, (0, 0) if none."""
    w = int(_f["qsa_debug_bounds_status"]())
    return w >> 48, w & ((1 << 48) - 1)


def qsa_debug_bounds_enabled() -> bool:
    return bool(_f["qsa_debug_bounds_enabled"]())


def qsa_costmodel_init(seed: int) -> np.ndarray:
    p = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(_f["qsa_costmodel_init"](_c.c_uint64(seed), p.ctypes.data_as(_fp)))
    return p


def qsa_mlp_workspace_bytes(n: int) -> int:
    return int(_f["qsa_mlp_workspace_bytes"](n))


def qsa_mlp_forward(params_dev: int, X_dev: int, n: int, y_dev: int, ws_dev: int, stream: int = 0) -> None:
    _check(_f["qsa_mlp_forward"](_vp(params_dev), _vp(X_dev), n, _vp(y_dev), _vp(ws_dev), _vp(stream)))


def qsa_mlp_loss_grad(params_dev: int, X_dev: int, t_dev: int, n: int, grads_dev: int, loss_dev: int, ws_dev: int,
                      stream: int = 0) -> None:
    _check(_f["qsa_mlp_loss_grad"](_vp(params_dev), _vp(X_dev), _vp(t_dev), n, _vp(grads_dev), _vp(loss_dev),
                                   _vp(ws_dev), _vp(stream)))


def qsa_mlp_adam_step(params_dev: int, grads_dev: int, m_dev: int, v_dev: int, count: int, step: int,
                      lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                      stream: int = 0) -> None:
    _check(_f["qsa_mlp_adam_step"](_vp(params_dev), _vp(grads_dev), _vp(m_dev), _vp(v_dev), count, step, lr, beta1,
                                   beta2, eps, _vp(stream)))


def qsa_costmodel_collect(s: int, n_samples: int, reps: int = 3, precision: int = QSA_PREC_FP32,
                          seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    X = np.zeros((n_samples, MLP_IN), dtype=np.float32)
    y = np.zeros(n_samples, dtype=np.float32)
    _check(_f["qsa_costmodel_collect"](_vp(s), n_samples, reps, precision, _c.c_uint64(seed),
                                       X.ctypes.data_as(_fp), y.ctypes.data_as(_fp)))
    return X, y


def qsa_costmodel_train(X: np.ndarray, y: np.ndarray, epochs: int = 200, batch: int = 64, lr: float = 1e-3,
                        seed: int = 0, params: Optional[np.ndarray] = None,
                        weight_decay: float = 1e-2) -> Tuple[np.ndarray, np.ndarray]:
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    p = qsa_costmodel_init(seed) if params is None else np.ascontiguousarray(params, dtype=np.float32).copy()
    losses = np.zeros(epochs, dtype=np.float32)
    _check(_f["qsa_costmodel_train"](X.ctypes.data_as(_fp), y.ctypes.data_as(_fp), X.shape[0], epochs, batch, lr,
                                     weight_decay, _c.c_uint64(seed), p.ctypes.data_as(_fp),
                                     losses.ctypes.data_as(_fp)))
    return p, losses


_f["qsa_batch_create"] = _sig("qsa_batch_create", [_c.c_int, _c.c_int, _c.POINTER(qsa_op), _szp,
                                                   _c.POINTER(qsa_plan_opts), _c.POINTER(_vp)])
_f["qsa_batch_info"] = _sig("qsa_batch_info", [_vp, _szp, _szp, _u64p])
_f["qsa_batch_run"] = _sig("qsa_batch_run", [_vp, _vp, _c.c_size_t, _c.c_uint64, _c.c_uint64, _c.c_uint64, _c.c_int,
                                             _vp, _c.POINTER(qsa_run_stats)])
_f["qsa_batch_counts"] = _sig("qsa_batch_counts", [_vp, _vp, _vp, _vp])
_f["qsa_batch_destroy"] = _sig("qsa_batch_destroy", [_vp])


def qsa_batch_create(n_qubits: int, trajectories, opts: Optional[qsa_plan_opts] = None) -> int:
    """``trajectories``: list of op lists."""
    flat = [op for t in trajectories for op in t]
    offs = np.zeros(len(trajectories) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(t) for t in trajectories])
    oa = OpArray(flat)
    h = _vp()
    _check(_f["qsa_batch_create"](n_qubits, len(trajectories), oa.arr, offs.ctypes.data_as(_szp),
                                  _c.byref(opts) if opts else None, _c.byref(h)))
    return h.value


def qsa_batch_info(b: int) -> dict:
    tb, to = _c.c_size_t(), _c.c_size_t()
    la = _c.c_uint64()
    _check(_f["qsa_batch_info"](_vp(b), _c.byref(tb), _c.byref(to), _c.byref(la)))
    return {"blocks": tb.value, "ops": to.value, "launches": la.value}


def qsa_batch_run(b: int, states_ptr: int, nbytes: int, shots: int, seed: int, budget_cycles: int = 0,
                  use_graph: int = 1, stream: int = 0) -> dict:
    st = qsa_run_stats()
    _check(_f["qsa_batch_run"](_vp(b), _vp(states_ptr), nbytes, shots, _c.c_uint64(seed), _c.c_uint64(budget_cycles),
                               use_graph, _vp(stream), _c.byref(st)))
    return st.as_dict()


def qsa_batch_counts(b: int, n_traj: int, shots: int):
    """Per trajectory: (outcomes ascending, counts) as uint32 arrays."""
    outc = np.zeros(n_traj * shots, dtype=np.uint32)
    cnt = np.zeros(n_traj * shots, dtype=np.uint32)
    nd = np.zeros(n_traj, dtype=np.uint32)
    _check(_f["qsa_batch_counts"](_vp(b), _vp(outc.ctypes.data), _vp(cnt.ctypes.data), _vp(nd.ctypes.data)))
    return [(outc[t * shots: t * shots + nd[t]].copy(), cnt[t * shots: t * shots + nd[t]].copy())
            for t in range(n_traj)]


def qsa_batch_destroy(b: int) -> None:
    _check(_f["qsa_batch_destroy"](_vp(b)))


def exported_symbols() -> List[str]:
    return sorted(k for k in _f)
