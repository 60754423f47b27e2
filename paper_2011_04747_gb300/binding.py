"""Thin ctypes binding of libdaeti (argument marshalling only).

Every ``daeti_*`` function here has the name and meaning of the C entry point
declared in ``include/daeti.h`` and only converts Python arguments (numpy
arrays, torch tensors, streams) into pointers and sizes.  All computation runs
in the library's CUDA kernels; there is no Python or CPU fallback, and
importing the binding without a built ``libdaeti.so`` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdaeti.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, EUNSTABLE, ENONFINITE = range(7)
EUNSUPPORTED = 8   # 7 is unused
FP64, FP32_KAHAN, FP32 = 0, 1, 2
SCHEME_DAETI, SCHEME_OSTAR, SCHEME_OST = 0, 1, 2
L_FLOOR, L_CEIL = 0, 1
MODEL_MS, MODEL_TP06 = 1, 2
DTYPE_F64, DTYPE_F32 = 0, 1
KERNEL_REACTION, KERNEL_DIFFUSION, KERNEL_OTHER = 0, 1, 2
ADJ_RECORD, ADJ_REPLAY, ADJ_NO_GRADIENT, NODAL_GRADIENT = 1, 2, 4, 8
K_TOTAL, K_REACTION = 0, 1

_PREC = {"fp64": FP64, "fp32_kahan": FP32_KAHAN, "fp32": FP32}
_SCHEME = {"daeti": SCHEME_DAETI, "ostar": SCHEME_OSTAR, "ost": SCHEME_OST}
_MODEL = {"ms": MODEL_MS, "tp06": MODEL_TP06}


class DaetiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libdaeti error {code}: {msg}")
        self.code = code


class daeti_options(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
        ("l_rounding", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("dt0", ctypes.c_double),
        ("v_threshold", ctypes.c_double),
        ("gate_rush_larsen", ctypes.c_int32),
        ("bucket_k", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("react_block", ctypes.c_int32),
        ("diff_block", ctypes.c_int32),
        ("fuse_diffusion", ctypes.c_int32),
        ("k_rule", ctypes.c_int32),
    ]


class daeti_tuning(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int32),
        ("react_block", ctypes.c_int32),
        ("react_min_blocks", ctypes.c_int32),
        ("diff_block", ctypes.c_int32),
        ("fuse_diffusion", ctypes.c_int32),
        ("bucket_k", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("pdl", ctypes.c_int32),
        ("diff_rows", ctypes.c_int32),
    ]


TUNING_FIELDS = ("react_block", "react_min_blocks", "diff_block", "fuse_diffusion", "bucket_k", "graph_steps",
                 "pdl", "diff_rows")

_lib = None

_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

_SIGNATURES = {
    "daeti_default_options": (None, [ctypes.POINTER(daeti_options)]),
    "daeti_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(daeti_options)]),
    "daeti_destroy": (ctypes.c_int, [_VP]),
    "daeti_last_error": (ctypes.c_char_p, [_VP]),
    "daeti_set_stream": (ctypes.c_int, [_VP, _VP]),
    "daeti_set_mesh_grid": (ctypes.c_int, [_VP, ctypes.c_int, _I64P, ctypes.c_double]),
    "daeti_set_mesh_tet": (ctypes.c_int, [_VP, ctypes.c_int64, _DP, ctypes.c_int64, _I64P]),
    "daeti_set_conductivity": (ctypes.c_int, [_VP, ctypes.c_int64, _DP, _DP, _DP]),
    "daeti_set_conductivity_nodal": (ctypes.c_int, [_VP, ctypes.c_int64, _DP, _DP, _DP]),
    "daeti_set_cell_model": (ctypes.c_int, [_VP, ctypes.c_int, _DP, ctypes.c_int]),
    "daeti_set_cell_types": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint8)]),
    "daeti_add_stimulus": (ctypes.c_int, [_VP, _I64P, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int]),
    "daeti_prepare": (ctypes.c_int, [_VP]),
    "daeti_get_stability": (ctypes.c_int, [_VP, _DP, _DP, _IP, _IP, _DP]),
    "daeti_get_sizes": (ctypes.c_int, [_VP, _I64P, _IP]),
    "daeti_init_state": (ctypes.c_int, [_VP, _DP]),
    "daeti_advance": (ctypes.c_int, [_VP, ctypes.c_double]),
    "daeti_synchronize": (ctypes.c_int, [_VP]),
    "daeti_get_time": (ctypes.c_int, [_VP, _DP, _I64P]),
    "daeti_read_v": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int]),
    "daeti_read_activation": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int]),
    "daeti_read_v_nodes": (ctypes.c_int, [_VP, _I64P, ctypes.c_int64, _DP]),
    "daeti_read_state": (ctypes.c_int, [_VP, _DP]),
    "daeti_state_bytes": (ctypes.c_int, [_VP, _I64P]),
    "daeti_save_state": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
    "daeti_load_state": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
    "daeti_get_substeps": (ctypes.c_int, [_VP, _I64P]),
    "daeti_get_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(daeti_tuning)]),
    "daeti_set_tuning": (ctypes.c_int, [_VP, ctypes.POINTER(daeti_tuning)]),
    "daeti_set_profiling": (ctypes.c_int, [_VP, ctypes.c_int]),
    "daeti_time_launches": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _DP]),
    "daeti_update_cell_params": (ctypes.c_int, [_VP, _DP, ctypes.c_int]),
    "daeti_get_kernel_time": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _I64P]),
    "daeti_kernel_work": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _DP]),
    "daeti_update_conductivity": (ctypes.c_int, [_VP, ctypes.c_int64, _DP, _DP, _DP]),
    "daeti_update_conductivity_nodal": (ctypes.c_int, [_VP, ctypes.c_int64, _DP, _DP, _DP]),
    "daeti_adjoint": (ctypes.c_int, [_VP, _I64P, ctypes.c_int, ctypes.c_int, _DP, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_int, _DP, _DP, _DP]),
    "daeti_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(daeti_options)]),
    "daeti_batch_destroy": (ctypes.c_int, [_VP]),
    "daeti_batch_last_error": (ctypes.c_char_p, [_VP]),
    "daeti_batch_set_stream": (ctypes.c_int, [_VP, _VP]),
    "daeti_batch_add": (ctypes.c_int, [_VP, _VP]),
    "daeti_batch_prepare": (ctypes.c_int, [_VP]),
    "daeti_batch_advance": (ctypes.c_int, [_VP, ctypes.c_double]),
    "daeti_batch_synchronize": (ctypes.c_int, [_VP]),
    "daeti_batch_info": (ctypes.c_int, [_VP, _I64P, _IP, _IP, _DP]),
    "daeti_batch_read_v": (ctypes.c_int, [_VP, ctypes.c_int, _DP]),
    "daeti_batch_read_activation": (ctypes.c_int, [_VP, ctypes.c_int, _DP]),
    "daeti_grid_stability_noalloc": (ctypes.c_int, [ctypes.c_int, _I64P, ctypes.c_double, ctypes.c_int64, _DP, _DP,
                                                    _DP, _VP, _DP, _DP, ctypes.c_char_p, ctypes.c_int]),
}


def load_library(path: str = LIB_PATH):
    """Load libdaeti.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdaeti.so not built at {path}; run paper_2011_04747_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    return sorted(_SIGNATURES)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _cond(d_long, d_trans, fibre, n_fibre=None):
    """Conductivity arrays as float64, with the lengths the C side reads
    checked here (it reads d_trans[e] for every entry of d_long and three
    fibre components for each of n_fibre elements, default len(d_long))."""
    dl = _f64(d_long).reshape(-1)
    dtr = _f64(d_trans).reshape(-1) if d_trans is not None else None
    fb = _f64(fibre).reshape(-1) if fibre is not None else None
    if dtr is not None and dtr.shape != dl.shape:
        raise DaetiError(EINVAL, f"d_trans has {dtr.shape[0]} entries, d_long {dl.shape[0]}")
    nf = dl.shape[0] if n_fibre is None else int(n_fibre)
    if fb is not None and fb.shape[0] != 3 * nf:
        raise DaetiError(EINVAL, f"fibre needs 3 x {nf} entries, got {fb.shape[0]}")
    return dl, dtr, fb


class Solver:
    """One tissue on the GPU: owns a ``daeti_ctx``.

    Methods map one to one onto the C entry points of the same name.
    """

    def __init__(self, precision="fp32_kahan", scheme="daeti", dt=0.1, dt0=0.01, l_rounding="floor",
                 v_threshold: Optional[float] = None, gate_rush_larsen=True, bucket_k=True, graph_steps=20,
                 react_block=0, diff_block=0, fuse_diffusion=True, k_rule="total", stream=None):
        self.lib = load_library()
        o = daeti_options()
        self.lib.daeti_default_options(ctypes.byref(o))
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.scheme = _SCHEME[scheme] if isinstance(scheme, str) else int(scheme)
        o.l_rounding = L_FLOOR if l_rounding == "floor" else L_CEIL
        o.dt = float(dt)
        o.dt0 = float(dt0)
        o.v_threshold = float("nan") if v_threshold is None else float(v_threshold)
        o.gate_rush_larsen = int(bool(gate_rush_larsen))
        o.bucket_k = int(bool(bucket_k))
        o.graph_steps = int(graph_steps)
        o.react_block = int(react_block)
        o.diff_block = int(diff_block)
        o.fuse_diffusion = int(bool(fuse_diffusion))
        o.k_rule = {"total": 0, "reaction": 1}[k_rule] if isinstance(k_rule, str) else int(k_rule)
        self.options = o
        self.precision = o.precision
        h = _VP()
        rc = self.lib.daeti_create(ctypes.byref(h), ctypes.byref(o))
        if rc != OK:
            raise DaetiError(rc, "daeti_create failed")
        self.ctx = h
        self.n_nodes = 0
        self.n_elem = 0
        self.n_states = 0
        if stream is not None:
            self.daeti_set_stream(stream)

    # -- helpers --------------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            msg = self.lib.daeti_last_error(self.ctx)
            raise DaetiError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.daeti_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points -----------------------------------------------------------
    def daeti_set_stream(self, stream):
        """stream: torch.cuda.Stream, a raw cudaStream_t int, or None (legacy default)."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.daeti_set_stream(self.ctx, _VP(int(handle) if handle else 0)))

    def daeti_set_mesh_grid(self, dim, n, h):
        nn = _i64(list(n) + [1] * (3 - len(n)))
        self._check(self.lib.daeti_set_mesh_grid(self.ctx, int(dim), _ptr(nn, ctypes.c_int64), float(h)))
        self.n_elem = int(np.prod([int(nn[d]) - 1 for d in range(int(dim))]))
        self._sizes()

    def daeti_set_mesh_tet(self, xyz, tets):
        x = _f64(xyz)
        t = _i64(tets)
        self._check(self.lib.daeti_set_mesh_tet(self.ctx, x.shape[0], _ptr(x, ctypes.c_double), t.shape[0],
                                                _ptr(t, ctypes.c_int64)))
        self.n_elem = int(t.shape[0])
        self._sizes()

    def daeti_set_conductivity(self, d_long, d_trans=None, fibre=None):
        dl, dtr, fb = _cond(d_long, d_trans, fibre)
        self._check(self.lib.daeti_set_conductivity(self.ctx, dl.shape[0], _ptr(dl, ctypes.c_double),
                                                    _ptr(dtr, ctypes.c_double), _ptr(fb, ctypes.c_double)))

    def daeti_set_cell_model(self, model, params=()):
        m = _MODEL[model] if isinstance(model, str) else int(model)
        p = _f64(params) if len(params) else None
        self._check(self.lib.daeti_set_cell_model(self.ctx, m, _ptr(p, ctypes.c_double), 0 if p is None else len(p)))
        self._sizes()

    def daeti_set_cell_types(self, types):
        """TP06 cell type per node (0 endo, 1 epi, 2 mid-myocardial)."""
        t = np.ascontiguousarray(types, dtype=np.uint8).reshape(-1)
        self._check(self.lib.daeti_set_cell_types(self.ctx, t.shape[0], _ptr(t, ctypes.c_uint8)))

    def daeti_add_stimulus(self, nodes, t_start, duration, amplitude, period=0.0, count=1):
        nd = _i64(nodes)
        self._check(self.lib.daeti_add_stimulus(self.ctx, _ptr(nd, ctypes.c_int64), nd.shape[0], float(t_start),
                                                float(duration), float(amplitude), float(period), int(count)))

    def daeti_prepare(self):
        self._check(self.lib.daeti_prepare(self.ctx))
        self._sizes()

    def daeti_get_stability(self):
        dts, lam, dte = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        l, km = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.daeti_get_stability(self.ctx, ctypes.byref(dts), ctypes.byref(lam), ctypes.byref(l),
                                                 ctypes.byref(km), ctypes.byref(dte)))
        return {"dt_s": dts.value, "lambda_max": lam.value, "l": l.value, "k_max": km.value, "dt": dte.value}

    def _sizes(self):
        n = ctypes.c_int64()
        s = ctypes.c_int()
        if self.lib.daeti_get_sizes(self.ctx, ctypes.byref(n), ctypes.byref(s)) == OK:
            self.n_nodes, self.n_states = n.value, s.value

    def daeti_init_state(self, state=None):
        st = None if state is None else _f64(state).reshape(-1)
        self._check(self.lib.daeti_init_state(self.ctx, _ptr(st, ctypes.c_double)))

    def daeti_advance(self, t_end):
        self._check(self.lib.daeti_advance(self.ctx, float(t_end)))

    def daeti_synchronize(self):
        self._check(self.lib.daeti_synchronize(self.ctx))

    def daeti_get_time(self):
        t = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self.lib.daeti_get_time(self.ctx, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def _read(self, fn, out, dtype):
        if out is not None and hasattr(out, "data_ptr"):           # torch tensor
            if out.is_cuda:
                dt = DTYPE_F32 if str(out.dtype) == "torch.float32" else DTYPE_F64
                self._check(fn(self.ctx, _VP(out.data_ptr()), dt, 1))
                return out
            arr = out.numpy()
            self._check(fn(self.ctx, arr.ctypes.data_as(_VP), DTYPE_F32 if arr.dtype == np.float32 else DTYPE_F64, 0))
            return out
        if out is None:
            out = np.empty(self.n_nodes, dtype=np.dtype(dtype))
        dt = DTYPE_F32 if out.dtype == np.float32 else DTYPE_F64
        self._check(fn(self.ctx, out.ctypes.data_as(_VP), dt, 0))
        return out

    def daeti_read_v(self, out=None, dtype=np.float64):
        return self._read(self.lib.daeti_read_v, out, dtype)

    def daeti_read_activation(self, out=None, dtype=np.float64):
        return self._read(self.lib.daeti_read_activation, out, dtype)

    def daeti_read_v_nodes(self, nodes):
        """V (double) at the given node indices."""
        idx = np.ascontiguousarray(nodes, dtype=np.int64)
        out = np.empty(idx.size, dtype=np.float64)
        self._check(self.lib.daeti_read_v_nodes(self.ctx, _ptr(idx, ctypes.c_int64), idx.size,
                                                _ptr(out, ctypes.c_double)))
        return out

    def daeti_read_state(self):
        out = np.empty(self.n_states * self.n_nodes, dtype=np.float64)
        self._check(self.lib.daeti_read_state(self.ctx, _ptr(out, ctypes.c_double)))
        return out.reshape(self.n_states, self.n_nodes)

    def daeti_save_state(self):
        nb = ctypes.c_int64()
        self._check(self.lib.daeti_state_bytes(self.ctx, ctypes.byref(nb)))
        buf = np.empty(nb.value, dtype=np.uint8)
        self._check(self.lib.daeti_save_state(self.ctx, buf.ctypes.data_as(_VP), nb.value))
        return buf

    def daeti_load_state(self, buf):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.lib.daeti_load_state(self.ctx, b.ctypes.data_as(_VP), b.shape[0]))

    def daeti_set_conductivity_nodal(self, d_long, d_trans=None, fibre=None):
        """Per-node d_long, d_trans (element value = mean of its nodes); fibre per element."""
        dl, dtr, fb = _cond(d_long, d_trans, fibre, self.n_elem)
        self._check(self.lib.daeti_set_conductivity_nodal(self.ctx, dl.shape[0], _ptr(dl, ctypes.c_double),
                                                          _ptr(dtr, ctypes.c_double), _ptr(fb, ctypes.c_double)))

    def daeti_update_conductivity_nodal(self, d_long, d_trans=None, fibre=None):
        dl, dtr, fb = _cond(d_long, d_trans, fibre, self.n_elem)
        self._check(self.lib.daeti_update_conductivity_nodal(self.ctx, dl.shape[0], _ptr(dl, ctypes.c_double),
                                                             _ptr(dtr, ctypes.c_double),
                                                             _ptr(fb, ctypes.c_double)))

    def daeti_update_conductivity(self, d_long, d_trans=None, fibre=None):
        dl, dtr, fb = _cond(d_long, d_trans, fibre)
        self._check(self.lib.daeti_update_conductivity(self.ctx, dl.shape[0], _ptr(dl, ctypes.c_double),
                                                       _ptr(dtr, ctypes.c_double), _ptr(fb, ctypes.c_double)))

    def daeti_adjoint(self, sensors, data, n_steps, sample_every, n_slots=32, flags=0, n_elem=None, nodal=False):
        """Returns (loss, dL/dD_e (n_elem,) or None, dL/dtau_close or None); with nodal,
        the gradient is per node (n_nodes,) for element D = mean of nodal D."""
        sn = _i64(sensors)
        dd = _f64(data).reshape(-1)
        loss = ctypes.c_double()
        gt = ctypes.c_double()
        grad = None if flags else np.empty(int(self.n_nodes if nodal else n_elem), dtype=np.float64)
        if nodal:
            flags |= NODAL_GRADIENT
        self._check(self.lib.daeti_adjoint(self.ctx, _ptr(sn, ctypes.c_int64), sn.shape[0], int(sample_every),
                                           _ptr(dd, ctypes.c_double), int(n_steps), int(n_slots), int(flags),
                                           ctypes.byref(loss), _ptr(grad, ctypes.c_double), ctypes.byref(gt)))
        return loss.value, grad, (None if grad is None else gt.value)

    def daeti_get_substeps(self):
        n = ctypes.c_int64()
        self._check(self.lib.daeti_get_substeps(self.ctx, ctypes.byref(n)))
        return n.value

    def daeti_get_tuning(self):
        t = daeti_tuning()
        self._check(self.lib.daeti_get_tuning(self.ctx, ctypes.byref(t)))
        return {f: getattr(t, f) for f in TUNING_FIELDS}

    def daeti_set_tuning(self, **changes):
        """Change launch shapes (keys of TUNING_FIELDS); returns the new tuning."""
        cur = self.daeti_get_tuning()
        cur.update(changes)
        t = daeti_tuning()
        t.struct_size = ctypes.sizeof(daeti_tuning)
        for f in TUNING_FIELDS:
            setattr(t, f, int(cur[f]))
        self._check(self.lib.daeti_set_tuning(self.ctx, ctypes.byref(t)))
        return self.daeti_get_tuning()

    def daeti_update_cell_params(self, params):
        p = _f64(params).reshape(-1)
        self._check(self.lib.daeti_update_cell_params(self.ctx, _ptr(p, ctypes.c_double), p.shape[0]))

    def daeti_time_launches(self, which, count=20):
        """ms per launch of `count` back-to-back launches in a graph (changes the state)."""
        ms = ctypes.c_double()
        self._check(self.lib.daeti_time_launches(self.ctx, int(which), int(count), ctypes.byref(ms)))
        return ms.value

    def daeti_set_profiling(self, enable=True):
        """True/1: events around plain launches; 2: event-record nodes inside graphs; False/0: off."""
        mode = enable if isinstance(enable, int) and not isinstance(enable, bool) else int(bool(enable))
        self._check(self.lib.daeti_set_profiling(self.ctx, mode))

    def daeti_get_kernel_time(self, which):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self.lib.daeti_get_kernel_time(self.ctx, int(which), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def daeti_kernel_work(self, which):
        b, f = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.daeti_kernel_work(self.ctx, int(which), ctypes.byref(b), ctypes.byref(f)))
        return b.value, f.value

    # -- convenience --------------------------------------------------------------
    @property
    def time(self):
        return self.daeti_get_time()[0]


class Batch:
    """Many tissues advanced together (daeti_batch_*).  Tissues are added as
    unprepared Solver descriptions (mesh, conductivity, model, stimuli)."""

    def __init__(self, precision="fp32_kahan", dt=0.1, dt0=0.01, graph_steps=20, stream=None, **opts):
        self.lib = load_library()
        o = daeti_options()
        self.lib.daeti_default_options(ctypes.byref(o))
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.dt, o.dt0, o.graph_steps = float(dt), float(dt0), int(graph_steps)
        for k, v in opts.items():
            setattr(o, k, v)
        h = _VP()
        rc = self.lib.daeti_batch_create(ctypes.byref(h), ctypes.byref(o))
        if rc != OK:
            raise DaetiError(rc, "daeti_batch_create failed")
        self.b = h
        self.sizes = []
        if stream is not None:
            handle = getattr(stream, "cuda_stream", stream)
            self._check(self.lib.daeti_batch_set_stream(self.b, _VP(int(handle) if handle else 0)))

    def _check(self, rc):
        if rc != OK:
            msg = self.lib.daeti_batch_last_error(self.b)
            raise DaetiError(rc, msg.decode() if msg else "")

    def daeti_batch_add(self, solver):
        self._check(self.lib.daeti_batch_add(self.b, solver.ctx))
        self.sizes.append(solver.n_nodes)

    def daeti_batch_prepare(self):
        self._check(self.lib.daeti_batch_prepare(self.b))

    def daeti_batch_advance(self, t_end):
        self._check(self.lib.daeti_batch_advance(self.b, float(t_end)))

    def daeti_batch_synchronize(self):
        self._check(self.lib.daeti_batch_synchronize(self.b))

    def daeti_batch_info(self):
        n, t, l, dt = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.daeti_batch_info(self.b, ctypes.byref(n), ctypes.byref(t), ctypes.byref(l),
                                              ctypes.byref(dt)))
        return {"n_nodes": n.value, "n_tissues": t.value, "l": l.value, "dt": dt.value}

    def daeti_batch_read_v(self, tissue):
        out = np.empty(self.sizes[tissue], dtype=np.float64)
        self._check(self.lib.daeti_batch_read_v(self.b, int(tissue), _ptr(out, ctypes.c_double)))
        return out

    def daeti_batch_read_activation(self, tissue):
        out = np.empty(self.sizes[tissue], dtype=np.float64)
        self._check(self.lib.daeti_batch_read_activation(self.b, int(tissue), _ptr(out, ctypes.c_double)))
        return out

    def close(self):
        if getattr(self, "b", None):
            self.lib.daeti_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def describe_workload(wl, **options) -> Solver:
    """An unprepared Solver holding a workload's description (for Batch)."""
    opts = dict(dt=wl.dt, dt0=wl.dt0, v_threshold=wl.v_threshold)
    opts.update(options)
    s = Solver(**opts)
    s.daeti_set_mesh_grid(wl.dim, wl.n, wl.h)
    s.daeti_set_conductivity(wl.d_long, wl.d_trans, wl.fibre)
    if getattr(wl, "cell_type", None) is not None:
        raise ValueError("a batch tissue takes one cell type (per-node cell types need a Solver)")
    s.daeti_set_cell_model(wl.model, tuple(wl.model_params))
    for st in wl.stimuli:
        s.daeti_add_stimulus(st.nodes, st.t_start, st.duration, st.amplitude, st.period, st.count)
    return s


def daeti_grid_stability_noalloc(dim, n, h, d_long, d_trans=None, fibre=None, stream=None):
    """Allocation-free (dt_s, lambda_max) of a layered structured grid; raises DaetiError."""
    lib = load_library()
    nn = _i64(list(n) + [1] * (3 - len(n)))
    dl, dtr, fb = _cond(d_long, d_trans, fibre)
    handle = getattr(stream, "cuda_stream", stream)
    dts, lam = ctypes.c_double(), ctypes.c_double()
    err = ctypes.create_string_buffer(256)
    rc = lib.daeti_grid_stability_noalloc(int(dim), _ptr(nn, ctypes.c_int64), float(h), dl.shape[0],
                                          _ptr(dl, ctypes.c_double), _ptr(dtr, ctypes.c_double),
                                          _ptr(fb, ctypes.c_double), _VP(int(handle) if handle else 0),
                                          ctypes.byref(dts), ctypes.byref(lam), err, 256)
    if rc != OK:
        raise DaetiError(rc, err.value.decode())
    return dts.value, lam.value


def solver_from_workload(wl, **options) -> Solver:
    """Build and prepare a Solver from a workload description.

    ``wl`` needs the attributes of ``inputs.Workload`` (dim, n, h or xyz/tets,
    d_long, d_trans, fibre, model, model_params, stimuli, dt, dt0,
    v_threshold); the description is only copied into the library.
    """
    opts = dict(dt=wl.dt, dt0=wl.dt0, v_threshold=wl.v_threshold)
    opts.update(options)
    s = Solver(**opts)
    if getattr(wl, "tets", None) is not None:
        s.daeti_set_mesh_tet(wl.xyz, wl.tets)
    else:
        s.daeti_set_mesh_grid(wl.dim, wl.n, wl.h)
    s.daeti_set_conductivity(wl.d_long, wl.d_trans, wl.fibre)
    s.daeti_set_cell_model(wl.model, tuple(wl.model_params))
    if getattr(wl, "cell_type", None) is not None:
        s.daeti_set_cell_types(wl.cell_type)
    for st in wl.stimuli:
        s.daeti_add_stimulus(st.nodes, st.t_start, st.duration, st.amplitude, st.period, st.count)
    s.daeti_prepare()
    return s

