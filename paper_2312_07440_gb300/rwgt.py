"""Thin Python binding of librwgt.so (include/rwgt.h): argument marshalling only.

Every step of the reweighting path runs in the library's CUDA kernels; this
module converts Python/torch arguments to the C ABI's plain pointers and
sizes.  There is no CPU fallback: if the library is missing or fails to load,
``load()`` raises.  torch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librwgt.so")

RW_OK = 0
RW_WARN_BAD_EVENTS = 1
ERRORS = {-1: "RW_ERR_NULL", -2: "RW_ERR_ARG", -3: "RW_ERR_MODE", -4: "RW_ERR_PARAM", -5: "RW_ERR_CUDA",
          -6: "RW_ERR_STATE", -7: "RW_ERR_ALIGN", -8: "RW_ERR_WORKSPACE"}
PROCESS = {"ee_mumu": 0, "gg_tt": 1, "gg_ttg": 2, "gg_ttgg": 3, "ee_5a": 4}
MODE = {"fp64": 0, "fp32": 1, "mixed_fp16": 2, "mixed_bf16": 3}
MAX_POINTS = 256
PARAM_FIELDS = ("alpha_s", "m_t", "w_t", "yt_scale", "alpha_em_inv", "G_F", "m_Z", "w_Z")


class RwParams(ctypes.Structure):
    _fields_ = [(f, ctypes.c_double) for f in PARAM_FIELDS]


class RwProcessInfo(ctypes.Structure):
    _fields_ = [("n_external", ctypes.c_int), ("n_helicities", ctypes.c_int), ("n_colour_flows", ctypes.c_int),
                ("n_diagrams", ctypes.c_int), ("colour_den", ctypes.c_int), ("flops_hel_sum", ctypes.c_longlong)]


class RwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Load librwgt.so (built by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    P, i, d, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "rw_create": ([ctypes.POINTER(P), i, P], i),
        "rw_destroy": ([P], i),
        "rw_last_error": ([P], ctypes.c_char_p),
        "rw_process_info_get": ([i, ctypes.POINTER(RwProcessInfo)], i),
        "rw_set_process": ([P, i, i], i),
        "rw_set_params": ([P, ctypes.POINTER(RwParams)], i),
        "rw_set_reweight_points": ([P, P, i], i),
        "rw_set_tuning": ([P, i, i], i),
        "rw_workspace_bytes": ([P, i64], sz),
        "rw_load_events": ([P, P, P, i64, P, sz], i),
        "rw_eval_me": ([P, i, P], i),
        "rw_reweight_async": ([P, P, P, P, P], i),
        "rw_get_results": ([P, P, P, P], i),
        "rw_get_result_pairs": ([P, P, P, P], i),
        "rw_reweight": ([P, P, P, P, P, P], i),
        "rw_workspace_bytes_host": ([P, i64], sz),
        "rw_reweight_host": ([P, P, P, i64, P, P, P, P, P, sz], i),
        "rw_get_tuning": ([P, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "rw_mlp_create": ([ctypes.POINTER(P), i, P, i, i, i, i, ctypes.c_uint64], i),
        "rw_mlp_destroy": ([P], i),
        "rw_mlp_last_error": ([P], ctypes.c_char_p),
        "rw_mlp_n_params": ([P], i64),
        "rw_mlp_info": ([P, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(P)], i),
        "rw_mlp_get_state": ([P, P, P, P, ctypes.POINTER(i64)], i),
        "rw_mlp_set_state": ([P, P, P, P, i64], i),
        "rw_mlp_forward": ([P, P, i64, P], i),
        "rw_mlp_gradient": ([P, P, P, i64, ctypes.c_float, ctypes.c_float, P, ctypes.POINTER(ctypes.c_float)], i),
        "rw_mlp_train": ([P, P, P, i64, i, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_uint64], i),
        "rw_mlp_set_gemm": ([P, i], i),
        "rw_mlp_status": ([P], i),
        "rw_mlp_hidden_layer": ([P, i, P, i64, P, P], i),
        "rw_surrogate_features": ([P, i, d, d, P, P, P], i),
        "rw_surrogate_workspace_bytes": ([P, i], sz),
        "rw_surrogate_reweight": ([P, P, d, d, d, P, P, P, P, P, sz], i),
        "rw_graph_begin": ([P], i),
        "rw_graph_end": ([P, ctypes.POINTER(P)], i),
        "rw_graph_launch": ([P, P], i),
        "rw_graph_destroy": ([P], i),
        "rw_autotune": ([P, i64, ctypes.c_char_p, ctypes.POINTER(d)], i),
        "rw_split_double": ([P, i64, P, P, P], i),
        "rw_interp_workspace_bytes": ([P], sz),
        "rw_lhe_open": ([ctypes.POINTER(P), ctypes.c_char_p], i),
        "rw_lhe_close": ([P], i),
        "rw_lhe_last_error": ([P], ctypes.c_char_p),
        "rw_lhe_n_events": ([P], i64),
        "rw_lhe_read": ([P, i, i64, i64, P, i64, P, i], i),
        "rw_lhe_write": ([P, ctypes.c_char_p, P, i, i64, P], i),
        "rw_lhe_classify": ([P, P, i, P, i], i),
        "rw_lhe_write_begin": ([P, ctypes.c_char_p, i, P], i),
        "rw_lhe_write_events": ([P, i64, i64, P, i64], i),
        "rw_lhe_write_end": ([P], i),
        "rw_lhe_workspace_bytes": ([P, i64], sz),
        "rw_lhe_reweight": ([P, P, ctypes.c_char_p, P, i64, i, P, sz, P, P, P], i),
        "rw_lhe_read_list": ([P, i, P, i64, P, i64, P, i], i),
        "rw_reweight_interp": ([P, i, d, P, P, P, P, P, P, P, sz], i),
        "rw_alu_peak": ([i, P, i, ctypes.POINTER(d), ctypes.POINTER(d)], i),
        "rw_multi_create": ([ctypes.POINTER(P), i, P], i),
        "rw_multi_destroy": ([P], i),
        "rw_multi_last_error": ([P], ctypes.c_char_p),
        "rw_multi_add": ([P, P, P, P], i),
        "rw_multi_workspace_bytes": ([P], sz),
        "rw_multi_reweight_async": ([P, P, sz], i),
        "rw_multi_get_results": ([P, P, P, P], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _check_buffer(x, name, min_elems=0, dtype="float64"):
    """Check a torch tensor or numpy array before its address goes to the
    library, which takes plain pointers and cannot see their type or size:
    element type, C-contiguity and at least min_elems elements.  None and raw
    integer addresses pass unchecked."""
    if x is None or isinstance(x, int):
        return
    if isinstance(x, np.ndarray):
        kind, contiguous, n = str(x.dtype), bool(x.flags.c_contiguous), int(x.size)
    else:
        kind, contiguous, n = str(x.dtype).replace("torch.", ""), bool(x.is_contiguous()), int(x.numel())
    if kind != dtype:
        raise ValueError(f"{name}: expected {dtype} elements, got {kind}")
    if not contiguous:
        raise ValueError(f"{name}: must be C-contiguous")
    if n < min_elems:
        raise ValueError(f"{name}: {n} elements, need at least {min_elems}")


class Multi:
    """Several prepared contexts (one process each) reweighted by one
    persistent launch (rw_multi_*).  add() the contexts with their W' and r
    outputs, then reweight_async(); each context's own sums come from
    ctx.get_results(), the sample's totals from get_results()."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        self.h = ctypes.c_void_p()
        self._keep = []
        rc = self.lib.rw_multi_create(ctypes.byref(self.h), device, stream)
        if rc:
            self.h = None
            raise RwError(rc, "rw_multi_create")

    def _check(self, rc, what):
        if rc < 0:
            raise RwError(rc, f"{what}: {self.lib.rw_multi_last_error(self.h).decode()}")
        return rc

    def add(self, ctx, wnew=None, ratio=None):
        P, E = ctx.n_points, ctx.n_events
        _check_buffer(wnew, "wnew", P * E)
        _check_buffer(ratio, "ratio", P * E)
        self._keep.append((ctx, wnew, ratio))
        self._check(self.lib.rw_multi_add(self.h, ctx.h, _ptr(wnew), _ptr(ratio)), "rw_multi_add")

    def workspace_bytes(self) -> int:
        return int(self.lib.rw_multi_workspace_bytes(self.h))

    def reweight_async(self, workspace, workspace_bytes: int):
        _check_buffer(workspace, "workspace", workspace_bytes, dtype="uint8")
        self._check(self.lib.rw_multi_reweight_async(self.h, _ptr(workspace), workspace_bytes),
                    "rw_multi_reweight_async")

    def get_results(self, n_points: int):
        sig = np.zeros(n_points)
        so = ctypes.c_double()
        nb = ctypes.c_int64()
        rc = self._check(self.lib.rw_multi_get_results(self.h, sig.ctypes.data, ctypes.byref(so), ctypes.byref(nb)),
                         "rw_multi_get_results")
        return sig, so.value, nb.value, rc

    def close(self):
        if self.h:
            self.lib.rw_multi_destroy(self.h)
            self.h = None
        self._keep = []

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def lhe_workspace_bytes(ctx, chunk: int) -> int:
    return int(ctx.lib.rw_lhe_workspace_bytes(ctx.h, int(chunk)))


def lhe_reweight(ctx, lhe, out_path, ids, chunk: int, workspace, workspace_bytes: int, threads: int = 8):
    """rw_lhe_reweight: the context's process and points applied to every
    event of the open event file `lhe`, written to out_path with the weight
    ids, host parsing and writing overlapped with the GPU.  Returns
    (sigma [P], sigma_orig, n_bad, status)."""
    P = ctx.n_points
    if len(ids) != P:
        raise ValueError(f"need {P} weight ids, got {len(ids)}")
    _check_buffer(workspace, "workspace", workspace_bytes, dtype="uint8")
    enc = [i.encode() for i in ids]
    arr = (ctypes.c_char_p * P)(*enc)
    sig = np.zeros(P)
    so = ctypes.c_double()
    nb = ctypes.c_int64()
    rc = ctx._check(ctx.lib.rw_lhe_reweight(ctx.h, lhe.h, os.fsencode(os.fspath(out_path)), arr, int(chunk),
                                            int(threads), _ptr(workspace), int(workspace_bytes), sig.ctypes.data,
                                            ctypes.byref(so), ctypes.byref(nb)), "rw_lhe_reweight")
    return sig, so.value, nb.value, rc


def alu_peak(kind, device=0, stream=None):
    """rw_alu_peak: measured FP64 (kind "fp64") or FP32 ("fp32") FMA throughput
    of the device in TFLOP/s, and the timed launch's milliseconds."""
    lib = load()
    t, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.rw_alu_peak(device, stream, {"fp64": 0, "fp32": 1}[kind], ctypes.byref(t), ctypes.byref(ms))
    if rc:
        raise RwError(rc, "rw_alu_peak")
    return t.value, ms.value


def split_double(d_x, d_hi, d_lo, stream=None):
    """rw_split_double: the FP32 modes' FP64 -> (hi, lo) float split of the
    device array d_x into d_hi, d_lo (same length), asynchronous on stream."""
    n = int(d_x.numel())
    if d_hi.numel() != n or d_lo.numel() != n:
        raise ValueError("d_hi and d_lo must have the length of d_x")
    _check_buffer(d_x, "d_x", n)
    _check_buffer(d_hi, "d_hi", n, "float32")
    _check_buffer(d_lo, "d_lo", n, "float32")
    rc = load().rw_split_double(_ptr(d_x), n, _ptr(d_hi), _ptr(d_lo), stream)
    if rc:
        raise RwError(rc, "rw_split_double")


def process_info(process: str) -> RwProcessInfo:
    info = RwProcessInfo()
    rc = load().rw_process_info_get(PROCESS[process], ctypes.byref(info))
    if rc:
        raise RwError(rc, "rw_process_info_get")
    return info


def params_struct(vec) -> RwParams:
    v = np.asarray(vec, dtype=np.float64).reshape(8)
    return RwParams(*[float(x) for x in v])


class Context:
    """One rw_ctx: process, precision mode, parameter points, attached events."""

    def __init__(self, device: int = 0, stream=None):
        self.h = None
        self.n_external = 0  # of the process set, for the buffer checks
        self.n_points = 0
        self.n_events = 0
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.rw_create(ctypes.byref(h), int(device), stream)
        if rc:
            raise RwError(rc, "rw_create failed")
        self.h = h

    def close(self):
        if self.h:
            self.lib.rw_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self) -> str:
        return self.lib.rw_last_error(self.h).decode()

    def _check(self, rc, what):
        if rc < 0:
            raise RwError(rc, f"{what}: {self.last_error()}")
        return rc

    def set_process(self, process: str, mode: str = "fp64"):
        rc = self._check(self.lib.rw_set_process(self.h, PROCESS[process], MODE[mode]), "rw_set_process")
        self.n_external = process_info(process).n_external
        return rc

    def set_params(self, vec):
        p = params_struct(vec)
        return self._check(self.lib.rw_set_params(self.h, ctypes.byref(p)), "rw_set_params")

    def set_reweight_points(self, pts):
        arr = np.ascontiguousarray(np.atleast_2d(pts), dtype=np.float64)
        rc = self._check(self.lib.rw_set_reweight_points(self.h, arr.ctypes.data, arr.shape[0]),
                         "rw_set_reweight_points")
        self.n_points = arr.shape[0]
        return rc

    def set_tuning(self, lane_bits: int = -1, block: int = 0):
        return self._check(self.lib.rw_set_tuning(self.h, int(lane_bits), int(block)), "rw_set_tuning")

    def get_tuning(self):
        lb, bl = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.rw_get_tuning(self.h, ctypes.byref(lb), ctypes.byref(bl)), "rw_get_tuning")
        return lb.value, bl.value

    def autotune(self, max_events: int = 1 << 18, cache_path: str | None = None) -> float:
        """Time every compiled launch shape on the attached events; keep the fastest."""
        ms = ctypes.c_double()
        self._check(self.lib.rw_autotune(self.h, int(max_events), cache_path.encode() if cache_path else None,
                                         ctypes.byref(ms)), "rw_autotune")
        return ms.value

    def workspace_bytes(self, n_events: int) -> int:
        return int(self.lib.rw_workspace_bytes(self.h, int(n_events)))

    def surrogate_workspace_bytes(self, n_in: int = 32) -> int:
        return int(self.lib.rw_surrogate_workspace_bytes(self.h, int(n_in)))

    def workspace_bytes_host(self, n_events: int) -> int:
        return int(self.lib.rw_workspace_bytes_host(self.h, int(n_events)))

    def load_events(self, mom, w, n_events: int, workspace, workspace_bytes: int):
        E = max(int(n_events), 0)
        _check_buffer(mom, "mom", self.n_external * 4 * E)
        _check_buffer(w, "w", E)
        rc = self._check(self.lib.rw_load_events(self.h, _ptr(mom), _ptr(w), int(n_events), _ptr(workspace),
                                                 int(workspace_bytes)), "rw_load_events")
        self.n_events = E
        return rc

    def eval_me(self, point: int, out):
        _check_buffer(out, "out", self.n_events)
        return self._check(self.lib.rw_eval_me(self.h, int(point), _ptr(out)), "rw_eval_me")

    def reweight_async(self, wnew=None, ratio=None, me0=None, me_pts=None):
        PE = self.n_points * self.n_events
        for x, name, n in ((wnew, "wnew", PE), (ratio, "ratio", PE), (me0, "me0", self.n_events),
                           (me_pts, "me_pts", PE)):
            _check_buffer(x, name, n)
        return self._check(self.lib.rw_reweight_async(self.h, _ptr(wnew), _ptr(ratio), _ptr(me0), _ptr(me_pts)),
                           "rw_reweight_async")

    def get_results(self, n_points: int):
        sig = np.zeros(n_points)
        so = ctypes.c_double()
        nb = ctypes.c_int64()
        rc = self._check(self.lib.rw_get_results(self.h, sig.ctypes.data, ctypes.byref(so), ctypes.byref(nb)),
                         "rw_get_results")
        return sig, so.value, nb.value, rc

    def get_result_pairs(self, n_points: int):
        """(sum[P+1], compensation[P+1], n_bad) of the last reweight; index P
        is the original sample's sigma."""
        s = np.zeros(n_points + 1)
        c = np.zeros(n_points + 1)
        nb = ctypes.c_int64()
        self._check(self.lib.rw_get_result_pairs(self.h, s.ctypes.data, c.ctypes.data, ctypes.byref(nb)),
                    "rw_get_result_pairs")
        return s, c, nb.value

    def reweight(self, n_points: int, wnew=None, ratio=None):
        sig = np.zeros(n_points)
        so = ctypes.c_double()
        nb = ctypes.c_int64()
        rc = self._check(self.lib.rw_reweight(self.h, _ptr(wnew), _ptr(ratio), sig.ctypes.data, ctypes.byref(so),
                                              ctypes.byref(nb)), "rw_reweight")
        return sig, so.value, nb.value, rc

    def reweight_host(self, h_mom, h_w, n_events: int, h_wnew, n_points: int, workspace, workspace_bytes: int):
        E = max(int(n_events), 0)
        _check_buffer(h_mom, "h_mom", self.n_external * 4 * E)
        _check_buffer(h_w, "h_w", E)
        _check_buffer(h_wnew, "h_wnew", int(n_points) * E)
        sig = np.zeros(n_points)
        so = ctypes.c_double()
        nb = ctypes.c_int64()
        rc = self._check(self.lib.rw_reweight_host(self.h, _ptr(h_mom), _ptr(h_w), int(n_events), _ptr(h_wnew),
                                                   sig.ctypes.data, ctypes.byref(so), ctypes.byref(nb),
                                                   _ptr(workspace), int(workspace_bytes)), "rw_reweight_host")
        return sig, so.value, nb.value, rc


def reweight_interp(ctx, n_nodes, tol, d_wnew, d_fallback=None):
    """rw_reweight_interp on a Context with events and points attached:
    returns dict(sigma[P], sigma_orig, n_fallback, n_bad, status); W' and the
    fallback flags go to the given device tensors."""
    lib = ctx.lib
    nb = int(lib.rw_interp_workspace_bytes(ctx.h))
    import torch
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=d_wnew.device)
    P = ctx.n_points
    _check_buffer(d_wnew, "d_wnew", P * ctx.n_events)
    _check_buffer(d_fallback, "d_fallback", ctx.n_events, "uint8")
    sig = np.zeros(max(P, 1))
    so = ctypes.c_double()
    nfb = ctypes.c_int64()
    nbad = ctypes.c_int64()
    rc = ctx._check(lib.rw_reweight_interp(ctx.h, int(n_nodes), float(tol), _ptr(d_wnew), _ptr(d_fallback),
                                           sig.ctypes.data, ctypes.byref(so), ctypes.byref(nfb), ctypes.byref(nbad),
                                           _ptr(ws), nb), "rw_reweight_interp")
    return {"sigma": sig, "sigma_orig": so.value, "n_fallback": int(nfb.value), "n_bad": int(nbad.value),
            "status": rc}


class Lhe:
    """A Les Houches Event file: read events into the library's layout, write
    it back with new weights (rw_lhe_*; host only, no GPU needed).  A gzip
    file (.lhe.gz) is decompressed to a temporary file first, and write() to a
    path ending in .gz compresses its output."""

    def __init__(self, path):
        self.h = None
        self._tmp = None
        self.lib = load()
        src = os.fspath(path)
        try:
            with open(src, "rb") as f:
                gz = f.read(2) == b"\x1f\x8b"
        except OSError:
            gz = False  # the library reports the missing or unreadable file
        if gz:
            import gzip
            import shutil
            import tempfile
            fd, self._tmp = tempfile.mkstemp(suffix=".lhe")
            with os.fdopen(fd, "wb") as out, gzip.open(src, "rb") as inp:
                shutil.copyfileobj(inp, out, 1 << 22)
            src = self._tmp
        h = ctypes.c_void_p()
        rc = self.lib.rw_lhe_open(ctypes.byref(h), os.fsencode(src))
        # the library holds the whole text in memory now: the plain copy of a
        # compressed file is not needed any more
        self._drop_tmp()
        if rc:
            raise RwError(rc, f"rw_lhe_open: cannot read {path} (or an <event> or XML comment is not closed)")
        self.h = h

    def _drop_tmp(self):
        if self._tmp:
            os.unlink(self._tmp)
            self._tmp = None

    def close(self):
        if self.h:
            self.lib.rw_lhe_close(self.h)
            self.h = None
        self._drop_tmp()

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return int(self.lib.rw_lhe_n_events(self.h))

    def _check(self, rc, what):
        if rc < 0:
            raise RwError(rc, f"{what}: {self.lib.rw_lhe_last_error(self.h).decode()}")
        return rc

    def read(self, process: str, first: int = 0, n=None, threads: int = 8):
        """(mom [N][4][n] float64, w [n]) for events [first, first + n)."""
        n = len(self) - first if n is None else int(n)
        N = process_info(process).n_external
        mom = np.empty((N, 4, n))
        w = np.empty(n)
        self._check(self.lib.rw_lhe_read(self.h, PROCESS[process], int(first), n, mom.ctypes.data, n,
                                         w.ctypes.data, int(threads)), "rw_lhe_read")
        return mom, w

    def classify(self, processes, threads: int = 8) -> np.ndarray:
        """Process index into ``processes`` (names) of every event, -1 if it
        matches none: int32 [len(self)]."""
        ids = np.array([PROCESS[p] for p in processes], dtype=np.int32)
        out = np.empty(len(self), dtype=np.int32)
        self._check(self.lib.rw_lhe_classify(self.h, ids.ctypes.data, len(ids), out.ctypes.data, int(threads)),
                    "rw_lhe_classify")
        pos = {int(v): i for i, v in enumerate(ids)}
        return np.array([pos.get(int(v), -1) for v in out], dtype=np.int32)

    def read_list(self, process: str, idx, threads: int = 8):
        """(mom [N][4][n], w [n]) for the events idx (file indices, any order)."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        n = idx.shape[0]
        N = process_info(process).n_external
        mom = np.empty((N, 4, n))
        w = np.empty(n)
        self._check(self.lib.rw_lhe_read_list(self.h, PROCESS[process], idx.ctypes.data, n, mom.ctypes.data, n,
                                              w.ctypes.data, int(threads)), "rw_lhe_read_list")
        return mom, w

    def write(self, path, wnew, ids):
        """Write the file to ``path`` with wnew[P][E] (E = all events) added as
        <wgt id=...> lines of each event's <rwgt> block."""
        wnew = np.ascontiguousarray(wnew, dtype=np.float64)
        P, ld = wnew.shape
        if len(ids) != P:
            raise ValueError(f"{len(ids)} weight ids for {P} rows of wnew")
        arr = (ctypes.c_char_p * P)(*[str(x).encode() for x in ids])
        dst = os.fspath(path)
        if not dst.endswith(".gz"):
            self._check(self.lib.rw_lhe_write(self.h, os.fsencode(dst), wnew.ctypes.data, P, ld, arr), "rw_lhe_write")
            return
        import gzip
        import shutil
        import tempfile
        fd, tmp = tempfile.mkstemp(suffix=".lhe")
        os.close(fd)
        try:
            self._check(self.lib.rw_lhe_write(self.h, os.fsencode(tmp), wnew.ctypes.data, P, ld, arr), "rw_lhe_write")
            with open(tmp, "rb") as inp, gzip.open(dst, "wb", compresslevel=6) as out:
                shutil.copyfileobj(inp, out, 1 << 22)
        finally:
            os.unlink(tmp)


class Mlp:
    """rw_mlp: the surrogate network (n_in -> hidden x n_layers SiLU -> (mu, s))."""

    def __init__(self, device: int = 0, stream=None, n_in: int = 32, hidden: int = 256, n_layers: int = 4,
                 max_batch: int = 16384, seed: int = 1):
        self.h = None
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.rw_mlp_create(ctypes.byref(h), int(device), stream, n_in, hidden, n_layers, max_batch, seed)
        if rc:
            raise RwError(rc, "rw_mlp_create failed")
        self.h = h
        self.n_in, self.hidden, self.n_layers, self.max_batch = n_in, hidden, n_layers, max_batch
        self.n_params = int(self.lib.rw_mlp_n_params(h))

    def close(self):
        if self.h:
            self.lib.rw_mlp_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, what):
        if rc < 0:
            raise RwError(rc, f"{what}: {self.lib.rw_mlp_last_error(self.h).decode()}")
        return rc

    def get_state(self):
        p = np.empty(self.n_params, np.float32)
        m1 = np.empty_like(p)
        m2 = np.empty_like(p)
        st = ctypes.c_int64()
        self._check(self.lib.rw_mlp_get_state(self.h, p.ctypes.data, m1.ctypes.data, m2.ctypes.data,
                                              ctypes.byref(st)), "rw_mlp_get_state")
        return {"params": p, "m1": m1, "m2": m2, "step": st.value}

    def set_state(self, params, m1=None, m2=None, step=0):
        p = np.ascontiguousarray(params, np.float32)
        a = np.ascontiguousarray(m1, np.float32) if m1 is not None else None
        b = np.ascontiguousarray(m2, np.float32) if m2 is not None else None
        self._check(self.lib.rw_mlp_set_state(self.h, p.ctypes.data, _ptr(a), _ptr(b), int(step)),
                    "rw_mlp_set_state")

    def forward(self, x, out):
        n = int(x.shape[0])
        _check_buffer(x, "x", n * self.n_in, "float32")
        _check_buffer(out, "out", 2 * n, "float32")
        self._check(self.lib.rw_mlp_forward(self.h, _ptr(x), int(x.shape[0]), _ptr(out)), "rw_mlp_forward")

    def gradient(self, x, y, tau: float, lam: float):
        n = int(x.shape[0])
        _check_buffer(x, "x", n * self.n_in, "float32")
        _check_buffer(y, "y", n, "float32")
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_float()
        self._check(self.lib.rw_mlp_gradient(self.h, _ptr(x), _ptr(y), int(x.shape[0]), tau, lam, g.ctypes.data,
                                             ctypes.byref(loss)), "rw_mlp_gradient")
        return loss.value, g

    def train(self, x, y, batch: int, n_steps: int, lr: float, tau: float, lam: float, seed: int = 7):
        n = int(x.shape[0])
        _check_buffer(x, "x", n * self.n_in, "float32")
        _check_buffer(y, "y", n, "float32")
        self._check(self.lib.rw_mlp_train(self.h, _ptr(x), _ptr(y), int(x.shape[0]), int(batch), int(n_steps), lr,
                                          tau, lam, int(seed)), "rw_mlp_train")

    def set_gemm(self, kind: str):
        """Forward GEMMs: "tcgen05" (5th-generation tensor cores; inference of
        the whole network in one kernel where the shape allows), "tcgen05_layers"
        (tensor cores, one kernel per layer) or "mma_sync" (the legacy path)."""
        self._check(self.lib.rw_mlp_set_gemm(self.h, {"tcgen05": 0, "mma_sync": 1, "tcgen05_layers": 2}[kind]),
                    "rw_mlp_set_gemm")

    def status(self):
        """Synchronise and raise if a tensor-core pipeline wait gave up."""
        self._check(self.lib.rw_mlp_status(self.h), "rw_mlp_status")

    def hidden_layer(self, layer: int, h_in, z_out, h_out):
        """One hidden layer: z_out = h_in W_layer + b (FP32), h_out = bf16(SiLU(z_out));
        h_in, h_out: [n][hidden] torch.bfloat16, z_out: [n][hidden] float32 (device)."""
        n = int(h_in.shape[0])
        _check_buffer(h_in, "h_in", n * self.hidden, "bfloat16")
        _check_buffer(h_out, "h_out", n * self.hidden, "bfloat16")
        _check_buffer(z_out, "z_out", n * self.hidden, "float32")
        self._check(self.lib.rw_mlp_hidden_layer(self.h, int(layer), _ptr(h_in), n, _ptr(z_out), _ptr(h_out)),
                    "rw_mlp_hidden_layer")


class Graph:
    """Record rw_* calls queued on `stream` between begin() and end(); replay with launch()."""

    def __init__(self, stream):
        self.lib = load()
        self.stream = stream
        self.h = None

    def begin(self):
        rc = self.lib.rw_graph_begin(self.stream)
        if rc:
            raise RwError(rc, "rw_graph_begin")

    def end(self):
        h = ctypes.c_void_p()
        rc = self.lib.rw_graph_end(self.stream, ctypes.byref(h))
        if rc:
            raise RwError(rc, "rw_graph_end")
        self.h = h

    def launch(self):
        rc = self.lib.rw_graph_launch(self.h, self.stream)
        if rc:
            raise RwError(rc, "rw_graph_launch")

    def close(self):
        if self.h:
            self.lib.rw_graph_destroy(self.h)
            self.h = None

    __del__ = close


def surrogate_features(ctx: "Context", n_in, p_scale, k_scale, ratio, x, y):
    PE = ctx.n_points * ctx.n_events
    _check_buffer(ratio, "ratio", PE)
    _check_buffer(x, "x", PE * int(n_in), "float32")
    _check_buffer(y, "y", PE, "float32")
    return ctx._check(ctx.lib.rw_surrogate_features(ctx.h, int(n_in), float(p_scale), float(k_scale), _ptr(ratio),
                                                    _ptr(x), _ptr(y)), "rw_surrogate_features")


def surrogate_reweight(ctx: "Context", mlp: Mlp, p_scale, k_scale, s_max, wnew, fallback, n_points, ws, ws_bytes):
    P = max(int(n_points), ctx.n_points)  # the library writes one sum per attached point
    _check_buffer(wnew, "wnew", ctx.n_points * ctx.n_events)
    _check_buffer(fallback, "fallback", ctx.n_points * ctx.n_events, "uint8")
    sig = np.zeros(P)
    nf = np.zeros(P, np.int64)
    ctx._check(ctx.lib.rw_surrogate_reweight(ctx.h, mlp.h, float(p_scale), float(k_scale), float(s_max), _ptr(wnew),
                                             _ptr(fallback), sig.ctypes.data, nf.ctypes.data, _ptr(ws),
                                             int(ws_bytes)), "rw_surrogate_reweight")
    return sig, nf


def reweight(process: str, mode: str, mom, w, p0, points, *, lane_bits: int = -1, block: int = 0,
             want_me: bool = True, device=None):
    """Convenience: reweight a device batch (torch float64 tensors mom[N][4][E],
    w[E]) for P points; returns a dict of torch tensors and the sums."""
    import torch
    dev = mom.device if device is None else device
    E = mom.shape[-1]
    pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
    P = pts.shape[0]
    stream = torch.cuda.current_stream(dev).cuda_stream
    with Context(dev.index or 0, stream) as c:
        c.set_process(process, mode)
        c.set_params(p0)
        c.set_reweight_points(pts)
        c.set_tuning(lane_bits, block)
        nb = c.workspace_bytes(E)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        c.load_events(mom, w, E, ws, nb)
        out = {"wnew": torch.empty((P, E), dtype=torch.float64, device=dev),
               "ratio": torch.empty((P, E), dtype=torch.float64, device=dev)}
        if want_me:
            out["me0"] = torch.empty(E, dtype=torch.float64, device=dev)
            out["me"] = torch.empty((P, E), dtype=torch.float64, device=dev)
        c.reweight_async(out["wnew"], out["ratio"], out.get("me0"), out.get("me"))
        sig, so, nbad, rc = c.get_results(P)
        out.update(sigma=sig, sigma_orig=so, n_bad=nbad, status=rc)
        return out
