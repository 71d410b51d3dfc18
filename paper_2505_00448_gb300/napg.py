"""Python binding of libnapg.so (include/napg.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. PyTorch provides device
memory and the CUDA stream. Importing this module loads the library and raises
ImportError when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import time
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnapg.so")

PEARSON, SPEARMAN, CHI2, ANOVA, TTEST, MWU, KRUSKAL = range(7)
TESTS = {"pearson": PEARSON, "spearman": SPEARMAN, "chi2": CHI2, "anova": ANOVA, "ttest": TTEST,
         "mwu": MWU, "kruskal": KRUSKAL}
FP64_PLAIN, MIXED = 0, 1
F32, F64 = 0, 1
STATUS = {0: "OK", 1: "E_ARG", 2: "E_OOM", 3: "E_CUDA", 4: "E_LABEL", 5: "E_NONFINITE",
          6: "E_TIMEOUT", 7: "E_UNSUPPORTED", 8: "E_BUSY"}
E_ARG, E_OOM, E_CUDA, E_LABEL, E_NONFINITE, E_TIMEOUT, E_UNSUPPORTED, E_BUSY = range(1, 9)
MWU_MODES = {"auto": 0, "exact": 1, "asymptotic": 2}

# every symbol include/napg.h declares
EXPORTS = ["napg_default_options", "napg_create", "napg_destroy", "napg_last_error", "napg_sync", "napg_release_cache",
           "napg_load_cohort", "napg_run", "napg_run_batch", "napg_debug_integers", "napg_debug_pvalues", "napg_serve_start",
           "napg_serve_submit", "napg_serve_poll", "napg_serve_stop", "napg_serve_plan", "napg_version", "napg_trace_enable",
           "napg_trace_read", "napg_kernel_launches", "napg_tune_enable", "napg_tune_read", "napg_tune_pin", "napg_pearson_fp64_noalloc",
           "napg_run_ex", "napg_adjust"]
ADJUST = {"bonferroni": 0, "bh": 1, "by": 2}


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("welch", C.c_int32), ("yates_2x2", C.c_int32),
                ("mwu_mode", C.c_int32), ("mwu_continuity", C.c_int32), ("debug_checks", C.c_int32),
                ("async_host_outputs", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("test", C.c_int32), ("opt", Options), ("sample_mask", C.c_void_p),
                ("vars_a", C.c_void_p), ("n_a", C.c_int32), ("vars_b", C.c_void_p), ("n_b", C.c_int32),
                ("stat", C.c_void_p), ("pval", C.c_void_p), ("n", C.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    L = C.CDLL(LIB_PATH)
    p, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    L.napg_default_options.argtypes = [p]
    L.napg_default_options.restype = None
    L.napg_create.argtypes = [p, C.c_int, p]
    L.napg_create.restype = C.c_int
    L.napg_destroy.argtypes = [p]
    L.napg_destroy.restype = None
    L.napg_last_error.argtypes = [p]
    L.napg_last_error.restype = C.c_char_p
    L.napg_sync.argtypes = [p]
    L.napg_sync.restype = C.c_int
    L.napg_release_cache.argtypes = [p]
    L.napg_release_cache.restype = C.c_int
    L.napg_load_cohort.argtypes = [p, p, i32, i64, i64, i32, d, p, p]
    L.napg_load_cohort.restype = C.c_int
    L.napg_run.argtypes = [p, i32, p, p, p, i32, p, i32, p, p, p]
    L.napg_run.restype = C.c_int
    L.napg_run_ex.argtypes = [p, i32, p, p, p, i32, p, i32, p, p, p, p, p]
    L.napg_run_ex.restype = C.c_int
    L.napg_run_part.argtypes = [p, i32, p, p, p, i32, p, i32, i32, i32, p, p, p]
    L.napg_run_part.restype = C.c_int
    L.napg_adjust.argtypes = [p, i32, p, i64, i64, i32, p]
    L.napg_adjust.restype = C.c_int
    L.napg_run_batch.argtypes = [p, i32, p, i32, p, p, i32, p, i32, p, p, p]
    L.napg_run_batch.restype = C.c_int
    L.napg_debug_integers.argtypes = [p, i32, p, i32, i32, p, i64, p]
    L.napg_debug_integers.restype = C.c_int
    L.napg_debug_pvalues.argtypes = [p, i32, p, p, p, i64, p]
    L.napg_debug_pvalues.restype = C.c_int
    L.napg_serve_start.argtypes = [p, C.c_size_t, i32]
    L.napg_serve_start.restype = C.c_int
    L.napg_serve_submit.argtypes = [p, p, p]
    L.napg_serve_submit.restype = C.c_int
    L.napg_serve_poll.argtypes = [p, C.c_uint64, p, p, p]
    L.napg_serve_poll.restype = C.c_int
    L.napg_serve_stop.argtypes = [p]
    L.napg_serve_stop.restype = C.c_int
    L.napg_serve_plan.argtypes = [p, p, i32, p, p, i32, C.c_uint64, p]
    L.napg_serve_plan.restype = C.c_int
    L.napg_tune_enable.argtypes = [p, i32]
    L.napg_tune_enable.restype = C.c_int
    L.napg_tune_read.argtypes = [p, p, C.c_size_t]
    L.napg_tune_read.restype = C.c_int
    L.napg_tune_pin.argtypes = [p, C.c_char_p, i32]
    L.napg_tune_pin.restype = C.c_int
    L.napg_version.argtypes = []
    L.napg_version.restype = C.c_char_p
    L.napg_trace_enable.argtypes = [p, i32]
    L.napg_trace_enable.restype = C.c_int
    L.napg_trace_read.argtypes = [p, p, C.c_size_t]
    L.napg_trace_read.restype = C.c_int
    L.napg_kernel_launches.argtypes = []
    L.napg_kernel_launches.restype = C.c_uint64
    L.napg_pearson_fp64_noalloc.argtypes = [p, i32, i32, d, p, p, p, p]
    L.napg_pearson_fp64_noalloc.restype = C.c_int
    return L


lib = _load()


class NapgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"napg {STATUS.get(code, code)}: {msg}")
        self.code = code


def options(precision="fp64", welch=True, yates=False, mwu_mode="auto", mwu_continuity=True):
    o = Options()
    lib.napg_default_options(C.byref(o))
    o.precision = MIXED if precision in ("mixed", MIXED) else FP64_PLAIN
    o.welch = 1 if welch else 0
    o.yates_2x2 = 1 if yates else 0
    o.mwu_mode = MWU_MODES[mwu_mode] if isinstance(mwu_mode, str) else int(mwu_mode)
    o.mwu_continuity = 1 if mwu_continuity else 0
    return o


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _i32(v):
    return None if v is None else np.ascontiguousarray(np.asarray(v, dtype=np.int32))


class Context:
    """One library context (device cohort + work memory) on one CUDA stream."""

    def __init__(self, device=0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
            if stream.cuda_stream == 0:
                # the legacy default stream has handle 0, which the C ABI reads as
                # "no stream": give the context a stream of its own
                stream = torch.cuda.Stream(device)
        self.stream = stream
        h = C.c_void_p()
        rc = lib.napg_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if rc:
            raise NapgError(rc, "napg_create failed")
        self.h = h
        self.F = self.S = 0
        self.vtype = self.nlev = None

    def _check(self, rc):
        if rc:
            raise NapgError(rc, lib.napg_last_error(self.h).decode())

    def close(self):
        if self.h:
            lib.napg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self):
        self._check(lib.napg_sync(self.h))

    def load_cohort(self, X, vtype, nlev, missing=math.nan, samples_major=False):
        """X: (F, S) (or (S, F) with samples_major) float32/float64, numpy or torch (any device)."""
        torch = self.torch
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X)
            dt = F32 if X.dtype == np.float32 else F64
            if X.dtype not in (np.float32, np.float64):
                X = X.astype(np.float64)
                dt = F64
        else:
            X = X.contiguous()
            dt = F32 if X.dtype == torch.float32 else F64
        F, S = (X.shape[1], X.shape[0]) if samples_major else (X.shape[0], X.shape[1])
        vt = np.ascontiguousarray(vtype, dtype=np.uint8)
        nl = np.ascontiguousarray(nlev, dtype=np.int32)
        self._check(lib.napg_load_cohort(self.h, _ptr(X), dt, F, S, 1 if samples_major else 0, float(missing),
                                         _ptr(vt), _ptr(nl)))
        self.F, self.S, self.vtype, self.nlev = F, S, vt, nl
        return self

    def run(self, test, vars_a, vars_b=None, mask=None, out="cuda", outputs=None, sync=True, effects=False, **opt):
        """One test over all pairs vars_a x vars_b (vars_a x vars_a when vars_b is None).

        out="cuda": torch tensors on the device (stream-ordered; synchronised unless
        sync=False); out="numpy": host numpy arrays, written before the call returns,
        or with sync=False once sync() returns (the copies then overlap the next
        call's kernels; pinned arrays let them run asynchronously). `outputs` may
        supply the dict(stat, p, n[, effect, effect2]) buffers to write. Returns
        dict(stat, p, n), plus effect and effect2 (Table 2's effect sizes; Cramer's
        V for chi-squared, the t distribution's degrees of freedom for the t-test)
        with effects=True.
        """
        torch = self.torch
        t = TESTS[test] if isinstance(test, str) else int(test)
        va, vb = _i32(vars_a), _i32(vars_b)
        na = len(va)
        nb = na if vb is None else len(vb)
        o = options(**opt)
        if not sync and (out == "numpy" or (outputs is not None and isinstance(outputs.get("stat", outputs.get("p")), np.ndarray))):
            o.async_host_outputs = 1
        e1 = e2 = None
        if outputs is not None:
            stat, p, n = outputs.get("stat"), outputs.get("p"), outputs.get("n")
            e1, e2 = outputs.get("effect"), outputs.get("effect2")
        elif out == "numpy":
            stat = np.empty((na, nb), np.float64)
            p = np.empty((na, nb), np.float64)
            n = np.empty((na, nb), np.int32)
            if effects:
                e1, e2 = np.empty((na, nb), np.float64), np.empty((na, nb), np.float64)
        else:
            dev = torch.device("cuda", self.device)
            stat = torch.empty((na, nb), dtype=torch.float64, device=dev)
            p = torch.empty((na, nb), dtype=torch.float64, device=dev)
            n = torch.empty((na, nb), dtype=torch.int32, device=dev)
            if effects:
                e1 = torch.empty((na, nb), dtype=torch.float64, device=dev)
                e2 = torch.empty((na, nb), dtype=torch.float64, device=dev)
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask, dtype=np.uint8) if isinstance(mask, np.ndarray) else mask
        self._check(lib.napg_run_ex(self.h, t, C.byref(o), _ptr(m), _ptr(va), na, _ptr(vb), 0 if vb is None else nb,
                                    _ptr(stat), _ptr(p), _ptr(n), _ptr(e1), _ptr(e2)))
        if out != "numpy" and sync:
            self.sync()
        res = {"stat": stat, "p": p, "n": n}
        if e1 is not None or e2 is not None:
            res["effect"], res["effect2"] = e1, e2
        return res

    def run_part(self, test, vars_a, vars_b=None, part=0, nparts=1, mask=None, outputs=None, out="numpy", **opt):
        """One part of a call split over `nparts` (napg_run_part): the pairs of the
        output rows this part owns (rows in blocks of PART_ROWS dealt back and
        forth to the parts). `outputs` may supply dict(stat, p, n) buffers (entries
        of other parts are left as they are); otherwise new arrays are made,
        filled with NaN (stat, p) and -1 (n) where this part writes nothing."""
        torch = self.torch
        t = TESTS[test] if isinstance(test, str) else int(test)
        va, vb = _i32(vars_a), _i32(vars_b)
        na = len(va)
        nb = na if vb is None else len(vb)
        o = options(**opt)
        if outputs is not None:
            stat, p, n = outputs.get("stat"), outputs.get("p"), outputs.get("n")
        elif out == "numpy":
            stat = np.full((na, nb), np.nan)
            p = np.full((na, nb), np.nan)
            n = np.full((na, nb), -1, np.int32)
        else:
            dev = torch.device("cuda", self.device)
            stat = torch.full((na, nb), float("nan"), dtype=torch.float64, device=dev)
            p = torch.full((na, nb), float("nan"), dtype=torch.float64, device=dev)
            n = torch.full((na, nb), -1, dtype=torch.int32, device=dev)
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask, dtype=np.uint8) if isinstance(mask, np.ndarray) else mask
        self._check(lib.napg_run_part(self.h, t, C.byref(o), _ptr(m), _ptr(va), na, _ptr(vb),
                                      0 if vb is None else nb, int(part), int(nparts), _ptr(stat), _ptr(p), _ptr(n)))
        return {"stat": stat, "p": p, "n": n}

    def adjust(self, p, method="bh", symmetric=False, out=None):
        """Multiple-testing correction (Sec. 3.4) of a p-value matrix (numpy or
        device tensor): method "bonferroni", "bh" or "by"; symmetric=True for a
        variable set against itself (each pair i < j one test, NaN diagonal).
        Returns the adjusted matrix (numpy for numpy input, a device tensor
        otherwise), or writes `out`."""
        torch = self.torch
        mth = ADJUST[method] if isinstance(method, str) else int(method)
        if isinstance(p, np.ndarray):
            p = np.ascontiguousarray(p, dtype=np.float64)
            res = np.empty(p.shape, np.float64) if out is None else out
        else:
            p = p.contiguous()
            res = torch.empty(p.shape, dtype=torch.float64, device=p.device) if out is None else out
        rows, cols = (int(p.shape[0]), int(p.shape[1])) if len(p.shape) == 2 else (1, int(p.shape[0]))
        self._check(lib.napg_adjust(self.h, mth, _ptr(p), rows, cols, 1 if symmetric else 0, _ptr(res)))
        return res

    def release_cache(self):
        """Mark the cached planes and presort stale (the next run rebuilds them)."""
        self._check(lib.napg_release_cache(self.h))

    def tune(self, on=True):
        """Enable or disable the launch-shape autotuner (on by default)."""
        self._check(lib.napg_tune_enable(self.h, 1 if on else 0))

    def tune_pin(self, kind, choice):
        """Fix the launch-shape candidate of one kind (0-3 for the stacked
        contractions, 0-1 for the others); -1 unpins."""
        self._check(lib.napg_tune_pin(self.h, kind.encode(), int(choice)))

    def tune_read(self):
        import json
        buf = C.create_string_buffer(1 << 16)
        self._check(lib.napg_tune_read(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def trace(self, on=True):
        self._check(lib.napg_trace_enable(self.h, 1 if on else 0))

    def trace_read(self):
        import json
        buf = C.create_string_buffer(1 << 16)
        self._check(lib.napg_trace_read(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def run_batch(self, test, masks, vars_a, vars_b=None, out="numpy", outputs=None, sync=True, **opt):
        """One test for several sample contexts (a list of uint8 masks, host or
        device; None = every sample). Returns a list of dict(stat, p, n): numpy
        arrays (out="numpy"), or device tensors (out="cuda", stream-ordered;
        synchronised unless sync=False). Either way the batch runs as one captured
        CUDA graph; host outputs are written to a device region first and copied
        back. `outputs` may supply the per-context dict buffers to write."""
        torch = self.torch
        t = TESTS[test] if isinstance(test, str) else int(test)
        va, vb = _i32(vars_a), _i32(vars_b)
        na = len(va)
        nb = na if vb is None else len(vb)
        o = options(**opt)
        ms = [np.ascontiguousarray(m, dtype=np.uint8) if isinstance(m, np.ndarray) else m for m in masks]
        K = len(ms)
        if outputs is not None:
            outs = outputs
        elif out == "numpy":
            outs = [{"stat": np.empty((na, nb)), "p": np.empty((na, nb)), "n": np.empty((na, nb), np.int32)}
                    for _ in range(K)]
        else:
            dev = torch.device("cuda", self.device)
            outs = [{"stat": torch.empty((na, nb), dtype=torch.float64, device=dev),
                     "p": torch.empty((na, nb), dtype=torch.float64, device=dev),
                     "n": torch.empty((na, nb), dtype=torch.int32, device=dev)} for _ in range(K)]
        mp = (C.c_void_p * max(K, 1))(*[_ptr(m) for m in ms])
        sp = (C.c_void_p * max(K, 1))(*[_ptr(r.get("stat")) for r in outs])
        pp = (C.c_void_p * max(K, 1))(*[_ptr(r.get("p")) for r in outs])
        npp = (C.c_void_p * max(K, 1))(*[_ptr(r.get("n")) for r in outs])
        self._check(lib.napg_run_batch(self.h, t, C.byref(o), K, mp, _ptr(va), na, _ptr(vb),
                                       0 if vb is None else nb, sp, pp, npp))
        if out != "numpy" and sync:
            self.sync()
        return outs

    # ------------------------------------------------------------ serving --
    def serve_start(self, mem_budget=0, slots=4):
        """Start the request loop on the resident cohort (`slots` concurrent requests)."""
        self._serve_out = {}
        self._check(lib.napg_serve_start(self.h, int(mem_budget), int(slots)))

    def serve_submit(self, test, vars_a, vars_b=None, mask=None, **opt):
        """Queue one request; returns its ticket. Outputs are host arrays kept until done."""
        t = TESTS[test] if isinstance(test, str) else int(test)
        va, vb = _i32(vars_a), _i32(vars_b)
        na = len(va)
        nb = na if vb is None else len(vb)
        outs = {"stat": np.empty((na, nb)), "p": np.empty((na, nb)), "n": np.empty((na, nb), np.int32)}
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        r = Request()
        r.test = t
        r.opt = options(**opt)
        r.sample_mask = _ptr(m)
        r.vars_a = _ptr(va)
        r.n_a = na
        r.vars_b = _ptr(vb)
        r.n_b = 0 if vb is None else nb
        r.stat = _ptr(outs["stat"])
        r.pval = _ptr(outs["p"])
        r.n = _ptr(outs["n"])
        tk = C.c_uint64()
        self._check(lib.napg_serve_submit(self.h, C.byref(r), C.byref(tk)))
        self._serve_out[tk.value] = outs
        return tk.value

    def serve_poll(self, ticket):
        """(done, latency_ms, status, outputs-or-None); a finished ticket is reported once."""
        done, lat, st = C.c_int32(), C.c_double(), C.c_int32()
        self._check(lib.napg_serve_poll(self.h, C.c_uint64(ticket), C.byref(done), C.byref(lat), C.byref(st)))
        if not done.value:
            return False, None, None, None
        return True, lat.value, st.value, self._serve_out.pop(ticket, None)

    def serve_wait(self, ticket, poll_s=2e-4):
        while True:
            d, lat, st, out = self.serve_poll(ticket)
            if d:
                return lat, st, out
            time.sleep(poll_s)

    def serve_stop(self):
        self._check(lib.napg_serve_stop(self.h))

    def debug_integers(self, test, a, b, mask=None):
        t = TESTS[test] if isinstance(test, str) else int(test)
        out = np.zeros(4 + 2 * 64 + 64 * 64, np.int64)
        w = C.c_int64()
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self._check(lib.napg_debug_integers(self.h, t, _ptr(m), int(a), int(b), _ptr(out), len(out), C.byref(w)))
        return out[:w.value].copy()

    PVALUE_KINDS = {"corr": 0, "t": 1, "f": 2, "chi2": 3, "norm": 4, "ibeta": 5, "gamma_q": 6,
                    "erfcx_sqrt": 7, "erfcx_sqrt_cuda": 8}

    def debug_pvalues(self, kind, s, a=None, b=None):
        """The device p-value functions on given values (host float64 arrays)."""
        k = self.PVALUE_KINDS[kind] if isinstance(kind, str) else int(kind)
        s = np.ascontiguousarray(s, dtype=np.float64)
        a = None if a is None else np.ascontiguousarray(np.broadcast_to(a, s.shape), dtype=np.float64)
        b = None if b is None else np.ascontiguousarray(np.broadcast_to(b, s.shape), dtype=np.float64)
        out = np.empty_like(s)
        self._check(lib.napg_debug_pvalues(self.h, k, _ptr(s), _ptr(a), _ptr(b), s.size, _ptr(out)))
        return out


def serve_plan(est, age_ms, slot_mem, slot_busy, budget):
    """The serving loop's admission policy on given numbers (host only): the
    queue index each slot would take (-1 = none)."""
    e = np.ascontiguousarray(est, dtype=np.uint64)
    a = np.ascontiguousarray(age_ms, dtype=np.float64)
    m = np.ascontiguousarray(slot_mem, dtype=np.uint64)
    b = np.ascontiguousarray(slot_busy, dtype=np.int32)
    out = np.empty(len(m), np.int32)
    rc = lib.napg_serve_plan(_ptr(e), _ptr(a), len(e), _ptr(m), _ptr(b), len(m), int(budget), _ptr(out))
    if rc:
        raise NapgError(rc, "napg_serve_plan")
    return out


def version() -> str:
    return lib.napg_version().decode()


def kernel_launches() -> int:
    return int(lib.napg_kernel_launches())
