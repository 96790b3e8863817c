"""Thin ctypes binding of libcfust (include/cfust.h).

Argument marshalling only: every step of the E-step, M-step and fit runs in
the library's CUDA kernels.  PyTorch supplies device memory and the stream.
Loading fails loudly when the library is missing and cannot be built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CFUST_FP64 = 0
CFUST_FP32 = 1
STATUS = {0: "CFUST_OK", -1: "CFUST_EINVAL", -2: "CFUST_ENOTPD", -3: "CFUST_ENUMERIC",
          -4: "CFUST_EDEGENERATE", -5: "CFUST_ETIMEOUT", -6: "CFUST_ECUDA", -7: "CFUST_ENOMEM"}

EXPORTED = ["cfust_create", "cfust_destroy", "cfust_loglik", "cfust_estep", "cfust_mstep",
            "cfust_fit", "cfust_fit_begin", "cfust_fit_step", "cfust_fit_end", "cfust_fit_trace",
            "cfust_fit_batched", "cfust_batched_shape",
            "cfust_last_rescued", "cfust_last_sweep_ms", "cfust_normal_f32", "cfust_mstep_noalloc",
            "cfust_last_error",
            "cfust_surrogate_create", "cfust_surrogate_destroy", "cfust_surrogate_label",
            "cfust_surrogate_predict", "cfust_surrogate_gradient", "cfust_surrogate_get_params",
            "cfust_surrogate_set_params", "cfust_surrogate_train", "cfust_surrogate_last_error",
            "cfust_set_surrogate", "cfust_last_fallback", "cfust_surrogate_problems",
            "cfust_surrogate_finetune", "cfust_fit_multistart", "cfust_kmeans", "cfust_init_partition",
            "cfust_multistart_partitions", "cfust_loglik_shifts", "cfust_last_mstep_ms", "cfust_mstep_sums", "cfust_mstep_apply", "cfust_surrogate_inputs"]

SURROGATE_NPARAM = 35338


class CfustError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class cfust_params(ctypes.Structure):
    _fields_ = [("g", ctypes.c_int), ("p", ctypes.c_int), ("r", ctypes.c_int),
                ("pi", ctypes.POINTER(ctypes.c_double)), ("mu", ctypes.POINTER(ctypes.c_double)),
                ("Sigma", ctypes.POINTER(ctypes.c_double)), ("Delta", ctypes.POINTER(ctypes.c_double)),
                ("nu", ctypes.POINTER(ctypes.c_double))]


class cfust_lattice(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("dim", ctypes.c_int),
                ("z", ctypes.POINTER(ctypes.c_int64)), ("shift", ctypes.POINTER(ctypes.c_double))]


class cfust_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("lattice", cfust_lattice), ("e2_mode", ctypes.c_int),
                ("nu_min", ctypes.c_double), ("nu_max", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("use_graph", ctypes.c_int),
                ("timing", ctypes.c_int), ("pairs_per_warp", ctypes.c_int), ("autotune", ctypes.c_int),
                ("triage_nats", ctypes.c_double), ("prioritise", ctypes.c_int),
                ("test_wait_polls", ctypes.c_int), ("fused", ctypes.c_int), ("shared_points", ctypes.c_int)]


_LIB = None


def load(build_if_missing: bool = True, path: str | None = None) -> ctypes.CDLL:
    """Load libcfust.so (building it in-tree with nvcc when absent or stale).
    `path` loads another build of the same library instead."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    if path is None:
        path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libcfust.so not found at {path}")
    lib = ctypes.CDLL(path)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    P = ctypes.POINTER(cfust_params)
    sig = {
        "cfust_create": ([ctypes.POINTER(vp), ctypes.POINTER(cfust_opts), vp], ctypes.c_int),
        "cfust_destroy": ([vp], ctypes.c_int),
        "cfust_loglik": ([vp, vp, i64, P, dp], ctypes.c_int),
        "cfust_estep": ([vp, vp, i64, P, vp, vp, vp, vp, vp, vp, dp], ctypes.c_int),
        "cfust_mstep": ([vp, vp, i64, vp, vp, vp, vp, vp, P], ctypes.c_int),
        "cfust_fit": ([vp, vp, i64, P, dp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_fit_begin": ([vp, vp, i64, P], ctypes.c_int),
        "cfust_fit_step": ([vp, ctypes.c_int], ctypes.c_int),
        "cfust_fit_end": ([vp, P, dp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_fit_trace": ([vp, dp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_fit_batched": ([vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(i64), P, dp,
                               ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_batched_shape": ([vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_last_rescued": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
        "cfust_last_sweep_ms": ([vp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "cfust_last_mstep_ms": ([vp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "cfust_last_error": ([vp], ctypes.c_char_p),
        "cfust_normal_f32": ([vp, vp, i64, ctypes.c_int, vp], ctypes.c_int),
        "cfust_mstep_noalloc": ([ctypes.c_int, vp, i64, vp, vp, vp, vp, vp, ctypes.c_double,
                                 ctypes.c_double, P, vp], ctypes.c_int),
        "cfust_surrogate_create": ([ctypes.POINTER(vp), ctypes.c_uint64, ctypes.POINTER(cfust_lattice), vp],
                                   ctypes.c_int),
        "cfust_surrogate_destroy": ([vp], ctypes.c_int),
        "cfust_surrogate_label": ([vp, vp, vp, i64], ctypes.c_int),
        "cfust_surrogate_predict": ([vp, vp, vp, i64], ctypes.c_int),
        "cfust_surrogate_gradient": ([vp, vp, vp, i64, dp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "cfust_surrogate_get_params": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
                                       ctypes.c_int),
        "cfust_surrogate_set_params": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
                                       ctypes.c_int),
        "cfust_surrogate_train": ([vp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
        "cfust_surrogate_last_error": ([vp], ctypes.c_char_p),
        "cfust_set_surrogate": ([vp, vp], ctypes.c_int),
        "cfust_last_fallback": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
        "cfust_surrogate_problems": ([vp, vp, i64, P, i64, vp, i64, ctypes.POINTER(i64)], ctypes.c_int),
        "cfust_fit_multistart": ([vp, vp, i64, P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp,
                                  ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_kmeans": ([vp, vp, i64, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, vp,
                          ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_init_partition": ([vp, vp, i64, vp, ctypes.c_double, ctypes.c_double, P], ctypes.c_int),
        "cfust_loglik_shifts": ([vp, vp, i64, P, ctypes.c_int, dp, dp], ctypes.c_int),
        "cfust_multistart_partitions": ([vp, vp, i64, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, P, ctypes.POINTER(ctypes.c_int), dp,
                                         ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cfust_surrogate_inputs": ([vp, vp, i64, P, vp, vp], ctypes.c_int),
        "cfust_mstep_sums": ([vp, vp, i64, vp, vp, vp, vp, vp, P, dp], ctypes.c_int),
        "cfust_mstep_apply": ([vp, dp, i64, P], ctypes.c_int),
        "cfust_surrogate_finetune": ([vp, vp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


class _HostParams:
    """cfust_params view over contiguous float64 numpy copies (kept alive here)."""

    def __init__(self, params):
        self.arrays = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in params.as_arrays()]
        pi, mu, Sigma, Delta, nu = self.arrays
        dp = ctypes.POINTER(ctypes.c_double)
        self.c = cfust_params(int(pi.shape[0]), int(mu.shape[1]), int(Delta.shape[2]),
                              pi.ctypes.data_as(dp), mu.ctypes.data_as(dp), Sigma.ctypes.data_as(dp),
                              Delta.ctypes.data_as(dp), nu.ctypes.data_as(dp))

    def to_params(self):
        from .synth import Params
        return Params(*(a.copy() for a in self.arrays))


def _zero_params(g, p, r):
    from .synth import Params
    return Params(np.zeros(g), np.zeros((g, p)), np.zeros((g, p, p)), np.zeros((g, p, r)), np.zeros(g))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _check_mstep_inputs(Y, E, params, dtype):
    """Shapes, dtypes, contiguity and device of the M-step's device inputs
    (Y [n][p] float64; tau, e1, e2 [g][n], e3 [g][r][n], e4 [g][r(r+1)/2][n]
    in the E-step's element type), so that a mismatch raises here instead of
    letting a kernel read past a buffer."""
    import torch
    g, r = params.g, params.r
    p = params.mu.shape[1]
    if Y.dim() != 2 or Y.shape[1] != p or Y.dtype != torch.float64:
        raise ValueError(f"Y must be float64 [n][{p}], got {Y.dtype} {tuple(Y.shape)}")
    n = Y.shape[0]
    want = {"tau": (g, n), "e1": (g, n), "e2": (g, n), "e3": (g, r, n), "e4": (g, r * (r + 1) // 2, n)}
    dev = torch.device("cuda", torch.cuda.current_device())
    for k, shp in want.items():
        t = E[k]
        if tuple(t.shape) != shp or t.dtype != dtype:
            raise ValueError(f"{k} must be {dtype} {shp}, got {t.dtype} {tuple(t.shape)}")
    for k, t in [("Y", Y)] + [(k, E[k]) for k in want]:
        if not t.is_contiguous() or t.device != dev:
            raise ValueError(f"{k} must be contiguous and on the current CUDA device {dev}")
    return n


class Context:
    """A cfust_ctx bound to the current CUDA device and a torch stream."""

    def __init__(self, lattice, precision=CFUST_FP32, e2_mode=0, nu_min=0.0, nu_max=0.0,
                 max_iter=0, tol=0.0, use_graph=True, timing=False, pairs_per_warp=0, autotune=False,
                 stream=None, triage_nats=0.0, prioritise=False, test_wait_polls=0, fused=False,
                 shared_points=False):
        import torch
        self.lib = load()
        self._z = np.ascontiguousarray(lattice.z, dtype=np.int64)
        self._shift = np.ascontiguousarray(lattice.shift, dtype=np.float64)
        lat = cfust_lattice(int(lattice.n), int(self._z.shape[0]),
                            self._z.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            self._shift.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self.opts = cfust_opts(int(precision), lat, int(e2_mode), float(nu_min), float(nu_max),
                               int(max_iter), float(tol), 1 if use_graph else 0, 1 if timing else 0,
                               int(pairs_per_warp), 1 if autotune else 0, float(triage_nats),
                               1 if prioritise else 0, int(test_wait_polls), 1 if fused else 0,
                               1 if shared_points else 0)
        self.precision = int(precision)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.lattice_n = int(lattice.n)
        h = ctypes.c_void_p()
        st = self.lib.cfust_create(ctypes.byref(h), ctypes.byref(self.opts),
                                   ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise CfustError(st, self.lib.cfust_last_error(None).decode())
        self.h = h

    # -- helpers ---------------------------------------------------------
    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == CFUST_FP64 else torch.float32

    def _check(self, st):
        if st != 0:
            raise CfustError(st, self.lib.cfust_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.cfust_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- ABI calls (same names as the C entry points) ----------------------
    def cfust_loglik(self, Y, params) -> float:
        hp = _HostParams(params)
        out = ctypes.c_double()
        self._check(self.lib.cfust_loglik(self.h, _ptr(Y), Y.shape[0], ctypes.byref(hp.c), ctypes.byref(out)))
        return out.value

    def alloc_estep(self, n, g, r, device=None):
        import torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        kw = dict(dtype=self.dtype, device=dev)
        rp = r * (r + 1) // 2
        return dict(logf=torch.empty((g, n), **kw), tau=torch.empty((g, n), **kw),
                    e1=torch.empty((g, n), **kw), e2=torch.empty((g, n), **kw),
                    e3=torch.empty((g, r, n), **kw), e4=torch.empty((g, rp, n), **kw))

    def cfust_estep(self, Y, params, out=None):
        """Returns dict(logf, tau, e1, e2, e3[g,r,n], e4[g,r(r+1)/2,n], loglik)."""
        n = Y.shape[0]
        if out is None:
            out = self.alloc_estep(n, params.g, params.r, Y.device)
        hp = _HostParams(params)
        ll = ctypes.c_double()
        self._check(self.lib.cfust_estep(self.h, _ptr(Y), n, ctypes.byref(hp.c), _ptr(out["logf"]),
                                         _ptr(out["tau"]), _ptr(out["e1"]), _ptr(out["e2"]),
                                         _ptr(out["e3"]), _ptr(out["e4"]), ctypes.byref(ll)))
        out = dict(out)
        out["loglik"] = ll.value
        return out

    def cfust_mstep(self, Y, E, params):
        _check_mstep_inputs(Y, E, params, self.dtype)
        hp = _HostParams(params)
        self._check(self.lib.cfust_mstep(self.h, _ptr(Y), Y.shape[0], _ptr(E["tau"]), _ptr(E["e1"]),
                                         _ptr(E["e2"]), _ptr(E["e3"]), _ptr(E["e4"]), ctypes.byref(hp.c)))
        return hp.to_params()

    def cfust_mstep_sums(self, Y, E, params):
        """The eight per-component sums over Y's rows: float64 [g][K] (numpy)."""
        _check_mstep_inputs(Y, E, params, self.dtype)
        hp = _HostParams(params)
        sums = np.zeros((params.g, sums_width(params.mu.shape[1], params.r)))
        self._check(self.lib.cfust_mstep_sums(self.h, _ptr(Y), Y.shape[0], _ptr(E["tau"]), _ptr(E["e1"]),
                                              _ptr(E["e2"]), _ptr(E["e3"]), _ptr(E["e4"]), ctypes.byref(hp.c),
                                              sums.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return sums

    def cfust_mstep_apply(self, sums, n_total, params):
        """Algorithm 3's update from sums totalled over every worker's rows."""
        hp = _HostParams(params)
        sums = np.ascontiguousarray(sums, dtype=np.float64)
        if sums.shape != (params.g, sums_width(params.mu.shape[1], params.r)):
            raise ValueError(f"sums must be [g][K], got {sums.shape}")
        self._check(self.lib.cfust_mstep_apply(self.h, sums.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               int(n_total), ctypes.byref(hp.c)))
        return hp.to_params()

    def cfust_fit(self, Y, params, max_iter=None):
        if max_iter is not None and max_iter != self.opts.max_iter:
            raise ValueError("max_iter is fixed at context creation")
        hp = _HostParams(params)
        trace = np.zeros(self.opts.max_iter + 1)
        done = ctypes.c_int()
        self._check(self.lib.cfust_fit(self.h, _ptr(Y), Y.shape[0], ctypes.byref(hp.c),
                                       trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(done)))
        return hp.to_params(), trace[:done.value + 1], done.value

    def cfust_fit_begin(self, Y, params):
        self._fit_hp = _HostParams(params)
        self._fit_Y = Y  # keep the device buffer alive until cfust_fit_end
        self._check(self.lib.cfust_fit_begin(self.h, _ptr(Y), Y.shape[0], ctypes.byref(self._fit_hp.c)))

    def cfust_fit_step(self, iters=1):
        self._check(self.lib.cfust_fit_step(self.h, int(iters)))

    def cfust_fit_trace(self):
        buf = np.zeros(max(1, self.opts.max_iter))
        cnt = ctypes.c_int()
        self._check(self.lib.cfust_fit_trace(self.h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             ctypes.byref(cnt)))
        return buf[:cnt.value]

    def cfust_fit_end(self):
        hp = self._fit_hp
        trace = np.zeros(self.opts.max_iter + 1)
        done = ctypes.c_int()
        self._check(self.lib.cfust_fit_end(self.h, ctypes.byref(hp.c),
                                           trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.byref(done)))
        self._fit_Y = None
        return hp.to_params(), trace[:done.value + 1], done.value

    def cfust_fit_batched(self, Ys, params_list):
        """Fit every (Y, params) pair together.  Returns (params list, traces
        [nfits][max_iter+1], per-fit status list)."""
        nf = len(Ys)
        hps = [_HostParams(p) for p in params_list]
        arr = (cfust_params * nf)(*[h.c for h in hps])
        yp = (ctypes.c_void_p * nf)(*[y.data_ptr() for y in Ys])
        ns = (ctypes.c_int64 * nf)(*[int(y.shape[0]) for y in Ys])
        trace = np.zeros((nf, self.opts.max_iter + 1))
        st = (ctypes.c_int * nf)()
        rc = self.lib.cfust_fit_batched(self.h, nf, yp, ns, arr, trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        st)
        self._check(rc)
        # the library wrote the updated parameters through the struct pointers
        return [h.to_params() for h in hps], trace, list(st)

    def cfust_fit_multistart(self, Y, starts, burn_in):
        """Returns (index of the chosen start, its fitted params, trace, iterations,
        the burned-in params of every start)."""
        ns = len(starts)
        hps = [_HostParams(p) for p in starts]
        arr = (cfust_params * ns)(*[h.c for h in hps])
        trace = np.zeros(self.opts.max_iter + 1)
        best, done = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.cfust_fit_multistart(self.h, _ptr(Y), Y.shape[0], arr, ns, int(burn_in),
                                                  ctypes.byref(best), trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                  ctypes.byref(done)))
        out = [h.to_params() for h in hps]
        return best.value, out[best.value], trace[:done.value + 1], done.value, out

    def cfust_loglik_shifts(self, Y, params, shifts):
        """l(Psi) under each shift (rows of `shifts`, [M][dim]) of the context's
        lattice; returns float64 [M].  Mean and sd / sqrt(M) estimate l and
        the rule's integration error."""
        hp = _HostParams(params)
        S = np.ascontiguousarray(shifts, dtype=np.float64)
        out = np.zeros(S.shape[0])
        dpp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.cfust_loglik_shifts(self.h, _ptr(Y), Y.shape[0], ctypes.byref(hp.c), S.shape[0],
                                                 S.ctypes.data_as(dpp), out.ctypes.data_as(dpp)))
        return out

    def cfust_kmeans(self, Y, centers0, max_iter, labels=None):
        """Lloyd's k-means from host centres [g][p].  Returns (labels: device
        int32 tensor [n], final centres, assignment passes)."""
        import torch
        C = np.ascontiguousarray(centers0, dtype=np.float64).copy()
        g, p = C.shape
        if labels is None:
            labels = torch.empty(Y.shape[0], dtype=torch.int32, device=Y.device)
        it = ctypes.c_int()
        self._check(self.lib.cfust_kmeans(self.h, _ptr(Y), Y.shape[0], p, g,
                                          C.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(max_iter),
                                          _ptr(labels), ctypes.byref(it)))
        return labels, C, it.value

    def cfust_init_partition(self, Y, labels, g, r, nu0=10.0, lam=0.5):
        """Psi^(0) of the partition `labels` (device int32 [n]) by moments."""
        hp = _HostParams(_zero_params(g, Y.shape[1], r))
        self._check(self.lib.cfust_init_partition(self.h, _ptr(Y), Y.shape[0], _ptr(labels), float(nu0),
                                                  float(lam), ctypes.byref(hp.c)))
        return hp.to_params()

    def cfust_multistart_partitions(self, Y, labels, g, r, nu0=10.0, lam=0.5, burn_in=0):
        """Algorithm 1 from partitions (device int32 [m][n]).  Returns (index of
        the chosen partition, its fitted params, trace, iterations, every
        start's initial (or burned-in) params)."""
        m = labels.shape[0]
        hps = [_HostParams(_zero_params(g, Y.shape[1], r)) for _ in range(m)]
        arr = (cfust_params * m)(*[h.c for h in hps])
        trace = np.zeros(self.opts.max_iter + 1)
        best, done = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.cfust_multistart_partitions(
            self.h, _ptr(Y), Y.shape[0], _ptr(labels), m, float(nu0), float(lam), int(burn_in), arr,
            ctypes.byref(best), trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(done)))
        out = [h.to_params() for h in hps]
        return best.value, out[best.value], trace[:done.value + 1], done.value, out

    def cfust_batched_shape(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.cfust_batched_shape(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def cfust_last_sweep_ms(self) -> float:
        v = ctypes.c_float()
        self._check(self.lib.cfust_last_sweep_ms(self.h, ctypes.byref(v)))
        return v.value

    def cfust_last_mstep_ms(self) -> float:
        v = ctypes.c_float()
        self._check(self.lib.cfust_last_mstep_ms(self.h, ctypes.byref(v)))
        return v.value

    def cfust_last_rescued(self) -> int:
        v = ctypes.c_int64()
        self._check(self.lib.cfust_last_rescued(self.h, ctypes.byref(v)))
        return v.value

    def cfust_set_surrogate(self, sur):
        """Attach a Surrogate (None detaches); the context keeps a reference."""
        self._sur = sur
        self._check(self.lib.cfust_set_surrogate(self.h, None if sur is None else sur.h))

    def cfust_last_fallback(self) -> int:
        v = ctypes.c_int64()
        self._check(self.lib.cfust_last_fallback(self.h, ctypes.byref(v)))
        return v.value

    def cfust_surrogate_inputs(self, Y, params):
        """Both network inputs of every pair as the surrogate E-step forms them:
        (x [g][n][2][7] float32 (BF16-rounded), kind [g][n] int32) on the device."""
        import torch
        n, g = Y.shape[0], params.g
        x = torch.empty((g, n, 2, 7), dtype=torch.float32, device=Y.device)
        kind = torch.empty((g, n), dtype=torch.int32, device=Y.device)
        hp = _HostParams(params)
        self._check(self.lib.cfust_surrogate_inputs(self.h, _ptr(Y), n, ctypes.byref(hp.c), _ptr(x), _ptr(kind)))
        return x, kind

    def cfust_surrogate_problems(self, Y, params, stride=1, max_rows=None):
        """Standardised problems (float32 CUDA tensor [rows, 7]) of every
        stride-th pair in the surrogate's domain at `params` (r = 3)."""
        import torch
        if max_rows is None:
            max_rows = 2 * ((params.g * Y.shape[0] + stride - 1) // stride)
        x = torch.empty((max_rows, 7), dtype=torch.float32, device=Y.device)
        hp = _HostParams(params)
        rows = ctypes.c_int64()
        self._check(self.lib.cfust_surrogate_problems(self.h, _ptr(Y), Y.shape[0], ctypes.byref(hp.c), int(stride),
                                                      _ptr(x), int(max_rows), ctypes.byref(rows)))
        return x[:rows.value]


class Surrogate:
    """A cfust_surrogate (learned form of the r = 3 lattice integrals)."""

    def __init__(self, lattice, seed=0, stream=None):
        import torch
        self.lib = load()
        self._z = np.ascontiguousarray(lattice.z, dtype=np.int64)
        self._shift = np.ascontiguousarray(lattice.shift, dtype=np.float64)
        lat = cfust_lattice(int(lattice.n), int(self._z.shape[0]),
                            self._z.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            self._shift.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.cfust_surrogate_create(ctypes.byref(h), int(seed), ctypes.byref(lat),
                                             ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise CfustError(st, self.lib.cfust_surrogate_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != 0:
            raise CfustError(st, self.lib.cfust_surrogate_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.cfust_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, x, cols):
        import torch
        return torch.empty((x.shape[0], cols), dtype=torch.float32, device=x.device)

    def cfust_surrogate_label(self, x):
        y = self._out(x, 10)
        self._check(self.lib.cfust_surrogate_label(self.h, _ptr(x), _ptr(y), x.shape[0]))
        return y

    def cfust_surrogate_predict(self, x):
        y = self._out(x, 10)
        self._check(self.lib.cfust_surrogate_predict(self.h, _ptr(x), _ptr(y), x.shape[0]))
        return y

    def cfust_surrogate_gradient(self, x, y):
        loss = ctypes.c_double()
        g = np.zeros(SURROGATE_NPARAM, dtype=np.float32)
        self._check(self.lib.cfust_surrogate_gradient(self.h, _ptr(x), _ptr(y), x.shape[0], ctypes.byref(loss),
                                                      g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return loss.value, g

    def cfust_surrogate_get_params(self):
        th = np.zeros(SURROGATE_NPARAM, dtype=np.float32)
        nm = np.zeros(20, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(self.lib.cfust_surrogate_get_params(self.h, th.ctypes.data_as(fp), nm.ctypes.data_as(fp)))
        return th, nm

    def cfust_surrogate_set_params(self, theta, norm=None):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        nm = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
        self._check(self.lib.cfust_surrogate_set_params(self.h, th.ctypes.data_as(fp),
                                                        None if nm is None else nm.ctypes.data_as(fp)))

    def cfust_surrogate_finetune(self, x, epochs, batch=16384, lr=5e-4, seed=1):
        trace = np.zeros(epochs, dtype=np.float32)
        self._check(self.lib.cfust_surrogate_finetune(self.h, _ptr(x), x.shape[0], int(epochs), int(batch),
                                                      float(lr), int(seed),
                                                      trace.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return trace

    def cfust_surrogate_train(self, n_train, epochs, batch=4096, lr=2e-3, seed=1):
        trace = np.zeros(epochs, dtype=np.float32)
        self._check(self.lib.cfust_surrogate_train(self.h, int(n_train), int(epochs), int(batch), float(lr),
                                                   int(seed), trace.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return trace


def cfust_normal_f32(x, which, stream=None):
    """Evaluate one of the library's single-precision normal functions on a
    float32 CUDA tensor (see include/cfust.h for `which`)."""
    import torch
    lib = load()
    out = torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.cfust_normal_f32(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.numel(),
                              int(which), ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise CfustError(rc, "cfust_normal_f32 failed")
    st.synchronize()
    return out


def cfust_mstep_noalloc(precision, Y, E, params, nu_min=0.0, nu_max=0.0, stream=None):
    """M-step through the allocation-free entry point (no context; scratch in a
    static device array, see include/cfust.h).  Returns the updated params."""
    import torch
    if precision not in (CFUST_FP64, CFUST_FP32):
        raise ValueError("precision must be CFUST_FP64 or CFUST_FP32")
    _check_mstep_inputs(Y, E, params, torch.float64 if precision == CFUST_FP64 else torch.float32)
    lib = load()
    hp = _HostParams(params)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.cfust_mstep_noalloc(int(precision), _ptr(Y), Y.shape[0], _ptr(E["tau"]), _ptr(E["e1"]),
                                 _ptr(E["e2"]), _ptr(E["e3"]), _ptr(E["e4"]), float(nu_min), float(nu_max),
                                 ctypes.byref(hp.c), ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise CfustError(rc, lib.cfust_last_error(None).decode())
    return hp.to_params()


def sums_width(p, r):
    """Doubles in one component's sums vector (S1..S8 of Section 3.2)."""
    return 3 + p + r + p * r + r * (r + 1) // 2 + p * (p + 1) // 2


def unpack_e4(e4, r):
    """[.., r(r+1)/2, n] packed lower triangle -> [.., n, r, r] symmetric (numpy)."""
    e4 = np.asarray(e4)
    lead = e4.shape[:-2]
    n = e4.shape[-1]
    full = np.zeros(lead + (n, r, r))
    for t in range(r):
        for h in range(t + 1):
            v = e4[..., t * (t + 1) // 2 + h, :]
            full[..., :, t, h] = v
            full[..., :, h, t] = v
    return full
