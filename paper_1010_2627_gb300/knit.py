"""Thin ctypes binding of the C-ABI in ``include/knit.h`` (libknit.so).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C entry points.  The functions keep the C names
(``knit_system_create``, ``knit_lead_selfenergy``, ``knit_transmission``,
``knit_transmission_sigma``, ``knit_ldos``, ...); arrays may be numpy arrays
(host memory) or torch CUDA tensors (device memory), and ``stream`` may be a
``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer.

The library must have been built (``paper_1010_2627_gb300.build.build()``);
loading fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

KNIT_OK, KNIT_ERR_INVALID, KNIT_ERR_OOM, KNIT_ERR_CUDA = 0, 1, 2, 3
KNIT_ERR_SINGULAR, KNIT_ERR_NOCONVERGE, KNIT_ERR_TIMEOUT, KNIT_ERR_NONFINITE = 4, 5, 6, 7
KNIT_FP64, KNIT_MIXED, KNIT_MIXED_CUDACORE = 0, 1, 2
KNIT_LEAD_AUTO, KNIT_LEAD_MODES, KNIT_LEAD_DECIMATION, KNIT_LEAD_LEARNED = 0, 1, 2, 3
KNIT_PEAK_MMA_BF16, KNIT_PEAK_MMA_TF32, KNIT_PEAK_DFMA, KNIT_PEAK_FFMA = 0, 1, 2, 3
KNIT_PEAK_MMA_N64, KNIT_PEAK_MMA_N16, KNIT_PEAK_MMA_RESIDUAL = 4, 5, 6
KNIT_PEAK_MMA_RESIDUAL_TF32 = 7
KNIT_SWEEP_FP64, KNIT_SWEEP_MIXED_NARROW, KNIT_SWEEP_MIXED_CUDACORE = 0, 1, 2
KNIT_SWEEP_MIXED_TC128, KNIT_SWEEP_MIXED_HALF_ROWS = 3, 4

P = ctypes.c_void_p
i32, f64 = ctypes.c_int32, ctypes.c_double


class knit_system_desc(ctypes.Structure):
    _fields_ = [("M", i32), ("L", i32), ("block", i32), ("onsite_sign", P), ("H0", P),
                ("onsite", P), ("V", P), ("Vperiod", i32), ("lead_H0", P * 2), ("lead_V", P * 2),
                ("lead_Vperiod", i32 * 2)]


class knit_lead_opts(ctypes.Structure):
    _fields_ = [("method", i32), ("eta", f64), ("tol", f64), ("maxit", i32), ("model", P * 2)]


class knit_graph_desc(ctypes.Structure):
    _fields_ = [("N", i32), ("H", P), ("n_lead_sites", i32 * 2), ("lead_sites", P * 2)]


class knit_graph_multi_desc(ctypes.Structure):
    _fields_ = [("N", i32), ("H", P), ("n_leads", i32), ("n_lead_sites", P), ("lead_sites", P)]


class KnitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"knit error {code}: {msg}")
        self.code = code


_lib = None

# every entry point the header declares, with its ctypes signature
_SIGS = {
    "knit_system_create": (i32, [P, P]),
    "knit_system_destroy": (i32, [P]),
    "knit_lead_selfenergy": (i32, [P, i32, P, i32, P, P, P, P, P]),
    "knit_transmission": (i32, [P, P, i32, P, i32, f64, i32, P, P, P, P]),
    "knit_transmission_sigma": (i32, [P, P, i32, P, i32, f64, P, P, i32, P, P, P]),
    "knit_ldos": (i32, [P, P, i32, P, i32, f64, i32, i32, P, P, P, P, P]),
    "knit_transmission_eigenvalues": (i32, [P, P, i32, P, i32, f64, i32, P, P, P, P, P, P]),
    "knit_lesser": (i32, [P, P, i32, P, i32, f64, i32, P, P, P, P, P, P, P, P]),
    "knit_system_num_edges": (i32, [P, P]),
    "knit_system_info": (i32, [P, i32, P, P]),
    "knit_graph_create": (i32, [P, P]),
    "knit_graph_destroy": (i32, [P]),
    "knit_graph_slices": (i32, [P, P, P, P]),
    "knit_graph_transmission": (i32, [P, P, i32, P, P, P, P, P]),
    "knit_graph_create_multi": (i32, [P, P]),
    "knit_graph_plan": (i32, [P, P, P]),
    "knit_debug_fail_alloc_after": (i32, [ctypes.c_int64]),
    "knit_graph_conductance": (i32, [P, P, i32, P, P, P, P]),
    "knit_lead_decimation_noalloc": (i32, [P, P, i32, i32, P, i32, f64, f64, i32, P, P, P, P]),
    "knit_batch_create": (i32, [P, i32, P, i32, i32, P]),
    "knit_lead_model_train": (i32, [P, i32, P, i32, i32, i32, ctypes.c_float, ctypes.c_uint64,
                                    P, P, P, P]),
    "knit_lead_model_destroy": (i32, [P]),
    "knit_lead_model_num_params": (ctypes.c_int64, [P]),
    "knit_lead_model_num_outputs": (ctypes.c_int64, [P]),
    "knit_lead_model_get_params": (i32, [P, P]),
    "knit_lead_model_set_params": (i32, [P, P]),
    "knit_lead_model_forward": (i32, [P, P, i32, P, P]),
    "knit_lead_model_gradient": (i32, [P, P, P, i32, P, P, P]),
    "knit_batch_destroy": (i32, [P]),
    "knit_batch_transmission": (i32, [P, P, P, P, P, P, P, P]),
    "knit_batch_buckets": (i32, [P, P, P, P, P, P]),
    "knit_batch_configure": (i32, [P, P]),
    "knit_batch_autotune": (i32, [P, P, P, P, P, P, P]),
    "knit_peak_probe": (i32, [i32, ctypes.c_int64, i32, P, P, P]),
    "knit_debug_wait_probe": (i32, [ctypes.c_int64, P, P]),
    "knit_last_error": (ctypes.c_char_p, []),
    "knit_version": (ctypes.c_char_p, []),
}


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libknit.so (must be built).  Raises if it is missing."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: the CUDA library must be built "
                               "(paper_1010_2627_gb300.build.build()); there is no fallback")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def knit_last_error() -> str:
    return load().knit_last_error().decode()


def knit_version() -> str:
    return load().knit_version().decode()


def _check(rc: int):
    if rc != KNIT_OK:
        raise KnitError(rc, knit_last_error())


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return P(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return P(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return P(stream.cuda_stream)
    return P(int(stream))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _opts(method=KNIT_LEAD_AUTO, eta=0.0, tol=0.0, maxit=0, models=(None, None)):
    o = knit_lead_opts(int(method), float(eta), float(tol), int(maxit))
    for p in range(2):
        o.model[p] = models[p]
    return o


# ---------------------------------------------------------------------------
# C entry points with the C names

def knit_system_create(M, L, H0, V, block=1, onsite_sign=None, onsite=None, lead_H0=(None, None),
                       lead_V=(None, None), lead_Vperiod=(0, 0)):
    """Create a system (see include/knit.h); returns an opaque handle (int).
    A lead_V[p] of shape (2, M, M) is a period-2 lead [V_first, V_second]."""
    H0 = _c128(H0)
    V = _c128(V)
    Vp = 1 if V.ndim == 2 else V.shape[0]
    keep = [H0, V]
    d = knit_system_desc()
    d.M, d.L, d.block, d.Vperiod = int(M), int(L), int(block), int(Vp)
    d.H0, d.V = _ptr(H0), _ptr(V)
    if onsite_sign is not None:
        s = np.ascontiguousarray(onsite_sign, dtype=np.float64)
        keep.append(s)
        d.onsite_sign = _ptr(s)
    if onsite is not None:
        o = np.ascontiguousarray(onsite, dtype=np.float64)
        keep.append(o)
        d.onsite = _ptr(o)
    for p in range(2):
        if lead_H0[p] is not None:
            h = _c128(lead_H0[p])
            keep.append(h)
            d.lead_H0[p] = h.ctypes.data
        d.lead_Vperiod[p] = int(lead_Vperiod[p])
        if lead_V[p] is not None:
            v = _c128(lead_V[p])
            keep.append(v)
            d.lead_V[p] = v.ctypes.data
            if v.ndim == 3 and v.shape[0] == 2:
                d.lead_Vperiod[p] = 2
    h = P()
    _check(load().knit_system_create(ctypes.byref(d), ctypes.byref(h)))
    return h.value


def knit_system_destroy(handle):
    _check(load().knit_system_destroy(P(handle)))


def knit_lead_selfenergy(handle, lead, E, sigma, opts=None, iters=None, residual=None,
                         stream=None):
    o = opts if opts is not None else None
    _check(load().knit_lead_selfenergy(P(handle), int(lead), _ptr(E), int(len(E)),
                                       None if o is None else ctypes.byref(o), _ptr(sigma),
                                       _ptr(iters), _ptr(residual), _stream(stream)))


def knit_transmission(handle, E, seeds, W, precision, T, status=None, opts=None, nE=None, nS=None,
                      stream=None):
    nE = len(E) if nE is None else nE
    nS = (1 if seeds is None else len(seeds)) if nS is None else nS
    _check(load().knit_transmission(P(handle), _ptr(E), int(nE), _ptr(seeds), int(nS), float(W),
                                    int(precision), None if opts is None else ctypes.byref(opts),
                                    _ptr(T), _ptr(status), _stream(stream)))


def knit_transmission_sigma(handle, E, seeds, W, sigmaL, sigmaR, precision, T, status=None,
                            nE=None, nS=None, stream=None):
    nE = len(E) if nE is None else nE
    nS = (1 if seeds is None else len(seeds)) if nS is None else nS
    _check(load().knit_transmission_sigma(P(handle), _ptr(E), int(nE), _ptr(seeds), int(nS),
                                          float(W), _ptr(sigmaL), _ptr(sigmaR), int(precision),
                                          _ptr(T), _ptr(status), _stream(stream)))


def knit_transmission_eigenvalues(handle, E, seeds, W, precision, tau, noise=None, T=None,
                                  status=None, opts=None, nE=None, nS=None, stream=None):
    nE = len(E) if nE is None else nE
    nS = (1 if seeds is None else len(seeds)) if nS is None else nS
    _check(load().knit_transmission_eigenvalues(P(handle), _ptr(E), int(nE), _ptr(seeds), int(nS),
                                                float(W), int(precision),
                                                None if opts is None else ctypes.byref(opts),
                                                _ptr(tau), _ptr(noise), _ptr(T), _ptr(status),
                                                _stream(stream)))


def knit_lesser(handle, E, seeds, W, saving_level, rhoL=None, rhoR=None, jx=None, jt=None,
                T=None, status=None, opts=None, nE=None, nS=None, stream=None):
    nE = len(E) if nE is None else nE
    nS = (1 if seeds is None else len(seeds)) if nS is None else nS
    _check(load().knit_lesser(P(handle), _ptr(E), int(nE), _ptr(seeds), int(nS), float(W),
                              int(saving_level), None if opts is None else ctypes.byref(opts),
                              _ptr(rhoL), _ptr(rhoR), _ptr(jx), _ptr(jt), _ptr(T), _ptr(status),
                              _stream(stream)))


def knit_graph_create(H, lead0, lead1):
    """Handle of an arbitrary two-lead geometry (H: N x N complex128)."""
    H = np.ascontiguousarray(H, dtype=np.complex128)
    l0 = np.ascontiguousarray(lead0, dtype=np.int32)
    l1 = np.ascontiguousarray(lead1, dtype=np.int32)
    d = knit_graph_desc()
    d.N = H.shape[0]
    d.H = _ptr(H)
    d.n_lead_sites[0], d.n_lead_sites[1] = len(l0), len(l1)
    d.lead_sites[0], d.lead_sites[1] = _ptr(l0), _ptr(l1)
    out = P()
    _check(load().knit_graph_create(ctypes.byref(d), ctypes.byref(out)))
    return out.value


def _multi_desc(H, leads):
    H = np.ascontiguousarray(H, dtype=np.complex128)
    ls = [np.ascontiguousarray(l, dtype=np.int32) for l in leads]
    n = np.array([len(l) for l in ls], np.int32)
    ptrs = (P * len(ls))(*[l.ctypes.data for l in ls])
    d = knit_graph_multi_desc()
    d.N = H.shape[0]
    d.H = _ptr(H)
    d.n_leads = len(ls)
    d.n_lead_sites = _ptr(n)
    d.lead_sites = ctypes.cast(ptrs, P)
    return d, (H, ls, n, ptrs)   # keep the arrays alive with the descriptor


def knit_graph_plan(H, leads):
    """(nslices, slice_of) of the slicing, computed on the host."""
    d, keep = _multi_desc(H, leads)
    k = ctypes.c_int32(0)
    so = np.empty(d.N, np.int32)
    _check(load().knit_graph_plan(ctypes.byref(d), ctypes.byref(k), _ptr(so)))
    return int(k.value), so


def knit_debug_fail_alloc_after(n):
    """Make the n-th device allocation from now on fail (n < 0: off)."""
    _check(load().knit_debug_fail_alloc_after(int(n)))


def knit_graph_create_multi(H, leads):
    """Handle of an arbitrary geometry with several leads (site lists)."""
    d, keep = _multi_desc(H, leads)
    out = P()
    _check(load().knit_graph_create_multi(ctypes.byref(d), ctypes.byref(out)))
    return out.value


def knit_graph_conductance(handle, E, sigmas, Tmat, status=None, nE=None, stream=None):
    """sigmas: one (nE, w_p, w_p) complex128 array (or device tensor) per lead."""
    nE = len(E) if nE is None else nE
    ptrs = (P * len(sigmas))(*[_ptr(s) for s in sigmas])
    _check(load().knit_graph_conductance(P(handle), _ptr(E), int(nE), ctypes.cast(ptrs, P),
                                         _ptr(Tmat), _ptr(status), _stream(stream)))


def knit_graph_destroy(handle):
    _check(load().knit_graph_destroy(P(handle)))


def knit_graph_slices(handle, N):
    """(widths, slice_of) of the slicing."""
    k = ctypes.c_int32(0)
    _check(load().knit_graph_slices(P(handle), ctypes.byref(k), None, None))
    w = np.empty(k.value, np.int32)
    so = np.empty(N, np.int32)
    _check(load().knit_graph_slices(P(handle), ctypes.byref(k), _ptr(w), _ptr(so)))
    return w, so


def knit_graph_transmission(handle, E, sigma0, sigma1, T, status=None, nE=None, stream=None):
    nE = len(E) if nE is None else nE
    _check(load().knit_graph_transmission(P(handle), _ptr(E), int(nE), _ptr(sigma0), _ptr(sigma1),
                                          _ptr(T), _ptr(status), _stream(stream)))


class Graph:
    """Owns one knit_graph: Graph(H, lead0, lead1) or Graph(H, leads=[...])."""

    def __init__(self, H, lead0=None, lead1=None, leads=None):
        self.N = np.asarray(H).shape[0]
        if leads is None:
            self.handle = knit_graph_create(H, lead0, lead1)
            self.P = 2
        else:
            self.handle = knit_graph_create_multi(H, leads)
            self.P = len(leads)

    def close(self):
        if self.handle:
            knit_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def slices(self):
        return knit_graph_slices(self.handle, self.N)

    def transmission(self, E, sigma0, sigma1):
        E = np.ascontiguousarray(E, dtype=np.float64)
        T = np.empty(len(E))
        st = np.empty(len(E), np.int32)
        knit_graph_transmission(self.handle, E, _c128(sigma0), _c128(sigma1), T, st)
        return T, st

    def conductance(self, E, sigmas):
        """(Tmat (nE, P, P), status): T_kl between every pair of leads."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        Tm = np.empty((len(E), self.P, self.P))
        st = np.empty(len(E), np.int32)
        sig = [_c128(s) for s in sigmas]
        knit_graph_conductance(self.handle, E, sig, Tm, st)
        return Tm, st


def knit_system_info(handle, precision):
    """(sweep kernel KNIT_SWEEP_*, [lead blocks left, right]) of a system."""
    sw = ctypes.c_int32()
    lb = (ctypes.c_int32 * 2)()
    _check(load().knit_system_info(P(handle), int(precision), ctypes.byref(sw), lb))
    return sw.value, [lb[0], lb[1]]


def knit_system_num_edges(handle) -> int:
    c = ctypes.c_int32(0)
    _check(load().knit_system_num_edges(P(handle), ctypes.byref(c)))
    return int(c.value)


def knit_ldos(handle, E, seeds, W, saving_level, ldos, T=None, status=None, opts=None, nE=None,
              nS=None, stream=None, precision=KNIT_FP64):
    nE = len(E) if nE is None else nE
    nS = (1 if seeds is None else len(seeds)) if nS is None else nS
    _check(load().knit_ldos(P(handle), _ptr(E), int(nE), _ptr(seeds), int(nS), float(W),
                            int(precision), int(saving_level),
                            None if opts is None else ctypes.byref(opts),
                            _ptr(ldos), _ptr(T), _ptr(status), _stream(stream)))


def knit_lead_decimation_noalloc(H0, V, M, lead, E, sigma, eta=0.0, tol=0.0, maxit=0, iters=None,
                                 status=None, nE=None, stream=None):
    """Decimation into caller-provided device arrays; the library allocates
    nothing (fixed internal scratch, M <= 64)."""
    nE = len(E) if nE is None else nE
    _check(load().knit_lead_decimation_noalloc(_ptr(H0), _ptr(V), int(M), int(lead), _ptr(E),
                                               int(nE), float(eta), float(tol), int(maxit),
                                               _ptr(sigma), _ptr(iters), _ptr(status),
                                               _stream(stream)))


def knit_peak_probe(kind, iters, nsm, stream=None, check=False):
    """Launch one peak-rate loop (KNIT_PEAK_*) on nsm SMs; returns its flop
    count (the caller times the launch).  With check=True the call waits and
    raises KnitError(KNIT_ERR_TIMEOUT) if a tensor-core wait ran out."""
    flop = ctypes.c_double(0.0)
    flag = ctypes.c_int32(0)
    _check(load().knit_peak_probe(int(kind), int(iters), int(nsm), ctypes.byref(flop),
                                  ctypes.byref(flag) if check else None, _stream(stream)))
    if check and flag.value:
        raise KnitError(KNIT_ERR_TIMEOUT, "peak probe: a tensor-core wait ran out")
    return flop.value


def knit_debug_wait_probe(polls):
    """Run the bounded tensor-core wait on a barrier nothing completes;
    returns (wait status, cleanup completed)."""
    ws, cd = ctypes.c_int32(-1), ctypes.c_int32(-1)
    _check(load().knit_debug_wait_probe(int(polls), ctypes.byref(ws), ctypes.byref(cd)))
    return ws.value, cd.value


def knit_batch_create(handles, sys_index, precision):
    """Plan a heterogeneous batch over system handles; returns the plan handle."""
    arr = (P * len(handles))(*[P(h) for h in handles])
    idx = np.ascontiguousarray(sys_index, dtype=np.int32)
    out = P()
    _check(load().knit_batch_create(arr, len(handles), _ptr(idx), len(idx), int(precision),
                                    ctypes.byref(out)))
    return out.value


def knit_batch_destroy(plan):
    _check(load().knit_batch_destroy(P(plan)))


def knit_batch_transmission(plan, E, seeds, W, T, status=None, opts=None, stream=None):
    _check(load().knit_batch_transmission(P(plan), _ptr(E), _ptr(seeds), _ptr(W),
                                          None if opts is None else ctypes.byref(opts), _ptr(T),
                                          _ptr(status), _stream(stream)))


def knit_batch_buckets(plan):
    """[(kind, Mmax, count, max_ctas)] per kernel variant, in launch order."""
    nb = ctypes.c_int32()
    _check(load().knit_batch_buckets(P(plan), ctypes.byref(nb), None, None, None, None))
    a = [np.zeros(nb.value, np.int32) for _ in range(4)]
    _check(load().knit_batch_buckets(P(plan), ctypes.byref(nb), *[_ptr(x) for x in a]))
    return [tuple(int(x[q]) for x in a) for q in range(nb.value)]


def knit_batch_configure(plan, config):
    c = np.ascontiguousarray(config, dtype=np.int32)
    _check(load().knit_batch_configure(P(plan), _ptr(c)))


def knit_batch_autotune(plan, E, seeds, W, opts=None):
    """(CTAs per SM, ms) chosen per kernel variant."""
    nb = len(knit_batch_buckets(plan))
    cfg = np.zeros(nb, np.int32)
    ms = np.zeros(nb, np.float32)
    _check(load().knit_batch_autotune(P(plan), _ptr(E), _ptr(seeds), _ptr(W),
                                      None if opts is None else ctypes.byref(opts), _ptr(cfg),
                                      _ptr(ms)))
    return cfg, ms


class LeadModel:
    """A learned warm start for one lead of a System (see include/knit.h)."""

    def __init__(self, system, lead, E_train, epochs=200, batch=256, lr=1e-3, seed=0, eta=0.0):
        self.system = system
        self.lead = lead
        E = np.ascontiguousarray(E_train, dtype=np.float64)
        self.loss = np.zeros(epochs, np.float32)
        out = P()
        o = _opts(KNIT_LEAD_DECIMATION, eta)
        _check(load().knit_lead_model_train(P(system.handle), int(lead), _ptr(E), len(E),
                                            int(epochs), int(batch), ctypes.c_float(lr),
                                            ctypes.c_uint64(seed), ctypes.byref(o),
                                            _ptr(self.loss), ctypes.byref(out), None))
        self.handle = out.value

    def close(self):
        if self.handle:
            _check(load().knit_lead_model_destroy(P(self.handle)))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(load().knit_lead_model_num_params(P(self.handle)))

    def get_params(self):
        out = np.empty(self.num_params, np.float32)
        _check(load().knit_lead_model_get_params(P(self.handle), _ptr(out)))
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().knit_lead_model_set_params(P(self.handle), _ptr(p)))

    @property
    def num_outputs(self):
        return int(load().knit_lead_model_num_outputs(P(self.handle)))

    def forward(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        out = np.empty((len(E), self.num_outputs), np.float32)
        _check(load().knit_lead_model_forward(P(self.handle), _ptr(E), len(E), _ptr(out), None))
        return out

    def gradient(self, E, target):
        E = np.ascontiguousarray(E, dtype=np.float64)
        t = np.ascontiguousarray(target, dtype=np.float32)
        grad = np.empty(self.num_params, np.float32)
        loss = np.zeros(1, np.float32)
        _check(load().knit_lead_model_gradient(P(self.handle), _ptr(E), _ptr(t), len(E),
                                               _ptr(grad), _ptr(loss), None))
        return grad, float(loss[0])


class Batch:
    """A heterogeneous batch plan over ``System`` objects (kept alive here)."""

    def __init__(self, systems, sys_index, precision=KNIT_MIXED):
        self.systems = list(systems)
        self.n = len(sys_index)
        self.handle = knit_batch_create([s.handle for s in self.systems], sys_index, precision)

    def buckets(self):
        return knit_batch_buckets(self.handle)

    def autotune(self, E, seeds=None, W=None, cache=None):
        """Tune CTAs per SM per kernel variant (knit_batch_autotune), or take
        them from the JSON file `cache`, whose entries are keyed by the
        variants' (kind, Mmax, count, max_ctas) and the instance count;
        returns the configuration."""
        import json
        key = repr((self.n, self.buckets()))
        table = {}
        if cache is not None and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                cfg = table[key]["ctas_per_sm"]
                knit_batch_configure(self.handle, cfg)
                return cfg
        E = np.ascontiguousarray(E, dtype=np.float64)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        Wv = None if W is None else np.ascontiguousarray(np.broadcast_to(W, (self.n,)),
                                                          dtype=np.float64)
        cfg, ms = knit_batch_autotune(self.handle, E, sd, Wv)
        if cache is not None:
            table[key] = {"ctas_per_sm": [int(c) for c in cfg], "ms": [float(m) for m in ms]}
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        return [int(c) for c in cfg]

    def close(self):
        if self.handle:
            knit_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def transmission(self, E, seeds=None, W=None, method=KNIT_LEAD_AUTO):
        E = np.ascontiguousarray(E, dtype=np.float64)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        Wv = None if W is None else np.ascontiguousarray(np.broadcast_to(W, (self.n,)),
                                                          dtype=np.float64)
        T = np.empty(self.n)
        st = np.empty(self.n, np.int32)
        knit_batch_transmission(self.handle, E, sd, Wv, T, st, _opts(method))
        return T, st


# ---------------------------------------------------------------------------
# Convenience wrapper over a SliceSystem (paper_1010_2627_gb300.inputs)

class System:
    """Owns one knit_system built from an ``inputs.SliceSystem``."""

    def __init__(self, ss, onsite=None):
        self.M, self.L = ss.M, ss.L
        self.handle = knit_system_create(ss.M, ss.L, ss.H0, ss.V, block=ss.block,
                                         onsite_sign=ss.sign, onsite=onsite,
                                         lead_H0=ss.lead_H0, lead_V=ss.lead_V)

    def info(self, precision=KNIT_MIXED):
        """(sweep kernel KNIT_SWEEP_*, [lead blocks left, right])"""
        return knit_system_info(self.handle, precision)

    def close(self):
        if self.handle:
            knit_system_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lead_selfenergy(self, lead, E, method=KNIT_LEAD_AUTO, eta=0.0, want_residual=False,
                        models=(None, None)):
        """(Sigma (nE, M, M), iterations (nE,), residual (nE,) or None) of lead
        0 (left) or 1 (right) at the energies E."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        S = np.empty((len(E), self.M, self.M), np.complex128)
        it = np.zeros(len(E), np.int32)
        res = np.zeros(len(E)) if want_residual else None
        mods = tuple(None if m is None else m.handle for m in models)
        knit_lead_selfenergy(self.handle, lead, E, S, _opts(method, eta, models=mods), it, res)
        return S, it, res

    def transmission(self, E, seeds=None, W=0.0, precision=KNIT_FP64, method=KNIT_LEAD_AUTO):
        """(T (nE, nS), status (nE, nS)) for every energy x disorder seed;
        W is the disorder strength, precision KNIT_FP64 or KNIT_MIXED."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        nS = 1 if sd is None else len(sd)
        T = np.empty(len(E) * nS)
        st = np.empty(len(E) * nS, np.int32)
        knit_transmission(self.handle, E, sd, W, precision, T, st, _opts(method))
        return T.reshape(len(E), nS), st.reshape(len(E), nS)

    def transmission_sigma(self, E, SL, SR, seeds=None, W=0.0, precision=KNIT_FP64):
        """As transmission, with the lead self-energies SL, SR (nE, M, M) given."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        nS = 1 if sd is None else len(sd)
        T = np.empty(len(E) * nS)
        st = np.empty(len(E) * nS, np.int32)
        knit_transmission_sigma(self.handle, E, sd, W, _c128(SL), _c128(SR), precision, T, st)
        return T.reshape(len(E), nS), st.reshape(len(E), nS)

    def transmission_eigenvalues(self, E, seeds=None, W=0.0, precision=KNIT_FP64,
                                 method=KNIT_LEAD_AUTO):
        """(tau, noise, T, status): tau (nE, nS, M) in decreasing order,
        noise = sum tau (1 - tau), T and status as for transmission."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        nS = 1 if sd is None else len(sd)
        n = len(E) * nS
        tau = np.empty((n, self.M))
        noise = np.empty(n)
        T = np.empty(n)
        st = np.empty(n, np.int32)
        knit_transmission_eigenvalues(self.handle, E, sd, W, precision, tau, noise, T, st,
                                      _opts(method))
        return (tau.reshape(len(E), nS, self.M), noise.reshape(len(E), nS),
                T.reshape(len(E), nS), st.reshape(len(E), nS))

    def lesser(self, E, seeds=None, W=0.0, saving_level=-1, method=KNIT_LEAD_AUTO):
        """dict(rhoL, rhoR (nE, nS, L, M), jx (nE, nS, L-1, M), jt (nE, nS, L, nedge),
        T, status): lead-resolved densities and left-injected bond currents."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        nS = 1 if sd is None else len(sd)
        n = len(E) * nS
        ne = knit_system_num_edges(self.handle)
        rl = np.empty((n, self.L, self.M))
        rr = np.empty((n, self.L, self.M))
        jx = np.empty((n, max(self.L - 1, 0), self.M))
        jt = np.empty((n, self.L, ne))
        T = np.empty(n)
        st = np.empty(n, np.int32)
        knit_lesser(self.handle, E, sd, W, saving_level, rl, rr, jx if jx.size else None,
                    jt if jt.size else None, T, st, _opts(method))
        sh = (len(E), nS)
        return dict(rhoL=rl.reshape(sh + rl.shape[1:]), rhoR=rr.reshape(sh + rr.shape[1:]),
                    jx=jx.reshape(sh + jx.shape[1:]), jt=jt.reshape(sh + jt.shape[1:]),
                    T=T.reshape(sh), status=st.reshape(sh))

    def ldos(self, E, seeds=None, W=0.0, saving_level=-1, method=KNIT_LEAD_AUTO,
             precision=KNIT_FP64):
        """(LDOS (nE, nS, L, M), T (nE, nS), status (nE, nS)); saving_level k
        keeps every k-th slice's g and recomputes the rest (-1: keep all)."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        nS = 1 if sd is None else len(sd)
        out = np.empty((len(E) * nS, self.L, self.M))
        T = np.empty(len(E) * nS)
        st = np.empty(len(E) * nS, np.int32)
        knit_ldos(self.handle, E, sd, W, saving_level, out, T, st, _opts(method),
                  precision=precision)
        return (out.reshape(len(E), nS, self.L, self.M), T.reshape(len(E), nS),
                st.reshape(len(E), nS))
