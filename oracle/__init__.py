"""Plain FP64 CPU oracle for the two-terminal KNIT problem -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_1010_2627_gb300`` and imports nothing
from it; both sides only read inputs produced by
``paper_1010_2627_gb300.inputs``, which holds no arithmetic of the method.

The arithmetic lives in ``knit_oracle.c`` (plain C, FP64, own complex LU, no
BLAS).  This module compiles it with gcc on first use and calls it through
ctypes:

* ``sigma_square``   closed-form lead self-energy of a clean square lead
                     (KNIT user guide Sec. 5.3 B lead construction; textbook
                     transverse modes)
* ``decimation``     Sancho-Rubio surface Green function and self-energy of
                     a general lead (Sec. 5.3 B)
* ``dense``          the plain definition, Eq. (2) and the Sec. 2.3
                     transmission formula, by dense LU of the whole system
* ``dense_general``  the same for an arbitrary site graph with two leads
                     (the Sec. 2.2 worked example)
* ``rgf``            the slice form of the method (Sec. 5.3 D knitting and
                     sewing), plain loops
* ``rgf_batch``      ``rgf`` over many instances on all host cores (the CPU
                     baseline)
* ``transmission_matrix``
                     T_kl between every pair of several leads of a site
                     graph (Sec. 2.3), dense numpy inverse
* ``lesser_parts``   lead-resolved densities and bond currents from
                     G^<_l = i G Gamma_l G^+ (Sec. 2.3), dense numpy inverse
* ``graph_lesser``   the same lead-resolved densities, LDOS and bond currents
                     for an arbitrary site graph with several leads
* ``transmission_eigenvalues``, ``shot_noise``
                     the eigenvalues of the matrix inside Sec. 2.3's
                     transmission trace, and sum tau (1 - tau)
* ``onsite``         counter-based Anderson disorder (Sec. 6.1)

Parity status: every function here is pinned by ``tests/test_oracle.py`` and
``tests/test_oracle_scattering.py`` (closed forms, the paper's printed Fig. 3
values, brute force, identities, scattering states by mode matching).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knit_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_OOM, ERR_SINGULAR, ERR_NOCONVERGE = 0, 1, 2, 4, 5


def build(force: bool = False) -> str:
    """Compile knit_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, f64, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_uint64
            lib.orc_splitmix64.restype = u64
            lib.orc_splitmix64.argtypes = [u64]
            lib.orc_onsite.restype = f64
            lib.orc_onsite.argtypes = [u64, i32, i32, f64]
            lib.orc_onsite_fill.argtypes = [u64, i32, i32, i32, P, f64, P]
            lib.orc_sigma_square.argtypes = [i32, f64, f64, P]
            lib.orc_lead_decimation.restype = i32
            lib.orc_lead_decimation.argtypes = [i32, P, P, f64, f64, i32, f64, i32, P, P, P]
            lib.orc_dense_flat.restype = i32
            lib.orc_dense_flat.argtypes = [i32, i32, P, P, P, i32, f64, P, P, P, P, P, P, P]
            lib.orc_rgf_flat.restype = i32
            lib.orc_rgf_flat.argtypes = [i32, i32, P, P, P, i32, f64, P, P, P, P, P, P]
            lib.orc_dense_general.restype = i32
            lib.orc_dense_general.argtypes = [i32, P, f64, i32, P, P, i32, P, P, P]
            lib.orc_rgf_batch.restype = i32
            lib.orc_rgf_batch.argtypes = [i32, i32, P, P, i32, i32, P, i32, P, P, P, P, P, P,
                                          i32, P, P]
            lib.orc_max_threads.restype = i32
            lib.orc_lu_factor.restype = i32
            lib.orc_lu_factor.argtypes = [i32, P, P]
            lib.orc_lu_solve.argtypes = [i32, P, P, P, i32]
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def splitmix64(z: int) -> int:
    return int(_load().orc_splitmix64(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def onsite(seed: int, L: int, M: int, W: float, block: int = 1, sign=None) -> np.ndarray:
    """(L, M) on-site energies W (r - 1/2), r from the (seed, n, site) counter."""
    sign = _c([1.0] * block if sign is None else sign, np.float64)
    out = np.empty((L, M), dtype=np.float64)
    _load().orc_onsite_fill(ctypes.c_uint64(seed), L, M, block, _p(sign), W, _p(out))
    return out


def sigma_square(M: int, t: float, E: float) -> np.ndarray:
    """Closed-form self-energy (M x M) of a clean square lead of width M, hopping t."""
    out = np.empty((M, M), dtype=np.complex128)
    _load().orc_sigma_square(M, t, E, _p(out))
    return out


def _retarded_fixed_point(H0, V, g, z, side):
    """Is g the retarded solution of its lead's fixed point at the complex
    energy z: g = (z - H0 - V g V^dagger)^{-1} (left; right with V^dagger,
    V) to 1e-5 relative max-norm, and i(g - g^dagger) positive semidefinite?"""
    if not np.isfinite(g).all():
        return False
    M = H0.shape[0]
    W = V @ g @ V.conj().T if side == 0 else V.conj().T @ g @ V
    A = np.linalg.inv(z * np.eye(M) - H0 - W)
    if not np.abs(A - g).max() <= 1e-5 * np.abs(g).max():
        return False
    G = 1j * (g - g.conj().T)
    ev = np.linalg.eigvalsh((G + G.conj().T) / 2)
    return ev.min() >= -1e-9 * max(ev.max(), 0.0)


def decimation(H0, V, E: float, side: int, eta: float = 1e-12, tol: float = 1e-15,
               maxit: int = 200):
    """Sancho-Rubio surface g and self-energy of a lead (side 0 left, 1 right)
    at E + i eta.  The retarded solution of the fixed point is wanted (a
    reading of Sec. 5.3 B): when the doubling loses enough precision to end on
    anything else (non-finite, not a fixed point at its own eta to 1e-5, or
    i(g - g^dagger) not positive semidefinite), it is run again at 100x eta,
    up to eta * 1e6.

    Returns (g, Sigma, iterations)."""
    H0 = _c(H0, np.complex128)
    V = _c(V, np.complex128)
    M = H0.shape[0]
    for k in range(4):
        eta_k = eta * 100.0 ** k
        g = np.empty((M, M), dtype=np.complex128)
        S = np.empty((M, M), dtype=np.complex128)
        it = ctypes.c_int(0)
        rc = _load().orc_lead_decimation(M, _p(H0), _p(V), E, eta_k, side, tol, maxit, _p(g),
                                         _p(S), ctypes.byref(it))
        if rc == OK and _retarded_fixed_point(H0, V, g, E + 1j * eta_k, side):
            return g, S, it.value
    raise OracleError(rc if rc != OK else ERR_NOCONVERGE, "decimation")


def decimation_period2(H0, V_first, V_second, E: float, side: int, eta: float = 1e-12,
                       tol: float = 1e-15, maxit: int = 200):
    """Self-energy on the system's end slice of a lead whose inter-slice
    couplings alternate V_first, V_second going outward (V_first couples the
    end slice to the lead's surface slice; slice-forward orientation
    H_{n,n-1}), from the surface function of the lead's two-slice cell
    (Sec. 5.3 B with a cell of two slices).  Returns Sigma (M x M)."""
    H0 = np.asarray(H0, np.complex128)
    Vf = np.asarray(V_first, np.complex128)
    Vs = np.asarray(V_second, np.complex128)
    M = H0.shape[0]
    Hc = np.zeros((2 * M, 2 * M), np.complex128)
    Vc = np.zeros_like(Hc)
    Hc[:M, :M] = H0
    Hc[M:, M:] = H0
    if side == 0:
        # cell (s_-1, s_-2): H_{s-1,s-2} = V_second; next cell couples via H_{s-2,s-3} = V_first
        Hc[:M, M:] = Vs
        Hc[M:, :M] = Vs.conj().T
        Vc[M:, :M] = Vf
    else:
        # cell (s_L, s_L+1): H_{s_L+1,s_L} = V_second; next cell via H_{s_L+2,s_L+1} = V_first
        Hc[M:, :M] = Vs
        Hc[:M, M:] = Vs.conj().T
        Vc[:M, M:] = Vf
    g, _, _ = decimation(Hc, Vc, E, side, eta=eta, tol=tol, maxit=maxit)
    g11 = g[:M, :M]
    return Vf @ g11 @ Vf.conj().T if side == 0 else Vf.conj().T @ g11 @ Vf


def _sys_arrays(H0, V, eps, L):
    H0 = _c(H0, np.complex128)
    M = H0.shape[0]
    V = _c(V, np.complex128)
    if V.ndim == 2:
        V = V[None]
    eps = None if eps is None else _c(eps, np.float64).reshape(L, M)
    return H0, V, eps, M


def dense(H0, V, eps, L: int, E: float, SigL, SigR, want_ldos: bool = False):
    """Dense-LU solution of Eq. (2) for a slice system.

    V is (M, M) or (P, M, M) with H_{n,n-1} = V[n % P]; eps is (L, M) or None.
    Returns dict(T_LR, T_RL, G11, G1L, GL1, ldos)."""
    H0, V, eps, M = _sys_arrays(H0, V, eps, L)
    SigL = _c(SigL, np.complex128)
    SigR = _c(SigR, np.complex128)
    T = np.empty(2)
    G11 = np.empty((M, M), np.complex128)
    G1L = np.empty((M, M), np.complex128)
    GL1 = np.empty((M, M), np.complex128)
    ldos = np.empty((L, M)) if want_ldos else None
    rc = _load().orc_dense_flat(M, L, _p(H0), _p(eps), _p(V), V.shape[0], E, _p(SigL), _p(SigR),
                                _p(T), _p(G11), _p(G1L), _p(GL1), _p(ldos))
    if rc != OK:
        raise OracleError(rc, "dense")
    return dict(T_LR=float(T[0]), T_RL=float(T[1]), G11=G11, G1L=G1L, GL1=GL1, ldos=ldos)


def dense_general(H, E: float, idx0, Sig0, idx1, Sig1):
    """Two-lead transmission of an arbitrary site graph: (T_{1<-0}, T_{0<-1})."""
    H = _c(H, np.complex128)
    idx0 = _c(idx0, np.int32)
    idx1 = _c(idx1, np.int32)
    Sig0 = _c(Sig0, np.complex128)
    Sig1 = _c(Sig1, np.complex128)
    T = np.empty(2)
    rc = _load().orc_dense_general(H.shape[0], _p(H), E, len(idx0), _p(idx0), _p(Sig0),
                                   len(idx1), _p(idx1), _p(Sig1), _p(T))
    if rc != OK:
        raise OracleError(rc, "dense_general")
    return float(T[0]), float(T[1])


def rgf(H0, V, eps, L: int, E: float, SigL, SigR, want_ldos: bool = False):
    """The slice-by-slice method: returns dict(T, ldos, G11, G1L)."""
    H0, V, eps, M = _sys_arrays(H0, V, eps, L)
    SigL = _c(SigL, np.complex128)
    SigR = _c(SigR, np.complex128)
    T = np.empty(1)
    ldos = np.empty((L, M)) if want_ldos else None
    G11 = np.empty((M, M), np.complex128) if want_ldos else None
    G1L = np.empty((M, M), np.complex128)
    rc = _load().orc_rgf_flat(M, L, _p(H0), _p(eps), _p(V), V.shape[0], E, _p(SigL), _p(SigR),
                              _p(T), _p(ldos), _p(G11), _p(G1L))
    if rc != OK:
        raise OracleError(rc, "rgf")
    return dict(T=float(T[0]), ldos=ldos, G11=G11, G1L=G1L)


def _gamma(Sig):
    Sig = np.asarray(Sig, dtype=np.complex128)
    return 1j * (Sig - Sig.conj().T)


def _psd_sqrt(G):
    w, U = np.linalg.eigh((G + G.conj().T) / 2)
    return (U * np.sqrt(np.clip(w, 0.0, None))) @ U.conj().T


def transmission_eigenvalues(G1L, SigL, SigR):
    """Transmission eigenvalues tau_n, decreasing (M values).

    Sec. 2.3 writes T_kl as the trace of G_kl Gamma_l G_kl^+ Gamma_k; with
    k = L (slice 1), l = R (slice L) its eigenvalues are the tau_n, taken here
    in the Hermitian form Gamma_L^{1/2} G_1L Gamma_R G_1L^+ Gamma_L^{1/2}
    (same spectrum; Gamma^{1/2} and the eigenvalues by numpy's Hermitian
    eigensolver).  Gamma = i (Sigma - Sigma^+)."""
    S = _psd_sqrt(_gamma(SigL))
    G1L = np.asarray(G1L, dtype=np.complex128)
    H = S @ G1L @ _gamma(SigR) @ G1L.conj().T @ S
    return np.linalg.eigvalsh((H + H.conj().T) / 2)[::-1].copy()


def transmission_matrix(H, E: float, lead_sites, sigmas):
    """Multi-terminal transmissions T_kl = Re Tr[Gamma_k G_kl Gamma_l G_kl^+]
    (Sec. 2.3, G^+_lk = (G_kl)^dagger for the retarded G) of an arbitrary
    site graph with leads k attached to the sites lead_sites[k] through
    self-energies sigmas[k], by the plain dense inverse of E - H - sum Sigma
    (numpy).  Returns a (P, P) array with a zero diagonal."""
    H = np.asarray(H, dtype=np.complex128)
    N = H.shape[0]
    A = E * np.eye(N) - H
    idx = [np.asarray(s, dtype=int) for s in lead_sites]
    for s, S in zip(idx, sigmas):
        A[np.ix_(s, s)] -= np.asarray(S, dtype=np.complex128)
    G = np.linalg.inv(A)
    P = len(idx)
    T = np.zeros((P, P))
    for k in range(P):
        for l in range(P):
            if k != l:
                B = G[np.ix_(idx[k], idx[l])]
                T[k, l] = np.real(np.trace(_gamma(sigmas[k]) @ B @ _gamma(sigmas[l]) @ B.conj().T))
    return T


def lesser_parts(H0, V, eps, L: int, E: float, SigL, SigR):
    """Lead-resolved parts of the lesser function, G^<_l = i G Gamma_l G^+
    (Sec. 2.3, with Gamma_l = i (Sigma_l - Sigma_l^+)), from the plain dense
    inverse of E - H - Sigma_L - Sigma_R (numpy).  Returns a dict of

    rhoL, rhoR (L, M): A^l_xx / (2 pi) with A^l = G Gamma_l G^+ -- the density
        of states injected by lead l (the non-equilibrium density is
        f_L rhoL + f_R rhoR);
    jx (L - 1, M): current carried by left-injected states from orbital x of
        slice n into slice n + 1, sum_y -2 Im[H_{(n,x),(n+1,y)} A^L_{(n+1,y),(n,x)}];
    jt (L, E_up): the same along the edges x < y of H0 inside each slice, in
        row-major order of H0's nonzero entries above the diagonal;
    ldos (L, M): -Im G_xx / pi, and T (Sec. 2.3 trace)."""
    H0, V, eps, M = _sys_arrays(H0, V, eps, L)
    N = M * L
    H = np.zeros((N, N), np.complex128)
    for n in range(L):
        H[n * M:(n + 1) * M, n * M:(n + 1) * M] = H0 + (np.diag(eps[n]) if eps is not None else 0)
        if n + 1 < L:
            Vn = V[(n + 1) % V.shape[0]]
            H[(n + 1) * M:(n + 2) * M, n * M:(n + 1) * M] = Vn
            H[n * M:(n + 1) * M, (n + 1) * M:(n + 2) * M] = Vn.conj().T
    A = E * np.eye(N) - H
    A[:M, :M] -= _c(SigL, np.complex128)
    A[N - M:, N - M:] -= _c(SigR, np.complex128)
    G = np.linalg.inv(A)
    GL, GR = _gamma(SigL), _gamma(SigR)
    AL = G[:, :M] @ GL @ G[:, :M].conj().T
    AR = G[:, N - M:] @ GR @ G[:, N - M:].conj().T
    rhoL = (np.real(np.diag(AL)) / (2 * np.pi)).reshape(L, M)
    rhoR = (np.real(np.diag(AR)) / (2 * np.pi)).reshape(L, M)
    jx = np.zeros((max(L - 1, 0), M))
    for n in range(L - 1):
        for x in range(M):
            a = n * M + x
            jx[n, x] = sum(-2 * np.imag(H[a, (n + 1) * M + y] * AL[(n + 1) * M + y, a])
                           for y in range(M))
    edges = [(x, y) for x in range(M) for y in range(x + 1, M) if H0[x, y] != 0]
    jt = np.zeros((L, len(edges)))
    for n in range(L):
        for e, (x, y) in enumerate(edges):
            a, b = n * M + x, n * M + y
            jt[n, e] = -2 * np.imag(H[a, b] * AL[b, a])
    ldos = (-np.imag(np.diag(G)) / np.pi).reshape(L, M)
    T = float(np.real(np.trace(GL @ G[:M, N - M:] @ GR @ G[:M, N - M:].conj().T)))
    return dict(rhoL=rhoL, rhoR=rhoR, jx=jx, jt=jt, edges=edges, ldos=ldos, T=T)


def graph_lesser(H, E: float, lead_sites, sigmas):
    """Lead-resolved local quantities of an arbitrary site graph with P leads
    (Sec. 2.3: G^<_l = i G Gamma_l G^+ is the part of the lesser function fed
    by lead l, Gamma_l = i (Sigma_l - Sigma_l^+); local currents between
    neighbouring sites), from the plain dense inverse of E - H - sum Sigma
    (numpy).  Returns a dict of

    rho (P, N): A^l_ii / (2 pi) with A^l = G Gamma_l G^+, the density of
        states injected by lead l;
    ldos (N): -Im G_ii / pi;
    edges (n_edge, 2): the pairs i < j with H_ij != 0, row-major;
    J (P, n_edge): current carried by lead-l-injected states from i to j
        along each edge, -2 Im[H_ij A^l_ji];
    T (P, P): T_kl = Re Tr[Gamma_k G_kl Gamma_l G_kl^+] (zero diagonal)."""
    H = np.asarray(H, dtype=np.complex128)
    N = H.shape[0]
    A = E * np.eye(N) - H
    idx = [np.asarray(s, dtype=int) for s in lead_sites]
    for s, S in zip(idx, sigmas):
        A[np.ix_(s, s)] -= np.asarray(S, dtype=np.complex128)
    G = np.linalg.inv(A)
    P = len(idx)
    edges = np.array([(i, j) for i in range(N) for j in range(i + 1, N) if H[i, j] != 0],
                     dtype=int).reshape(-1, 2)
    rho = np.zeros((P, N))
    J = np.zeros((P, len(edges)))
    T = np.zeros((P, P))
    for l in range(P):
        Gl = G[:, idx[l]]
        Al = Gl @ _gamma(sigmas[l]) @ Gl.conj().T
        rho[l] = np.real(np.diag(Al)) / (2 * np.pi)
        for e, (i, j) in enumerate(edges):
            J[l, e] = -2 * np.imag(H[i, j] * Al[j, i])
        for k in range(P):
            if k != l:
                B = G[np.ix_(idx[k], idx[l])]
                T[k, l] = np.real(np.trace(_gamma(sigmas[k]) @ B @ _gamma(sigmas[l]) @ B.conj().T))
    ldos = -np.imag(np.diag(G)) / np.pi
    return dict(rho=rho, ldos=ldos, edges=edges, J=J, T=T)


def shot_noise(tau):
    """sum_n tau_n (1 - tau_n): zero-temperature shot noise in units of 2 e^3 |V| / h."""
    tau = np.asarray(tau, dtype=np.float64)
    return float(np.sum(tau * (1.0 - tau)))


def rgf_batch(H0, V, L: int, E, seeds, W, SigL, SigR, sig_index, block: int = 1, sign=None,
              nthreads: int = 0):
    """``rgf`` over instances i with energy E[i], disorder (seeds[i], W[i]) and
    self-energies SigL[sig_index[i]], SigR[sig_index[i]].  Returns (T, status)."""
    H0 = _c(H0, np.complex128)
    M = H0.shape[0]
    V = _c(V, np.complex128)
    if V.ndim == 2:
        V = V[None]
    E = _c(E, np.float64)
    n = E.shape[0]
    seeds = _c(seeds, np.uint64)
    W = _c(np.broadcast_to(W, (n,)), np.float64)
    SigL = _c(SigL, np.complex128)
    SigR = _c(SigR, np.complex128)
    sig_index = _c(sig_index, np.int32)
    sign = _c([1.0] * block if sign is None else sign, np.float64)
    T = np.empty(n)
    st = np.zeros(n, np.int32)
    _load().orc_rgf_batch(M, L, _p(H0), _p(V), V.shape[0], block, _p(sign), n, _p(E), _p(seeds),
                          _p(W), _p(SigL), _p(SigR), _p(sig_index), nthreads, _p(T), _p(st))
    return T, st


def max_threads() -> int:
    return int(_load().orc_max_threads())


def lu_solve(A, B):
    """Solve A X = B with the oracle's own pivoted LU (for tests of the LU)."""
    A = np.array(A, dtype=np.complex128, order="C")
    B = np.array(B, dtype=np.complex128, order="C")
    if B.ndim == 1:
        B = B[:, None]
    N = A.shape[0]
    perm = np.empty(N, np.int32)
    rc = _load().orc_lu_factor(N, _p(A), _p(perm))
    if rc != 0:
        raise OracleError(ERR_SINGULAR, "lu_factor")
    _load().orc_lu_solve(N, _p(A), _p(perm), _p(B), B.shape[1])
    return B, perm
