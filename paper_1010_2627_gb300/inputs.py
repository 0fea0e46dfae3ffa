"""Seeded synthetic inputs shaped like the KNIT user guide's workloads.

This module builds tight-binding slice blocks (Eq. 1 of the user guide grouped
by slices), energy grids and instance lists.  It holds none of the method's
arithmetic (no self-energy, no inversion, no transmission): both the CUDA
library and the CPU oracle read what it produces, and it imports neither.

Conventions shared by every consumer:

* a slice system has L slices of M orbitals, ``block`` orbitals per site;
* ``H0`` (M, M) is the clean slice Hamiltonian (on-site + intra-slice hopping);
* ``V`` (P, M, M) holds the inter-slice couplings, H_{n,n-1} = V[n % P] and
  H_{n-1,n} = V[n % P]^dagger;
* each lead p is the semi-infinite repetition of a cell (``lead_H0[p]``,
  ``lead_V[p]``) whose hopping to the system equals its own inter-cell hopping
  (Sec. 5.3 B of the user guide);
* disorder: orbital c of site s in slice n gets ``sign[c] * W * (r - 1/2)``
  with r drawn from the (seed, n, s) counter of the method's generator
  (Sec. 6.1 "Introducing disorder"); ``sign`` = +1 for electrons, -1 for the
  hole components of a Nambu block.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class SliceSystem:
    M: int
    L: int
    H0: np.ndarray                 # (M, M) complex128
    V: np.ndarray                  # (P, M, M) complex128
    block: int = 1
    sign: np.ndarray = field(default_factory=lambda: np.ones(1))
    lead_H0: tuple = ()            # (left, right) cells, (M, M) each
    lead_V: tuple = ()             # (left, right) inter-cell couplings, (M, M) each, or
                                   # (2, M, M) for a period-2 lead [V_first, V_second]
    name: str = ""

    def __post_init__(self):
        self.H0 = np.ascontiguousarray(self.H0, dtype=np.complex128)
        V = np.ascontiguousarray(self.V, dtype=np.complex128)
        self.V = V[None] if V.ndim == 2 else V
        self.sign = np.ascontiguousarray(self.sign, dtype=np.float64)
        if not self.lead_H0:
            self.lead_H0 = (self.H0, self.H0)
        if not self.lead_V:
            self.lead_V = (self.V[0], self.V[0])
        self.lead_H0 = tuple(np.ascontiguousarray(h, dtype=np.complex128) for h in self.lead_H0)
        self.lead_V = tuple(np.ascontiguousarray(v, dtype=np.complex128) for v in self.lead_V)


def energy_grid(a: float, b: float, n: int) -> np.ndarray:
    """n energies evenly spaced in the open interval (a, b): the midpoints
    a + (b - a)(j + 1/2)/n, symmetric about (a + b)/2."""
    j = np.arange(n, dtype=np.float64)
    return a + (b - a) * (j + 0.5) / n


def square(M: int, L: int, t: float = 1.0) -> SliceSystem:
    """Square lattice, nearest-neighbour hopping t, slices = columns of M sites
    (user guide Sec. 2.2 / Sec. 5.3 A rectangles); clean leads of width M."""
    H0 = np.zeros((M, M), np.complex128)
    i = np.arange(M - 1)
    H0[i, i + 1] = t
    H0[i + 1, i] = t
    V = t * np.eye(M, dtype=np.complex128)
    return SliceSystem(M, L, H0, V, name=f"square M={M} L={L} t={t}")


def chain(L: int, t: float = 1.0) -> SliceSystem:
    """1D chain: the M = 1 square lattice."""
    return square(1, L, t)


def armchair(M: int, L: int, t: float = 2.7) -> SliceSystem:
    """Honeycomb ribbon as a brick wall: slice n = a zigzag row of M sites with
    in-row hopping t; vertical bonds between rows n-1 and n at sites x with
    (x + n) even, so V alternates with period 2.  The ribbon edges (x = 0 and
    x = M - 1) run along the armchair direction.  The leads are the same clean
    ribbon continued: period-2 leads whose couplings go on alternating
    (left: H_{0,-1} = V_0, then V_1; right: H_{L,L-1} = V_{L mod 2}, then
    V_{(L+1) mod 2})."""
    H0 = np.zeros((M, M), np.complex128)
    i = np.arange(M - 1)
    H0[i, i + 1] = t
    H0[i + 1, i] = t
    x = np.arange(M)
    V = np.stack([np.diag(t * ((x + k) % 2 == 0).astype(np.float64)) for k in range(2)])
    V = V.astype(np.complex128)
    left = np.stack([V[0], V[1]])
    right = np.stack([V[L % 2], V[(L + 1) % 2]])
    return SliceSystem(M, L, H0, V, lead_V=(left, right), name=f"armchair M={M} L={L} t={t}")


def armchair_half_sites(M: int, n: int):
    """Sites x of brick-wall row n split as (a_n, b_n): a_n couples to row
    n - 1 ((x + n) even), b_n to row n + 1 (the others), each in increasing
    x (M even)."""
    x = np.arange(M)
    a = x[(x + n) % 2 == 0]
    b = x[(x + n) % 2 == 1]
    return a, b


def armchair_halfslices(M: int, L: int, t: float = 2.7) -> SliceSystem:
    """The armchair ribbon of ``armchair(M, L, t)`` sliced by half-rows: row n
    splits into a_n (the sites coupled to row n - 1) and b_n (the rest), and
    the chain a_0, b_0, a_1, b_1, ... is block tridiagonal with blocks of
    M / 2 orbitals and no hopping inside a block.  Couplings (H_{m, m-1} =
    V[m % 4]): t I between b_{n-1} and a_n (the same x), and the in-row chain
    bonds between a_n and b_n, bidiagonal with a shape set by the parity of
    n.  The same physical system, so the same transmission; disorder must be
    given per half-row (``armchair_halfslice_onsite``), and the lead
    self-energies are the row picture's restricted to a_0 (left) and
    b_{L-1} (right) (``armchair_halfslice_sigma``)."""
    assert M % 2 == 0
    h = M // 2
    V = np.zeros((4, h, h), np.complex128)
    V[0] = t * np.eye(h)
    V[2] = t * np.eye(h)
    for n, q in ((0, 1), (1, 3)):
        a, b = armchair_half_sites(M, n)
        for i, xa in enumerate(a):
            for j, xb in enumerate(b):
                if abs(int(xa) - int(xb)) == 1:
                    V[q][j, i] = t          # H_{b_n, a_n}
    return SliceSystem(h, 2 * L, np.zeros((h, h), np.complex128), V,
                       name=f"armchair half-rows M={M} L={L} t={t}")


def armchair_halfslice_onsite(eps: np.ndarray) -> np.ndarray:
    """(2L, M / 2) on-site energies of the half-row slicing from the row
    picture's (L, M)."""
    L, M = eps.shape
    out = np.empty((2 * L, M // 2))
    for n in range(L):
        a, b = armchair_half_sites(M, n)
        out[2 * n] = eps[n, a]
        out[2 * n + 1] = eps[n, b]
    return out


def armchair_halfslice_sigma(SL: np.ndarray, SR: np.ndarray, M: int, L: int):
    """The row picture's self-energies (..., M, M) restricted to the half-rows
    they act on: a_0 (left lead) and b_{L-1} (right lead)."""
    a0, _ = armchair_half_sites(M, 0)
    _, bl = armchair_half_sites(M, L - 1)
    return (np.ascontiguousarray(SL[..., a0[:, None], a0[None, :]]),
            np.ascontiguousarray(SR[..., bl[:, None], bl[None, :]]))


_s0 = np.eye(2, dtype=np.complex128)
_sx = np.array([[0, 1], [1, 0]], np.complex128)
_sy = np.array([[0, -1j], [1j, 0]], np.complex128)


def _bdg_hop(tau):
    """Nambu hopping in the basis (c_up, c_dn, c_dn^+, -c_up^+)."""
    z = np.zeros((2, 2), np.complex128)
    return np.block([[tau, z], [z, -_sy @ tau.conj() @ _sy]])


def bdg(Ns: int, L: int, mu: float = -1.0, t: float = 1.0, delta: float = 0.1,
        alpha: float = 0.2, lead_delta: float = 0.0) -> SliceSystem:
    """Spinful Bogoliubov-de Gennes square lattice, 4 x 4 blocks per site
    (spin x Nambu, basis (c_up, c_dn, c_dn^+, -c_up^+)), Ns sites per slice.
    On-site h = -mu s0 (disorder adds +eps to electrons, -eps to holes),
    pairing delta s0 between the electron and hole blocks, hopping t s0 plus
    Rashba: bond between slices +i alpha s_y, bond within a slice -i alpha s_x.
    The leads are the same lattice with pairing ``lead_delta``."""
    M = 4 * Ns

    def cell(d):
        h = -mu * _s0
        onsite = np.block([[h, d * _s0], [np.conj(d) * _s0, -_sy @ h.conj() @ _sy]])
        H0 = np.zeros((M, M), np.complex128)
        hy = _bdg_hop(t * _s0 - 1j * alpha * _sx)
        for s in range(Ns):
            H0[4 * s:4 * s + 4, 4 * s:4 * s + 4] = onsite
            if s + 1 < Ns:
                H0[4 * (s + 1):4 * (s + 2), 4 * s:4 * s + 4] = hy
                H0[4 * s:4 * s + 4, 4 * (s + 1):4 * (s + 2)] = hy.conj().T
        return H0

    V = np.kron(np.eye(Ns), _bdg_hop(t * _s0 + 1j * alpha * _sy))
    Hl = cell(lead_delta)
    return SliceSystem(M, L, cell(delta), V, block=4, sign=np.array([1.0, 1.0, -1.0, -1.0]),
                       lead_H0=(Hl, Hl), lead_V=(V, V),
                       name=f"bdg Ns={Ns} L={L} mu={mu} delta={delta} alpha={alpha}")


def random_slice_system(rng: np.random.Generator, M: int, L: int, P: int = 1,
                        hermitian_V: bool = False) -> SliceSystem:
    """Random dense slice blocks (Hermitian H0, general complex V) for brute-force
    checks on tiny lattices."""
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    H0 = (A + A.conj().T) / 2
    V = rng.standard_normal((P, M, M)) + 1j * rng.standard_normal((P, M, M))
    if hermitian_V:
        V = (V + np.swapaxes(V.conj(), 1, 2)) / 2
    return SliceSystem(M, L, H0, V, name=f"random M={M} L={L}")


def random_retarded_sigma(rng: np.random.Generator, M: int) -> np.ndarray:
    """A random matrix with the retarded sign structure: Hermitian part plus
    -i times a positive semi-definite part."""
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    B = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    return (A + A.conj().T) / 4 - 0.5j * (B @ B.conj().T) / M


@dataclass
class Batch:
    """Instances of one geometry: energies E[i], disorder seeds[i], strengths W[i]."""
    E: np.ndarray
    seeds: np.ndarray
    W: np.ndarray


def energy_seed_batch(E: np.ndarray, seeds, W: float) -> Batch:
    """All (energy, seed) pairs, energy-major: instance i = (E[i // nS], seeds[i % nS])."""
    seeds = np.asarray(seeds, dtype=np.uint64)
    nE, nS = len(E), len(seeds)
    return Batch(np.repeat(np.asarray(E, np.float64), nS), np.tile(seeds, nE),
                 np.full(nE * nS, float(W)))


def uneven_instances(n: int = 4096, seed: int = 12345,
                     widths=(32, 48, 64, 96, 128), lengths=(128, 256, 512, 1024, 2048),
                     wmax: float = 4.0, emax: float = 3.9):
    """The uneven square-lattice batch: per instance M and L uniform over the
    given sets, W ~ U[0, wmax], E ~ U(-emax, emax), disorder seed = index."""
    rng = np.random.default_rng(seed)
    M = rng.choice(np.asarray(widths), size=n)
    L = rng.choice(np.asarray(lengths), size=n)
    W = rng.uniform(0.0, wmax, size=n)
    E = rng.uniform(-emax, emax, size=n)
    return dict(M=M.astype(np.int32), L=L.astype(np.int32), W=W, E=E,
                seeds=np.arange(n, dtype=np.uint64))


def lshape_example():
    """The two-lead L-shaped system of the user guide's Sec. 2.2 worked example:
    block A = 8 x 4 sites at (0, 3), block B = 3 x 7 at (5, 0) glued on A,
    nearest-neighbour hopping t = 1, on-site 0.  Lead 0 is attached to the
    column x = 0 (y = 3..6), lead 1 to the row y = 0 (x = 5..7), both clean
    square leads with the same hopping.  Returns (H, idx0, idx1, width0, width1)."""
    sites = set()
    for x in range(8):
        for y in range(3, 7):
            sites.add((x, y))
    for x in range(5, 8):
        for y in range(0, 7):
            sites.add((x, y))
    sites = sorted(sites)
    idx = {s: i for i, s in enumerate(sites)}
    N = len(sites)
    H = np.zeros((N, N), np.complex128)
    for (x, y), i in idx.items():
        for dx, dy in ((1, 0), (0, 1)):
            j = idx.get((x + dx, y + dy))
            if j is not None:
                H[i, j] = H[j, i] = 1.0
    idx0 = [idx[(0, y)] for y in range(3, 7)]
    idx1 = [idx[(x, 0)] for x in range(5, 8)]
    return H, np.array(idx0), np.array(idx1), 4, 3
