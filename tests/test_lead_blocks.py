"""The lead decimation by symmetry blocks (the library's reading of Sec. 5.3
B for a lead sector that splits in a mode basis), pinned on the CPU with the
oracle's own decimation: in the eigenbasis U of K = H0 + a (V + V^dagger) +
i b (V - V^dagger) the Rashba strip's electron sector is block-diagonal, and
U diag(Sigma_r) U^dagger over the blocks' decimations equals the decimation
of the whole sector.  Without the i b term (K even under time reversal)
Kramers pairs mix the blocks, which the first test also checks.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

KA, KB = 0.3711, 0.6180   # the constants of the library's split


def electron_sector(Ns, mu=-1.0, alpha=0.2):
    b = inputs.bdg(Ns, 1, mu=mu, delta=0.0, alpha=alpha)
    e = [i for i in range(b.M) if i % 4 < 2]
    return b.lead_H0[0][np.ix_(e, e)], b.lead_V[0][np.ix_(e, e)]


def blocks_of(H0, V, kb=KB):
    K = H0 + KA * (V + V.conj().T) + kb * 1j * (V - V.conj().T)
    w, U = np.linalg.eigh(K)
    Hh, Vh = U.conj().T @ H0 @ U, U.conj().T @ V @ U
    tol = 1e-11 * max(np.abs(H0).max(), np.abs(V).max())
    adj = (np.abs(Hh) > tol) | (np.abs(Vh) > tol) | (np.abs(Vh.conj().T) > tol)
    n = len(w)
    comp = -np.ones(n, int)
    c = 0
    for i in range(n):
        if comp[i] >= 0:
            continue
        stack, comp[i] = [i], c
        while stack:
            j = stack.pop()
            for k in np.nonzero(adj[j])[0]:
                if comp[k] < 0:
                    comp[k] = c
                    stack.append(k)
        c += 1
    return U, Hh, Vh, [np.nonzero(comp == a)[0] for a in range(c)]


@pytest.mark.parametrize("Ns", [2, 5, 8])
def test_rashba_sector_splits_in_two(Ns):
    H0, V = electron_sector(Ns)
    U, Hh, Vh, bl = blocks_of(H0, V)
    assert [len(b) for b in bl] == [Ns, Ns]
    # without the time-reversal-odd term, Kramers pairs mix the two classes
    assert len(blocks_of(H0, V, kb=0.0)[3]) == 1


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("E", [-0.9, 0.35, 2.1])
def test_block_decimation_equals_whole_sector(side, E):
    H0, V = electron_sector(4)
    U, Hh, Vh, bl = blocks_of(H0, V)
    Sh = np.zeros_like(H0)
    for b in bl:
        Sh[np.ix_(b, b)] = oracle.decimation(Hh[np.ix_(b, b)], Vh[np.ix_(b, b)], E, side)[1]
    S_blocks = U @ Sh @ U.conj().T
    S_whole = oracle.decimation(H0, V, E, side)[1]
    assert np.abs(S_blocks - S_whole).max() < 1e-9
