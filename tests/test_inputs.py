"""The seeded synthetic inputs have the shapes and structure the workloads
state: energy grids of midpoints, Hermitian slice blocks with the couplings
of each lattice (square: t I; graphene brick wall: alternating bond masks;
BdG: 4 x 4 spin x Nambu blocks with particle-hole structure), the uneven
batch's distributions, and the L-shaped example's geometry.  CPU only."""
import numpy as np
import pytest

from paper_1010_2627_gb300 import inputs


def herm(A):
    return np.allclose(A, A.conj().T)


def test_energy_grid_midpoints():
    E = inputs.energy_grid(-3.9, 3.9, 1024)
    assert len(E) == 1024 and np.allclose(np.diff(E), 7.8 / 1024)
    assert np.isclose(E[0], -3.9 + 3.9 / 1024) and np.allclose(E, -E[::-1])


def test_square_and_chain():
    s = inputs.square(64, 512)
    assert s.H0.shape == (64, 64) and s.V.shape == (1, 64, 64) and herm(s.H0)
    assert np.allclose(s.V[0], np.eye(64)) and np.count_nonzero(s.H0) == 2 * 63
    c = inputs.chain(7)
    assert c.M == 1 and c.H0[0, 0] == 0 and c.V[0, 0, 0] == 1


def test_armchair_brick_wall():
    a = inputs.armchair(8, 5)
    assert a.V.shape == (2, 8, 8) and herm(a.H0)
    m0, m1 = np.diag(a.V[0]).real, np.diag(a.V[1]).real
    assert np.allclose(m0 + m1, 2.7) and set(m0) == {0.0, 2.7}    # every other site, alternating
    assert np.allclose(np.abs(a.H0[np.arange(7), np.arange(1, 8)]), 2.7)
    # three bonds per interior site of the honeycomb: two in-row, one vertical
    L, M = 6, 8
    a = inputs.armchair(M, L)
    deg = np.zeros((L, M))
    for n in range(L):
        deg[n] += (np.abs(a.H0) > 0).sum(axis=1)
        if n > 0:
            deg[n] += np.diag(a.V[n % 2]).real != 0
        if n + 1 < L:
            deg[n] += np.diag(a.V[(n + 1) % 2]).real != 0
    assert (deg[1:-1, 1:-1] == 3).all()
    lv, rv = a.lead_V
    assert lv.shape == (2, M, M) and np.allclose(lv[0], a.V[0]) and np.allclose(rv[0], a.V[L % 2])


def test_bdg_blocks_and_particle_hole_structure():
    b = inputs.bdg(4, 6, mu=-1.0, t=1.0, delta=0.1, alpha=0.2)
    assert b.M == 16 and b.block == 4 and herm(b.H0)
    assert np.allclose(b.sign, [1, 1, -1, -1])
    V = b.V[0]
    for i in range(4):     # block-diagonal coupling, 4 x 4 per site
        for j in range(4):
            if i != j:
                assert not V[4 * i:4 * i + 4, 4 * j:4 * j + 4].any()
    # particle-hole: with (c_up, c_dn, c_dn^+, -c_up^+), C = i s_y tau_y K
    # maps the single-particle blocks to minus themselves
    sy = np.array([[0, -1j], [1j, 0]])
    C = np.kron(np.eye(4), np.kron(sy, sy))
    assert np.allclose(C @ b.H0.conj() @ C.conj().T, -b.H0)
    assert np.allclose(C @ V.conj() @ C.conj().T, -V)
    bn = inputs.bdg(4, 6, delta=0.1, alpha=0.2, lead_delta=0.0)
    e, h = [0, 1], [2, 3]
    for blk in (bn.lead_H0[0], bn.lead_V[0]):   # normal leads: no electron-hole entries
        assert not blk.reshape(4, 4, 4, 4)[:, e][:, :, :, h].any()


def test_uneven_batch_recipe():
    u = inputs.uneven_instances()
    assert len(u["M"]) == 4096 and set(u["M"]) == {32, 48, 64, 96, 128}
    assert set(u["L"]) == {128, 256, 512, 1024, 2048}
    assert (0 <= u["W"]).all() and (u["W"] <= 4).all() and np.abs(u["E"]).max() < 3.9
    assert np.array_equal(u["seeds"], np.arange(4096))
    v = inputs.uneven_instances()
    assert all(np.array_equal(u[k], v[k]) for k in u)       # seeded


def test_lshape_example_geometry():
    H, i0, i1, w0, w1 = inputs.lshape_example()
    assert H.shape == (41, 41) and herm(H) and (w0, w1) == (4, 3)   # 32 + 21 - 12 shared
    assert len(i0) == 4 and len(i1) == 3 and not set(i0) & set(i1)
    deg = (np.abs(H) > 0).sum(axis=1)
    assert deg.max() == 4 and deg.min() == 2


def test_armchair_halfslices_same_transmission_as_rows():
    """The half-row slicing of an armchair ribbon is the same system: the
    oracle's slice sweep gives the row picture's T, with the same disorder
    and the row picture's lead self-energies restricted to a_0 and b_{L-1}."""
    import oracle
    from paper_1010_2627_gb300 import inputs
    for M, L in ((6, 3), (12, 5), (10, 4)):
        ss = inputs.armchair(M, L)
        hs = inputs.armchair_halfslices(M, L)
        eps = oracle.onsite(7, L, M, 0.8)
        for E in (-1.7, 0.3, 2.1):
            SL = oracle.decimation_period2(ss.H0, *ss.lead_V[0], E, 0)
            SR = oracle.decimation_period2(ss.H0, *ss.lead_V[1], E, 1)
            Tr = oracle.dense(ss.H0, ss.V, eps, L, E, SL, SR)["T_LR"]
            hl, hr = inputs.armchair_halfslice_sigma(SL, SR, M, L)
            # the row picture's Sigma lives on those half-rows only
            a0, _ = inputs.armchair_half_sites(M, 0)
            assert np.abs(SL).sum() == pytest.approx(np.abs(hl).sum(), rel=1e-14)
            Th = oracle.rgf(hs.H0, hs.V, inputs.armchair_halfslice_onsite(eps), 2 * L, E, hl, hr)["T"]
            assert abs(Th - Tr) < 1e-10, (M, L, E, Th, Tr)
