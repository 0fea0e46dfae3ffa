"""GPU parity for honeycomb (armchair) ribbons up to 256 sites per row
(Sec. 6.3 geometry, Sec. 2.3 transmission): period-2 leads decimated block by
block in the eigenbasis of their cell Hamiltonian, and KNIT_MIXED run on the
half-row chain (width M / 2, tridiagonal couplings of period 4).  The lead
blocks are checked against the oracle's decimation of the whole two-slice
supercell where the oracle finishes in seconds (M <= 66) and, at M = 256,
by the fixed point and retarded branch of the assembled supercell g; the
half-row sweeps against the oracle's row-picture sweep given the same
self-energies and disorder.  Tolerances: 1e-8 relative on the self-energies
(the decimation tolerance of the other lead tests), |dT| <= 1e-6 per site of
the row (mixed) and 1e-8 (FP64)."""
import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


@pytest.mark.parametrize("M,E", [(16, (-4.1, -0.6, 0.35, 1.9, 5.2)), (66, (-2.3, 0.05, 0.77))])
def test_period2_lead_blocks_against_oracle(knit, M, E):
    """every mode pair (k, M + 1 - k) a 4 x 4 supercell of its own"""
    ss = inputs.armchair(M, 3)
    E = np.array(E)
    sysk = knit.System(ss)
    assert sysk.info()[1] == [M // 2, M // 2]
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, want_residual=True)
        for e, Ee in enumerate(E):
            So = oracle.decimation_period2(ss.H0, *ss.lead_V[lead], Ee, lead)
            assert np.abs(S[e] - So).max() < 1e-8 * max(1.0, np.abs(So).max()), (M, lead, Ee)
            assert res[e] < 1e-7, (M, lead, Ee, res[e])
    sysk.close()


def test_period2_lead_blocks_width_256(knit):
    """fixed point of the whole 512 x 512 supercell, retarded self-energy
    (Im Sigma_kk <= 0, Sigma restricted to the coupled sites), and a clean
    ribbon that transmits an integer number of channels"""
    M = 256
    ss = inputs.armchair(M, 6)
    E = np.array([-2.2, -0.41, 0.05, 0.77, 1.6])
    sysk = knit.System(ss)
    assert sysk.info()[1] == [M // 2, M // 2]
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, want_residual=True)
        assert (res < 1e-7).all(), (lead, res)
        Vf = ss.lead_V[lead][0]
        sup = np.abs(np.diag(Vf)) > 0
        for e in range(len(E)):
            assert np.diag(S[e]).imag.max() <= 1e-12
            assert np.abs(S[e][~sup]).max() == 0.0 and np.abs(S[e][:, ~sup]).max() == 0.0
    Tm, stm = sysk.transmission(E, precision=knit.KNIT_MIXED)
    Tf, stf = sysk.transmission(E, precision=knit.KNIT_FP64)
    sysk.close()
    assert (stm == 0).all() and (stf == 0).all()
    assert np.abs(Tf - np.round(Tf)).max() <= TOL_FP64 * M, Tf[:, 0]
    assert np.abs(Tm - Tf).max() <= TOL_MIXED * M


def test_half_rows_chosen_only_above_128(knit):
    wide = knit.System(inputs.armchair(200, 2))
    narrow = knit.System(inputs.armchair(128, 2))
    assert wide.info(knit.KNIT_MIXED)[0] == knit.KNIT_SWEEP_MIXED_HALF_ROWS
    assert wide.info(knit.KNIT_FP64)[0] == knit.KNIT_SWEEP_FP64
    assert narrow.info(knit.KNIT_MIXED)[0] == knit.KNIT_SWEEP_MIXED_TC128
    square = knit.System(inputs.square(200, 2))   # rows that do not split into halves
    assert square.info(knit.KNIT_MIXED)[0] == knit.KNIT_SWEEP_FP64
    for s in (wide, narrow, square):
        s.close()


@pytest.mark.parametrize("M,L", [(130, 5), (200, 3), (256, 4)])
def test_rows_mixed_by_half_rows_against_oracle(knit, M, L):
    """W = 1 disorder drawn per (row, site) on both sides, so the half-row
    chain sees the row picture's realisation; the oracle sweeps the row
    picture with the GPU's lead self-energies"""
    ss = inputs.armchair(M, L)
    E = np.array([-1.3, 0.21, 0.9])
    seeds = np.array([5, 9], np.uint64)
    sysk = knit.System(ss)
    SL = sysk.lead_selfenergy(0, E)[0]
    SR = sysk.lead_selfenergy(1, E)[0]
    Tm, stm = sysk.transmission(E, seeds, W=1.0, precision=knit.KNIT_MIXED)
    Tf, stf = sysk.transmission(E, seeds, W=1.0, precision=knit.KNIT_FP64)
    sysk.close()
    assert (stm == 0).all() and (stf == 0).all()
    for e, Ee in enumerate(E):
        for s, sd in enumerate(seeds):
            eps = oracle.onsite(int(sd), L, M, 1.0)
            To = oracle.rgf(ss.H0, ss.V, eps, L, Ee, SL[e], SR[e])["T"]
            assert abs(Tf[e, s] - To) <= TOL_FP64 * M, (M, Ee, int(sd), Tf[e, s], To)
            assert abs(Tm[e, s] - To) <= TOL_MIXED * M, (M, Ee, int(sd), Tm[e, s], To)


def test_rows_mixed_explicit_onsite_long(knit):
    """explicit on-site energies remapped to the half-rows; a longer ribbon
    against the FP64 row sweep"""
    M, L = 256, 40
    ss = inputs.armchair(M, L)
    eps = oracle.onsite(13, L, M, 1.0)
    E = np.array([-1.7, -0.2, 0.45, 1.1])
    sysk = knit.System(ss, onsite=eps)
    Tm, stm = sysk.transmission(E, precision=knit.KNIT_MIXED)
    Tf, stf = sysk.transmission(E, precision=knit.KNIT_FP64)
    sysk.close()
    assert (stm == 0).all() and (stf == 0).all()
    assert np.abs(Tm - Tf).max() <= TOL_MIXED * M, (Tm[:, 0], Tf[:, 0])


def test_half_rows_sigma_support_flag(knit):
    """a caller-supplied Sigma with entries outside the end half-rows cannot
    ride the half-row chain: those energies come back KNIT_ERR_INVALID"""
    M, L = 200, 2
    ss = inputs.armchair(M, L)
    E = np.array([-0.5, 0.6])
    sysk = knit.System(ss)
    SL = sysk.lead_selfenergy(0, E)[0]
    SR = sysk.lead_selfenergy(1, E)[0]
    T, st = sysk.transmission_sigma(E, SL, SR, precision=knit.KNIT_MIXED)
    Tf, stf = sysk.transmission_sigma(E, SL, SR, precision=knit.KNIT_FP64)
    assert (st == 0).all() and (stf == 0).all()
    assert np.abs(T - Tf).max() <= TOL_MIXED * M
    SL2 = SL.copy()
    SL2[1, 1, 1] += 0.1   # site 1 of row 0 is not coupled to the left lead
    T2, st2 = sysk.transmission_sigma(E, SL2, SR, precision=knit.KNIT_MIXED)
    sysk.close()
    assert st2[0, 0] == 0 and st2[1, 0] == knit.KNIT_ERR_INVALID
