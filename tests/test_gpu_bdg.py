"""GPU parity at the spinful BdG bar's width (32 sites x 4 = 128 orbitals
per slice, the Rashba bar of the BdG workload) against the oracle's dense
solve (Eq. 2, Sec. 2.3).

The sweep is checked on its own by giving the GPU the oracle's self-energies
(knit_transmission_sigma): |dT| / max(1, N_ch) <= 1e-8 in FP64 and <= 1e-6 in
the mixed mode, with N_ch the open channels of the clean BdG leads at E
(propagating incoming Bloch modes of the lead, counted by mode analysis).
End to end (the GPU's own lead decimation) the two sides also differ by their
decimations at eta = 1e-12: those agree to ~1e-8 in Sigma (the decimation
tolerance of the other lead tests), which moves T by up to ~1e-8 per open
channel, so the end-to-end bound is twice the sweep's."""
import numpy as np
import pytest

import oracle
import scattering as sc
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-8
TOL_MIXED = 1e-6
SEED, W = 4, 1.0


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def open_channels(b, E):
    """min over the two leads of the propagating incoming modes at E"""
    return min(len(sc.lead_modes(b.lead_H0[p], b.lead_V[p], E, p)[3]) for p in (0, 1))


@pytest.fixture(scope="module")
def bdg32_cases():
    """Ns = 32 bars of lengths 3 and 6 with the oracle's leads and dense T"""
    E = np.array([-0.17, -0.05, 0.04, 0.13])
    out = {}
    for L in (3, 6):
        b = inputs.bdg(32, L, mu=-1.0, delta=0.1, alpha=0.2)
        eps = oracle.onsite(SEED, L, b.M, W, block=4, sign=b.sign)
        SL = np.stack([oracle.decimation(b.lead_H0[0], b.lead_V[0], e, 0, eta=1e-12)[1] for e in E])
        SR = np.stack([oracle.decimation(b.lead_H0[1], b.lead_V[1], e, 1, eta=1e-12)[1] for e in E])
        To = np.array([oracle.dense(b.H0, b.V, eps, L, e, SL[k], SR[k])["T_LR"]
                       for k, e in enumerate(E)])
        nch = np.array([max(1, open_channels(b, e)) for e in E])
        out[L] = (b, E, SL, SR, To, nch)
    return out


@pytest.mark.parametrize("L", [3, 6])
@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_MIXED)])
def test_bdg32_sweep_with_oracle_leads(knit, bdg32_cases, L, precision, tol):
    b, E, SL, SR, To, nch = bdg32_cases[L]
    sysk = knit.System(b)
    T, st = sysk.transmission_sigma(E, SL, SR, seeds=[SEED], W=W, precision=precision)
    sysk.close()
    assert (st == 0).all()
    err = np.abs(T[:, 0] - To) / nch
    assert err.max() <= tol, (precision, L, err, T[:, 0], To)


@pytest.mark.parametrize("L", [3, 6])
@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_MIXED)])
def test_bdg32_end_to_end(knit, bdg32_cases, L, precision, tol):
    b, E, _, _, To, nch = bdg32_cases[L]
    sysk = knit.System(b)
    T, st = sysk.transmission(E, seeds=[SEED], W=W, precision=precision)
    sysk.close()
    assert (st == 0).all()
    err = np.abs(T[:, 0] - To) / nch
    assert err.max() <= 2 * tol, (precision, L, err)


def test_bdg3_sweep_fp64_with_oracle_leads(knit):
    """the small BdG bar of the block-coupling test, sweep alone at 1e-8"""
    b = inputs.bdg(3, 6, mu=-1.0, delta=0.1, alpha=0.2)
    E = np.array([-0.11, 0.05])
    eps = oracle.onsite(SEED, b.L, b.M, W, block=4, sign=b.sign)
    SL = np.stack([oracle.decimation(b.lead_H0[0], b.lead_V[0], e, 0, eta=1e-12)[1] for e in E])
    SR = np.stack([oracle.decimation(b.lead_H0[1], b.lead_V[1], e, 1, eta=1e-12)[1] for e in E])
    sysk = knit.System(b)
    for precision, tol in ((0, TOL_FP64), (1, TOL_MIXED)):
        T, st = sysk.transmission_sigma(E, SL, SR, seeds=[SEED], W=W, precision=precision)
        assert (st == 0).all()
        for k, e in enumerate(E):
            To = oracle.dense(b.H0, b.V, eps, b.L, e, SL[k], SR[k])["T_LR"]
            assert abs(T[k, 0] - To) <= tol * max(1, open_channels(b, e)), (precision, e)
    sysk.close()


@pytest.mark.parametrize("Ns,lead_delta", [(32, 0.0), (6, 0.0), (6, 0.05)])
def test_bdg_lead_sectors_against_oracle(knit, Ns, lead_delta):
    """Normal Nambu leads split into electron and hole sectors, and each of
    those into two blocks in a mode basis (the transverse mirror combined
    with a spin rotation commutes with the Rashba lead's H0 and V), which the
    GPU decimates one by one (Sec. 5.3 B on each decoupled block); a lead
    with pairing does not split.  Either way Sigma equals the oracle's
    decimation of the whole cell to the decimation tolerance (1e-8)."""
    b = inputs.bdg(Ns, 3, mu=-1.0, delta=0.1, alpha=0.2, lead_delta=lead_delta)
    E = np.array([-0.17, 0.04]) if Ns == 32 else np.array([-0.17, 0.04, 0.11])
    sysk = knit.System(b)
    assert sysk.info()[1] == ([1, 1] if lead_delta else [4, 4])
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, method=knit.KNIT_LEAD_DECIMATION, eta=1e-12,
                                          want_residual=True)
        for e, Ee in enumerate(E):
            So = oracle.decimation(b.lead_H0[lead], b.lead_V[lead], Ee, lead, eta=1e-12)[1]
            assert np.abs(S[e] - So).max() < 1e-8, (Ns, lead_delta, lead, Ee)
            assert res[e] < 1e-5
    sysk.close()


def test_bdg_lead_particle_hole_pairs_symmetric_grid(knit):
    """Normal Nambu leads: the hole sector is the particle-hole image of the
    electron sector, so on a grid symmetric about zero every hole block comes
    from the electron block at -E of the same list; both against the
    oracle's decimation of the whole cell (1e-8), and the end-to-end T with
    the mirror symmetry T(E) = T(-E) of a bar without disorder"""
    b = inputs.bdg(6, 4, mu=-1.0, delta=0.1, alpha=0.2)
    E = inputs.energy_grid(-0.16, 0.16, 6)
    assert np.array_equal(E, -E[::-1]) or np.abs(E + E[::-1]).max() < 1e-15
    sysk = knit.System(b)
    # electron and hole sectors, each two mode blocks (mirror x spin rotation)
    assert sysk.info()[1] == [4, 4]
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, method=knit.KNIT_LEAD_DECIMATION, eta=1e-12,
                                          want_residual=True)
        for e, Ee in enumerate(E):
            So = oracle.decimation(b.lead_H0[lead], b.lead_V[lead], Ee, lead, eta=1e-12)[1]
            assert np.abs(S[e] - So).max() < 1e-8, (lead, Ee)
            assert res[e] < 1e-5
    T, st = sysk.transmission(E, precision=knit.KNIT_FP64)
    sysk.close()
    assert (st == 0).all()
    assert np.abs(T[:, 0] - T[::-1, 0]).max() < 1e-8


def _rashba_electron_cell(Ns, mu, alpha):
    """the electron sector (c_up, c_dn per site) of the normal BdG lead"""
    b = inputs.bdg(Ns, 1, mu=mu, delta=0.0, alpha=alpha)
    e = [i for i in range(b.M) if i % 4 < 2]
    return b.lead_H0[0][np.ix_(e, e)], b.lead_V[0][np.ix_(e, e)]


def test_two_unrelated_sectors_split_in_mode_basis(knit):
    """A lead of two decoupled Rashba strips with different mu and alpha: two
    orbital sectors that are not particle-hole images of each other, so each
    is decimated by itself, and each splits again into two mode blocks.
    Sigma of both leads against the oracle's decimation of the whole cell
    (1e-8), and the FP64 transmission of a short bar against the oracle's
    dense solve with the oracle's self-energies."""
    Ns = 5
    ha, va = _rashba_electron_cell(Ns, -1.0, 0.2)
    hb, vb = _rashba_electron_cell(Ns, -0.7, 0.35)
    m = ha.shape[0]
    Z = np.zeros((m, m), np.complex128)
    H0 = np.block([[ha, Z], [Z, hb]])
    V = np.block([[va, Z], [Z, vb]])
    b = inputs.SliceSystem(2 * m, 3, H0, V, name="two Rashba strips")
    E = np.array([-0.9, 0.3, 1.7])
    sysk = knit.System(b)
    assert sysk.info()[1] == [4, 4]
    S_or = []
    for lead in (0, 1):
        S, it, res = sysk.lead_selfenergy(lead, E, method=knit.KNIT_LEAD_DECIMATION, eta=1e-12,
                                          want_residual=True)
        So = np.stack([oracle.decimation(b.lead_H0[lead], b.lead_V[lead], e, lead, eta=1e-12)[1]
                       for e in E])
        S_or.append(So)
        assert np.abs(S - So).max() < 1e-8, lead
        assert (res < 1e-5).all()
    T, st = sysk.transmission(E, precision=knit.KNIT_FP64)
    sysk.close()
    assert (st == 0).all()
    eps = np.zeros((b.L, b.M))
    To = np.array([oracle.dense(b.H0, b.V, eps, b.L, e, S_or[0][k], S_or[1][k])["T_LR"]
                   for k, e in enumerate(E)])
    assert np.abs(T[:, 0] - To).max() < 1e-8
