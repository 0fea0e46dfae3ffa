"""GPU parity for the lead-resolved lesser function (knit_lesser): injected
densities and left-injected bond currents against the oracle's dense
G Gamma_l G^+ (Sec. 2.3), plus the sum rule, current conservation and
Kirchhoff's law on the GPU output itself.  Both sides are FP64: with the
closed-form square-lead self-energy on both sides they agree to 1e-10 (only
the elimination order differs); with decimated leads (BdG, armchair) to
1e-7, the agreement of the two decimations (as for T)."""
import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def compare(out, ss, E, seeds, W, sig, tol=TOL):
    assert (out["status"] == 0).all()
    for e, Ee in enumerate(E):
        SL, SR = sig(Ee)
        for s, sd in enumerate(seeds):
            eps = oracle.onsite(int(sd), ss.L, ss.M, W, block=ss.block, sign=ss.sign) if W else None
            r = oracle.lesser_parts(ss.H0, ss.V, eps, ss.L, Ee, SL, SR)
            for k in ("rhoL", "rhoR", "jx", "jt"):
                d = np.abs(out[k][e, s] - r[k]).max() if r[k].size else 0.0
                assert d <= tol * max(1.0, np.abs(r[k]).max() if r[k].size else 1.0), (k, Ee, sd, d)
            assert abs(out["T"][e, s] - r["T"]) <= tol * max(1.0, r["T"])


def square_sig(M):
    return lambda E: (oracle.sigma_square(M, 1.0, E),) * 2


@pytest.mark.parametrize("saving_level", [-1, 1, 3, 8])
def test_lesser_square(knit, saving_level):
    ss = inputs.square(6, 9)
    E = np.array([-2.2, 0.35, 1.6])
    seeds = np.array([2, 5], np.uint64)
    out = knit.System(ss).lesser(E, seeds, W=2.0, saving_level=saving_level)
    compare(out, ss, E, seeds, 2.0, square_sig(6))


def test_lesser_conservation_and_kirchhoff(knit):
    """On the GPU output alone: every slice interface carries T; inflow equals
    outflow at every interior orbital (diagonal V); rhoL + rhoR = LDOS."""
    M, L = 10, 14
    ss = inputs.square(M, L)
    E = np.array([-1.3, 0.2, 2.7])
    sysk = knit.System(ss)
    out = sysk.lesser(E, [7], W=2.5, saving_level=4)
    ld, _, _ = sysk.ldos(E, [7], W=2.5, saving_level=4)
    for e in range(len(E)):
        jx, jt, T = out["jx"][e, 0], out["jt"][e, 0], out["T"][e, 0]
        assert np.abs(jx.sum(axis=1) - T).max() < 1e-10 * max(1.0, T)
        edges = [(x, x + 1) for x in range(M - 1)]
        net = np.zeros((L, M))
        net[:-1] += jx
        net[1:] -= jx
        for k, (x, y) in enumerate(edges):
            net[:, x] += jt[:, k]
            net[:, y] -= jt[:, k]
        assert np.abs(net[1:-1]).max() < 1e-10
        assert np.abs(out["rhoL"][e, 0] + out["rhoR"][e, 0] - ld[e, 0]).max() < 1e-10


def test_lesser_clean_chain_closed_form(knit):
    E = np.array([-1.5, 0.4, 1.8])
    out = knit.System(inputs.chain(7)).lesser(E)
    for e, Ee in enumerate(E):
        half = 1 / (2 * np.pi * np.sqrt(4 - Ee * Ee))
        assert np.abs(out["rhoL"][e, 0] - half).max() < 1e-12
        assert np.abs(out["rhoR"][e, 0] - half).max() < 1e-12
        assert np.abs(out["jx"][e, 0] - 1.0).max() < 1e-12
    assert out["jt"].shape[-1] == 0


def test_lesser_bdg_blocks(knit):
    """Spin x Nambu blocks: 4 x 4 inter-slice couplings and a complex H0
    (Rashba), so jx sums over a block and jt runs over complex edges."""
    b = inputs.bdg(3, 5, mu=-1.0, t=1.0, delta=0.2, alpha=0.3)
    E = np.array([-0.4, 0.25])

    def sig(Ee):
        return (oracle.decimation(b.lead_H0[0], b.lead_V[0], Ee, 0, eta=1e-12)[1],
                oracle.decimation(b.lead_H0[1], b.lead_V[1], Ee, 1, eta=1e-12)[1])

    out = knit.System(b).lesser(E, [3], W=0.8, saving_level=2)
    compare(out, b, E, np.array([3]), 0.8, sig, tol=1e-7)


def test_lesser_armchair_period2(knit):
    ss = inputs.armchair(8, 6)

    def sig(Ee):
        return (oracle.decimation_period2(ss.H0, *ss.lead_V[0], Ee, 0),
                oracle.decimation_period2(ss.H0, *ss.lead_V[1], Ee, 1))

    E = np.array([-1.9, 0.7])
    out = knit.System(ss).lesser(E, [4], W=1.0)
    compare(out, ss, E, np.array([4]), 1.0, sig, tol=1e-7)


def test_lesser_single_slice_and_invalid(knit):
    ss = inputs.square(5, 1)
    out = knit.System(ss).lesser(np.array([0.3, -1.1]), W=1.0)
    compare(out, ss, np.array([0.3, -1.1]), np.array([0]), 1.0, square_sig(5))
    assert out["jx"].shape[2] == 0
    sysk = knit.System(inputs.square(4, 3))
    with pytest.raises(Exception):
        knit.knit_lesser(sysk.handle, np.array([0.1]), None, 0.0, 0, np.empty(12))
    with pytest.raises(Exception):
        knit.knit_lesser(sysk.handle, np.array([0.1]), None, 0.0, -1)
