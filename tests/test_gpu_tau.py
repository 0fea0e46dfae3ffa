"""GPU parity for the transmission eigenvalues tau_n and the shot noise
sum tau (1 - tau) (knit_transmission_eigenvalues) against the oracle's
eigenvalues of the matrix inside Sec. 2.3's transmission trace.

Tolerance per eigenvalue: 1e-8 for KNIT_FP64 and 1e-6 for KNIT_MIXED, the
bounds the transmission itself meets (Weyl: an eigenvalue moves by at most
the norm of the perturbation of the Hermitian matrix, whose trace is T)."""
import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-8, 1: 1e-6}


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def oracle_tau(ss, E, seed, W, SL=None, SR=None):
    eps = oracle.onsite(seed, ss.L, ss.M, W, block=ss.block, sign=ss.sign) if W else None
    if SL is None:
        SL = SR = oracle.sigma_square(ss.M, ss.V[0][0, 0].real, E)
    r = oracle.rgf(ss.H0, ss.V, eps, ss.L, E, SL, SR)
    return oracle.transmission_eigenvalues(r["G1L"], SL, SR), r["T"]


def check(tau, noise, T, st, ss, E, seeds, W, precision, sig=None):
    assert (st == 0).all()
    tol = TOL[precision]
    for e, Ee in enumerate(E):
        SL, SR = (None, None) if sig is None else sig(Ee)
        for s, sd in enumerate(seeds):
            to, Tt = oracle_tau(ss, Ee, int(sd), W, SL, SR)
            g = tau[e, s]
            assert np.all(np.diff(g) <= 0), "decreasing order"
            assert np.abs(g - to).max() <= tol, (Ee, int(sd), np.abs(g - to).max())
            assert abs(noise[e, s] - oracle.shot_noise(to)) <= tol * ss.M
            # the same call's T is the trace of the diagonalised matrix
            assert abs(g.sum() - T[e, s]) <= 1e-9 * max(1.0, abs(T[e, s]))
            assert abs(T[e, s] - Tt) <= tol * max(1.0, Tt)


@pytest.mark.parametrize("precision", [0, 1])
def test_tau_small_config(knit, precision):
    ss = inputs.square(16, 24)
    E = np.array([-3.3, -1.45, -0.2, 0.65, 2.1, 3.7])
    seeds = np.array([0, 7], np.uint64)
    tau, noise, T, st = knit.System(ss).transmission_eigenvalues(E, seeds, W=1.5,
                                                                 precision=precision)
    check(tau, noise, T, st, ss, E, seeds, 1.5, precision)


# widths that select each sweep kernel: mixed CUDA-core (<= 32), tensor-core
# residual (33 .. 64, ragged 37 and 40), wide (96); FP64 at all of them
@pytest.mark.parametrize("M,L", [(1, 9), (5, 7), (37, 12), (40, 20), (64, 16), (96, 6)])
@pytest.mark.parametrize("precision", [0, 1])
def test_tau_widths(knit, M, L, precision):
    ss = inputs.square(M, L)
    E = np.array([-2.35, 0.4, 1.9])
    seeds = np.array([4, 9], np.uint64)
    tau, noise, T, st = knit.System(ss).transmission_eigenvalues(E, seeds, W=2.0,
                                                                 precision=precision)
    assert tau.shape == (3, 2, M)
    check(tau, noise, T, st, ss, E, seeds, 2.0, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_tau_clean_ribbon_zero_or_one(knit, precision):
    """Clean ribbon: N_ch eigenvalues 1, the rest 0, no shot noise."""
    M = 24
    ss = inputs.square(M, 30)
    ek = 2 * np.cos(np.arange(1, M + 1) * np.pi / (M + 1))
    E = inputs.energy_grid(-3.9, 3.9, 17)
    E = E[np.min(np.abs(np.abs(E[:, None] - ek[None]) - 2), axis=1) > 1e-3]
    tau, noise, T, st = knit.System(ss).transmission_eigenvalues(E, precision=precision)
    assert (st == 0).all()
    for e, Ee in enumerate(E):
        n = int(np.sum(np.abs(Ee - ek) < 2))
        want = np.r_[np.ones(n), np.zeros(M - n)]
        assert np.abs(tau[e, 0] - want).max() < TOL[precision]
        assert abs(noise[e, 0]) < TOL[precision] * M


def test_tau_armchair_period2_leads(knit):
    """Armchair ribbon with period-2 leads (mixed sweep): the right lead's
    Gamma^{1/2} comes from the supercell self-energy."""
    ss = inputs.armchair(24, 30)
    E = np.array([-2.9, 0.8])
    seeds = np.array([5], np.uint64)
    W = 0.5 * 2.7

    def sig(Ee):
        return (oracle.decimation_period2(ss.H0, *ss.lead_V[0], Ee, 0),
                oracle.decimation_period2(ss.H0, *ss.lead_V[1], Ee, 1))

    tau, noise, T, st = knit.System(ss).transmission_eigenvalues(E, seeds, W=W, precision=1)
    check(tau, noise, T, st, ss, E, seeds, W, 1, sig)


def test_tau_bench_workload_sampled(knit):
    """The 64 x 512 bench geometry (W = 2): instances across the band and at
    both edges, mixed sweep."""
    ss = inputs.square(64, 512)
    E = np.array([-3.85, -2.6, -0.9, 0.35, 1.8, 3.9])
    seeds = np.array([1, 6], np.uint64)
    tau, noise, T, st = knit.System(ss).transmission_eigenvalues(E, seeds, W=2.0, precision=1)
    check(tau, noise, T, st, ss, E, seeds, 2.0, 1)
    assert (tau >= -1e-6).all() and (tau <= 1 + 1e-6).all()


def test_tau_device_outputs_and_invalid(knit):
    """Device output buffers give the host result; NULL tau and M > 256 are rejected."""
    import torch
    ss = inputs.square(12, 10)
    sysk = knit.System(ss)
    E = np.array([-1.1, 0.3, 2.2])
    tau, noise, T, st = sysk.transmission_eigenvalues(E, [2, 3], W=1.0, precision=1)
    dtau = torch.empty((6, 12), dtype=torch.float64, device="cuda")
    dn = torch.empty(6, dtype=torch.float64, device="cuda")
    knit.knit_transmission_eigenvalues(sysk.handle, E, np.array([2, 3], np.uint64), 1.0, 1,
                                       dtau, dn)
    torch.cuda.synchronize()
    assert np.array_equal(dtau.cpu().numpy().reshape(3, 2, 12), tau)
    assert np.array_equal(dn.cpu().numpy().reshape(3, 2), noise)
    with pytest.raises(Exception):
        knit.knit_transmission_eigenvalues(sysk.handle, E, None, 1.0, 1, None)
