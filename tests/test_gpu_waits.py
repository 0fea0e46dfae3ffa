"""Failure detection on the GPU without a fault: the bounded tensor-core wait
is made to run out (a barrier that nothing completes), the kernel reports
KNIT_ERR_TIMEOUT, releases its tensor memory after a bounded wait for its
last commit, and the context stays usable for the next sweep.  Also the peak
loops that give the roofline denominators run to completion."""
import numpy as np
import pytest

import oracle
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def _small_mixed_sweep_matches_oracle(knit):
    M, L, W = 40, 6, 1.0          # width 40: the tensor-core sweep kernel
    ss = inputs.square(M, L)
    E = np.array([-1.3, 0.45])
    T, st = knit.System(ss).transmission(E, seeds=[3], W=W, precision=knit.KNIT_MIXED)
    assert (st == 0).all()
    for k, e in enumerate(E):
        S = oracle.sigma_square(M, 1.0, e)
        To = oracle.dense(ss.H0, ss.V, oracle.onsite(3, L, M, W), L, e, S, S)["T_LR"]
        assert abs(T[k, 0] - To) <= 1e-6 * M


@pytest.mark.parametrize("polls", [1, 1000])
def test_bounded_wait_runs_out_and_context_survives(knit, polls):
    ws, cleanup = knit.knit_debug_wait_probe(polls)
    assert ws == knit.KNIT_ERR_TIMEOUT
    assert cleanup == 1          # the committed MMA was waited for before the release
    _small_mixed_sweep_matches_oracle(knit)


def test_wait_probe_rejects_bad_bounds(knit):
    for polls in (0, 1 << 25):
        with pytest.raises(knit.KnitError) as ei:
            knit.knit_debug_wait_probe(polls)
        assert ei.value.code == knit.KNIT_ERR_INVALID


def test_peak_loops_complete(knit):
    torch = pytest.importorskip("torch")
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for kind, iters in ((knit.KNIT_PEAK_MMA_BF16, 2000), (knit.KNIT_PEAK_MMA_TF32, 2000),
                        (knit.KNIT_PEAK_DFMA, 10), (knit.KNIT_PEAK_FFMA, 10)):
        flop = knit.knit_peak_probe(kind, iters, nsm, check=True)
        assert flop > 0
    _small_mixed_sweep_matches_oracle(knit)
