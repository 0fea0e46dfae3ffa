"""Failure injection on the host: every device allocation of a create +
transmission sequence is made to fail in turn (knit_debug_fail_alloc_after).
Each failure must come back as KNIT_ERR_OOM, leave the context usable and
release what the call had allocated; the first run that no injection reaches
must give the undisturbed result.  No kernel is made to fault or wait.  Runs
last (file name) because it arms a process-wide switch."""
import gc

import numpy as np
import pytest

from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def run(knit, ss, E, seeds):
    sysk = knit.System(ss)
    try:
        T, st = sysk.transmission(E, seeds, W=1.5, precision=knit.KNIT_MIXED)
        T64, _ = sysk.transmission(E, seeds, W=1.5, precision=knit.KNIT_FP64)
    finally:
        sysk.close()
    return T, st, T64


def test_each_allocation_failure_reports_oom_and_recovers(knit):
    import torch
    ss = inputs.square(40, 12)
    E = np.array([-2.1, 0.4, 1.7])
    seeds = np.array([3, 8], np.uint64)
    ref = run(knit, ss, E, seeds)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    fired = 0
    try:
        for k in range(200):
            knit.knit_debug_fail_alloc_after(k)
            try:
                got = run(knit, ss, E, seeds)
            except knit.KnitError as e:
                assert e.code == knit.KNIT_ERR_OOM, (k, str(e))
                fired += 1
                continue
            break
        else:
            pytest.fail("every run hit an injected failure")
    finally:
        knit.knit_debug_fail_alloc_after(-1)
    assert fired >= 5
    assert (got[1] == 0).all()
    assert np.allclose(got[0], ref[0], rtol=0, atol=1e-12)
    assert np.allclose(got[2], ref[2], rtol=0, atol=1e-12)
    gc.collect()
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < 64 << 20
