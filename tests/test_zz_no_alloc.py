"""The allocation-free lead decimation entry point against the allocating one.

knit_lead_decimation_noalloc exists for callers that cannot let the library
allocate device memory; it takes its scratch from a fixed array inside the
library.  This file is named to be collected last so that a run stopping at
its first failure has already run every other test."""
import numpy as np
import pytest

from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-8   # the decimation tolerance used by the other lead tests


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


def _dev(torch, a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).copy()).cuda()


CELLS = {
    # name: (system, energies)
    "square12": (lambda: inputs.square(12, 3), lambda: inputs.energy_grid(-3.5, 3.5, 37)),
    "bdg2": (lambda: inputs.bdg(2, 3, delta=0.0), lambda: inputs.energy_grid(-0.5, 0.5, 21)),
    # the largest cell the fixed array holds (M = 64, every slot of a chunk
    # in use) with an energy count that leaves a ragged last chunk of 5
    "square64": (lambda: inputs.square(64, 3), lambda: inputs.energy_grid(-3.9, 3.9, 37)),
}


@pytest.mark.parametrize("cell", sorted(CELLS))
def test_noalloc_matches_allocating_entry_point_twice(knit, cell):
    torch = pytest.importorskip("torch")
    ss, E = CELLS[cell][0](), CELLS[cell][1]()
    M = ss.M
    sysk = knit.System(ss)
    stream = torch.cuda.Stream()
    for lead in (0, 1):
        S_ref, it_ref, _ = sysk.lead_selfenergy(lead, E, method=knit.KNIT_LEAD_DECIMATION,
                                                eta=1e-12)
        dH0 = _dev(torch, ss.lead_H0[lead])
        dV = _dev(torch, ss.lead_V[lead])
        dE = torch.tensor(E, dtype=torch.float64, device="cuda")
        dS = torch.empty(len(E) * M * M * 2, dtype=torch.float64, device="cuda")
        dit = torch.empty(len(E), dtype=torch.int32, device="cuda")
        dst = torch.empty(len(E), dtype=torch.int32, device="cuda")
        for call in range(2):            # two calls in a row share the scratch
            dS.fill_(float("nan"))
            dit.fill_(-1)
            # the fills and uploads above ran on the current stream: order the
            # entry point's stream after them
            stream.wait_stream(torch.cuda.current_stream())
            knit.knit_lead_decimation_noalloc(dH0, dV, M, lead, dE, dS, eta=1e-12, iters=dit,
                                             status=dst, stream=stream)
            torch.cuda.synchronize()
            S = dS.cpu().numpy().view(np.complex128).reshape(len(E), M, M)
            assert (dst.cpu().numpy() == 0).all()
            # the allocating path decimates a cell that splits into decoupled
            # sectors (the Nambu cell) sector by sector; each sector may stop
            # one doubling before the whole cell does
            assert np.abs(dit.cpu().numpy() - it_ref).max() <= 1
            assert np.abs(S - S_ref).max() <= TOL, (cell, lead, call)
    sysk.close()


def test_noalloc_rejects_what_it_cannot_hold(knit):
    torch = pytest.importorskip("torch")
    M = 65
    d = torch.zeros(M * M * 2, dtype=torch.float64, device="cuda")
    dE = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(knit.KnitError) as ei:
        knit.knit_lead_decimation_noalloc(d, d, M, 0, dE, d)
    assert ei.value.code == knit.KNIT_ERR_INVALID
    assert "64" in knit.knit_last_error()
    h = np.zeros((4, 4), np.complex128)
    with pytest.raises(knit.KnitError) as ei:
        knit.knit_lead_decimation_noalloc(h, h, 4, 0, np.zeros(1), h)
    assert ei.value.code == knit.KNIT_ERR_INVALID
