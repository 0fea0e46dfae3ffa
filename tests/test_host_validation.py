"""CPU-side checks of the boundary's argument validation.  Every entry point
checks its arguments on the host before it touches the device, so these run
without a GPU: a bad descriptor or a NULL handle returns KNIT_ERR_INVALID with
a message, never a CUDA error or a crash.  On a machine without a GPU a valid
descriptor gets past validation and then fails loudly at the first device
allocation (no CPU fallback)."""
import ctypes

import numpy as np
import pytest

from paper_1010_2627_gb300 import knit

INVALID = 1
CUDA = 3


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1010_2627_gb300 import build
    build.build()
    knit.load()


def chain(M):
    H0 = np.zeros((M, M), complex)
    for i in range(M - 1):
        H0[i, i + 1] = H0[i + 1, i] = -1.0
    return H0, -np.eye(M, dtype=complex)


def create_code(**kw):
    try:
        h = knit.knit_system_create(**kw)
    except knit.KnitError as e:
        return e.code, str(e)
    knit.knit_system_destroy(h)
    return 0, ""


def base(M=4, L=5):
    H0, V = chain(M)
    return dict(M=M, L=L, H0=H0, V=V)


def _no_gpu():
    try:
        import torch
        return not torch.cuda.is_available()
    except Exception:
        return True


@pytest.mark.parametrize("change, what", [
    (dict(M=0), "out of range"),
    (dict(M=300, H0=np.eye(300), V=np.eye(300)), "out of range"),
    (dict(L=0), "L = 0"),
    (dict(block=3), "block"),
    (dict(M=6, block=4, H0=np.eye(6), V=np.eye(6)), "multiple of block"),
])
def test_system_shape_checks(change, what):
    kw = base()
    kw.update(change)
    code, msg = create_code(**kw)
    assert code == INVALID and what in msg, msg


def test_system_hermiticity_and_structure_checks():
    kw = base()
    H = kw["H0"].copy()
    H[0, 1] = 0.5            # H0[1, 0] stays -1: not Hermitian
    code, msg = create_code(**dict(kw, H0=H))
    assert code == INVALID and "H0 is not Hermitian" in msg
    V = kw["V"].copy()
    V[0, 2] = 0.3            # block = 2 needs 2 x 2 diagonal blocks
    code, msg = create_code(**dict(kw, V=V, block=2))
    assert code == INVALID and "block-diagonal" in msg
    lh = kw["H0"].copy()
    lh[1, 2] = 1j
    code, msg = create_code(**dict(kw, lead_H0=(None, lh)))
    assert code == INVALID and "lead_H0[1]" in msg
    code, msg = create_code(**dict(kw, lead_Vperiod=(3, 0)))
    assert code == INVALID and "lead_Vperiod[0]" in msg
    on = np.zeros((kw["L"], kw["M"]))
    on[2, 1] = np.nan
    code, msg = create_code(**dict(kw, onsite=on))
    assert code == INVALID and "non-finite" in msg
    code, msg = create_code(**dict(kw, V=np.stack([kw["V"]] * 3)))
    assert code == INVALID and "Vperiod" in msg


@pytest.mark.skipif(not _no_gpu(), reason="a GPU is present: creation succeeds")
def test_valid_system_fails_loudly_without_gpu():
    code, msg = create_code(**base())
    assert code == CUDA, (code, msg)
    code, msg = create_code(**dict(base(), block=2, V=np.stack([-np.eye(4), -2 * np.eye(4)])))
    assert code == CUDA, (code, msg)


def test_null_handles_are_rejected():
    lib = knit.load()
    E = np.array([0.1])
    out = np.zeros(4)
    st = np.zeros(4, np.int32)
    seeds = np.zeros(1, np.uint64)
    calls = [
        lambda: lib.knit_transmission(None, knit._ptr(E), 1, knit._ptr(seeds), 1, 0.0, 0, None,
                                      knit._ptr(out), knit._ptr(st), None),
        lambda: lib.knit_ldos(None, knit._ptr(E), 1, knit._ptr(seeds), 1, 0.0, 0, 1,
                              knit._ptr(out), None, None, None, None),
        lambda: lib.knit_lead_selfenergy(None, 0, knit._ptr(E), 1, None, knit._ptr(out), None,
                                         None, None),
        lambda: lib.knit_system_num_edges(None, knit._ptr(st)),
        lambda: lib.knit_graph_slices(None, knit._ptr(st), None, None),
        lambda: lib.knit_graph_transmission(None, knit._ptr(E), 1, None, None, knit._ptr(out),
                                            None, None),
        lambda: lib.knit_batch_transmission(None, knit._ptr(E), None, None, knit._ptr(out), None,
                                            None, None),
        lambda: lib.knit_lead_model_get_params(None, knit._ptr(out)),
    ]
    for i, c in enumerate(calls):
        assert c() == INVALID, i
        assert knit.knit_last_error() != "no error"


def test_error_message_is_per_thread():
    """knit_last_error is thread-local: a failure on another thread does not
    overwrite this thread's message."""
    import threading
    create_code(**dict(base(), L=0))
    mine = knit.knit_last_error()
    t = threading.Thread(target=lambda: create_code(**dict(base(), block=3)))
    t.start()
    t.join()
    assert knit.knit_last_error() == mine and "L = 0" in mine


def test_injected_allocation_failure_is_reported_as_oom():
    """Host-side fault injection: the armed allocation fails as out of
    memory, the call reports KNIT_ERR_OOM, and the injection is one-shot."""
    knit.knit_debug_fail_alloc_after(0)
    code, msg = create_code(**base())
    assert code == 2 and "out of memory" in msg, (code, msg)
    code, _ = create_code(**base())
    assert code == (CUDA if _no_gpu() else 0)
    knit.knit_debug_fail_alloc_after(3)
    knit.knit_debug_fail_alloc_after(-1)          # disarmed before it fired
    code, _ = create_code(**base())
    assert code == (CUDA if _no_gpu() else 0)
