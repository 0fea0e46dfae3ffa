"""The learned lead warm start: the GPU network against its FP64 reference,
training, and what it gains over decimation alone."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1010_2627_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knit():
    from paper_1010_2627_gb300 import build, knit as k
    build.build()
    k.load()
    return k


@pytest.fixture(scope="module")
def square_lead_model(knit):
    """A square lead of width 4 (so the closed form is available as the arbiter)."""
    ss = inputs.square(4, 3)
    sysk = knit.System(ss)
    E_train = np.random.default_rng(0).uniform(-3.6, 3.6, 3000)
    model = knit.LeadModel(sysk, 0, E_train, epochs=400, batch=256, lr=1e-3, seed=1)
    model.E_train = E_train
    return ss, sysk, model


def test_gpu_gradient_matches_fp64_reference(knit, square_lead_model):
    ss, sysk, model = square_lead_model
    dims = [1, 128, 128, 128, 2 * 4 * 4]
    p = model.get_params()
    E = np.linspace(-3.0, 3.0, 64)
    lo, hi = model.E_train.min(), model.E_train.max()
    u = ((E - 0.5 * (lo + hi)) / (0.5 * (hi - lo))).reshape(-1, 1)
    rng = np.random.default_rng(4)
    target = rng.standard_normal((64, dims[-1])).astype(np.float32)
    y_gpu = model.forward(E)
    y_ref = mlp.forward(p.astype(np.float64), dims, u)[-1]
    assert np.abs(y_gpu - y_ref).max() < 1e-4 * max(1.0, np.abs(y_ref).max())
    g_gpu, loss_gpu = model.gradient(E, target)
    loss_ref, g_ref = mlp.loss_and_grad(p.astype(np.float64), dims, u, target)
    assert abs(loss_gpu - loss_ref) < 1e-5 * max(1.0, loss_ref)
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel < 1e-3, rel


def test_training_reduces_loss(square_lead_model):
    ss, sysk, model = square_lead_model
    assert model.loss[-1] < 0.05 * model.loss[0]
    assert np.isfinite(model.loss).all()


def test_learned_lead_reaches_fixed_point_and_gains_over_decimation(knit, square_lead_model):
    ss, sysk, model = square_lead_model
    E = inputs.energy_grid(-3.5, 3.5, 61)
    S_l, it_l, res_l = sysk.lead_selfenergy(0, E, method=knit.KNIT_LEAD_LEARNED, want_residual=True,
                                            models=(model, None))
    S_d, it_d, res_d = sysk.lead_selfenergy(0, E, method=knit.KNIT_LEAD_DECIMATION, eta=1e-13,
                                            want_residual=True)
    for e, Ee in enumerate(E):
        Sc = oracle.sigma_square(4, 1.0, Ee)
        assert np.abs(S_l[e] - Sc).max() < 1e-9, Ee
    newton = it_l <= 8     # energies settled by Newton (others fell back to decimation)
    assert newton.mean() >= 0.8
    # gain: a few Newton steps instead of ~45 doubling steps, and a fixed point
    # that is exact at eta = 0 rather than at the decimation's broadening
    assert np.median(it_l[newton]) <= 6 and np.median(it_d) >= 30
    assert np.median(res_l[newton]) < 1e-13
    assert np.median(res_l[newton]) < np.median(res_d)


def test_untrained_model_falls_back_to_decimation(knit):
    ss = inputs.square(3, 3)
    sysk = knit.System(ss)
    model = knit.LeadModel(sysk, 1, np.linspace(-3, 3, 64), epochs=1, batch=64, seed=3)
    E = np.array([-2.2, -0.3, 1.7])
    S, it, _ = sysk.lead_selfenergy(1, E, method=knit.KNIT_LEAD_LEARNED, models=(None, model))
    for e, Ee in enumerate(E):
        assert np.abs(S[e] - oracle.sigma_square(3, 1.0, Ee)).max() < 1e-8


def test_learned_lead_bdg_cell(knit):
    """Spin x Nambu lead cell with Rashba coupling (8 orbitals): the learned
    start + Newton agrees with the oracle's decimation."""
    b = inputs.bdg(2, 3, mu=-1.0, delta=0.1, alpha=0.2)
    sysk = knit.System(b)
    E_train = np.random.default_rng(5).uniform(-0.25, 0.25, 2000)
    model = knit.LeadModel(sysk, 0, E_train, epochs=300, batch=256, seed=2)
    E = inputs.energy_grid(-0.2, 0.2, 16)
    S, it, res = sysk.lead_selfenergy(0, E, method=knit.KNIT_LEAD_LEARNED, want_residual=True,
                                      models=(model, None))
    for e, Ee in enumerate(E):
        _, So, _ = oracle.decimation(b.lead_H0[0], b.lead_V[0], Ee, 0, eta=1e-12)
        assert np.abs(S[e] - So).max() < 1e-7


@pytest.fixture(scope="module")
def ribbon_lead_model(knit):
    """The armchair ribbon's period-2 lead (M = 64: 32 blocks of 4 x 4 in the
    eigenbasis of its cell), the network trained on 20 000 decimation samples
    over (-2, 2)"""
    ss = inputs.armchair(64, 3)
    sysk = knit.System(ss)
    E_train = np.random.default_rng(3).uniform(-2.0, 2.0, 20000)
    model = knit.LeadModel(sysk, 0, E_train, epochs=60, batch=256, lr=1e-3, seed=4)
    return ss, sysk, model


def test_learned_lead_mode_blocks_against_oracle(knit, ribbon_lead_model):
    ss, sysk, model = ribbon_lead_model
    assert sysk.info()[1] == [32, 32]
    assert model.num_outputs == 2 * 32 * 16
    assert np.isfinite(model.loss).all() and model.loss[-1] < model.loss[0]
    E = np.array([-1.7, -0.45, 0.31, 1.2])
    S, it, res = sysk.lead_selfenergy(0, E, method=knit.KNIT_LEAD_LEARNED, want_residual=True,
                                      models=(model, None))
    for e, Ee in enumerate(E):
        So = oracle.decimation_period2(ss.H0, *ss.lead_V[0], Ee, 0)
        assert np.abs(S[e] - So).max() < 1e-8 * max(1.0, np.abs(So).max()), Ee
        assert res[e] < 1e-7


def test_learned_lead_mode_blocks_time_to_fixed_point(knit):
    """Wall time for the self-energies of the 256-site ribbon's lead at 8192
    energies, with the network (Newton to max|A g - I| < 1e-12 at eta = 0 in
    every block, decimation where Newton does not settle) and without it
    (decimation at eta = 1e-12): the two agree to the decimation tolerance,
    most blocks settle by Newton, and the learned path is the faster one."""
    import time
    import torch
    ss = inputs.armchair(256, 3)
    sysk = knit.System(ss)
    t0 = time.perf_counter()
    model = knit.LeadModel(sysk, 0, np.random.default_rng(8).uniform(-2.0, 2.0, 20000), epochs=60,
                           batch=256, lr=1e-3, seed=5)
    train_s = time.perf_counter() - t0
    E = inputs.energy_grid(-2.0, 2.0, 8192)
    dE = torch.tensor(E, device="cuda")
    dS = torch.empty(8192 * 256 * 256 * 2, dtype=torch.float64, device="cuda")
    dit = torch.empty(8192, dtype=torch.int32, device="cuda")

    def run(method):
        opts = knit._opts(method, 0.0, models=(model.handle, None))
        knit.knit_lead_selfenergy(sysk.handle, 0, dE, dS, opts, dit)
        torch.cuda.synchronize()

    times = {}
    out = {}
    for method in (knit.KNIT_LEAD_DECIMATION, knit.KNIT_LEAD_LEARNED):
        run(method)   # warm-up
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            run(method)
            ts.append(time.perf_counter() - t0)
        times[method] = sorted(ts)[1]
        out[method] = (dS.view(8192, 256, 256, 2)[::97].cpu().numpy(), dit.cpu().numpy())
    Sd, itd = out[knit.KNIT_LEAD_DECIMATION]
    Sl, itl = out[knit.KNIT_LEAD_LEARNED]
    assert np.abs(Sl - Sd).max() < 1e-7 * max(1.0, np.abs(Sd).max())
    print(f"ribbon lead, 8192 energies: decimation {times[knit.KNIT_LEAD_DECIMATION]:.3f} s, "
          f"learned + Newton {times[knit.KNIT_LEAD_LEARNED]:.3f} s (training {train_s:.1f} s)")
    assert times[knit.KNIT_LEAD_LEARNED] < times[knit.KNIT_LEAD_DECIMATION]
    sysk.close()
