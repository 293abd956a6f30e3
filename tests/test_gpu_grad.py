"""The gain gradient (epic_grad, torch.autograd) against the FP64 oracle: the
FX closed-form gradient, central finite differences of the oracle loss, and the
autograd binding."""
import numpy as np
import pytest

import oracle
from paper_1904_11422_gb300 import build_lib, epic, synth

from _helpers import oracle_array

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build_lib.build()
    return epic.load_library()


def _gpu_grad(w, gains, model):
    import torch
    plan = epic.plan_for(w)  # the plan's own gains are not used by epic_grad
    dv = torch.from_numpy(np.ascontiguousarray(w.volts)).cuda()
    g = torch.from_numpy(np.ascontiguousarray(np.stack([gains.real, gains.imag], -1).astype(np.float32))).cuda()
    m = torch.from_numpy(np.ascontiguousarray(model.astype(np.float32))).cuda()
    grad = torch.empty_like(g)
    loss = torch.empty((), dtype=torch.float32, device="cuda")
    epic.epic_grad(plan, dv, w.n_time, g, m, grad, loss)
    epic.epic_sync(plan)
    plan.close()
    gr = grad.cpu().numpy().astype(np.float64)
    return float(loss.item()), gr[..., 0] + 1j * gr[..., 1]


CASES = [
    dict(seed=1301, n_ant=12, n_pol=2, n_chan=2, grid_n=64, support=3, n_time=6),
    dict(seed=1302, n_ant=9, n_pol=1, n_chan=3, grid_n=64, support=5, n_time=5),
    # more antennas than half the block: one thread per antenna in the degrid
    dict(seed=1306, n_ant=300, n_pol=2, n_chan=1, grid_n=64, support=3, n_time=3),
    # 32 x 32 grids (128-thread blocks, up to 128 antennas)
    dict(seed=1307, n_ant=20, n_pol=2, n_chan=2, grid_n=32, support=3, n_time=5),
    dict(seed=1308, n_ant=120, n_pol=1, n_chan=1, grid_n=32, support=5, n_time=3),
    # 128 x 128 grids folded into four 64 x 64 problems: the fold's adjoint
    dict(seed=1309, n_ant=24, n_pol=2, n_chan=2, grid_n=128, support=5, n_time=4),
    dict(seed=1310, n_ant=60, n_pol=1, n_chan=1, grid_n=128, support=3, n_time=3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c['seed']}")
def test_gradient_matches_fx_oracle(case):
    w = synth.random_small(**case)
    rng = np.random.default_rng(case["seed"])
    model = rng.standard_normal((w.n_chan, 2, w.grid_n, w.grid_n)) * 20.0
    loss, grad = _gpu_grad(w, w.gains, model)
    arr = oracle_array(w)
    loss_ref, grad_ref = oracle.grad_fx(arr, w.volts, model)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    err = np.abs(grad - grad_ref).max() / np.abs(grad_ref).max()
    assert err <= 1e-3, err


@pytest.mark.parametrize("grid_n", [64, 32, 128])
def test_gradient_matches_finite_differences(grid_n):
    w = synth.random_small(1303, n_ant=10, n_pol=2, n_chan=2, grid_n=grid_n, support=5, n_time=4)
    plan = epic.plan_for(w)
    assert plan.info["transforms_per_image"] == (4 if grid_n == 128 else 1)
    plan.close()
    rng = np.random.default_rng(7)
    model = rng.standard_normal((w.n_chan, 2, w.grid_n, w.grid_n)) * 20.0
    _, grad = _gpu_grad(w, w.gains, model)
    h = 1e-4
    scale = np.abs(grad).max()
    for _ in range(32):
        c, a, p = (int(rng.integers(n)) for n in (w.n_chan, w.n_ant, w.n_pol))
        fd = 0j
        for unit in (1.0, 1j):
            gp, gm = w.gains.copy(), w.gains.copy()
            gp[c, a, p] += h * unit
            gm[c, a, p] -= h * unit
            lp = oracle.loss_epic(oracle_array(w, gains=gp), w.volts, model)
            lm = oracle.loss_epic(oracle_array(w, gains=gm), w.volts, model)
            fd += unit * (lp - lm) / (2 * h)
        assert abs(grad[c, a, p] - fd) <= 1e-3 * scale, (c, a, p, grad[c, a, p], fd)


def test_station_gradient_sampled_finite_differences():
    """Differentiation config (station block, seeded gains, 5-source model) on
    three channels: GPU gradient vs central differences of the oracle loss."""
    import torch
    w, sky = synth.differentiation(n_chan=64)
    chans = [0, 40]
    sub = synth.Workload("sub", w.ant_xy, w.freq_hz[chans], 2, w.grid_n, w.support, w.cell_lambda,
                         w.sigma_cells, np.ascontiguousarray(w.volts[:, chans]), gains=w.gains[chans])
    sky_arr = oracle.OracleArray(sky.ant_xy, sky.freq_hz[chans], 2, sky.grid_n, sky.support, 0.5, sky.sigma_cells)
    model = oracle.image(sky_arr, np.ascontiguousarray(sky.volts[:, chans]), use_fft=True)[:, :2]
    loss, grad = _gpu_grad(sub, sub.gains, model)
    arr = oracle.OracleArray(sub.ant_xy, sub.freq_hz, 2, sub.grid_n, sub.support, 0.5, sub.sigma_cells,
                             gains=sub.gains)
    img = oracle.image(arr, sub.volts, use_fft=True)
    loss_ref = float(np.sum((img[:, :2] - model) ** 2))
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    rng = np.random.default_rng(11)
    scale = np.abs(grad).max()
    h = 1e-3
    for _ in range(3):
        c, a, p = int(rng.integers(2)), int(rng.integers(sub.n_ant)), int(rng.integers(2))
        fd = 0j
        for unit in (1.0, 1j):
            vals = []
            for sgn in (1, -1):
                g = sub.gains.copy()
                g[c, a, p] += sgn * h * unit
                a1 = oracle.OracleArray(sub.ant_xy, sub.freq_hz[c:c + 1], 2, sub.grid_n, sub.support, 0.5,
                                        sub.sigma_cells, gains=g[c:c + 1])
                im1 = oracle.image(a1, np.ascontiguousarray(sub.volts[:, c:c + 1]), use_fft=True)[0, :2]
                vals.append(float(np.sum((im1 - model[c]) ** 2)))
            fd += unit * (vals[0] - vals[1]) / (2 * h)
        assert abs(grad[c, a, p] - fd) <= 1e-3 * scale, (c, a, p, grad[c, a, p], fd)


def test_autograd_function():
    import torch
    from paper_1904_11422_gb300 import autograd
    w = synth.random_small(1304, n_ant=12, n_pol=2, n_chan=2, grid_n=64, support=3, n_time=5)
    rng = np.random.default_rng(3)
    model = torch.from_numpy((rng.standard_normal((w.n_chan, 2, w.grid_n, w.grid_n)) * 20.0).astype(np.float32)).cuda()
    plan = epic.plan_for(w)
    dv = torch.from_numpy(w.volts).cuda()
    g = torch.tensor(w.gains.astype(np.complex64), device="cuda", requires_grad=True)
    loss = autograd.calib_loss(plan, dv, g, model)
    loss.backward()
    _, grad_ref = _gpu_grad(w, w.gains, model.cpu().numpy().astype(np.float64))
    got = g.grad.detach().cpu().numpy()
    assert np.abs(got - grad_ref).max() <= 1e-6 * np.abs(grad_ref).max()
    # a few gradient steps lower the loss
    opt = torch.optim.SGD([g], lr=0.3 / float(np.abs(grad_ref).max()))
    losses = []
    for _ in range(4):
        opt.zero_grad()
        l = autograd.calib_loss(plan, dv, g, model)
        l.backward()
        opt.step()
        losses.append(float(l.detach()))
    assert losses[-1] < losses[0]
    plan.close()


@pytest.mark.parametrize("kind", ["tensor", "cluster128", "ants32"])
def test_grad_unsupported_plans(kind):
    """Tensor-core plans, 128 x 128 grids on two-CTA clusters and 32 x 32 grids
    with more antennas than the adjoint's threads are refused."""
    import torch
    if kind == "tensor":
        w = synth.random_small(1305, n_ant=6, n_pol=2, n_chan=1, grid_n=64, support=3, n_time=2)
        plan = epic.plan_for(w, epic.XFORMS["dft_bf16x3"])
    elif kind == "cluster128":
        w = synth.random_small(1311, n_ant=450, n_pol=2, n_chan=1, grid_n=128, support=5, n_time=2)
        plan = epic.plan_for(w)
        assert plan.info["cluster_dim"] == 2
    else:
        w = synth.random_small(1312, n_ant=129, n_pol=2, n_chan=1, grid_n=32, support=3, n_time=2)
        plan = epic.plan_for(w)
    z = torch.zeros((1, w.n_ant, 2, 2), dtype=torch.float32, device="cuda")
    m = torch.zeros((1, 2, w.grid_n, w.grid_n), dtype=torch.float32, device="cuda")
    with pytest.raises(epic.EpicError) as ei:
        epic.epic_grad(plan, torch.from_numpy(w.volts).cuda(), 2, z, m, torch.empty_like(z),
                       torch.empty((), device="cuda"))
    assert ei.value.status == epic.EPIC_ERR_UNSUPPORTED
    plan.close()
