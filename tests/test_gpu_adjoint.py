"""Discrete adjoint of the step (CUDA, FP64) against central finite
differences of the FP64 oracle.

  - one adjoint step, exhaustively per population at a 7 x 6 grid whose
    interface touches the bottom wall (every ghost-row and wrap rule is hit),
    and along random directions at 32 x 64;
  - the checkpointed run (lbe_adjoint) at 32 x 64: loss equal to the
    oracle's, parameter gradients and dT0 directions against FD, the
    32 x 64 per-cell reference gradient from tests/golden, independence of
    the checkpoint spacing, the state left in the handle;
  - the autograd Function;
  - the 256 x 512 differentiable-migration problem (2000 steps, checkpoints
    every 100, loss over the last 200 states) against FP64 FD of the oracle.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

from paper_1412_6238_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adjoint_32x64.json")


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _sim(w, storage="f64"):
    _torch()
    from paper_1412_6238_gb300.lbe import LBE
    return LBE(w, storage=storage)


def _with_params(w, **kw):
    p = dict(w.params)
    p.update(kw)
    return dataclasses.replace(w, params=p)


def _theta_params(p, j, x):
    """Parameters with theta_j set to x (sigmaT, eta2/eta1, lam2/lam1)."""
    q = dict(p)
    if j == 0:
        q["sigmaT"] = x
    elif j == 1:
        q["eta2"] = x * q["eta1"]
    else:
        q["lam2"] = x * q["lam1"]
    return q


def _theta0(p):
    return (p["sigmaT"], p["eta2"] / p["eta1"], p["lam2"] / p["lam1"])


def _one_step_J(orc, w, a, wl, params=None):
    """J(Q) = a . S(Q) + wl * l(Q) with the oracle's step S and observable l."""
    params = params or w.params

    def J(Q):
        S = orc.run(params, Q, w.Tbot, w.Ttop, 1)
        v = float((a * S).sum())
        if wl:
            v += wl * orc.centroid_velocity(params, Q, w.Tbot, w.Ttop)
        return v
    return J


def _small_wall_case(orc):
    """7 x 6 grid, drop of radius 2.5 centred at (3, 1.5): the interface
    crosses the bottom wall and wraps in x; unequal ratios; a few steps so
    that u, p and the temperature field are not at rest."""
    rng = np.random.default_rng(11)
    w = W.droplet(7, 6, 2.5, 3.0, 1.5, Re=1.0, Ma=10.0, Ca=0.05, eta_m=0.2,
                  eta_r=0.5, lam_r=2.0, dT0=rng.normal(0.0, 1e-3, size=(6, 7)))
    w = _with_params(w, ay=-2e-5)
    Q = orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
    Q = orc.run(w.params, Q, w.Tbot, w.Ttop, 5)
    return w, Q


def _tiny_case(orc, steps=300):
    w = W.migration_tiny(steps=steps)
    Q = orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
    return w, orc.run(w.params, Q, w.Tbot, w.Ttop, steps)


# ---------------------------------------------------------------- one step
def test_observable_matches_oracle(orc):
    torch = _torch()
    w, Q = _tiny_case(orc)
    sim = _sim(w)
    l_gpu = sim.observable(torch.from_numpy(Q).cuda())
    l_orc = orc.centroid_velocity(w.params, Q, w.Tbot, w.Ttop)
    assert abs(l_gpu - l_orc) <= 1e-11 * abs(l_orc)
    sim.close()


def test_adjoint_step_exhaustive_small_grid(orc):
    """Every component of (dS/dQ)^T a + wl dl/dQ against a central difference
    of the oracle's step (7 x 6, walls and x-wrap inside the stencils)."""
    torch = _torch()
    w, Q = _small_wall_case(orc)
    rng = np.random.default_rng(3)
    a = rng.standard_normal(Q.shape)
    wl = 0.7
    sim = _sim(w)
    a_out, grad = sim.adjoint_step(torch.from_numpy(Q).cuda(), torch.from_numpy(a).cuda(), wl)
    a_out = a_out.cpu().numpy()
    J = _one_step_J(orc, w, a, wl)
    h = 1e-6
    fd = np.empty(Q.size)
    flat = Q.reshape(-1)
    for j in range(Q.size):
        qp, qm = flat.copy(), flat.copy()
        qp[j] += h
        qm[j] -= h
        fd[j] = (J(qp.reshape(Q.shape)) - J(qm.reshape(Q.shape))) / (2 * h)
    fd = fd.reshape(Q.shape)
    err = np.abs(a_out - fd)
    scale = np.abs(fd).max()
    worst = np.unravel_index(err.argmax(), err.shape)
    assert err.max() <= 2e-7 * scale + 1e-9, (err.max(), scale, worst, a_out[worst], fd[worst])
    # parameter partials of the same J
    th = _theta0(w.params)
    for j in range(3):
        hx = 1e-6 * max(abs(th[j]), 1e-3)
        Jp = _one_step_J(orc, w, a, wl, _theta_params(w.params, j, th[j] + hx))
        Jm = _one_step_J(orc, w, a, wl, _theta_params(w.params, j, th[j] - hx))
        g_fd = (Jp(Q) - Jm(Q)) / (2 * hx)
        assert abs(grad[j] - g_fd) <= 1e-6 * abs(g_fd) + 1e-9, (j, grad[j], g_fd)
    sim.close()


def test_adjoint_step_directions_32x64(orc):
    """<a_out, V> against the central difference of J along V: V over the
    f, g and hbar planes separately and over all 27 planes."""
    torch = _torch()
    w, Q = _tiny_case(orc)
    rng = np.random.default_rng(5)
    a = rng.standard_normal(Q.shape)
    wl = 50.0
    sim = _sim(w)
    a_out, grad = sim.adjoint_step(torch.from_numpy(Q).cuda(), torch.from_numpy(a).cuda(), wl)
    a_out = a_out.cpu().numpy()
    J = _one_step_J(orc, w, a, wl)
    # the regularised normal n = grad c / sqrt(|grad c|^2 + eta_n^2) is
    # strongly nonlinear where |grad c| is small (hundreds of cells below 1e-6
    # here), so the step must be well below that for the central difference
    # to be in its asymptotic range
    h = 1e-7
    for planes in (slice(0, 9), slice(9, 18), slice(18, 27), slice(0, 27)):
        V = np.zeros_like(Q)
        V[planes] = rng.standard_normal(V[planes].shape)
        fd = (J(Q + h * V) - J(Q - h * V)) / (2 * h)
        ad = float((a_out * V).sum())
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-8, (planes, ad, fd)
    sim.close()


def test_adjoint_step_terminal_state(orc):
    """a_next = None: only the observable's gradient remains."""
    torch = _torch()
    w, Q = _small_wall_case(orc)
    sim = _sim(w)
    a_out, grad = sim.adjoint_step(torch.from_numpy(Q).cuda(), None, 1.0)
    a_out = a_out.cpu().numpy()
    rng = np.random.default_rng(9)
    V = rng.standard_normal(Q.shape)
    h = 1e-6
    lp = orc.centroid_velocity(w.params, Q + h * V, w.Tbot, w.Ttop)
    lm = orc.centroid_velocity(w.params, Q - h * V, w.Tbot, w.Ttop)
    fd = (lp - lm) / (2 * h)
    ad = float((a_out * V).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-10, (ad, fd)
    sim.close()


# ---------------------------------------------------------------- full run
TINY_STEPS, TINY_WINDOW, TINY_K = 300, 50, 40


@pytest.fixture(scope="module")
def tiny_adjoint():
    w = W.migration_tiny(steps=TINY_STEPS)
    sim = _sim(w)
    r = sim.adjoint(TINY_STEPS, TINY_WINDOW, TINY_K, want_dT0=True, want_dQ0=True)
    state = sim.get_state()
    steps_done = sim.steps_done
    sim.close()
    return w, r, state.numpy(), steps_done


def _loss(orc, w, params=None, T0=None):
    return orc.migration_loss(params or w.params, w.c0, w.T0 if T0 is None else T0, w.Tbot,
                              w.Ttop, TINY_STEPS, TINY_WINDOW)


def test_adjoint_loss_and_end_state(orc, tiny_adjoint):
    w, r, state, steps_done = tiny_adjoint
    L = _loss(orc, w)
    assert abs(r["loss"] - L) <= 1e-11 * abs(L)
    assert steps_done == TINY_STEPS
    ref = orc.run(w.params, orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop), w.Tbot, w.Ttop,
                  TINY_STEPS)
    assert np.array_equal(state, ref)  # the FP64 step is bitwise the oracle's


def test_adjoint_parameter_gradients_fd(orc, tiny_adjoint):
    w, r, _, _ = tiny_adjoint
    th = _theta0(w.params)
    for j in range(3):
        hx = 1e-5 * th[j]
        Lp = _loss(orc, w, _theta_params(w.params, j, th[j] + hx))
        Lm = _loss(orc, w, _theta_params(w.params, j, th[j] - hx))
        g_fd = (Lp - Lm) / (2 * hx)
        assert abs(r["grad"][j] - g_fd) <= 1e-6 * abs(g_fd) + 1e-12, (j, r["grad"][j], g_fd)


def test_adjoint_dT0_directions_fd(orc, tiny_adjoint):
    w, r, _, _ = tiny_adjoint
    g = r["dT0"].cpu().numpy()
    rng = np.random.default_rng(21)
    h = 1e-6
    for _ in range(2):
        d = rng.standard_normal(w.T0.shape)
        fd = (_loss(orc, w, T0=w.T0 + h * d) - _loss(orc, w, T0=w.T0 - h * d)) / (2 * h)
        ad = float((g * d).sum())
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-12, (ad, fd)


def test_adjoint_dT0_is_rho_cv_weighted_dQ0(tiny_adjoint):
    w, r, _, _ = tiny_adjoint
    dQ0 = r["dQ0"].cpu().numpy()
    wts = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    expect = w.params["rho"] * w.params["cv"] * np.tensordot(wts, dQ0[18:27], axes=1)
    np.testing.assert_allclose(r["dT0"].cpu().numpy(), expect, rtol=1e-13, atol=1e-300)


def test_adjoint_checkpoint_spacing_invariant(tiny_adjoint):
    """k = 40 (ragged last segment) and k = N give the same numbers."""
    w, r, _, _ = tiny_adjoint
    sim = _sim(w)
    r2 = sim.adjoint(TINY_STEPS, TINY_WINDOW, TINY_STEPS, want_dT0=True)
    sim.close()
    assert r2["loss"] == r["loss"]
    assert r2["grad"] == r["grad"]
    assert np.array_equal(r2["dT0"].cpu().numpy(), r["dT0"].cpu().numpy())


def test_adjoint_golden_reference_gradient_32x64():
    """The per-cell FD reference gradient (oracle only, tests/golden)."""
    if not os.path.exists(GOLDEN):
        pytest.skip("golden file missing")
    G = json.load(open(GOLDEN))
    w = W.migration_tiny(steps=G["steps"])
    sim = _sim(w)
    r = sim.adjoint(G["steps"], G["window"], 100, want_dT0=True)
    sim.close()
    assert abs(r["loss"] - G["loss_value"]) <= 1e-11 * abs(G["loss_value"])
    ref = np.asarray(G["dT0"]).reshape(G["ny"], G["nx"])
    g = r["dT0"].cpu().numpy()
    err = np.abs(g - ref).max()
    assert err <= 1e-6 * np.abs(ref).max(), (err, np.abs(ref).max())
    for j, key in enumerate(("dsigmaT", "deta_ratio", "dlam_ratio")):
        assert abs(r["grad"][j] - G[key]) <= 1e-6 * abs(G[key]), (key, r["grad"][j], G[key])


@pytest.mark.parametrize("storage", ["f32", "f16mix"])
def test_adjoint_f32_forward(orc, tiny_adjoint, storage):
    """FP32 (or F16MIX) storage forward (strip kernel), FP64 reverse sweep:
    within the trajectory error of the FP64 gradient."""
    w, r, _, _ = tiny_adjoint
    sim = _sim(w, storage)
    r32 = sim.adjoint(TINY_STEPS, TINY_WINDOW, TINY_K, want_dT0=True)
    sim.close()
    assert abs(r32["loss"] - r["loss"]) <= 1e-4 * abs(r["loss"])
    for j in range(3):
        assert abs(r32["grad"][j] - r["grad"][j]) <= 1e-3 * abs(r["grad"][j]), j
    g64 = r["dT0"].cpu().numpy()
    g32 = r32["dT0"].cpu().numpy()
    assert np.sqrt(((g32 - g64) ** 2).sum() / (g64 ** 2).sum()) <= 1e-3


def test_adjoint_rejects_bad_specs():
    from paper_1412_6238_gb300.lbe import LBEError
    w = W.migration_tiny(steps=10)
    sim = _sim(w)
    for steps, window, k in ((0, 1, 1), (10, 0, 1), (10, 11, 1), (10, 5, 0)):
        with pytest.raises(LBEError) as e:
            sim.adjoint(steps, window, k)
        assert e.value.status == -1
    sim.close()
    sim = _sim([w, w])
    with pytest.raises(LBEError):
        sim.adjoint(10, 5, 5)
    sim.close()


def test_migration_autograd_function(tiny_adjoint):
    torch = _torch()
    from paper_1412_6238_gb300.adjoint import LBEMigration, MigrationProblem
    w, r, _, _ = tiny_adjoint
    base = W.migration_tiny(steps=TINY_STEPS, amp=0.0)
    dT0 = torch.from_numpy(w.T0 - base.T0).cuda().requires_grad_(True)
    th = _theta0(w.params)
    s, e, l = (torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in th)
    prob = MigrationProblem(base, TINY_STEPS, TINY_WINDOW, TINY_K, "f64")
    L = LBEMigration.apply(s, e, l, dT0, prob)
    (3.0 * L).backward()
    assert abs(L.item() - r["loss"]) <= 1e-14 * abs(r["loss"]) + 1e-300
    for t, j in ((s, 0), (e, 1), (l, 2)):
        assert abs(t.grad.item() - 3.0 * r["grad"][j]) <= 1e-12 * abs(r["grad"][j])
    np.testing.assert_allclose(dT0.grad.cpu().numpy(), 3.0 * r["dT0"].cpu().numpy(),
                               rtol=1e-12, atol=0)


# ---------------------------------------------------------------- 256 x 512
@pytest.fixture(scope="module")
def migration_fd(orc):
    """FP64 central FD of the oracle's loss for the 256 x 512 problem:
    sigmaT, the viscosity ratio and one random dT0 direction."""
    w = W.migration_256x512(steps=2000)

    def L(params=None, T0=None):
        return orc.migration_loss(params or w.params, w.c0, w.T0 if T0 is None else T0,
                                  w.Tbot, w.Ttop, 2000, 200)

    th = _theta0(w.params)
    out = dict(w=w, L0=L(), grad={})
    for j in (0, 1):
        hx = 1e-5 * th[j]
        out["grad"][j] = (L(_theta_params(w.params, j, th[j] + hx)) -
                          L(_theta_params(w.params, j, th[j] - hx))) / (2 * hx)
    d = np.random.default_rng(2).standard_normal(w.T0.shape)
    h = 1e-6
    out["d"] = d
    out["dir"] = (L(T0=w.T0 + h * d) - L(T0=w.T0 - h * d)) / (2 * h)
    return out


@pytest.mark.slow
@pytest.mark.parametrize("storage,rtol", [("f64", 1e-6), ("f32", 1e-4)])
def test_migration_256x512_against_oracle_fd(migration_fd, storage, rtol):
    """The differentiable-migration problem: 2000 steps, checkpoints every
    100, loss over the last 200 states."""
    F = migration_fd
    w = F["w"]
    sim = _sim(w, storage)
    r = sim.adjoint(2000, 200, 100, want_dT0=True)
    sim.close()
    print("storage %s loss %.10e (oracle %.10e) grad %s fd %s dir %.10e fd %.10e" % (
        storage, r["loss"], F["L0"], r["grad"], F["grad"],
        float((r["dT0"].cpu().numpy() * F["d"]).sum()), F["dir"]))
    assert abs(r["loss"] - F["L0"]) <= (1e-11 if storage == "f64" else 1e-4) * abs(F["L0"])
    for j in (0, 1):
        assert abs(r["grad"][j] - F["grad"][j]) <= rtol * abs(F["grad"][j]), j
    ad = float((r["dT0"].cpu().numpy() * F["d"]).sum())
    assert abs(ad - F["dir"]) <= rtol * abs(F["dir"])
