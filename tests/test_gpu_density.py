"""Parity of the FP64 CUDA path with the oracle when the density varies with
the order parameter (rho(c) = rho1 + c (rho2 - rho1)): the grad(rho c_s^2)
source of Eq. 12, the corrected pressure of Eq. 13 (a pass of its own before
each step, since p needs u of every cell and the step takes grad p), grad(rho
c_s^2) in the thermal force, rho(c) in u, T, the relaxation times, the
equilibria, the body force and the walls' anti-bounce-back.

The FP64 path rounds operation by operation like the oracle: states agree to
1e-13 of each lattice's magnitude (bitwise in practice), fields to 1e-12.
"""
import numpy as np
import pytest

from paper_1412_6238_gb300 import workloads as wl

from helpers import field_errors, gpu_fields, oracle_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def LBE():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_6238_gb300.lbe import LBE
    return LBE


def state_err(a, b):
    out = []
    for k in range(3):
        s = np.abs(b[9 * k:9 * k + 9]).max()
        out.append(np.abs(a[9 * k:9 * k + 9] - b[9 * k:9 * k + 9]).max() / max(s, 1e-300))
    return max(out)


def drop(nx=70, ny=45, R=9.0, rho2=4.0, yc=None):
    w = wl.droplet(nx, ny, R, nx / 2.0 + 3.3, (ny / 2.0 - 1.7) if yc is None else yc, Re=1.0,
                   Ma=10.0, Ca=0.05, eta_m=0.2, eta_r=0.5, lam_r=2.0)
    w.params["rho2"] = rho2
    return w


@pytest.mark.parametrize("rho2", [4.0, 0.25])
def test_initial_state(LBE, orc, rho2):
    """hbar_i = w_i rho(c0) c_v T0 at rest, bitwise."""
    w = drop(rho2=rho2)
    got = LBE(w, storage="f64").get_state().numpy()
    ref = orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("nx,ny", [(5, 7), (33, 9), (100, 37), (130, 19)])
@pytest.mark.parametrize("rho2", [4.0, 0.25])
def test_one_step_from_same_state(LBE, orc, nx, ny, rho2):
    """Tiny and ragged grids, the drop reaching both walls: one GPU step from
    the oracle's state equals one oracle step."""
    R = max(1.5, min(nx, ny) / 2.5)
    w = drop(nx, ny, R, rho2, yc=ny / 2.0 - 0.2)
    w.params["ax"] = 1e-6
    pop0 = orc.run(w.params, orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop), w.Tbot, w.Ttop, 3)
    sim = LBE(w, storage="f64")
    sim.set_state(pop0)
    sim.step(1)
    ref = orc.run(w.params, pop0, w.Tbot, w.Ttop, 1)
    assert state_err(sim.get_state().numpy(), ref) < 1e-13


@pytest.mark.parametrize("rho2", [4.0, 0.25])
def test_drop_run(LBE, orc, rho2):
    """300 steps of a migrating drop four times denser (lighter) than its
    surroundings on a 70 x 45 grid: state and fields, p included."""
    w = drop(rho2=rho2)
    n = 300
    sim = LBE(w, storage="f64")
    sim.step(n)
    pop = orc.run(w.params, orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop), w.Tbot, w.Ttop, n)
    assert state_err(sim.get_state().numpy(), pop) < 1e-13
    e = field_errors(gpu_fields(sim), oracle_fields(orc, w, pop))
    print("density ratio", rho2, n, "steps:", e)
    assert max(e.values()) < 1e-12, e


def test_layered_poiseuille_density_ratio_3(LBE, orc):
    """4 x 101 two-layer channel, the upper (denser, rho2 = 3) phase against
    the top wall (the anti-bounce-back takes rho(c) there), 4000 steps."""
    w = wl.layered_poiseuille()
    w.params["rho2"] = 3.0
    sim = LBE(w, storage="f64")
    sim.step(4000)
    pop = orc.run(w.params, orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop), w.Tbot, w.Ttop, 4000)
    assert state_err(sim.get_state().numpy(), pop) < 1e-13
    e = field_errors(gpu_fields(sim), oracle_fields(orc, w, pop))
    assert max(e["u"], e["T"], e["c"]) < 1e-12, e


def test_batch_mixes_uniform_and_varying_density(LBE, orc):
    """A batch of a varying-density and a uniform-density instance: each
    equals its own oracle run (the correction pass leaves the uniform one
    alone)."""
    a = drop(60, 40, 8.0, 4.0)
    b = drop(50, 36, 7.0, 1.0)  # rho2 = rho
    n = 60
    sim = LBE([a, b], storage="f64")
    sim.step(n)
    for j, w in enumerate((a, b)):
        pop = orc.run(w.params, orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop), w.Tbot, w.Ttop, n)
        assert state_err(sim.get_state(j).numpy(), pop) < 1e-13, j


def test_adjoint_rejects_varying_density(LBE):
    import torch
    w = drop()
    sim = LBE(w, storage="f64")
    Q = sim.get_state(device="cuda")
    with pytest.raises(Exception, match="uniform-density"):
        sim.observable(Q)
    with pytest.raises(Exception, match="uniform-density"):
        sim.adjoint_step(Q, None, 1.0)
    # the handle stays usable
    sim.step(2)
    assert torch.isfinite(sim.fields(names=("ux",))["ux"]).all()
