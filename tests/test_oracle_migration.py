"""Pins of the oracle's drop-migration observable (Sec. IV.C) and loss.

The observable l = sum(c u_y)/sum(c) is the velocity of the phase-1
centroid Y = sum(c y)/sum(c).  Pins independent of its definition:
  - kinematics: over a window of steps, the mean of l equals the centroid
    displacement per step, up to the diffusive and forcing parts of the c
    flux that the advective c u misses (a few per cent here);
  - mirror symmetry: the x-reflected problem has the same l (u_y is
    even under x -> -x, u_x odd), which fails if l used u_x or mixed axes;
  - the loss over a window of one state is l of the last state.
"""
import numpy as np
import pytest

from paper_1412_6238_gb300 import workloads as W


@pytest.fixture(scope="module")
def tiny():
    return W.migration_tiny(steps=400)


def test_centroid_velocity_is_centroid_displacement(orc, tiny):
    w = tiny
    pop = orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop)
    pop = orc.run(w.params, pop, w.Tbot, w.Ttop, 300)
    Y0 = orc.migration_centroid(w.params, pop, w.Tbot, w.Ttop)
    vs = []
    for _ in range(100):
        pop = orc.run(w.params, pop, w.Tbot, w.Ttop, 1)
        vs.append(orc.centroid_velocity(w.params, pop, w.Tbot, w.Ttop))
    Y1 = orc.migration_centroid(w.params, pop, w.Tbot, w.Ttop)
    dY = (Y1 - Y0) / 100.0
    assert dY > 0  # the drop migrates toward the hot (top) wall
    assert abs(np.mean(vs) - dY) <= 0.05 * abs(dY)


def test_observable_mirror_symmetric(orc, tiny):
    w = tiny
    L1 = orc.migration_loss(w.params, w.c0, w.T0, w.Tbot, w.Ttop, 120, 20)
    L2 = orc.migration_loss(w.params, w.c0[:, ::-1].copy(), w.T0[:, ::-1].copy(),
                            w.Tbot[::-1].copy(), w.Ttop[::-1].copy(), 120, 20)
    assert abs(L1 - L2) <= 1e-12 * abs(L1)
    assert abs(L1) > 1e-4


def test_loss_window_of_one_is_last_state(orc, tiny):
    w = tiny
    L = orc.migration_loss(w.params, w.c0, w.T0, w.Tbot, w.Ttop, 30, 1)
    pop = orc.run(w.params, orc.init(w.params, w.c0, w.T0, w.Tbot, w.Ttop), w.Tbot, w.Ttop, 30)
    assert L == orc.centroid_velocity(w.params, pop, w.Tbot, w.Ttop)
    with pytest.raises(ValueError):
        orc.migration_loss(w.params, w.c0, w.T0, w.Tbot, w.Ttop, 10, 11)
