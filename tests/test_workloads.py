"""The input generator: its exp and cos from IEEE basic operations (bitwise
the same on every platform) against the C library, and the fields they
build against their definitions."""
import math

import numpy as np

from paper_1412_6238_gb300 import workloads as wl


def _ulps(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.spacing(np.maximum(np.abs(a), np.abs(b)))


def test_det_exp_within_two_ulps_of_libm():
    x = np.concatenate([np.linspace(-700.0, 700.0, 40001), np.linspace(-1.0, 1.0, 4001),
                        [-1e-300, 0.0, 1e-300, 0.5 * math.log(2.0), -0.5 * math.log(2.0)]])
    ref = np.array([math.exp(v) for v in x])
    assert _ulps(wl.det_exp(x), ref).max() <= 2.0
    # the ends: underflow through the subnormals, overflow to inf
    e = wl.det_exp(np.array([-745.2, -1e6, 710.0, 1e6]))
    assert e[0] == 0.0 and e[1] == 0.0 and np.isinf(e[2]) and np.isinf(e[3])
    assert wl.det_exp(np.array([-744.0]))[0] == math.exp(-744.0)  # a subnormal


def test_det_cos2pi_within_1e15_of_the_exact_value():
    mpmath = __import__("pytest").importorskip("mpmath")
    mpmath.mp.prec = 120
    q = np.concatenate([np.arange(1024) / 1024.0, np.linspace(-3.0, 3.0, 601)])
    ref = np.array([float(mpmath.cos(2 * mpmath.pi * mpmath.mpf(float(v)))) for v in q])
    assert np.abs(wl.det_cos2pi(q) - ref).max() < 1e-15
    # exact at the quarter turns
    assert wl.det_cos2pi(np.array([0.0]))[0] == 1.0
    assert wl.det_cos2pi(np.array([0.5]))[0] == -1.0


def test_tanh_profile_is_the_planar_equilibrium_profile():
    d = np.linspace(-60.0, 60.0, 24001)
    ref = np.array([0.5 * (1.0 + math.tanh(2.0 * v / 4.0)) for v in d])
    c = wl.tanh_profile(d, 4.0)
    assert np.abs(c - ref).max() < 3e-16
    assert 0.0 <= c[0] < 1e-25
    assert c[-1] == 1.0


def test_planar_wall_temperature_and_drop_profile():
    w = wl.planar_marangoni()
    x = np.arange(w.nx)
    ref = 20.0 + 4.0 * np.array([math.cos(2.0 * math.pi * v / w.nx) for v in x])
    assert np.abs(w.Tbot - ref).max() < 1e-14
    d = wl.droplet_512x1024()
    # c = 1/2 exactly on the circle of radius R through a grid node: (256, 288)
    assert d.c0[288, 256] == 0.5
    assert d.c0[256, 256] > 1.0 - 1e-12 and d.c0[1000, 10] < 1e-12
