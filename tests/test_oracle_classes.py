"""Pins of the oracle's polydisperse particle classes (Eqs. forceterm_poly, poly): each
class is transported with its own settling velocity and tallies its own deposit; the
force reads phi_tot = sum_k c_k.  Closed forms and exact reductions."""
import numpy as np
import pytest

import oracle


def test_empty_classes_reduce_to_the_single_class_step_bitwise():
    shape = (32, 48)
    c0 = np.random.default_rng(0).uniform(0, 1, (48, 32))
    kw = dict(tau=0.6, gravity=1e-3, diffusivity=0.01, lf_alpha=0.12, u_cap=0.1)
    a = oracle.OracleSim(shape, settling_velocity=0.02, **kw)
    a.init(c0)
    a.step(20)
    b = oracle.OracleSim(shape, class_vs=(0.02, 0.05, 0.001), **kw)
    b.init(c0)  # classes 1 and 2 start empty
    b.step(20)
    for fa, fb in zip(a.fields(), b.fields()):
        assert np.array_equal(fa, fb)
    assert a.deposit == b.deposit == b.class_deposit(0)
    assert np.all(b.class_field(1) == 0.0) and b.class_deposit(2) == 0.0


def test_uniform_columns_deposit_at_each_class_rate():
    # quiescent uniform columns: class k loses exactly Vs_k c_k nx per step through the floor
    nx, ny = 8, 64
    vs = (0.002, 0.005, 0.011)
    amp = (1.0, 0.5, 0.25)
    s = oracle.OracleSim((nx, ny), frozen_velocity=True, class_vs=vs, u_cap=0.1)
    s.init(np.full((ny, nx), amp[0]), np.zeros((2, ny, nx)))
    for k in (1, 2):
        s.set_class(k, np.full((ny, nx), amp[k]))
    s.step(3)
    for k in range(3):
        assert s.class_deposit(k) == pytest.approx(3 * vs[k] * amp[k] * nx, rel=1e-12)
    assert s.deposit == pytest.approx(sum(3 * v * a * nx for v, a in zip(vs, amp)), rel=1e-12)


def test_each_class_conserves_its_mass_plus_deposit():
    shape = (32, 64)
    rng = np.random.default_rng(1)
    s = oracle.OracleSim(shape, tau=0.6, gravity=1e-4, diffusivity=1e-3, class_vs=(0.001, 0.004))
    y = np.arange(64)[:, None] + 0.5
    c0 = 0.5 * (1 + np.tanh((y - 40) / 2)) * np.ones((1, 32)) + 1e-3 * rng.uniform(-1, 1, (64, 32))
    s.init(c0)
    s.set_class(1, 0.5 * c0)
    m = [c0.sum(), 0.5 * c0.sum()]
    s.step(60)
    for k in range(2):
        assert s.class_field(k).sum() + s.class_deposit(k) == pytest.approx(m[k], rel=1e-13)
    assert s.fields()[2].sum() == pytest.approx(s.class_field(0).sum() + s.class_field(1).sum(), rel=1e-14)


def test_force_reads_the_sum_of_the_classes():
    # periodic box: total momentum grows by the summed force -A sum_k c_k per step
    shape = (16, 16)
    rng = np.random.default_rng(2)
    c0, c1 = rng.uniform(0, 1, (2, 16, 16))
    g, R = 1e-4, 0.8
    s = oracle.OracleSim(shape, periodic_vertical=True, gravity=g, density_contrast=R, class_vs=(0.0, 0.0))
    s.init(c0)
    s.set_class(1, c1)
    m0 = s.population_moments()
    s.step(1)
    m1 = s.population_moments()
    assert m1[2] - m0[2] == pytest.approx(-g * R * np.sum(c0 + c1), rel=1e-11)


def test_faster_class_leaves_first():
    # two classes, same initial slab, no flow: the faster-settling class reaches the floor
    # first and has deposited more after the same time
    nx, ny = 8, 96
    y = np.arange(ny)[:, None] + 0.5
    slab = ((y > 40) & (y < 60)).astype(float) * np.ones((1, nx))
    s = oracle.OracleSim((nx, ny), frozen_velocity=True, class_vs=(0.01, 0.05), u_cap=0.1, diffusivity=1e-3)
    s.init(slab, np.zeros((2, ny, nx)))
    s.set_class(1, slab)
    s.step(1000)
    assert s.class_deposit(1) > 10 * s.class_deposit(0)
