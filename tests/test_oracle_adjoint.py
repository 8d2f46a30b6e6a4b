"""Pins of the oracle's reverse sweep (gradient of the deposited mass, Sec. 4 m_b, with
respect to the initial concentration and the settling velocity), on the CPU.

The reverse sweep transposes complex-step Jacobians of complex twins of the oracle's own
forward routines; these tests tie it to the forward oracle itself, independently of how
the Jacobians are formed: central differences of the forward deposit (h = 1e-6 per
component, 1e-7 in Vs) over every component of c0 on a small walled lattice with strong
buoyancy, so that the fluid part of the sweep carries weight.
"""
import numpy as np
import pytest

import oracle

ADJ = dict(tau=0.6, gravity=2e-3, density_contrast=1.0, settling_velocity=0.05, diffusivity=0.02,
           lf_alpha=0.25, u_cap=0.2)


def _J(shape, c0, nsteps, **kw):
    o = oracle.OracleSim(shape, **dict(ADJ, **kw))
    o.init(c0)
    o.step(nsteps)
    return o.deposit


def _fd(shape, c0, nsteps, h=1e-6, **kw):
    fd = np.zeros_like(c0)
    for k in range(c0.size):
        e = np.zeros(c0.size)
        e[k] = h
        e = e.reshape(c0.shape)
        fd.flat[k] = (_J(shape, c0 + e, nsteps, **kw) - _J(shape, c0 - e, nsteps, **kw)) / (2 * h)
    return fd


def test_reverse_sweep_every_component_vs_central_differences():
    shape, nsteps = (12, 16), 15
    c0 = 0.5 + 0.4 * np.random.default_rng(3).uniform(-1.0, 1.0, size=(16, 12))
    J, g, _ = oracle.deposit_gradient(shape, c0, nsteps, **ADJ)
    assert J == _J(shape, c0, nsteps)
    fd = _fd(shape, c0, nsteps)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(fd).max()
    assert np.linalg.norm(g - fd) <= 1e-7 * np.linalg.norm(fd)
    # the buoyancy-driven flow changes the gradient well beyond the tolerance
    g0 = oracle.deposit_gradient(shape, c0, nsteps, **dict(ADJ, gravity=0.0))[1]
    assert np.abs(g - g0).max() > 1e-3 * np.abs(fd).max()


def test_reverse_sweep_settling_velocity():
    shape, nsteps = (12, 16), 15
    c0 = 0.5 + 0.4 * np.random.default_rng(4).uniform(-1.0, 1.0, size=(16, 12))
    _, _, dvs = oracle.deposit_gradient(shape, c0, nsteps, **ADJ)
    vs, h = ADJ["settling_velocity"], 1e-7
    fd = (_J(shape, c0, nsteps, settling_velocity=vs + h) - _J(shape, c0, nsteps, settling_velocity=vs - h)) / (2 * h)
    assert dvs == pytest.approx(fd, rel=1e-8)


def test_reverse_sweep_linear_case_euler_and_support():
    # no flow, no diffusion: the transport is linear in c (the WENO weights are
    # scale-invariant only approximately, but with a uniform c0 every smoothness indicator
    # vanishes and the scheme reduces to its linear weights), so J is homogeneous of
    # degree one in c0 and Euler's relation gives sum_k c0_k dJ/dc0_k = J.  After one step
    # the deposit reads c, c1 and c2 on the floor row; c2 there depends on c1 up to row 3
    # and c1 on c up to row 6, so dJ/dc0 vanishes from row 7 on.
    shape = (8, 12)
    c0 = np.full((12, 8), 0.7)
    kw = dict(ADJ, gravity=0.0, diffusivity=0.0)
    J, g, _ = oracle.deposit_gradient(shape, c0, 1, **kw)
    assert J == _J(shape, c0, 1, gravity=0.0, diffusivity=0.0)
    assert 0.7 * np.sum(g) == pytest.approx(J, rel=1e-12)
    assert np.all(g[7:] == 0.0) and np.all(g[6] != 0.0)


def test_reverse_sweep_rejects_unsupported():
    c0 = np.full((16, 12), 0.5)
    for kw in (dict(lf_alpha=0.0), dict(periodic_vertical=True), dict(frozen_velocity=True)):
        with pytest.raises(ValueError):
            oracle.deposit_gradient((12, 16), c0, 2, **dict(ADJ, **kw))
    with pytest.raises(ValueError):
        oracle.deposit_gradient((8, 8, 8), np.zeros((8, 8, 8)), 2, **ADJ)
