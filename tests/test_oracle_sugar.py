"""Pins of the oracle's sugar scalar S (the paper's density-altering quantity): first-order
upwind transport (Supplement Eqs. S5, S6) with central diffusion, the force term
(Eq. forceterm with rho/rho0 - 1 = S* S) and the S-dependent settling velocity
(Eq. stokes_vel).  Closed forms and reductions to already-pinned cases only."""
import numpy as np
import pytest

import oracle


def _sim(shape, u0=None, **kw):
    o = oracle.OracleSim(shape, sugar=True, **kw)
    return o


def test_upwind_at_cfl_one_shifts_exactly_both_signs():
    nx, ny = 16, 12
    rng = np.random.default_rng(0)
    S0 = rng.uniform(0, 1, (ny, nx))
    for ux, shift in ((1.0, 1), (-1.0, -1)):
        o = _sim((nx, ny), frozen_velocity=True, u_cap=2.0)
        u0 = np.zeros((2, ny, nx))
        u0[0] = ux
        o.init(np.zeros((ny, nx)), u0)
        o.set_sugar(S0)
        o.step(5)
        assert np.array_equal(o.sugar(), np.roll(S0, 5 * shift, axis=1))  # S5 / S6 at dt/dx u = 1


def test_upwind_vertical_toward_the_floor_with_neumann_lid():
    nx, ny, k = 8, 12, 4
    S0 = np.random.default_rng(1).uniform(0, 1, (ny, nx))
    o = _sim((nx, ny), frozen_velocity=True, u_cap=2.0)
    u0 = np.zeros((2, ny, nx))
    u0[1] = -1.0
    o.init(np.zeros((ny, nx)), u0)
    o.set_sugar(S0)
    o.step(k)
    # S6 with u = -1: S_y <- S_{y+1}; the lid's ghost mirrors S_{ny-1}
    expect = S0[np.minimum(np.arange(ny) + k, ny - 1)]
    assert np.array_equal(o.sugar(), expect)


def test_diffusion_modes_decay_by_the_exact_discrete_factor():
    nx, ny, D, m = 32, 16, 0.1, 3
    x = np.arange(nx)
    y = np.arange(ny)
    # periodic x: sin(2 pi m x / nx); Neumann y (mirror ghosts): cos(pi m (y + 1/2) / ny)
    Sx = np.tile(np.sin(2 * np.pi * m * x / nx), (ny, 1))
    Sy = np.tile(np.cos(np.pi * m * (y + 0.5) / ny)[:, None], (1, nx))
    for S0, lam in ((Sx, 1 - 4 * D * np.sin(np.pi * m / nx) ** 2), (Sy, 1 - 4 * D * np.sin(np.pi * m / (2 * ny)) ** 2)):
        o = _sim((nx, ny), frozen_velocity=True, sugar_diffusivity=D)
        o.init(np.zeros((ny, nx)))
        o.set_sugar(S0)
        o.step(7)
        np.testing.assert_allclose(o.sugar(), S0 * lam ** 7, rtol=0, atol=1e-13)


def test_sugar_mass_conserved_by_diffusion_and_bounded_by_upwind():
    nx, ny = 24, 20
    rng = np.random.default_rng(2)
    S0 = rng.uniform(0, 1, (ny, nx))
    o = _sim((nx, ny), frozen_velocity=True, sugar_diffusivity=0.2)
    o.init(np.zeros((ny, nx)))
    o.set_sugar(S0)
    o.step(50)
    assert o.sugar().sum() == pytest.approx(S0.sum(), rel=1e-13)
    # random velocity with |ux| + |uy| + 4 D <= 1: every update is a convex combination
    u0 = rng.uniform(-0.3, 0.3, (2, ny, nx))
    o = _sim((nx, ny), frozen_velocity=True, sugar_diffusivity=0.1, u_cap=1.0)
    o.init(np.zeros((ny, nx)), u0)
    o.set_sugar(S0)
    o.step(40)
    S = o.sugar()
    assert S.min() >= S0.min() - 1e-15 and S.max() <= S0.max() + 1e-15


def test_sugar_off_terms_reduce_to_the_plain_step_bitwise():
    shape = (32, 48)
    c0 = np.random.default_rng(3).uniform(0, 1, (48, 32))
    kw = dict(tau=0.6, gravity=1e-3, settling_velocity=0.01, diffusivity=0.01)
    a = oracle.OracleSim(shape, **kw)
    a.init(c0)
    a.step(20)
    # S = 0 everywhere: the sugar force term and Vs(S) vanish, S stays 0
    b = oracle.OracleSim(shape, sugar=True, sugar_contrast=0.3, phi0=0.01, vs_sugar=0.5,
                         sugar_diffusivity=0.05, **kw)
    b.init(c0)
    b.step(20)
    for fa, fb in zip(a.fields(), b.fields()):
        assert np.array_equal(fa, fb)
    assert a.deposit == b.deposit
    assert np.all(b.sugar() == 0.0)


def test_settling_velocity_follows_sugar_uniform_column():
    nx, ny, s0, kS, vs = 16, 20, 0.6, 0.25, 0.02
    o = _sim((nx, ny), frozen_velocity=True, settling_velocity=vs, vs_sugar=kS)
    o.init(np.ones((ny, nx)))
    o.set_sugar(np.full((ny, nx), s0))
    o.step(1)
    # uniform c = 1: the floor loses exactly Vs (1 - kS S) per column per step
    assert o.deposit == pytest.approx(nx * vs * (1 - kS * s0), rel=1e-14)


def test_sugar_force_enters_the_momentum_budget():
    # periodic box: the populations' total momentum grows by exactly the summed force,
    # F_v = -g [R c + S* S (1 - phi0 c)] (Guo forcing, as in the plain case)
    shape = (16, 16)
    rng = np.random.default_rng(4)
    c0 = rng.uniform(0, 1, (16, 16))
    S0 = rng.uniform(0, 1, (16, 16))
    g, R, Ss, phi0 = 1e-4, 0.7, 0.4, 0.05
    o = oracle.OracleSim(shape, sugar=True, periodic_vertical=True, gravity=g, density_contrast=R,
                         sugar_contrast=Ss, phi0=phi0)
    o.init(c0)
    o.set_sugar(S0)
    m0 = o.population_moments()
    o.step(1)
    m1 = o.population_moments()
    expect = -g * np.sum(R * c0 + Ss * S0 * (1 - phi0 * c0))
    assert m1[2] - m0[2] == pytest.approx(expect, rel=1e-11)
    assert abs(m1[1] - m0[1]) < 1e-15


def test_heavy_sugar_layer_below_holds_the_interface():
    # particles above, sugar below: with S* = 2 against a particle contrast of 1 the
    # layering is statically stable and the x-dependent part of the vertical velocity
    # stays bounded (internal waves); without sugar it is Rayleigh-Taylor unstable and
    # grows.  (The x-uniform part is the hydrostatic adjustment of the lattice.)
    nx, ny = 64, 96
    rng = np.random.default_rng(5)
    y = np.arange(ny)[:, None] + 0.5
    c0 = 0.5 * (1 + np.tanh((y - ny / 2) / 2)) + 1e-3 * rng.uniform(-1, 1, (ny, nx))
    S0 = 0.5 * (1 - np.tanh((y - ny / 2) / 2)) * np.ones((1, nx))
    growth = {}
    for Ss in (0.0, 2.0):
        o = oracle.OracleSim((nx, ny), sugar=True, tau=0.6, gravity=1e-3, density_contrast=1.0,
                             sugar_contrast=Ss, settling_velocity=0.0, diffusivity=1e-3, u_cap=0.5)
        o.init(c0)
        o.set_sugar(S0)
        amps = []
        for _ in range(2):
            o.step(150 if not amps else 450)
            uy = o.fields()[1][1]
            amps.append(np.abs(uy - uy.mean(axis=1, keepdims=True)).max())
        growth[Ss] = amps[1] / amps[0]
    assert growth[0.0] > 8.0
    assert growth[2.0] < 3.0
