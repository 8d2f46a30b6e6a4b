"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
exact invariant, a textbook special case, a convergence order, or numbers the
paper prints (tests/golden).  Chosen so that a dropped term, a wrong sign or
index, or a transposed operand in any step a1..a9 fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- a5: WENO5 face value

def test_weno5_reduces_to_linear_upwind_scheme_when_eps_dominates():
    # With eps >> beta the nonlinear weights equal the linear ones (1/10, 6/10, 3/10) and
    # the face value is the textbook fifth-order upwind-biased formula (Jiang & Shu 1996):
    # (2 h_{i-2} - 13 h_{i-1} + 47 h_i + 27 h_{i+1} - 3 h_{i+2}) / 60.
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = rng.normal(size=5)
        got = oracle.weno5_left(v, 1e20)
        ref = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60.0
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))


def test_weno5_exact_for_quadratic_primitive_whatever_the_weights():
    # Finite-difference WENO reconstructs H with h = cell average of H.  Every
    # three-point candidate is exact for quadratic H, so the convex combination is exact
    # for any weights: H(x) = a x^2 + b x + c has cell averages H(x_i) + a/12.
    for (a, b, c0) in [(1.0, 0.0, 0.0), (-0.3, 2.0, 0.7), (5.0, -1.0, 3.0)]:
        for i in (0, 3, -7):
            x = np.arange(i - 2, i + 3, dtype=np.float64)
            h = a * x ** 2 + b * x + c0 + a / 12.0
            xf = i + 0.5
            exact = a * xf ** 2 + b * xf + c0
            for eps in (1e-40, 1e-6, 1e3):
                assert abs(oracle.weno5_left(h, eps) - exact) < 1e-12 * max(1.0, abs(exact))


def test_weno5_picks_the_smooth_stencil_next_to_a_jump():
    # ENO property: next to a jump the weight of the only smooth sub-stencil tends to 1.
    # Jump to the right: stencil {i-2, i-1, i} is flat, face value -> its candidate = 0.
    assert abs(oracle.weno5_left([0.0, 0.0, 0.0, 1.0, 1.0], 1e-6)) < 1e-10
    # Jump on the left: stencil {i, i+1, i+2} is flat, face value -> 1.
    assert abs(oracle.weno5_left([0.0, 0.0, 1.0, 1.0, 1.0], 1e-6) - 1.0) < 1e-10
    # Jump between i-2 and i-1: the two right stencils are flat; both give 1.
    assert abs(oracle.weno5_left([0.0, 1.0, 1.0, 1.0, 1.0], 1e-6) - 1.0) < 1e-10


# ---------------------------------------------------------------- a4-a8: transport operator

def _advect_periodic(N, w, axis, steps_frac=0.25):
    """Smooth periodic profile advected along `axis` by a frozen constant velocity."""
    shape = (N, 4) if axis == 0 else (4, N)
    kw = dict(periodic_vertical=True, frozen_velocity=True, lf_alpha=2 * abs(w), u_cap=0.1)
    if axis == 1:
        kw["settling_velocity"] = -w  # w_vertical = u - Vs
    s = oracle.OracleSim(shape, **kw)
    k = 2 * np.pi / N
    prof = lambda x: 0.5 + 0.25 * np.sin(k * x)
    x = np.arange(N, dtype=np.float64)
    u = np.zeros((2,) + s.grid)
    if axis == 0:
        u[0] = w
        c0 = np.tile(prof(x), (4, 1))
    else:
        c0 = np.tile(prof(x)[:, None], (1, 4))
    s.init(c0, u)
    nst = int(round(steps_frac * N / abs(w)))
    s.step(nst)
    _, _, c = s.fields()
    line = c[0] if axis == 0 else c[:, 0]
    return np.sqrt(np.mean((line - prof(x - w * nst)) ** 2))


@pytest.mark.parametrize("axis", [0, 1])
def test_weno5_rk3_fifth_order_on_smooth_advection(axis):
    # Frozen constant velocity, kappa = 0, periodic; alpha proportional to w and a small
    # CFL number so that the spatial error dominates; a quarter of the domain is
    # advected.  The observed order over N = 32..256 must be at least 4.7.
    w = 0.02
    errs = np.array([_advect_periodic(N, w, axis) for N in (32, 64, 128, 256)])
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all(orders > 4.7), orders


def test_settling_translates_profile_downwards_at_vs():
    # u = 0, kappa = 0, periodic vertical: c(y, t) = c0(y + Vs t); fifth-order error, and
    # the profile must move DOWN (a sign error in Vs moves it up and fails at O(1)).
    N, vs = 64, 0.01
    s = oracle.OracleSim((4, N), periodic_vertical=True, frozen_velocity=True,
                         settling_velocity=vs, lf_alpha=2 * vs, u_cap=0.1)
    y = np.arange(N, dtype=np.float64)
    k = 2 * np.pi / N
    prof = lambda y: 0.5 + 0.25 * np.sin(k * y)
    s.init(np.tile(prof(y)[:, None], (1, 4)), np.zeros((2, N, 4)))
    nst = 1600
    s.step(nst)
    c = s.fields()[2][:, 0]
    assert np.max(np.abs(c - prof(y + vs * nst))) < 2e-6
    assert np.max(np.abs(c - prof(y - vs * nst))) > 0.1


def test_transport_operator_mirror_symmetry():
    # Reflecting x and reversing the velocity must reflect L(c): checks the right-biased
    # (h-) reconstruction against the left-biased one, including the stencil indices.
    rng = np.random.default_rng(3)
    nx, ny = 16, 12
    s = oracle.OracleSim((nx, ny), settling_velocity=0.003, diffusivity=0.002, u_cap=0.1,
                         lf_alpha=0.05)
    c = rng.uniform(0, 1, size=(ny, nx))
    u = rng.uniform(-0.02, 0.02, size=(2, ny, nx))
    L = s.transport_rate(c, u)
    cm = c[:, ::-1].copy()
    um = u[:, :, ::-1].copy()
    um[0] *= -1.0
    Lm = s.transport_rate(cm, um)
    assert np.max(np.abs(Lm[:, ::-1] - L)) < 1e-15


def test_diffusion_fourier_mode_decays_by_discrete_rk3_factor():
    # w = 0 and alpha = 1e-16 (its O(alpha) dissipation is below rounding): L is kappa times the 5-point Laplacian, so a Fourier mode is
    # multiplied each step by G(lam) = 1 + lam + lam^2/2 + lam^3/6, with
    # lam = -kappa * sum_d 4 sin^2(k_d/2).  Pins a6, a7 and the RK3 coefficients.
    nx, ny, kappa = 16, 8, 0.05
    s = oracle.OracleSim((nx, ny), periodic_vertical=True, frozen_velocity=True,
                         diffusivity=kappa, lf_alpha=1e-16, u_cap=0.1)
    kx, ky = 2 * np.pi * 3 / nx, 2 * np.pi * 1 / ny
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    mode = np.cos(kx * X + ky * Y)
    s.init(1.0 + 0.1 * mode, np.zeros((2, ny, nx)))
    lam = -kappa * (4 * np.sin(kx / 2) ** 2 + 4 * np.sin(ky / 2) ** 2)
    G = 1 + lam + lam ** 2 / 2 + lam ** 3 / 6
    n = 40
    s.step(n)
    c = s.fields()[2]
    expect = 1.0 + 0.1 * G ** n * mode
    assert np.max(np.abs(c - expect)) < 1e-12


def test_rk3_stages_match_the_printed_shu_osher_coefficients():
    # Compose the stage coefficients printed in the paper (S21-S23) for the scalar test
    # equation a' = lam a and compare with the oracle's measured per-step factor on one
    # Fourier mode (diffusion only), for several lam.
    with open(os.path.join(GOLDEN, "ssp_rk3_shu_osher.json")) as fh:
        g = json.load(fh)
    for kappa in (0.01, 0.05, 0.1):
        nx = 8
        s = oracle.OracleSim((nx, 4), periodic_vertical=True, frozen_velocity=True,
                             diffusivity=kappa, lf_alpha=1e-16, u_cap=0.1)
        k = 2 * np.pi * 2 / nx
        mode = np.cos(k * np.arange(nx))
        s.init(np.tile(mode, (4, 1)), np.zeros((2, 4, nx)))
        s.step(1)
        measured = s.fields()[2][0, 0] / mode[0]
        lam = -kappa * 4 * np.sin(k / 2) ** 2
        vals = {"a": 1.0}
        for i, st in enumerate(g["stages"]):
            comb = sum(coef * vals[name] for name, coef in st["combine"].items())
            vals["a%d" % (i + 1)] = comb + st["rate_weight"] * lam * vals[st["rate_on"]]
        assert abs(measured - vals["a3"]) < 1e-14


def test_step_profile_creates_no_new_extrema():
    # Non-oscillation (TVD claim after S20): a unit step advected with WENO5 + RK3 stays
    # within [0, 1] up to 1e-3 of the jump.
    N = 64
    s = oracle.OracleSim((N, 4), periodic_vertical=True, frozen_velocity=True, u_cap=0.1)
    c0 = np.zeros((4, N))
    c0[:, 16:40] = 1.0
    u = np.zeros((2, 4, N))
    u[0] = 0.05
    s.init(c0, u)
    s.step(200)
    c = s.fields()[2]
    assert c.min() > -1e-3 and c.max() < 1.0 + 1e-3


# ---------------------------------------------------------------- a9: walls and deposit

def test_deposit_of_a_uniform_column_is_vs_nx_per_step():
    # u = 0, A = 0, kappa = 0, c = 1: interior faces carry -Vs, the floor face -Vs c_0 = -Vs,
    # so the floor row keeps c = 1 until the lid's depletion reaches it and the deposit
    # grows by exactly Vs nx per step (the constant individual-settling rate).
    nx, ny, vs, n = 8, 256, 2e-3, 10
    s = oracle.OracleSim((nx, ny), frozen_velocity=True, settling_velocity=vs, u_cap=0.1)
    s.init(np.ones((ny, nx)), np.zeros((2, ny, nx)))
    s.step(n)
    assert abs(s.deposit - vs * nx * n) < 1e-12 * vs * nx * n
    c = s.fields()[2]
    assert np.max(np.abs(c[:100] - 1.0)) < 1e-14
    assert c[-1].max() < 1.0  # the lid row empties


def test_lid_row_loses_exactly_the_settling_flux_first_step():
    # First stage at the lid: flux above is 0, flux below is -Vs (uniform), so
    # L = -Vs for the top row; after one RK3 step c_top = 1 - Vs exactly when the
    # row below is still uniform in every stage.
    nx, ny, vs = 8, 64, 1e-3
    s = oracle.OracleSim((nx, ny), frozen_velocity=True, settling_velocity=vs, u_cap=0.1)
    s.init(np.ones((ny, nx)), np.zeros((2, ny, nx)))
    L = s.transport_rate(np.ones((ny, nx)), np.zeros((2, ny, nx)))
    assert np.max(np.abs(L[-1] + vs)) < 1e-15
    assert np.max(np.abs(L[:-4])) < 1e-15


def test_mass_plus_deposit_is_invariant_in_the_coupled_step():
    # Sum c + deposit is conserved to rounding (conservative fluxes, RK3 b-weights for the
    # deposit); Sum f is conserved by collision and halfway bounce-back.
    s = oracle.OracleSim((32, 64), tau=0.6, gravity=1e-4, density_contrast=1.0,
                         settling_velocity=2e-3, diffusivity=1e-3)
    c0 = workloads.interface_field((32, 64), seed=5)
    s.init(c0)
    m0 = s.total_mass
    f0 = s.population_moments()[0]
    s.step(50)
    assert abs(s.total_mass + s.deposit - m0) < 1e-13 * m0
    assert s.deposit > 0
    assert abs(s.population_moments()[0] - f0) < 1e-13 * f0


# ---------------------------------------------------------------- a1-a3: fluid

def test_poiseuille_exact_at_the_magic_relaxation_time():
    # BGK with halfway bounce-back reproduces the parabolic profile exactly when
    # (tau - 1/2)^2 = 3/16; walls at v = -1/2 and N - 1/2, u = F/(2 nu) (v+1/2)(N-1/2-v).
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu, N, F = (tau - 0.5) / 3.0, 16, 1e-6
    s = oracle.OracleSim((4, N), tau=tau, body_force=(F, 0.0, 0.0))
    s.init(np.zeros((N, 4)))
    s.step(20000)
    u = s.fields()[1]
    v = np.arange(N)
    exact = F / (2 * nu) * (v + 0.5) * (N - 0.5 - v)
    assert np.max(np.abs(u[0][:, 0] - exact)) < 1e-10 * exact.max()
    assert np.max(np.abs(u[1])) < 1e-14


def test_poiseuille_second_order_at_tau_0_6():
    tau, F = 0.6, 1e-6
    nu = (tau - 0.5) / 3.0
    errs = []
    for N in (8, 16, 32):
        s = oracle.OracleSim((4, N), tau=tau, body_force=(F, 0.0, 0.0))
        s.init(np.zeros((N, 4)))
        s.step(int(8 * N * N / nu))
        v = np.arange(N)
        exact = F / (2 * nu) * (v + 0.5) * (N - 0.5 - v)
        errs.append(np.max(np.abs(s.fields()[1][0][:, 0] - exact)) / exact.max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.9), orders


def test_taylor_green_decay_rate_second_order():
    # Periodic box: the vortex decays as exp(-2 nu k^2 t); the relative error of the
    # measured rate falls by ~4x per doubling of N and is below 0.05% at N = 64.
    tau = 0.6
    nu = (tau - 0.5) / 3.0
    rel = []
    for N in (16, 32, 64):
        k = 2 * np.pi / N
        X, Y = np.meshgrid(np.arange(N), np.arange(N))
        ux = -1e-3 * np.cos(k * X) * np.sin(k * Y)
        uy = 1e-3 * np.sin(k * X) * np.cos(k * Y)
        s = oracle.OracleSim((N, N), tau=tau, periodic_vertical=True)
        s.init(np.zeros((N, N)), np.stack([ux, uy]))
        ts, amps = [], []
        for i in range(5):
            s.step(N * N // 8)
            ts.append(s.steps)
            amps.append(np.sum(s.fields()[1][0] * ux) / np.sum(ux * ux))
        rate = -np.polyfit(ts, np.log(amps), 1)[0]
        rel.append(rate / (2 * nu * k * k) - 1.0)
    rel = np.abs(np.array(rel))
    assert rel[-1] < 5e-4
    assert np.all(rel[:-1] / rel[1:] > 3.0), rel


def test_momentum_grows_by_the_total_force_each_step():
    # Guo forcing adds exactly F per node per step to sum_i f_i c_i (periodic box), so
    # the raw momentum after n steps is n * sum_x F(c) with F = body - A c e_v, and
    # sum c is conserved in a periodic box.
    nx, ny, A, bx = 16, 16, 3e-4, 2e-6
    s = oracle.OracleSim((nx, ny), tau=0.7, gravity=A, density_contrast=1.0,
                         body_force=(bx, 0.0, 0.0), settling_velocity=1e-3,
                         diffusivity=1e-3, periodic_vertical=True)
    c0 = workloads.interface_field((nx, ny), interface_frac=0.5, seed=2)
    s.init(c0)
    sum_c = c0.sum()
    n = 20
    s.step(n)
    m = s.population_moments()
    assert abs(m[1] - n * bx * nx * ny) < 1e-12 * n * bx * nx * ny
    assert abs(m[2] - (-n * A * sum_c)) < 1e-12 * n * A * sum_c


def test_d3q19_lattice_isotropy():
    # Standard D3Q19 set (the paper shows it in a figure only): sum w = 1,
    # sum w c c = cs^2 I, fourth moment isotropic, 19 velocities, all |c|^2 <= 2.
    s = oracle.OracleSim((4, 4, 4))
    ci, wi = s.lattice()
    assert ci.shape == (19, 3)
    assert abs(wi.sum() - 1.0) < 1e-15
    M2 = np.einsum("i,ia,ib->ab", wi, ci, ci)
    assert np.allclose(M2, np.eye(3) / 3.0, atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", wi, ci, ci, ci, ci)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) +
           np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(M4, iso, atol=1e-15)


def test_d3q19_poiseuille_matches_2d():
    # The 3D lattice on a channel uniform in x, y reproduces the magic-tau profile too.
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu, N, F = (tau - 0.5) / 3.0, 12, 1e-6
    s = oracle.OracleSim((4, 4, N), tau=tau, body_force=(F, 0.0, 0.0))
    s.init(np.zeros((N, 4, 4)))
    s.step(12000)
    u = s.fields()[1]
    v = np.arange(N)
    exact = F / (2 * nu) * (v + 0.5) * (N - 0.5 - v)
    assert np.max(np.abs(u[0][:, 0, 0] - exact)) < 1e-9 * exact.max()


def test_oracle_rejects_invalid_parameters():
    with pytest.raises(ValueError):
        oracle.OracleSim((16, 16), tau=0.5)
    with pytest.raises(ValueError):
        oracle.OracleSim((2, 16))


def test_status_flags_velocity_above_cap():
    s = oracle.OracleSim((8, 8), frozen_velocity=True, u_cap=0.01, periodic_vertical=True)
    u = np.zeros((2, 8, 8))
    u[0] = 0.02
    s.init(np.ones((8, 8)), u)
    assert s.step(1) != 0
