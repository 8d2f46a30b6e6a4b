"""Pins of the oracle's flux variants: the paper's third-order WENO (Supplement Eqs.
S10-S20) and the split by the sign of the face velocity (the paper's "upwind splitting of
the flux").  Closed forms, the printed candidate coefficients (tests/golden), limits,
convergence orders and exact reductions to the default scheme."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _coef(d):
    return np.array([d["i-1"], d["i"], d["i+1"]])


def test_weno3_candidates_are_the_printed_ones():
    g = json.load(open(os.path.join(GOLDEN, "weno3_candidates.json")))
    h1, h2, h3 = _coef(g["h1"]), _coef(g["h2"]), _coef(g["h3"])
    # the printed S13 identity: with gamma = (3/4, 1/4) the candidates give S12
    assert np.allclose(g["gamma"][0] * h1 + g["gamma"][1] * h2, h3, rtol=0, atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(10):
        a, b = rng.normal(size=2)
        # a huge jump on one side gives that side's indicator all the weight of the other
        # candidate: h_{i+1} far away -> candidate 2 alone (S11); h_{i-1} far away -> 1 (S10)
        assert oracle.weno3_left([a, b, 1e8], 1e-6) == pytest.approx(h2 @ [a, b, 1e8], rel=1e-12)
        assert oracle.weno3_left([1e8, a, b], 1e-6) == pytest.approx(h1 @ [1e8, a, b], rel=1e-12)


def test_weno3_linear_weights_give_the_third_order_upwind_formula():
    # eps >> beta: weights -> alpha = (2/3, 1/3) of Eq. S16, i.e. (-h_{i-1} + 5 h_i + 2 h_{i+1})/6
    g = json.load(open(os.path.join(GOLDEN, "weno3_candidates.json")))
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = rng.normal(size=3)
        ref = (-v[0] + 5 * v[1] + 2 * v[2]) / 6
        assert oracle.weno3_left(v, 1e20) == pytest.approx(ref, rel=1e-12, abs=1e-14)
        assert oracle.weno3_left(v, 1e20) == pytest.approx(
            g["alpha"][0] * (_coef(g["h1"]) @ v) + g["alpha"][1] * (_coef(g["h2"]) @ v), rel=1e-12, abs=1e-14)


def test_weno3_exact_for_linear_data_and_eno_next_to_a_jump():
    for (b, c0) in [(1.0, 0.0), (-0.7, 2.0)]:
        x = np.arange(-1, 2, dtype=np.float64)
        for eps in (1e-40, 1e-6, 1e3):
            assert oracle.weno3_left(b * x + c0, eps) == pytest.approx(b * 0.5 + c0, rel=1e-13, abs=1e-14)
    assert abs(oracle.weno3_left([0.0, 0.0, 1.0], 1e-6)) < 1e-10        # flat on the left
    assert abs(oracle.weno3_left([0.0, 1.0, 1.0], 1e-6) - 1.0) < 1e-10  # flat on the right


def _advect(N, w, axis, **kw):
    shape = (N, 4) if axis == 0 else (4, N)
    kw = dict(periodic_vertical=True, frozen_velocity=True, lf_alpha=2 * abs(w), u_cap=0.1, **kw)
    if axis == 1:
        kw["settling_velocity"] = -w
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
    nst = int(round(0.25 * N / abs(w)))
    s.step(nst)
    c = s.fields()[2]
    line = c[0] if axis == 0 else c[:, 0]
    return np.sqrt(np.mean((line - prof(x - w * nst)) ** 2))


@pytest.mark.parametrize("axis", [0, 1])
def test_convergence_orders_of_the_variants(axis):
    Ns = (32, 64, 128, 256)
    # WENO3: third order once the grid resolves the profile (JS weights cost order at
    # the coarsest grid's critical points)
    e3 = np.array([_advect(N, 0.02, axis, weno3=True) for N in Ns])
    assert np.all(np.log2(e3[1:-1] / e3[2:]) > 2.7), e3
    # sign split with WENO5: fifth order
    e5 = np.array([_advect(N, 0.02, axis, sign_split=True) for N in Ns])
    assert np.all(np.log2(e5[:-1] / e5[1:]) > 4.7), e5


@pytest.mark.parametrize("w", [0.03, -0.03])
@pytest.mark.parametrize("weno3", [False, True])
def test_sign_split_equals_lax_friedrichs_at_alpha_w_for_uniform_velocity(w, weno3):
    # uniform w: with alpha = |w| one Lax-Friedrichs half is w c and the other vanishes,
    # which is exactly the sign-split flux from the upwind side.  c is uniform along the
    # periodic vertical, so every vertical face of a column sees the same values and the
    # vertical divergence is exactly zero in both schemes.
    N = 48
    rng = np.random.default_rng(2)
    c0 = np.tile(rng.uniform(0, 1, N), (4, 1))
    u = np.zeros((2, 4, N))
    u[0] = w
    out = []
    for sign in (False, True):
        s = oracle.OracleSim((N, 4), periodic_vertical=True, frozen_velocity=True, lf_alpha=abs(w), u_cap=0.1,
                             diffusivity=1e-3, weno3=weno3, sign_split=sign)
        s.init(c0, u)
        s.step(30)
        out.append(s.fields()[2])
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("variant", [dict(weno3=True), dict(sign_split=True), dict(weno3=True, sign_split=True)])
def test_variants_conserve_mass_and_create_no_new_extrema(variant):
    s = oracle.OracleSim((32, 64), tau=0.6, gravity=1e-4, density_contrast=1.0, settling_velocity=2e-3,
                         diffusivity=1e-3, **variant)
    y = np.arange(64)[:, None] + 0.5
    c0 = 0.5 * (1 + np.tanh((y - 40) / 2)) * np.ones((1, 32))
    s.init(c0)
    m0 = s.total_mass
    s.step(60)
    assert abs(s.total_mass + s.deposit - m0) < 1e-13 * m0
    N = 64
    t = oracle.OracleSim((N, 4), periodic_vertical=True, frozen_velocity=True, u_cap=0.1, **variant)
    c1 = np.zeros((4, N))
    c1[:, 16:40] = 1.0
    u = np.zeros((2, 4, N))
    u[0] = 0.05
    t.init(c1, u)
    t.step(200)
    c = t.fields()[2]
    assert c.min() > -1e-3 and c.max() < 1.0 + 1e-3
