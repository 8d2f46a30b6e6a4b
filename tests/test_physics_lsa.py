"""Coupled early-time growth against linear stability analysis (Sec. 3, Sec. 4.1), without
and with the sugar scalar.

The paper validates its solver by comparing the early growth of the interface with the
dispersion relation of its LSA.  Here the LSA is the K/W eigenproblem with the density-
altering scalar removed (S* = 0), the base state an erf fit of the mean profile at the
onset (Eqs. phi_bs), and the simulated rate the exponential fit of the front-height
Fourier amplitude (front = lowest point with c = 1/2) in the linear regime, while the
amplitude stays below 40 % of the wavelength.
"""
import numpy as np
import pytest

import oracle
from oracle import lsa


def test_lsa_inviscid_thin_interface_limit():
    # Rayleigh-Taylor between two Boussinesq layers: sigma^2 = k A / 2 for a sharp interface
    # in an unbounded fluid; a thin erf profile at small k approaches it.
    A, H = 1e-3, 400.0
    k = 2 * np.pi / 200.0
    s = lsa.growth_rate(k, H, 0.0, A, 0.0, 0.0, lambda y: lsa.erf_profile(y, H / 2, 0.3), m=800)
    assert abs(s - np.sqrt(k * A / 2)) < 0.05 * np.sqrt(k * A / 2)


def test_lsa_stable_and_damped_cases():
    k, H = 2 * np.pi / 64, 128.0
    heavy_below = lsa.growth_rate(k, H, 1 / 30, 1e-3, 1e-3, 0.0,
                                  lambda y: 1.0 - lsa.erf_profile(y, 64.0, 2.0), m=200)
    assert heavy_below <= 1e-12            # light fluid on top: no growth
    inv = lsa.growth_rate(k, H, 0.0, 1e-3, 0.0, 0.0, lambda y: lsa.erf_profile(y, 64.0, 2.0), m=200)
    visc = lsa.growth_rate(k, H, 1 / 30, 1e-3, 0.0, 0.0, lambda y: lsa.erf_profile(y, 64.0, 2.0), m=200)
    wide = lsa.growth_rate(k, H, 0.0, 1e-3, 0.0, 0.0, lambda y: lsa.erf_profile(y, 64.0, 6.0), m=200)
    assert 0 < visc < inv and 0 < wide < inv  # viscosity and a wider interface slow the growth


def seeded_interface(nx, ny, mode, eps=0.05, width=2.0):
    """Heavy layer (c = 1) over c = 0 with the interface displaced by eps cos(k x)."""
    k = 2 * np.pi * mode / nx
    Y, X = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx), indexing="ij")
    return 0.5 * (1.0 + np.tanh((Y - 0.5 * ny - eps * np.cos(k * X)) / width))


def mode_growth(fields_at, steps_between, n_samples, nx, mode):
    """Fit of log |H~(k)| over the samples whose amplitude lies in [0.15, 0.4 lambda)."""
    k = 2 * np.pi * mode / nx
    x = np.arange(nx)
    ts, amps = [], []
    for i in range(n_samples):
        t, c = fields_at(i * steps_between)
        H = lsa.front_height(c)
        ts.append(t)
        amps.append(abs(np.sum(H * np.exp(-1j * k * x))) * 2 / nx)
    ts, amps = np.array(ts), np.array(amps)
    sel = (amps > 0.15) & (amps < 0.4 * nx / mode)
    assert sel.sum() >= 5
    return np.polyfit(ts[sel], np.log(amps[sel]), 1)[0]


PHYS_LSA = dict(tau=0.6, gravity=1e-3, density_contrast=1.0, settling_velocity=1e-3, diffusivity=1e-3)


@pytest.mark.slow
def test_oracle_growth_rate_matches_lsa_within_10_percent():
    nx, ny, mode = 64, 128, 1
    c0 = seeded_interface(nx, ny, mode)
    s = oracle.OracleSim((nx, ny), u_cap=0.5, **PHYS_LSA)
    s.init(c0)

    def at(t):
        s.step(t - s.steps)
        return s.steps, s.fields()[2]
    sigma_sim = mode_growth(at, 50, 26, nx, mode)
    # base state: erf fit of the mean profile at the onset of growth (step 300)
    s2 = oracle.OracleSim((nx, ny), u_cap=0.5, **PHYS_LSA)
    s2.init(c0)
    s2.step(300)
    y = np.arange(ny) + 0.5
    yc, delta = lsa.fit_erf(y, s2.fields()[2].mean(axis=1))
    nu = (PHYS_LSA["tau"] - 0.5) / 3.0
    sigma_lsa = lsa.growth_rate(2 * np.pi * mode / nx, ny, nu, PHYS_LSA["gravity"], PHYS_LSA["diffusivity"],
                                PHYS_LSA["settling_velocity"], lambda yy: lsa.erf_profile(yy, yc, delta), m=256)
    assert abs(sigma_sim - sigma_lsa) < 0.10 * sigma_lsa, (sigma_sim, sigma_lsa)


# ---- with the sugar scalar (the paper's full K/W problem) --------------------------------

def test_lsa_sugar_reductions():
    k, H, nu = 2 * np.pi / 64, 128.0, 1 / 30
    cb = lambda y: lsa.erf_profile(y, 64.0, 3.0)
    zero = lambda y: np.zeros_like(y)
    # S* = 0: the one-scalar problem
    a = lsa.growth_rate(k, H, nu, 1e-3, 1e-3, 1e-3, cb, m=128)
    b = lsa.growth_rate_sugar(k, H, nu, 1e-3, 1e-3, 1e-3, cb, m=128)
    assert b == pytest.approx(a, rel=1e-10)
    # sugar alone, heavy on top: the one-scalar problem with A -> g S*, kappa -> D_s, Vs -> 0
    Sb = lambda y: lsa.erf_profile(y, 64.0, 3.0)
    s1 = lsa.growth_rate_sugar(k, H, nu, 0.0, 1e-3, 0.0, zero, gS=2e-3, Ds=5e-4, Sbar_fn=Sb, m=128)
    s2 = lsa.growth_rate(k, H, nu, 2e-3, 5e-4, 0.0, Sb, m=128)
    assert s1 == pytest.approx(s2, rel=1e-10) and s1 > 0
    # sugar alone, heavy below: statically stable, nothing grows
    stable = lsa.growth_rate_sugar(k, H, nu, 0.0, 1e-3, 0.0, zero, gS=2e-3, Ds=5e-4,
                                   Sbar_fn=lambda y: 1 - Sb(y), m=128)
    assert stable <= 1e-12


def test_lsa_sugar_layer_below_slows_then_stops_the_growth():
    k, H, nu = 2 * np.pi / 64, 128.0, 1 / 30
    cb = lambda y: lsa.erf_profile(y, 64.0, 3.0)
    Sb = lambda y: 1 - lsa.erf_profile(y, 64.0, 3.0)
    rates = [lsa.growth_rate_sugar(k, H, nu, 1e-3, 1e-3, 1e-3, cb, gS=g, Ds=5e-4, Sbar_fn=Sb, phi0=0.01, m=128)
             for g in (0.0, 0.5e-3, 1e-3, 2e-3)]
    assert rates[0] > rates[1] > rates[2] > 0 >= rates[3]


SUGAR_LSA = dict(PHYS_LSA, sugar=True, sugar_contrast=0.5, sugar_diffusivity=1e-3, phi0=0.0, vs_sugar=0.0)


def sugar_layer(nx, ny):
    """Sugar (S = 1) below the interface of seeded_interface, S = 0 above."""
    y = np.arange(ny)[:, None] + 0.5
    return 0.5 * (1.0 - np.tanh((y - 0.5 * ny) / 2.0)) * np.ones((1, nx))


def sugar_lsa_rate(c_mean, S_mean, ny, nx, mode, kw):
    y = np.arange(ny) + 0.5
    yc, delta = lsa.fit_erf(y, c_mean)
    ys, ds = lsa.fit_erf(y, 1.0 - S_mean)
    nu = (kw["tau"] - 0.5) / 3.0
    return lsa.growth_rate_sugar(2 * np.pi * mode / nx, ny, nu, kw["gravity"] * kw["density_contrast"],
                                 kw["diffusivity"], kw["settling_velocity"], lambda yy: lsa.erf_profile(yy, yc, delta),
                                 gS=kw["gravity"] * kw["sugar_contrast"], Ds=kw["sugar_diffusivity"],
                                 Sbar_fn=lambda yy: 1.0 - lsa.erf_profile(yy, ys, ds), phi0=kw["phi0"], m=256)


@pytest.mark.slow
def test_oracle_growth_rate_with_sugar_matches_lsa_within_10_percent():
    # particles over a lighter-than-them sugar layer (S* g = A/2): still unstable, slower
    nx, ny, mode = 64, 128, 1
    c0 = seeded_interface(nx, ny, mode)
    S0 = sugar_layer(nx, ny)
    s = oracle.OracleSim((nx, ny), u_cap=0.5, **SUGAR_LSA)
    s.init(c0)
    s.set_sugar(S0)

    def at(t):
        s.step(t - s.steps)
        return s.steps, s.fields()[2]
    sigma_sim = mode_growth(at, 50, 40, nx, mode)
    s2 = oracle.OracleSim((nx, ny), u_cap=0.5, **SUGAR_LSA)
    s2.init(c0)
    s2.set_sugar(S0)
    s2.step(300)
    sigma_lsa = sugar_lsa_rate(s2.fields()[2].mean(axis=1), s2.sugar().mean(axis=1), ny, nx, mode, SUGAR_LSA)
    no_sugar = lsa.growth_rate(2 * np.pi * mode / nx, ny, (PHYS_LSA["tau"] - 0.5) / 3.0, PHYS_LSA["gravity"],
                               PHYS_LSA["diffusivity"], PHYS_LSA["settling_velocity"],
                               lambda yy: lsa.erf_profile(yy, 57.0, 3.0), m=256)
    assert sigma_lsa < 0.85 * no_sugar  # the sugar term matters at this contrast
    assert abs(sigma_sim - sigma_lsa) < 0.10 * sigma_lsa, (sigma_sim, sigma_lsa)
