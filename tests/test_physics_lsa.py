"""Coupled early-time growth against linear stability analysis (Sec. 3, Sec. 4.1).

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
