"""Pins of the host-side mapping of the paper's physical parameters to lattice units:
Table 1's volume fractions (printed values), the Stokes velocity against the drag and
net-gravity balance it solves (Eq. stokes_vel), the relaxation time of Eq. tau at the
workloads' tau = 0.6 (nu = 1/30), and the constants of the two-layer workload."""
import json
import os

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2106_07694_gb300 import units, workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_volume_fraction.json")


def test_table1_volume_fractions():
    t = json.load(open(GOLDEN))
    for conc, phi in zip(t["concentration_g_per_l"], t["volume_fraction"]):
        assert float(f"{units.volume_fraction(conc, t['rho_p']):.3g}") == phi


@pytest.mark.parametrize("diameter", [25e-6, 40e-6, 115e-6, 160e-6])
def test_stokes_velocity_balances_drag_and_net_gravity(diameter):
    rho_p, rho_f, mu, g = 2519.4, 1000.0, 1.0e-3, 9.81
    vol = np.pi / 6.0 * diameter ** 3

    def net_force(v):  # Stokes drag 3 pi mu D v against (rho_p - rho_f) V g
        return (rho_p - rho_f) * vol * g - 3.0 * np.pi * mu * diameter * v

    v = brentq(net_force, 0.0, 1.0, xtol=1e-18, rtol=1e-15)
    assert units.stokes_velocity(diameter, rho_p, rho_f, mu, g) == pytest.approx(v, rel=1e-12)


def test_relaxation_time():
    assert units.tau_from_viscosity(1.0 / 30.0) == pytest.approx(0.6, rel=1e-15)
    for tau in (0.51, 0.6, 0.5 + np.sqrt(3.0 / 16.0), 1.0):
        assert units.tau_from_viscosity(units.viscosity_from_tau(tau)) == pytest.approx(tau, rel=1e-14)
    with pytest.raises(ZeroDivisionError):
        units.LatticeScale.from_tau(1e-4, 0.0, 0.6)


def test_lattice_scale_round_trip():
    nu = 1.0e-6
    s = units.LatticeScale.from_tau(dx=2.0e-4, nu=nu, tau=0.6)
    assert units.tau_from_viscosity(s.viscosity(nu)) == pytest.approx(0.6, rel=1e-13)
    # halving dx at fixed tau divides dt by four (diffusive scaling)
    s2 = units.LatticeScale.from_tau(dx=1.0e-4, nu=nu, tau=0.6)
    assert s2.dt == pytest.approx(s.dt / 4.0, rel=1e-13)
    assert s2.velocity(1.0) == pytest.approx(s.velocity(1.0) / 2.0, rel=1e-13)
    assert s2.acceleration(9.81) == pytest.approx(s.acceleration(9.81) / 8.0, rel=1e-13)


def test_two_layer_workload_constants():
    """The sugar workload's lattice constants follow from the experiment's values: glass beads
    (2519.4 kg/m^3) at 3 g/l above the 1008.4 kg/m^3 sugar solution."""
    s = units.LatticeScale.from_tau(dx=1.0e-4, nu=1.0e-6, tau=0.6)
    p = units.lattice_params(s, 40e-6, 3.0, 2519.4, 1008.4, 1.0e-3, sugar=True)
    sw = workloads.SUGAR_2D.sugar
    assert p["phi0"] == pytest.approx(sw["phi0"], rel=1e-3)
    assert p["sugar_contrast"] == pytest.approx(sw["sugar_contrast"], rel=1e-12)
    assert p["vs_sugar"] == pytest.approx(sw["vs_sugar"], rel=1e-3)
    assert p["density_contrast"] == pytest.approx(workloads.SUGAR_2D.density_contrast, rel=1e-3)
    assert p["tau"] == pytest.approx(0.6, rel=1e-13)
    assert 0.0 < p["settling_velocity"] < 0.1  # a stable lattice velocity at this scale
