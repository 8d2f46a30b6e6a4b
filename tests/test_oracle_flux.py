"""Pins of the oracle's particle mass below a horizontal plane (Sec. 4.2.3, Eq. flux:
J = Delta m / (A Delta t), m the mass in the volume below the plane; the deposit counts as
below every plane).  Closed forms: the plane index convention at both ends, and the
individual settling rate Vs A of a uniform suspension at rest (the paper's constant
settling flux of individually settling particles) through every interior plane."""
import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads


def test_plane_at_the_floor_is_the_deposit_and_at_the_lid_the_whole_mass():
    shape = (24, 20)
    o = oracle.OracleSim(shape, tau=0.6, gravity=1e-3, density_contrast=1.0, settling_velocity=0.02,
                         diffusivity=0.01)
    o.init(workloads.interface_field(shape, interface_frac=0.5, amplitude=0.02, seed=3))
    o.step(15)
    assert o.deposit > 0.0
    assert o.mass_below(0) == o.deposit
    assert o.mass_below(shape[1]) == pytest.approx(o.total_mass + o.deposit, rel=1e-15)
    # one level: the bottom row's mass plus the deposit
    c = o.fields()[2]
    assert o.mass_below(1) == pytest.approx(c[0].sum() + o.deposit, rel=1e-14)
    assert np.isnan(o.mass_below(-1)) and np.isnan(o.mass_below(shape[1] + 1))


@pytest.mark.parametrize("shape", [(16, 64), (8, 6, 48)])
def test_uniform_suspension_settles_through_every_plane_at_vs(shape):
    """c = 1 everywhere, no buoyancy and no diffusion: the fluid stays at rest, and until
    the clear layer that opens under the lid reaches it, every plane passes Vs per unit
    area and step (the floor too: the deposit grows by Vs A per step)."""
    vs = 0.02
    area = int(np.prod(shape[:-1]))
    o = oracle.OracleSim(shape, tau=0.6, gravity=0.0, density_contrast=1.0, settling_velocity=vs,
                         diffusivity=0.0)
    o.init(np.ones(shape[::-1]))
    planes = (1, shape[-1] // 4, shape[-1] // 2)
    prev = [o.mass_below(v) for v in planes]
    for _ in range(40):
        o.step(1)
        cur = [o.mass_below(v) for v in planes]
        for a, b in zip(prev, cur):
            assert (b - a) / area == pytest.approx(vs, rel=1e-12)
        prev = cur
