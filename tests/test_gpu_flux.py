"""Particle mass below a horizontal plane (Sec. 4.2.3, Eq. flux) through the C ABI: parity
with the FP64 oracle at several planes (FP64 to 1e-12, FP32 to 2e-6), 2D and 3D, with
particle classes; the individual settling rate Vs A through every plane of a uniform
suspension at rest on the FP32 production kernels; and error codes."""
import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

STRONG = dict(tau=0.6, gravity=1e-3, density_contrast=1.0, settling_velocity=0.02, diffusivity=0.01)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def _pair(shape, fp64, steps, classes=None, **kw):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.02, seed=21)
    if not fp64:
        c0 = c0.astype(np.float32).astype(np.float64)
    g = Simulation(shape, fp64=fp64, **kw)
    o = oracle.OracleSim(shape, **kw)
    g.init(c0)
    o.init(c0)
    for k, ck in enumerate(classes or []):
        g.set_class(k, ck)
        o.set_class(k, ck)
    g.step(steps)
    o.step(steps)
    return g, o


@pytest.mark.parametrize("shape,fp64,tol", [((132, 64), True, 1e-12), ((132, 64), False, 2e-6),
                                            ((36, 20, 40), False, 2e-6), ((16, 12, 24), True, 1e-12)])
def test_mass_below_matches_oracle(shape, fp64, tol):
    g, o = _pair(shape, fp64, 25, **STRONG)
    nv = shape[-1]
    for level in (0, 1, nv // 3, nv - 1, nv):
        assert g.mass_below(level) == pytest.approx(o.mass_below(level), rel=tol, abs=1e-15)
    assert g.mass_below(nv) == pytest.approx(g.total_mass + g.deposit, rel=1e-14)


def test_mass_below_with_classes():
    shape = (64, 48)
    base = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.02, seed=22)
    cls = [base, 0.5 * base, 0.25 * base]
    kw = dict(STRONG)
    kw.pop("settling_velocity")
    g, o = _pair(shape, True, 20, classes=cls, class_vs=(0.005, 0.02, 0.04), **kw)
    for level in (0, 5, 24, 48):
        assert g.mass_below(level) == pytest.approx(o.mass_below(level), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("shape", [(256, 96), (64, 32, 40)])
def test_uniform_suspension_settles_through_planes_at_vs_fp32(shape):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    vs = 0.02
    area = int(np.prod(shape[:-1]))
    g = Simulation(shape, fp64=False, tau=0.6, gravity=0.0, density_contrast=1.0, settling_velocity=vs,
                   diffusivity=0.0)
    g.init(np.ones(shape[::-1]))
    planes = (1, shape[-1] // 4, shape[-1] // 2)
    prev = [g.mass_below(v) for v in planes]
    for _ in range(10):
        g.step(3)
        cur = [g.mass_below(v) for v in planes]
        for a, b in zip(prev, cur):
            assert (b - a) / (3 * area) == pytest.approx(vs, rel=1e-5)
        prev = cur


def test_mass_below_errors():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    g = lw.Simulation((32, 16), **STRONG)
    with pytest.raises(lw.LbmWenocError) as e:
        g.mass_below(0)
    assert e.value.code == lw.LW_ESTATE
    g.init(np.zeros((16, 32)))
    for bad in (-1, 17):
        with pytest.raises(lw.LbmWenocError) as e:
            g.mass_below(bad)
        assert e.value.code == lw.LW_EINVAL
    assert g.mass_below(16) == 0.0
