"""Parity of the flux variants (the paper's third-order WENO, Supplement Eqs. S10-S20, and
the split by the sign of the face velocity) with the FP64 oracle, through the C ABI:
FP64 to 1e-12, FP32 to 1e-5 before the flow saturates, 2D walls with a ragged width (the
FP32 row-sweep stage kernels, several segment heights), D3Q19 (FP64 generic kernels; FP32
tiled z-sweep), and with the sugar scalar (the generic stage kernels)."""
import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads
from tests.helpers import PHYS, rel_l2, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VARIANTS = [dict(weno3=True), dict(sign_split=True), dict(weno3=True, sign_split=True)]
STRONG = dict(tau=0.6, gravity=1e-3, density_contrast=1.0, settling_velocity=0.02, diffusivity=0.01)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def _run(shape, c0, steps, fp64, **kw):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    if not fp64:
        c0 = c0.astype(np.float32).astype(np.float64)
    g = Simulation(shape, fp64=fp64, **kw)
    g.init(c0)
    o = oracle.OracleSim(shape, **kw)
    o.init(c0)
    g.step(steps)
    o.step(steps)
    return g, o


def _check(g, o, tol, u_floor):
    rho, u, c = (to_np(t) for t in g.fields())
    orho, ou, oc = o.fields()
    assert rel_l2(c, oc) <= tol
    du = np.linalg.norm((u - ou).ravel())
    assert du <= tol * np.linalg.norm(ou.ravel()) + u_floor * np.sqrt(ou.size)
    assert g.deposit == pytest.approx(o.deposit, rel=max(tol, 1e-13), abs=1e-15)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_variant_2d_matches_oracle(variant, fp64, tol):
    shape = (132, 64)
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.02, seed=7)
    g, o = _run(shape, c0, 40, fp64, **STRONG, **variant)
    _check(g, o, tol, 1e-15 if fp64 else 1e-12)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_2d_fp32_row_segments(variant):
    """The FP32 row-sweep stage kernels with a variant: three strips (the last 4 columns
    wide), 16-row and ragged 5-row segments; both match the oracle to 1e-5 and each other
    bit for bit (every face is computed once, whatever the segmentation)."""
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    shape = (260, 96)
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.02, seed=11)
    c0 = c0.astype(np.float32).astype(np.float64)
    o = oracle.OracleSim(shape, **STRONG, **variant)
    o.init(c0)
    o.step(30)
    out = []
    for rows in (16, 5):
        g = lw.Simulation(shape, fp64=False, **STRONG, **variant)
        lw.lbm_wenoc_set_segment_rows(g.handle, rows)
        g.init(c0)
        g.step(30)
        _check(g, o, 1e-5, 1e-12)
        out.append(to_np(g.fields()[2]))
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_d3q19_matches_oracle(variant):
    shape = (16, 12, 24)
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.02, seed=8)
    g, o = _run(shape, c0, 12, True, **STRONG, **variant)
    _check(g, o, 1e-12, 1e-15)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_d3q19_fp32_sweep(variant):
    """The FP32 tiled z-sweep stage kernels with a variant: ragged tiles in x and y, 24- and
    7-level segments; both match the oracle to 1e-5 and each other bit for bit."""
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    shape = (36, 20, 40)
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.02, seed=12)
    c0 = c0.astype(np.float32).astype(np.float64)
    o = oracle.OracleSim(shape, **STRONG, **variant)
    o.init(c0)
    o.step(12)
    out = []
    for rows in (24, 7):
        g = lw.Simulation(shape, fp64=False, **STRONG, **variant)
        lw.lbm_wenoc_set_segment_rows(g.handle, rows)
        g.init(c0)
        g.step(12)
        _check(g, o, 1e-5, 1e-12)
        out.append(to_np(g.fields()[2]))
    assert np.array_equal(out[0], out[1])


def test_variant_with_sugar_matches_oracle():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    shape = (64, 48)
    c0 = workloads.interface_field(shape, interface_frac=0.5, amplitude=0.02, seed=9)
    S0 = 1.0 - workloads.interface_field(shape, interface_frac=0.5, amplitude=0.0, seed=9)
    kw = dict(STRONG, weno3=True, sign_split=True, sugar=True, sugar_contrast=0.5, sugar_diffusivity=0.02,
              phi0=0.05, vs_sugar=0.3)
    g = Simulation(shape, fp64=True, **kw)
    g.init(c0)
    g.set_sugar(S0)
    o = oracle.OracleSim(shape, **kw)
    o.init(c0)
    o.set_sugar(S0)
    g.step(25)
    o.step(25)
    _check(g, o, 1e-12, 1e-15)
    assert rel_l2(to_np(g.sugar()), o.sugar()) <= 1e-12


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("shape", [(132, 64), (36, 20, 40)])
def test_variant_with_sugar_fp32_sweep_kernels(variant, shape):
    """The variants combined with the sugar scalar on the FP32 row-sweep (2D) and z-sweep (3D)
    stage kernels, against the oracle to 1e-5 (c, u, S)."""
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    c0 = workloads.interface_field(shape, interface_frac=0.5, amplitude=0.02, seed=13).astype(np.float32)
    S0 = (1.0 - workloads.interface_field(shape, interface_frac=0.5, amplitude=0.0, seed=13)).astype(np.float32)
    c0, S0 = c0.astype(np.float64), S0.astype(np.float64)
    kw = dict(STRONG, sugar=True, sugar_contrast=0.5, sugar_diffusivity=0.02, phi0=0.05, vs_sugar=0.3, **variant)
    g = Simulation(shape, fp64=False, **kw)
    g.init(c0)
    g.set_sugar(S0)
    o = oracle.OracleSim(shape, **kw)
    o.init(c0)
    o.set_sugar(S0)
    steps = 20 if len(shape) == 2 else 8
    g.step(steps)
    o.step(steps)
    _check(g, o, 1e-5, 1e-12)
    assert rel_l2(to_np(g.sugar()), o.sugar()) <= 1e-5


def test_variant_errors():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    for variant in VARIANTS:
        with pytest.raises(lw.LbmWenocError) as e:
            lw.Simulation((64, 64), fused_rk3=True, **variant)
        assert e.value.code == lw.LW_EINVAL
        s = lw.Simulation((32, 32), lf_alpha=0.2, **PHYS, **variant)
        with pytest.raises(lw.LbmWenocError) as e:
            s.deposit_gradient(np.zeros((32, 32)), 4, 2)
        assert e.value.code == lw.LW_EINVAL
