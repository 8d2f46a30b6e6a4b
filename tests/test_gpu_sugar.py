"""Parity of the sugar path (the paper's density-altering scalar S: force term, S-dependent
settling velocity, first-order upwind transport) with the FP64 oracle, through the C ABI.

FP64 to 1e-12 (c, S; u with the rounding floor of the other parity tests), FP32 to 1e-5
before the flow saturates, D3Q19 both ways, periodic vertical, the exact upwind shift at
CFL 1 with a frozen velocity, graphs against direct launches bitwise, and error codes.
"""
import numpy as np
import pytest

import oracle
from tests.helpers import rel_l2, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# every sugar term well above rounding: strong force, strong Vs(S) dependence
SUG = dict(tau=0.6, gravity=1e-3, density_contrast=1.0, settling_velocity=0.02, diffusivity=0.01,
           sugar=True, sugar_contrast=0.5, sugar_diffusivity=0.02, phi0=0.05, vs_sugar=0.3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def _layers(shape, seed):
    grid = tuple(reversed(shape))
    rng = np.random.default_rng(seed)
    v = np.arange(grid[0]).reshape((-1,) + (1,) * (len(grid) - 1)) + 0.5
    h = grid[0] / 2
    c0 = 0.5 * (1 + np.tanh((v - h) / 2)) + 0.02 * rng.uniform(-1, 1, grid)
    S0 = 0.5 * (1 - np.tanh((v - h) / 2)) * np.ones(grid) + 0.02 * rng.uniform(-1, 1, grid)
    return c0, S0


def _pair(shape, c0, S0, fp64=True, **kw):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    if not fp64:
        c0 = c0.astype(np.float32).astype(np.float64)
        S0 = S0.astype(np.float32).astype(np.float64)
    g = Simulation(shape, fp64=fp64, **kw)
    g.init(c0)
    g.set_sugar(S0)
    o = oracle.OracleSim(shape, **kw)
    o.init(c0)
    o.set_sugar(S0)
    return g, o


def _check(g, o, tol, u_floor):
    rho, u, c = (to_np(t) for t in g.fields())
    orho, ou, oc = o.fields()
    assert rel_l2(c, oc) <= tol
    assert rel_l2(to_np(g.sugar()), o.sugar()) <= tol
    du = np.linalg.norm((u - ou).ravel())
    assert du <= tol * np.linalg.norm(ou.ravel()) + u_floor * np.sqrt(ou.size)
    assert g.deposit == pytest.approx(o.deposit, rel=max(tol, 1e-13), abs=1e-15)


@pytest.mark.parametrize("steps", [1, 2, 40])
def test_fp64_sugar_2d_matches_oracle(steps):
    shape = (64, 96)
    c0, S0 = _layers(shape, 1)
    g, o = _pair(shape, c0, S0, **SUG)
    g.step(steps)
    o.step(steps)
    _check(g, o, 1e-12, 1e-15)


def test_fp32_sugar_2d_matches_oracle():
    shape = (132, 80)  # ragged against the 128-wide blocks
    c0, S0 = _layers(shape, 2)
    g, o = _pair(shape, c0, S0, fp64=False, **SUG)
    g.step(30)
    o.step(30)
    _check(g, o, 1e-5, 1e-12)


@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_sugar_d3q19_matches_oracle(fp64, tol):
    shape = (16, 12, 24)
    c0, S0 = _layers(shape, 3)
    g, o = _pair(shape, c0, S0, fp64=fp64, **SUG)
    g.step(12)
    o.step(12)
    _check(g, o, tol, 1e-15 if fp64 else 1e-12)


def test_fp64_sugar_periodic_vertical():
    shape = (32, 48)
    c0, S0 = _layers(shape, 4)
    kw = dict(SUG, periodic_vertical=True)
    g, o = _pair(shape, c0, S0, **kw)
    g.step(20)
    o.step(20)
    _check(g, o, 1e-12, 1e-15)


def test_sugar_upwind_shift_frozen_velocity():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    nx, ny = 16, 12
    S0 = np.random.default_rng(5).uniform(0, 1, (ny, nx))
    u0 = np.zeros((2, ny, nx))
    u0[0] = 1.0
    g = Simulation((nx, ny), fp64=True, sugar=True, frozen_velocity=True, u_cap=2.0)
    g.init(np.zeros((ny, nx)), u0)
    g.set_sugar(S0)
    g.step(5)  # an odd count: S ends in the second buffer
    np.testing.assert_allclose(to_np(g.sugar()), np.roll(S0, 5, axis=1), rtol=0, atol=1e-15)


def test_sugar_graph_and_direct_launches_bitwise():
    shape = (64, 48)
    c0, S0 = _layers(shape, 6)
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    out = []
    for graphs in (True, False):
        g = Simulation(shape, graphs=graphs, **SUG)
        g.init(c0.astype(np.float32))
        g.set_sugar(S0.astype(np.float32))
        g.step(37)
        out.append([to_np(t) for t in g.fields()] + [to_np(g.sugar()), g.deposit])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_sugar_errors():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    with pytest.raises(lw.LbmWenocError) as e:
        lw.Simulation((32, 32), fused_rk3=True, **SUG)
    assert e.value.code == lw.LW_EINVAL
    plain = lw.Simulation((32, 32))
    plain.init(np.zeros((32, 32)))
    with pytest.raises(lw.LbmWenocError) as e:
        plain.set_sugar(np.zeros((32, 32)))
    assert e.value.code == lw.LW_EINVAL
    s = lw.Simulation((32, 32), lf_alpha=0.2, **SUG)
    with pytest.raises(lw.LbmWenocError) as e:
        s.set_sugar(np.zeros((32, 32)))  # before init
    assert e.value.code == lw.LW_ESTATE
    with pytest.raises(lw.LbmWenocError) as e:
        s.deposit_gradient(np.zeros((32, 32)), 4, 2)
    assert e.value.code == lw.LW_EINVAL
    with pytest.raises(lw.LbmWenocError):
        lw.Batch([dict(shape=(64, 64), **SUG)])
