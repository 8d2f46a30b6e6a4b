"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 build: <= 1e-12 relative L2 per step.  FP32 build (populations as f - w_i):
<= 1e-5 relative L2 on c and u before the instability saturates; rho to 1e-6
absolute.  Deposit and mass read back in FP64 on both builds.
"""
import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads
from tests.helpers import PHYS, rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def _pair(shape, c0, u0=None, fp64=True, fused_rk3=False, **kw):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    g = Simulation(shape, fp64=fp64, fused_rk3=fused_rk3, **kw)
    if not fp64:
        c0 = c0.astype(np.float32).astype(np.float64)
        if u0 is not None:
            u0 = u0.astype(np.float32).astype(np.float64)
    g.init(c0, u0)
    o = oracle.OracleSim(shape, **kw)
    o.init(c0, u0)
    return g, o


def _compare(g, o, tol_c, tol_u, tol_rho_abs, u_floor=None):
    """Relative L2 on c; on u relative L2 plus an absolute floor: the oracle keeps f_i
    (about w_i ~ 0.1-0.4) in FP64, so each of its velocities carries ~1e-17 of rounding
    while |u| is ~1e-6 early on -- the floor is 1e-15 RMS per node for FP64, 1e-12 for FP32."""
    rg, ug, cg = (to_np(t) for t in g.fields())
    ro, uo, co = o.fields()
    assert rel_l2(cg, co) <= tol_c, rel_l2(cg, co)
    if u_floor is None:
        u_floor = 1e-15 if g.fp64 else 1e-12
    du = np.linalg.norm((ug - uo).ravel())
    assert du <= tol_u * np.linalg.norm(uo.ravel()) + u_floor * np.sqrt(uo.size), \
        (rel_l2(ug, uo), du / np.sqrt(uo.size))
    assert np.max(np.abs(rg - ro)) <= tol_rho_abs
    return rel_l2(cg, co), rel_l2(ug, uo)


# ------------------------------------------------------------------ FP64: per step

@pytest.mark.parametrize("shape", [(128, 256), (36, 20)])
def test_fp64_first_steps_match_oracle(shape):
    c0 = workloads.interface_field(shape, seed=7)
    g, o = _pair(shape, c0, fp64=True, **PHYS)
    for _ in range(3):  # both AA parities and back
        g.step(1)
        o.step(1)
        _compare(g, o, 1e-12, 1e-12, 1e-14)
    assert abs(g.deposit - o.deposit) <= 1e-12 * abs(o.deposit)


def test_fp64_strong_forcing_steps_match_oracle():
    # Larger buoyancy so velocities are not tiny: exercises every Guo/equilibrium term.
    shape = (64, 64)
    c0 = workloads.interface_field(shape, interface_frac=0.5, amplitude=0.05, seed=3)
    kw = dict(PHYS, gravity=2e-3, settling_velocity=2e-3, diffusivity=2e-3)
    g, o = _pair(shape, c0, fp64=True, **kw)
    g.step(40)
    o.step(40)
    _compare(g, o, 1e-12, 1e-11, 1e-13)
    assert abs(g.deposit - o.deposit) <= 1e-12 * abs(o.deposit)


@pytest.mark.slow
def test_fp64_small_workload_1000_steps():
    # The 128 x 256 FP64 workload, 1000 steps.
    wl = workloads.SMALL_2D
    c0 = wl.initial_c()
    kw = dict(tau=wl.tau, gravity=wl.gravity, density_contrast=wl.density_contrast,
              settling_velocity=wl.settling_velocity, diffusivity=wl.diffusivity)
    g, o = _pair(wl.shape, c0, fp64=True, **kw)
    g.step(wl.steps)
    o.step(wl.steps)
    _compare(g, o, 1e-12, 1e-11, 1e-13)
    assert abs(g.deposit - o.deposit) <= 1e-12 * abs(o.deposit)
    m0 = c0.sum()
    assert abs(g.total_mass + g.deposit - m0) <= 1e-13 * m0


def test_fp64_periodic_vertical_and_frozen_velocity():
    rng = np.random.default_rng(11)
    shape = (132, 24)  # ragged x: not a multiple of the 128-wide blocks
    c0 = rng.uniform(0, 1, size=(24, 132))
    u0 = rng.uniform(-0.03, 0.03, size=(2, 24, 132))
    kw = dict(settling_velocity=3e-3, diffusivity=2e-3, periodic_vertical=True, frozen_velocity=True)
    g, o = _pair(shape, c0, u0, fp64=True, **kw)
    g.step(5)
    o.step(5)
    _compare(g, o, 1e-13, 1e-15, 0.0)


def test_fp64_frozen_velocity_with_walls():
    rng = np.random.default_rng(12)
    shape = (40, 33)
    c0 = rng.uniform(0, 1, size=(33, 40))
    u0 = rng.uniform(-0.03, 0.03, size=(2, 33, 40))
    kw = dict(settling_velocity=4e-3, diffusivity=1e-3, frozen_velocity=True)
    g, o = _pair(shape, c0, u0, fp64=True, **kw)
    g.step(7)
    o.step(7)
    _compare(g, o, 1e-13, 1e-15, 0.0)
    assert abs(g.deposit - o.deposit) <= 1e-13 * abs(o.deposit)


# ------------------------------------------------------------------ FP32

@pytest.mark.parametrize("fused", [False, True])
def test_fp32_small_workload_before_saturation(fused):
    wl = workloads.SMALL_2D
    c0 = wl.initial_c()
    kw = dict(tau=wl.tau, gravity=wl.gravity, density_contrast=wl.density_contrast,
              settling_velocity=wl.settling_velocity, diffusivity=wl.diffusivity)
    g, o = _pair(wl.shape, c0, fp64=False, fused_rk3=fused, **kw)
    for n in (1, 1, 98, 200):
        g.step(n)
        o.step(n)
        _compare(g, o, 1e-5, 1e-5, 1e-6)
    m0 = c0.astype(np.float32).astype(np.float64).sum()
    assert abs(g.total_mass + g.deposit - m0) <= 1e-6 * m0
    assert abs(g.deposit - o.deposit) <= 1e-5 * abs(o.deposit)


@pytest.mark.parametrize("A,vs", workloads.MAIN_2D_SWEEP)
def test_fp32_sweep_grid_before_saturation(A, vs):
    # the buoyancy x settling-velocity grid of the 2048 x 4096 workload, on the small lattice
    wl = workloads.SMALL_2D
    c0 = wl.initial_c()
    kw = dict(tau=wl.tau, gravity=A, density_contrast=1.0, settling_velocity=vs, diffusivity=wl.diffusivity)
    g, o = _pair(wl.shape, c0, fp64=False, **kw)
    g.step(300)
    o.step(300)
    _compare(g, o, 1e-5, 1e-5, 1e-6)
    assert abs(g.deposit - o.deposit) <= 1e-5 * abs(o.deposit) + 1e-9


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("shape", [(132, 40), (260, 70), (4, 8)])
def test_fp32_ragged_shapes_frozen_velocity(shape, fused):
    rng = np.random.default_rng(shape[0])
    nx, ny = shape
    c0 = rng.uniform(0, 1, size=(ny, nx))
    u0 = rng.uniform(-0.05, 0.05, size=(2, ny, nx))
    kw = dict(settling_velocity=2e-3, diffusivity=1e-3, frozen_velocity=True)
    g, o = _pair(shape, c0, u0, fp64=False, fused_rk3=fused, **kw)
    g.step(3)
    o.step(3)
    _compare(g, o, 2e-6, 1e-7, 0.0)
    assert abs(g.deposit - o.deposit) <= 1e-5 * abs(o.deposit)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("shape", [(128, 70), (500, 37)])
def test_fp32_sweep_segments_are_bitwise_invariant(shape, fused):
    # The 2D FP32 transport (three row-sweep stage kernels, or the fused sweep) splits
    # rows into CTA segments with primed pipelines; any segment height must give the same
    # bits as the default.
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    c0 = workloads.interface_field(shape, amplitude=0.05, seed=9)
    kw = dict(PHYS, gravity=5e-4, settling_velocity=3e-3, fused_rk3=fused)
    ref = Simulation(shape, fp64=False, **kw)
    ref.init(c0)
    ref.step(6)
    want = [to_np(t) for t in ref.fields()]
    for rows in (1, 2, 3, 4, 5, 7, 13, 64):
        s = Simulation(shape, fp64=False, **kw)
        lw.lbm_wenoc_set_segment_rows(s.handle, rows)
        s.init(c0)
        s.step(6)
        got = [to_np(t) for t in s.fields()]
        for g_, w_ in zip(got, want):
            assert np.array_equal(g_, w_), rows
        assert s.deposit == ref.deposit
    kwo = {k: v for k, v in kw.items() if k != "fused_rk3"}
    o = oracle.OracleSim(shape, **kwo)
    o.init(c0.astype(np.float32).astype(np.float64))
    o.step(6)
    assert rel_l2(want[2], o.fields()[2]) < 1e-6


# ------------------------------------------------------------------ 3D D3Q19

@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_d3q19_steps_match_oracle(fp64, tol):
    shape = (16, 12, 20)
    c0 = workloads.interface_field(shape, amplitude=0.02, seed=4)
    kw = dict(PHYS, gravity=5e-4)
    g, o = _pair(shape, c0, fp64=fp64, **kw)
    for n in (1, 1, 10):
        g.step(n)
        o.step(n)
        _compare(g, o, tol, tol * 10, 1e-14 if fp64 else 1e-6)
    assert abs(g.deposit - o.deposit) <= tol * abs(o.deposit)


@pytest.mark.parametrize("shape", [(64, 16, 40), (40, 20, 24)])
def test_d3q19_fp32_sweep_segments_bitwise_and_parity(shape):
    # The 3D FP32 stage kernels sweep z in segments (priming level, carried face);
    # any segment depth gives the same bits, and the result matches the oracle.
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    c0 = workloads.interface_field(shape, amplitude=0.03, seed=6)
    kw = dict(PHYS, gravity=5e-4, settling_velocity=3e-3)
    ref = Simulation(shape, fp64=False, **kw)
    ref.init(c0)
    ref.step(4)
    want = [to_np(t) for t in ref.fields()]
    for rows in (1, 3, 7, 64):
        s = Simulation(shape, fp64=False, **kw)
        lw.lbm_wenoc_set_segment_rows(s.handle, rows)
        s.init(c0)
        s.step(4)
        for g_, w_ in zip((to_np(t) for t in s.fields()), want):
            assert np.array_equal(g_, w_), rows
        assert s.deposit == ref.deposit
    o = oracle.OracleSim(shape, **kw)
    o.init(c0.astype(np.float32).astype(np.float64))
    o.step(4)
    ro, uo, co = o.fields()
    assert rel_l2(want[2], co) < 1e-6
    assert abs(ref.deposit - o.deposit) <= 1e-5 * abs(o.deposit)


# ------------------------------------------------------------------ physics on the GPU

def test_gpu_poiseuille_exact_at_magic_tau():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu, N, F = (tau - 0.5) / 3.0, 16, 1e-6
    g = Simulation((4, N), tau=tau, body_force=(F, 0.0, 0.0), fp64=True)
    g.init(np.zeros((N, 4)))
    g.step(20000)
    u = to_np(g.fields()[1])
    v = np.arange(N)
    exact = F / (2 * nu) * (v + 0.5) * (N - 0.5 - v)
    assert np.max(np.abs(u[0][:, 0] - exact)) < 1e-10 * exact.max()


# ------------------------------------------------------------------ host-side behaviour

def test_host_and_device_buffers_give_the_same_state():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    shape = (64, 32)
    c0 = workloads.interface_field(shape, seed=1)
    a = Simulation(shape, fp64=False, **PHYS)
    b = Simulation(shape, fp64=False, **PHYS)
    a.init(torch.tensor(c0, dtype=torch.float32).pin_memory())      # host (pinned)
    b.init(torch.tensor(c0, dtype=torch.float32, device="cuda"))   # device
    a.step(10)
    b.step(10)
    fa = [to_np(t) for t in a.fields("cpu")]
    fb = [to_np(t) for t in b.fields("cuda")]
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    assert a.deposit == b.deposit


def test_graph_and_direct_launches_agree_bitwise():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    shape = (128, 64)
    c0 = workloads.interface_field(shape, seed=2)
    a = Simulation(shape, fp64=False, graphs=True, **PHYS)
    b = Simulation(shape, fp64=False, graphs=False, **PHYS)
    a.init(c0)
    b.init(c0)
    a.step(37)
    b.step(37)
    for x, y in zip(a.fields(), b.fields()):
        assert torch.equal(x, y)
    assert a.deposit == b.deposit


def test_errors_are_returned_not_raised_on_device():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    s = Simulation((32, 32), fp64=False, **PHYS)
    with pytest.raises(lw.LbmWenocError) as e:
        s.step(1)
    assert e.value.code == lw.LW_ESTATE
    c0 = np.ones((32, 32))
    c0[5, 5] = np.nan
    s.init(c0)
    s.step(2)
    assert s.status() == lw.LW_EUNSTABLE
    with pytest.raises(lw.LbmWenocError) as e:
        _ = s.deposit
    assert e.value.code == lw.LW_EUNSTABLE
    # re-init clears the status; the handle stays usable
    s.init(np.ones((32, 32)))
    s.step(2)
    assert s.status() == lw.LW_OK


def test_velocity_cap_sets_unstable():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    s = Simulation((16, 16), fp64=True, u_cap=0.01, periodic_vertical=True)
    u0 = np.zeros((2, 16, 16))
    u0[0] = 0.02
    s.init(np.ones((16, 16)), u0)
    s.step(1)
    assert s.status() == lw.LW_EUNSTABLE
