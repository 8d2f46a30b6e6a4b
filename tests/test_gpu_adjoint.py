"""Gradient of the deposited mass (Sec. 4, m_b) by the hand-written adjoint of the 2D
coupled step, checked against central finite differences of the FP64 oracle and against
the oracle's own reverse sweep.

J(c0, Vs) = mass through the floor after N steps from c0 with the fluid at rest.  The
adjoint (reverse sweep with checkpoint-and-recompute) is exact up to rounding, so:
  * FP64, tiny lattice: every component of dJ/dc0 against the oracle's central
    difference (h = 1e-6) to 1e-6 of the largest component, relative L2 <= 1e-7;
  * FP64, a lattice spanning two 128-column blocks with a ragged tail and a ragged last
    segment: directional derivative and dJ/dVs (lf_alpha held fixed) to 1e-7;
  * 64 x 128, 100 steps: element by element against the oracle's reverse sweep, FP64 to
    1e-10, FP32 to 1e-3;
  * FP32 against the FP64 adjoint: relative L2 <= 1e-3;
  * the checkpoint spacing does not change the result (bitwise, FP64 and FP32); autograd
    wraps the same numbers;
  * the 512 x 1024 FP32 gradient over 2000 steps (checkpoint every 100) against central
    differences of the FP64 forward on 32 random unit directions, 1e-4 relative each.
"""

import numpy as np
import pytest

import oracle
from tests.helpers import rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# strong buoyancy so that the fluid adjoint matters within a few dozen steps
ADJ = dict(tau=0.6, gravity=2e-3, density_contrast=1.0, settling_velocity=0.05, diffusivity=0.02,
           lf_alpha=0.25, u_cap=0.2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def _c0(shape, seed):
    nx, ny = shape
    rng = np.random.default_rng(seed)
    return 0.5 + 0.4 * rng.uniform(-1.0, 1.0, size=(ny, nx))


def _oracle_J(shape, c0, nsteps, **kw):
    o = oracle.OracleSim(shape, **kw)
    o.init(c0)
    o.step(nsteps)
    return o.deposit


def _gpu_grad(shape, c0, nsteps, segment, fp64=True, **kw):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    s = Simulation(shape, fp64=fp64, **kw)
    J, g, dvs = s.deposit_gradient(c0, nsteps, segment)
    torch.cuda.synchronize()
    return J, to_np(g), dvs


def test_adjoint_every_component_vs_oracle_fd():
    shape, nsteps = (16, 24), 30
    c0 = _c0(shape, 11)
    J, g, _ = _gpu_grad(shape, c0, nsteps, segment=7, **ADJ)  # 4 segments + ragged 2
    assert J == pytest.approx(_oracle_J(shape, c0, nsteps, **ADJ), rel=1e-12)
    h = 1e-6
    fd = np.zeros_like(c0)
    for k in range(c0.size):
        e = np.zeros(c0.size)
        e[k] = h
        e = e.reshape(c0.shape)
        fd.flat[k] = (_oracle_J(shape, c0 + e, nsteps, **ADJ) - _oracle_J(shape, c0 - e, nsteps, **ADJ)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0.1
    # the buoyancy-driven flow changes the gradient far above the tolerance, so the
    # comparison covers the fluid part of the adjoint
    fd0 = np.zeros_like(c0)
    kw0 = dict(ADJ, gravity=0.0)
    for k in range(0, c0.size, 7):
        e = np.zeros(c0.size)
        e[k] = h
        e = e.reshape(c0.shape)
        fd0.flat[k] = (_oracle_J(shape, c0 + e, nsteps, **kw0) - _oracle_J(shape, c0 - e, nsteps, **kw0)) / (2 * h)
    assert np.abs(fd - fd0).flat[::7].max() > 1e-3 * scale
    assert np.abs(g - fd).max() <= 1e-6 * scale
    assert rel_l2(g, fd) <= 1e-7


def test_adjoint_vs_oracle_reverse_sweep_64x128():
    # the oracle's own reverse sweep (complex-step Jacobians of its forward routines),
    # element by element: FP64 to rounding, FP32 to its precision
    shape, nsteps = (64, 128), 100
    c0 = _c0(shape, 21)
    Jo, go, vo = oracle.deposit_gradient(shape, c0, nsteps, **ADJ)
    J, g, dvs = _gpu_grad(shape, c0, nsteps, segment=30, **ADJ)
    assert J == pytest.approx(Jo, rel=1e-12)
    assert rel_l2(g, go) <= 1e-10
    assert np.abs(g - go).max() <= 1e-10 * np.abs(go).max()
    assert dvs == pytest.approx(vo, rel=1e-10)
    c32 = c0.astype(np.float32).astype(np.float64)
    Jo32, go32, vo32 = oracle.deposit_gradient(shape, c32, nsteps, **ADJ)
    J, g, dvs = _gpu_grad(shape, c32, nsteps, segment=30, fp64=False, **ADJ)
    assert J == pytest.approx(Jo32, rel=1e-5)
    assert rel_l2(g, go32) <= 1e-3
    assert dvs == pytest.approx(vo32, rel=1e-3)


def test_adjoint_directional_and_vs_ragged():
    shape, nsteps = (196, 40), 45
    c0 = _c0(shape, 12)
    J, g, dvs = _gpu_grad(shape, c0, nsteps, segment=10, **ADJ)
    rng = np.random.default_rng(13)
    d = rng.standard_normal(c0.shape)
    h = 1e-6
    fd = (_oracle_J(shape, c0 + h * d, nsteps, **ADJ) - _oracle_J(shape, c0 - h * d, nsteps, **ADJ)) / (2 * h)
    got = float(np.sum(g * d))
    assert got == pytest.approx(fd, rel=1e-7, abs=1e-9 * np.abs(g).sum())
    kv = dict(ADJ)
    vs = kv.pop("settling_velocity")
    fdv = (_oracle_J(shape, c0, nsteps, settling_velocity=vs + h, **kv) -
           _oracle_J(shape, c0, nsteps, settling_velocity=vs - h, **kv)) / (2 * h)
    assert dvs == pytest.approx(fdv, rel=1e-7)


def test_adjoint_fp32_matches_fp64():
    shape, nsteps = (64, 48), 40
    c0 = _c0(shape, 14).astype(np.float32).astype(np.float64)
    J64, g64, v64 = _gpu_grad(shape, c0, nsteps, segment=6, fp64=True, **ADJ)
    J32, g32, v32 = _gpu_grad(shape, c0, nsteps, segment=6, fp64=False, **ADJ)
    assert J32 == pytest.approx(J64, rel=1e-5)
    assert rel_l2(g32, g64) <= 1e-3
    assert v32 == pytest.approx(v64, rel=1e-3)


def test_adjoint_segment_invariance():
    shape, nsteps = (32, 32), 24
    c0 = _c0(shape, 15)
    Ja, ga, va = _gpu_grad(shape, c0, nsteps, segment=1, **ADJ)
    Jb, gb, vb = _gpu_grad(shape, c0, nsteps, segment=5, **ADJ)
    Jc, gc, vc = _gpu_grad(shape, c0, nsteps, segment=nsteps, **ADJ)
    assert Ja == Jb == Jc
    # no atomics anywhere in the reverse sweep: bitwise the same for any spacing
    assert np.array_equal(ga, gb) and np.array_equal(ga, gc)
    assert va == vb == vc


def test_adjoint_fp32_deterministic():
    shape, nsteps = (256, 100), 12
    c0 = _c0(shape, 18).astype(np.float32)
    a = _gpu_grad(shape, c0, nsteps, segment=5, fp64=False, **ADJ)
    b = _gpu_grad(shape, c0, nsteps, segment=12, fp64=False, **ADJ)
    assert a[0] == b[0] and a[2] == b[2]
    assert np.array_equal(a[1], b[1])


def test_autograd_function():
    from paper_2106_07694_gb300.autograd import deposited_mass
    shape, nsteps = (32, 32), 20
    c0n = _c0(shape, 16)
    kw = dict(ADJ)
    vs0 = kw.pop("settling_velocity")
    J, g, dvs = _gpu_grad(shape, c0n, nsteps, segment=4, settling_velocity=vs0, **kw)
    c0 = torch.tensor(c0n, dtype=torch.float64, device="cuda", requires_grad=True)
    vs = torch.tensor(vs0, dtype=torch.float64, requires_grad=True)
    out = deposited_mass(c0, vs, nsteps, shape, segment=4, fp64=True, **kw)
    assert float(out.detach()) == J
    (3.0 * out).backward()
    assert np.array_equal(to_np(c0.grad), 3.0 * g)
    assert float(vs.grad) == 3.0 * dvs
    with torch.no_grad():
        plain = deposited_mass(c0, vs0, nsteps, shape, fp64=True, **kw)
    assert float(plain) == J


def test_adjoint_rejects_unsupported_and_restores_state():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    c0 = _c0((32, 32), 17)
    for kw in (dict(lf_alpha=0.0), dict(periodic_vertical=True), dict(fused_rk3=True), dict(frozen_velocity=True)):
        p = dict(ADJ)
        p.update(kw)
        s = lw.Simulation((32, 32), **p)
        with pytest.raises(lw.LbmWenocError) as e:
            s.deposit_gradient(c0, 4, 2)
        assert e.value.code == lw.LW_EINVAL
    s3 = lw.Simulation((16, 16, 16), **ADJ)
    with pytest.raises(lw.LbmWenocError):
        s3.deposit_gradient(np.zeros((16, 16, 16)), 4, 2)
    s = lw.Simulation((32, 32), fp64=True, **ADJ)
    nb = lw.lbm_wenoc_gradient_workspace_bytes(s.params, 8, 3)
    small = torch.empty(nb - 256, dtype=torch.uint8, device="cuda")
    grad = torch.empty((32, 32), dtype=torch.float64, device="cuda")
    ct = torch.tensor(c0, dtype=torch.float64, device="cuda")
    with pytest.raises(lw.LbmWenocError) as e:
        lw.lbm_wenoc_deposit_gradient(s.handle, ct, 8, 3, small, nb - 256, grad)
    assert e.value.code == lw.LW_ENOMEM
    s.deposit_gradient(c0, 8, 3)
    with pytest.raises(lw.LbmWenocError) as e:
        s.step(1)
    assert e.value.code == lw.LW_ESTATE
    s.init(c0)
    s.step(8)
    assert s.deposit == pytest.approx(_oracle_J((32, 32), c0, 8, **ADJ), rel=1e-12)


# ---- the 512 x 1024 FP32 gradient over 2000 steps (state kept every 100) -------------
# Expected values: central differences of the FP64 forward along 32 random unit directions
# d (seed 1), J(c0 + 1e-3 d) - J(c0 - 1e-3 d) over 2e-3, i.e. about 1.4e-6 per node
# (WENO5's eps = 1e-6 makes J strongly nonlinear for c near 0: a per-node step of 1e-5
# already leaves a 1e-3 relative truncation error), and in Vs with step 1e-7.  Bound: 1e-4
# relative to each direction's difference quotient, no absolute floor.  Measured: the FP32
# gradient within 2e-6 .. 7.7e-5 of the quotients (median 2.4e-5; the FP64 gradient within
# 5e-6), dJ/dVs within 4e-7.

def test_adjoint_512x1024_2000_steps_fd_32_directions():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300 import workloads
    wl = workloads.ADJOINT_2D
    kw = dict(tau=wl.tau, gravity=wl.gravity, density_contrast=wl.density_contrast,
              diffusivity=wl.diffusivity, lf_alpha=wl.extra["lf_alpha"])
    vs = wl.settling_velocity
    c0 = wl.initial_c().astype(np.float32).astype(np.float64)
    s32 = lw.Simulation(wl.shape, settling_velocity=vs, **kw)
    J, g, dvs = s32.deposit_gradient(c0, wl.steps, wl.extra["segment"])
    g = to_np(g)
    s64 = lw.Simulation(wl.shape, fp64=True, settling_velocity=vs, **kw)

    def J64(c, sim=s64):
        sim.init(c)
        sim.step(wl.steps)
        return sim.deposit

    assert J == pytest.approx(J64(c0), rel=1e-5, abs=1e-9)
    rng = np.random.default_rng(1)
    h = 1e-3
    worst = 0.0
    for i in range(32):
        d = rng.standard_normal(c0.shape)
        d /= np.linalg.norm(d)
        fd = (J64(c0 + h * d) - J64(c0 - h * d)) / (2 * h)
        got = float(np.sum(g * d))
        rel = abs(got - fd) / abs(fd)
        worst = max(worst, rel)
        assert rel <= 1e-4, (i, got, fd, rel)
    print(f"worst |g.d - fd| / |fd| over 32 directions: {worst:.3g}")
    hv = 1e-7
    sp = lw.Simulation(wl.shape, fp64=True, settling_velocity=vs + hv, **kw)
    sm = lw.Simulation(wl.shape, fp64=True, settling_velocity=vs - hv, **kw)
    fdv = (J64(c0, sp) - J64(c0, sm)) / (2 * hv)
    assert dvs == pytest.approx(fdv, rel=1e-5)
