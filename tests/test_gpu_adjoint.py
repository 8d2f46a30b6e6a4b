"""Gradient of the deposited mass (Sec. 4, m_b) by the hand-written adjoint of the 2D
coupled step, checked against central finite differences of the FP64 oracle.

J(c0, Vs) = mass through the floor after N steps from c0 with the fluid at rest.  The
adjoint (reverse sweep with checkpoint-and-recompute) is exact up to rounding, so:
  * FP64, tiny lattice: every component of dJ/dc0 against the oracle's central
    difference (h = 1e-6) to 1e-6 of the largest component, relative L2 <= 1e-7;
  * FP64, a lattice spanning two 128-column blocks with a ragged tail and a ragged last
    segment: directional derivative and dJ/dVs (lf_alpha held fixed) to 1e-7;
  * FP32 against the FP64 adjoint: relative L2 <= 1e-3;
  * the checkpoint spacing does not change the result; autograd wraps the same numbers.
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
    # only the atomic accumulation order differs
    assert rel_l2(gb, ga) <= 1e-13 and rel_l2(gc, ga) <= 1e-13
    assert vb == pytest.approx(va, rel=1e-13) and vc == pytest.approx(va, rel=1e-13)


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
    assert rel_l2(to_np(c0.grad), 3.0 * g) <= 1e-13
    assert float(vs.grad) == pytest.approx(3.0 * dvs, rel=1e-13)
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
