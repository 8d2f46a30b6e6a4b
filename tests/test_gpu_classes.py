"""Parity of polydisperse particle classes (Eqs. forceterm_poly, poly) with the FP64 oracle
through the C ABI: every class field, each class's deposit and the summed fields, FP64 to
1e-12 and FP32 to 1e-5 (the 2D FP32 path runs the row-sweep stage kernels per class),
D3Q19, with sugar; and error codes."""
import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads
from tests.helpers import rel_l2, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CLS = dict(tau=0.6, gravity=1e-3, density_contrast=1.0, diffusivity=0.01, class_vs=(0.005, 0.02, 0.04))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def _fields(shape, seed):
    base = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.02, seed=seed)
    return [base, 0.5 * workloads.interface_field(shape, interface_frac=0.7, amplitude=0.02, seed=seed + 1),
            0.25 * workloads.interface_field(shape, interface_frac=0.5, amplitude=0.02, seed=seed + 2)]


def _pair(shape, cs, fp64, S0=None, **kw):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    if not fp64:
        cs = [c.astype(np.float32).astype(np.float64) for c in cs]
        if S0 is not None:
            S0 = S0.astype(np.float32).astype(np.float64)
    g = Simulation(shape, fp64=fp64, **kw)
    o = oracle.OracleSim(shape, **kw)
    g.init(cs[0])
    o.init(cs[0])
    for k in range(1, len(cs)):
        g.set_class(k, cs[k])
        o.set_class(k, cs[k])
    if S0 is not None:
        g.set_sugar(S0)
        o.set_sugar(S0)
    return g, o


def _check(g, o, n, tol, u_floor):
    rho, u, c = (to_np(t) for t in g.fields())
    orho, ou, oc = o.fields()
    assert rel_l2(c, oc) <= tol
    du = np.linalg.norm((u - ou).ravel())
    assert du <= tol * np.linalg.norm(ou.ravel()) + u_floor * np.sqrt(ou.size)
    for k in range(n):
        assert rel_l2(to_np(g.class_field(k)), o.class_field(k)) <= tol
        assert g.class_deposit(k) == pytest.approx(o.class_deposit(k), rel=max(tol, 1e-13), abs=1e-15)
    assert g.deposit == pytest.approx(o.deposit, rel=max(tol, 1e-13))
    assert g.total_mass == pytest.approx(o.total_mass, rel=max(tol, 1e-13))


@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_classes_2d_match_oracle(fp64, tol):
    shape = (132, 64)
    g, o = _pair(shape, _fields(shape, 11), fp64, **CLS)
    g.step(40)
    o.step(40)
    _check(g, o, 3, tol, 1e-15 if fp64 else 1e-12)


def test_classes_d3q19_match_oracle():
    shape = (16, 12, 24)
    g, o = _pair(shape, _fields(shape, 21), True, **CLS)
    g.step(12)
    o.step(12)
    _check(g, o, 3, 1e-12, 1e-15)


@pytest.mark.parametrize("fp64,tol", [(True, 1e-12), (False, 1e-5)])
def test_classes_with_sugar_match_oracle(fp64, tol):
    shape = (64, 48)
    S0 = 1.0 - workloads.interface_field(shape, interface_frac=0.5, amplitude=0.0, seed=3)
    kw = dict(CLS, sugar=True, sugar_contrast=0.5, sugar_diffusivity=0.02, phi0=0.05, vs_sugar=0.3)
    g, o = _pair(shape, _fields(shape, 31), fp64, S0=S0, **kw)
    g.step(25)
    o.step(25)
    _check(g, o, 3, tol, 1e-15 if fp64 else 1e-12)
    assert rel_l2(to_np(g.sugar()), o.sugar()) <= tol


def test_class_errors():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    p = lw.make_params((64, 64), class_vs=(0.01, 0.02))
    p.n_classes = 9  # more classes than the parameter block holds
    with pytest.raises(lw.LbmWenocError) as e:
        lw.lbm_wenoc_workspace_bytes(p)
    assert e.value.code == lw.LW_EINVAL
    with pytest.raises(lw.LbmWenocError) as e:
        lw.Simulation((64, 64), fused_rk3=True, class_vs=(0.01, 0.02))
    assert e.value.code == lw.LW_EINVAL
    one = lw.Simulation((32, 32))
    one.init(np.zeros((32, 32)))
    with pytest.raises(lw.LbmWenocError) as e:
        one.set_class(1, np.zeros((32, 32)))
    assert e.value.code == lw.LW_EINVAL
    s = lw.Simulation((32, 32), lf_alpha=0.2, class_vs=(0.01, 0.02))
    s.init(np.zeros((32, 32)))
    with pytest.raises(lw.LbmWenocError) as e:
        s.set_class(2, np.zeros((32, 32)))
    assert e.value.code == lw.LW_EINVAL
    with pytest.raises(lw.LbmWenocError) as e:
        s.deposit_gradient(np.zeros((32, 32)), 4, 2)
    assert e.value.code == lw.LW_EINVAL
