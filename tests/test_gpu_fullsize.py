"""Parity at the full benchmark sizes, in the launch configuration the benchmark times
(FP32 populations as f - w_i, CUDA graphs, the default segment heights):

  * 2048 x 4096 D2Q9: three coupled steps of the whole lattice from the workload's initial
    state against the FP64 oracle (relative L2 <= 1e-5 on c and u, deposit), for the default
    workload and for its sugar, WENO3, sign-split and three-class variants;
  * 256 x 256 x 512 D3Q19: one step of the whole lattice.  The oracle computes a 32-level
    slab around the interface with a periodic vertical axis; one step moves information
    at most ten nodes (one for the fluid step, three per RK stage), so the levels more
    than ten nodes from the slab's ends must agree with the full lattice;
  * at both sizes: total mass + deposit conserved (FP64 reductions) and the result
    independent of the segment height, bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads
from tests.helpers import rel_l2, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def _kw(wl):
    kw = dict(tau=wl.tau, gravity=wl.gravity, density_contrast=wl.density_contrast,
              settling_velocity=wl.settling_velocity, diffusivity=wl.diffusivity, **wl.sugar, **wl.scheme)
    if wl.class_vs:
        kw["class_vs"] = wl.class_vs
    return kw


def _setup(sim, wl, to):
    """Sugar and class fields of a workload (after init)."""
    if wl.sugar:
        sim.set_sugar(to(wl.initial_S()))
    for k, ck in enumerate(wl.initial_classes() if wl.class_vs else []):
        sim.set_class(k, to(ck))


def _f32(a):
    return a.astype(np.float32).astype(np.float64)


def _run_gpu(wl, c0, steps, rows=0):
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    g = lw.Simulation(wl.shape, fp64=False, **_kw(wl))
    if rows:
        lw.lbm_wenoc_set_segment_rows(g.handle, rows)
    g.init(torch.from_numpy(c0.astype(np.float32)).cuda())
    _setup(g, wl, lambda a: torch.from_numpy(a.astype(np.float32)).cuda())
    m0 = g.total_mass + g.deposit
    g.step(steps)
    return g, m0


def _u_ok(ug, uo):
    du = np.linalg.norm((ug - uo).ravel())
    return du <= 1e-5 * np.linalg.norm(uo.ravel()) + 1e-12 * np.sqrt(uo.size)


@pytest.mark.parametrize("wl", [workloads.MAIN_2D, workloads.SUGAR_2D, workloads.WENO3_2D,
                                workloads.SIGN_SPLIT_2D, workloads.CLASSES_2D], ids=lambda w: w.name)
def test_d2q9_2048x4096_three_steps_whole_lattice(wl):
    c0 = _f32(wl.initial_c())
    g, m0 = _run_gpu(wl, c0, 3)
    _, ug, cg = (to_np(t) for t in g.fields())
    dep = g.deposit
    assert (g.total_mass + g.deposit) == pytest.approx(m0, rel=1e-6)
    o = oracle.OracleSim(wl.shape, **_kw(wl))
    o.init(c0)
    _setup(o, wl, _f32)
    o.step(3)
    _, uo, co = o.fields()
    assert rel_l2(cg, co) <= 1e-5
    assert _u_ok(ug, uo)
    assert dep == pytest.approx(o.deposit, rel=1e-4, abs=1e-12)
    g.close()
    # a ragged segment height gives the same bits
    g5, _ = _run_gpu(wl, c0, 3, rows=5)
    assert np.array_equal(to_np(g5.fields()[2]), cg)
    assert g5.deposit == dep


def test_d3q19_256x256x512_one_step_interface_slab():
    wl = workloads.MAIN_3D
    nz = wl.shape[2]
    c0 = wl.initial_c().astype(np.float32).astype(np.float64)  # [nz][ny][nx]
    g, m0 = _run_gpu(wl, c0, 1)
    _, ug, cg = (to_np(t) for t in g.fields())
    assert (g.total_mass + g.deposit) == pytest.approx(m0, rel=1e-6)
    g.close()
    z0, depth, margin = int(0.75 * nz) - 16, 32, 11
    slab = wl.with_(shape=(wl.shape[0], wl.shape[1], depth))
    o = oracle.OracleSim(slab.shape, periodic_vertical=True, **_kw(wl))
    o.init(c0[z0:z0 + depth])
    o.step(1)
    _, uo, co = o.fields()
    inner = slice(margin, depth - margin)
    glob = slice(z0 + margin, z0 + depth - margin)
    assert rel_l2(cg[glob], co[inner]) <= 1e-5
    assert _u_ok(ug[:, glob], uo[:, inner])
    # the comparison sees the interface: c spans both layers inside the compared levels
    assert co[inner].min() < 0.1 and co[inner].max() > 0.9
    # a ragged segment height gives the same bits
    g7, _ = _run_gpu(wl, c0, 1, rows=7)
    assert np.array_equal(to_np(g7.fields()[2]), cg)
