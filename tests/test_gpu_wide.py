"""The 2D FP32 stage kernels with four columns per thread against the one-column ones.

Both compute every WENO5 face once with the same arithmetic, so c, u and rho must agree
bit for bit after many coupled steps, whatever the strip raggedness (nx not a multiple
of the 256-column strip, a strip narrower than one warp) and the row segmentation; the
deposit's FP64 partial sums are grouped per strip, so it agrees to rounding.  Each side
is also held to the FP64 oracle (the fifth-order WENO, Supplement Eqs. S9-S16 raised to
fifth order, SSP-RK3 Eqs. S21-S23).
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


STRONG = dict(PHYS, gravity=5e-4, settling_velocity=3e-3)


def _run(shape, c0, steps, rows=0, **kw):
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    s = lw.Simulation(shape, fp64=False, **STRONG, **kw)
    if rows:
        lw.lbm_wenoc_set_segment_rows(s.handle, rows)
    s.init(c0)
    s.step(steps)
    return [to_np(t) for t in s.fields()], s.deposit


@pytest.mark.parametrize("shape", [(260, 96), (512, 70), (4, 12), (132, 40), (768, 33)])
def test_four_column_kernel_bitwise_equal_to_one_column(shape):
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.03, seed=21)
    steps = 25
    wide, dep_w = _run(shape, c0, steps)
    narrow, dep_n = _run(shape, c0, steps, one_column=True)
    for a, b in zip(wide, narrow):
        assert np.array_equal(a, b)
    assert abs(dep_w - dep_n) <= 1e-13 * abs(dep_n)
    o = oracle.OracleSim(shape, **STRONG)
    o.init(c0.astype(np.float32).astype(np.float64))
    o.step(steps)
    assert rel_l2(wide[2], o.fields()[2]) < 1e-5
    assert abs(dep_w - o.deposit) <= 1e-5 * abs(o.deposit)


@pytest.mark.parametrize("shape", [(520, 90), (256, 64)])
def test_four_column_kernel_segments_bitwise(shape):
    c0 = workloads.interface_field(shape, interface_frac=0.5, amplitude=0.03, seed=22)
    ref, dep = _run(shape, c0, 12)
    for rows in (1, 2, 5, 17, 64, 200):
        got, d = _run(shape, c0, 12, rows=rows)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), rows
        assert d == dep, rows


@pytest.mark.parametrize("shape", [(64, 48, 40), (36, 20, 24), (96, 40, 70)])
def test_four_column_3d_kernel_bitwise_equal_to_one_column(shape):
    # 3D: four x columns per thread on 32 x 16 tiles, ragged in x and y, several z segments
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.03, seed=24)
    out = {}
    for one in (False, True):
        s = lw.Simulation(shape, fp64=False, one_column=one, **STRONG)
        s.init(c0)
        s.step(9)
        out[one] = ([to_np(t) for t in s.fields()], s.deposit)
    for a, b in zip(out[False][0], out[True][0]):
        assert np.array_equal(a, b)
    assert out[False][1] == out[True][1]
    o = oracle.OracleSim(shape, **STRONG)
    o.init(c0.astype(np.float32).astype(np.float64))
    o.step(9)
    assert rel_l2(out[False][0][2], o.fields()[2]) < 1e-5


def test_four_column_3d_kernel_segments_bitwise():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    shape = (64, 32, 50)
    c0 = workloads.interface_field(shape, interface_frac=0.5, amplitude=0.03, seed=25)
    ref, dep = _run(shape, c0, 6)
    for rows in (1, 3, 7, 32, 200):
        got, d = _run(shape, c0, 6, rows=rows)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), rows
        assert d == dep, rows


@pytest.mark.parametrize("shape", [(260, 90), (128, 64)])
def test_fp64_row_sweep_segments_bitwise(shape):
    # the FP64 build runs the same one-column row sweep: segment heights change nothing,
    # and it stays on the FP64 oracle to rounding
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    c0 = workloads.interface_field(shape, interface_frac=0.5, amplitude=0.03, seed=26)
    out = []
    for rows in (0, 1, 3, 16, 200):
        s = lw.Simulation(shape, fp64=True, **STRONG)
        if rows:
            lw.lbm_wenoc_set_segment_rows(s.handle, rows)
        s.init(c0)
        s.step(10)
        out.append(([to_np(t) for t in s.fields()], s.deposit))
    for got, d in out[1:]:
        for a, b in zip(got, out[0][0]):
            assert np.array_equal(a, b)
        assert d == out[0][1]
    o = oracle.OracleSim(shape, **STRONG)
    o.init(c0)
    o.step(10)
    assert rel_l2(out[0][0][2], o.fields()[2]) < 1e-12
    assert abs(out[0][1] - o.deposit) <= 1e-12 * abs(o.deposit)
