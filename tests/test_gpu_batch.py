"""Batched simulations (many instances of different size and parameters in one persistent
launch with grid barriers between the phases of a step, or one launch per kernel type)
give the same bits as running each instance alone; a barrier wait that runs out ends the
launch with LW_ETIMEOUT instead of hanging."""
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


SPECS = [
    dict(shape=(256, 96), tau=0.6, gravity=3e-4, settling_velocity=1e-3, diffusivity=1e-3),
    dict(shape=(132, 200), tau=0.7, gravity=1e-4, settling_velocity=3e-3, diffusivity=5e-4),
    dict(shape=(64, 40), tau=0.55, gravity=5e-4, settling_velocity=5e-4, diffusivity=2e-3),
]


def _inits():
    return [workloads.interface_field(sp["shape"], amplitude=0.02, seed=10 + i) for i, sp in enumerate(SPECS)]


def _alone(steps):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    out = []
    for sp, c0 in zip(SPECS, _inits()):
        s = Simulation(sp["shape"], **{k: v for k, v in sp.items() if k != "shape"})
        s.init(c0)
        s.step(steps)
        out.append(([to_np(t) for t in s.fields()], s.deposit))
    return out


@pytest.mark.parametrize("persistent,tune", [(1, False), (1, True), (2, False), (2, True), (0, False)])
def test_batch_matches_instances_run_alone_bitwise(persistent, tune):
    from paper_2106_07694_gb300.lbm_wenoc import Batch
    b = Batch(SPECS)
    b.set_persistent(persistent)
    if tune:
        rows = b.autotune(2)
        assert len(rows) == len(SPECS) and all(2 <= r <= 64 for r in rows)
    for inst, c0 in zip(b.instances, _inits()):
        inst.init(c0)
    b.step(21)  # 16-step graph + 5 single steps, both AA parities
    assert b.status() == 0
    want = _alone(21)
    for inst, (fields, dep) in zip(b.instances, want):
        got = [to_np(t) for t in inst.fields()]
        for g_, w_ in zip(got, fields):
            assert np.array_equal(g_, w_)
        assert inst.deposit == dep
        assert inst.steps == 21


def test_persistent_batch_of_many_instances_bitwise():
    # more items than CTAs in every phase: twelve instances from 64 x 16 to 1024 x 160
    from paper_2106_07694_gb300.lbm_wenoc import Batch, Simulation
    specs = [dict(shape=(64 * (1 + (5 * i) % 16), 16 + 12 * i), tau=0.6 + 0.01 * i, gravity=1e-4 * (1 + i % 3),
                  settling_velocity=1e-3 * (1 + i % 4), diffusivity=1e-3) for i in range(12)]
    inits = [workloads.interface_field(sp["shape"], amplitude=0.02, seed=40 + i) for i, sp in enumerate(specs)]
    b = Batch(specs)
    for inst, c0 in zip(b.instances, inits):
        inst.init(c0)
    b.step(18)
    assert b.status() == 0
    for sp, c0, inst in zip(specs, inits, b.instances):
        s = Simulation(sp["shape"], **{k: v for k, v in sp.items() if k != "shape"})
        s.init(c0)
        s.step(18)
        for g_, w_ in zip((to_np(t) for t in inst.fields()), (to_np(t) for t in s.fields())):
            assert np.array_equal(g_, w_)
        assert inst.deposit == s.deposit


@pytest.mark.parametrize("mode", [1, 2])
def test_persistent_batch_barrier_wait_times_out_and_recovers(mode):
    # One CTA is told to leave before its first barrier; the others' bounded waits (about
    # 10 ms here) run out, the launch ends and the batch reports LW_ETIMEOUT once.  After
    # re-initialisation the batch steps normally again, bit for bit as before.
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Batch
    b = Batch(SPECS)
    b.set_persistent(mode)
    for inst, c0 in zip(b.instances, _inits()):
        inst.init(c0)
    lw.lbm_wenoc_batch_set_wait_limit(b.handle, 20_000_000, 0)
    b.step(1)
    assert b.status() == lw.LW_ETIMEOUT
    assert b.status() == lw.LW_OK  # reported once
    lw.lbm_wenoc_batch_set_wait_limit(b.handle, 1 << 31, -1)
    for inst, c0 in zip(b.instances, _inits()):
        inst.init(c0)
    b.step(5)
    assert b.status() == lw.LW_OK
    want = _alone(5)
    for inst, (fields, dep) in zip(b.instances, want):
        for g_, w_ in zip((to_np(t) for t in inst.fields()), fields):
            assert np.array_equal(g_, w_)
        assert inst.deposit == dep
    with pytest.raises(lw.LbmWenocError) as e:
        lw.lbm_wenoc_batch_set_wait_limit(b.handle, 0, -1)
    assert e.value.code == lw.LW_EINVAL


def test_batch_instance_matches_oracle():
    from paper_2106_07694_gb300.lbm_wenoc import Batch
    b = Batch(SPECS)
    c0s = _inits()
    for inst, c0 in zip(b.instances, c0s):
        inst.init(c0)
    b.step(10)
    sp = SPECS[1]
    o = oracle.OracleSim(sp["shape"], **{k: v for k, v in sp.items() if k != "shape"})
    o.init(c0s[1].astype(np.float32).astype(np.float64))
    o.step(10)
    assert rel_l2(to_np(b.instances[1].fields()[2]), o.fields()[2]) < 1e-5
    assert abs(b.instances[1].deposit - o.deposit) <= 1e-5 * abs(o.deposit)


def test_batch_state_errors():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Batch
    b = Batch(SPECS)
    with pytest.raises(lw.LbmWenocError) as e:
        b.step(1)                       # not initialised
    assert e.value.code == lw.LW_ESTATE
    for inst, c0 in zip(b.instances, _inits()):
        inst.init(c0)
    lw.lbm_wenoc_step(b.instances[0].handle, 1)  # one instance alone: out of step
    with pytest.raises(lw.LbmWenocError) as e:
        b.step(1)
    assert e.value.code == lw.LW_ESTATE
    bad = [dict(SPECS[0], fp64=True)]
    with pytest.raises(lw.LbmWenocError) as e:
        lw.lbm_wenoc_batch_workspace_bytes([lw.make_params(sp["shape"], fp64=True) for sp in bad])
    assert e.value.code == lw.LW_EINVAL
