"""Checkpoint and resume through the C ABI (lbm_wenoc_save_state / lbm_wenoc_load_state).

A handle that loads a saved state continues bit for bit as the saved handle does: the fields
c, u, rho and the FP64 deposit after the remaining steps are identical, over both AA
parities, with the state in device or host memory, for the default 2D path, the FP64 build,
the fused three-stage sweep (whose c ping-pongs between two buffers), the sugar scalar,
particle classes and D3Q19.  Mismatched parameters and short buffers are refused.
"""
import numpy as np
import pytest

from paper_2106_07694_gb300 import workloads
from tests.helpers import PHYS, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


STRONG = dict(PHYS, gravity=5e-4, settling_velocity=3e-3)
SUGAR = dict(sugar=True, sugar_contrast=0.5, sugar_diffusivity=0.02, phi0=0.05, vs_sugar=0.3)
CASES = {
    "2d_f32": ((260, 96), dict(STRONG)),
    "2d_f64": ((128, 64), dict(STRONG, fp64=True)),
    "2d_fused": ((256, 64), dict(STRONG, fused_rk3=True)),
    "2d_sugar": ((128, 64), dict(STRONG, **SUGAR)),
    "2d_classes": ((128, 64), dict(PHYS, gravity=5e-4, class_vs=(1e-3, 3e-3, 6e-3))),
    "3d_f32": ((32, 24, 40), dict(STRONG)),
}


def _outputs(s):
    out = [to_np(t) for t in s.fields()]
    if s.params.flags & 0x20:  # LW_SUGAR
        out.append(to_np(s.sugar()))
    return out, s.deposit, s.steps


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("where", ["cuda", "cpu"])
def test_resumed_run_is_bitwise_the_continuous_one(name, where):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    shape, kw = CASES[name]
    c0 = workloads.interface_field(shape, interface_frac=0.6, amplitude=0.03, seed=31)
    a = Simulation(shape, **kw)
    a.init(c0)
    if kw.get("sugar"):
        a.set_sugar(1.0 - workloads.interface_field(shape, interface_frac=0.6, amplitude=0.0, seed=31))
    a.step(37)  # odd: the saved state is at the other AA parity
    state = a.save_state(device=where)
    a.step(21)
    want = _outputs(a)
    b = Simulation(shape, **kw)
    b.load_state(state)
    assert b.steps == 37
    b.step(21)
    got = _outputs(b)
    for g_, w_ in zip(got[0], want[0]):
        assert np.array_equal(g_, w_)
    assert got[1] == want[1] and got[2] == want[2] == 58
    assert b.status() == 0


def test_state_of_other_parameters_or_short_buffer_is_refused():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    shape = (64, 32)
    a = Simulation(shape, **STRONG)
    with pytest.raises(lw.LbmWenocError) as e:
        a.save_state()  # before init
    assert e.value.code == lw.LW_ESTATE
    a.init(workloads.interface_field(shape, seed=1))
    a.step(3)
    state = a.save_state()
    with pytest.raises(lw.LbmWenocError) as e:
        lw.lbm_wenoc_save_state(a.handle, state, state.numel() - 1)
    assert e.value.code == lw.LW_ENOMEM
    other = Simulation(shape, **dict(STRONG, settling_velocity=1e-3))
    with pytest.raises(lw.LbmWenocError) as e:
        other.load_state(state)
    assert e.value.code == lw.LW_EINVAL
    bad = state.clone()
    bad[:4] = 0  # not a state header
    with pytest.raises(lw.LbmWenocError) as e:
        Simulation(shape, **STRONG).load_state(bad)
    assert e.value.code == lw.LW_EINVAL
    # the same parameters with graphs off take it
    c = Simulation(shape, graphs=False, **STRONG)
    c.load_state(state)
    assert c.steps == 3
