"""The allocation-free total-mass entry point against the workspace-based one.

Some callers cannot allocate device memory (a fixed arena owned by the host
application, a plugin inside another framework's allocator, a tool that only holds
a pointer to a field).  lbm_wenoc_total_mass_noalloc() serves them with scratch in a
static device array.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2106_07694_gb300 import workloads
from tests.helpers import PHYS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


@pytest.mark.parametrize("fp64,shape", [(False, (260, 70)), (True, (128, 256)), (False, (2048, 4096))])
def test_noalloc_total_mass_matches_workspace_reduction(fp64, shape):
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    sim = Simulation(shape, fp64=fp64, **PHYS)
    sim.init(workloads.interface_field(shape, seed=3))
    sim.step(5)
    want = sim.total_mass                      # existing entry point (handle + workspace)
    c = sim.fields(device="cuda")[2].contiguous()
    stream = torch.cuda.current_stream()
    for _ in range(2):                          # two calls in a row share the scratch
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        lw.lbm_wenoc_total_mass_noalloc(c, c.numel(), fp64, stream.cuda_stream, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - want) <= 1e-12 * abs(want), (got, want)


def test_noalloc_rejects_fields_beyond_the_scratch():
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    c = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lw.LbmWenocError) as e:
        lw.lbm_wenoc_total_mass_noalloc(c, 2048 * 32768 + 1, False, None, out)
    assert e.value.code == lw.LW_EINVAL
    with pytest.raises(lw.LbmWenocError):
        lw.lbm_wenoc_total_mass_noalloc(c, 0, False, None, out)


@pytest.mark.parametrize("n", [3 * 32768 + 17, 2048 * 32768])
def test_noalloc_partial_last_block_and_the_limit(n):
    # several blocks with a partial last one, and the largest accepted size, against an
    # FP64 sum of the same numbers
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    g = torch.Generator(device="cuda").manual_seed(7)
    c = torch.rand(n, dtype=torch.float32, device="cuda", generator=g)
    want = float(c.double().sum().item())
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    lw.lbm_wenoc_total_mass_noalloc(c, n, False, torch.cuda.current_stream().cuda_stream, out)
    torch.cuda.synchronize()
    assert abs(float(out.item()) - want) <= 1e-12 * abs(want)
    del c
    torch.cuda.empty_cache()


def test_noalloc_calls_on_two_streams_ordered_by_an_event():
    # The second call, on another stream, waits for the first through an event: the scratch
    # (its ticket cleared at the start of each call) is then reused safely.
    from paper_2106_07694_gb300 import lbm_wenoc as lw
    a = torch.arange(5 * 32768 + 3, dtype=torch.float32, device="cuda") * 1e-3
    b = torch.ones(70000, dtype=torch.float32, device="cuda")
    oa = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    ob = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    lw.lbm_wenoc_total_mass_noalloc(a, a.numel(), False, s1.cuda_stream, oa)
    ev = torch.cuda.Event()
    ev.record(s1)
    s2.wait_event(ev)
    lw.lbm_wenoc_total_mass_noalloc(b, b.numel(), False, s2.cuda_stream, ob)
    torch.cuda.synchronize()
    assert abs(float(oa.item()) - float(a.double().sum().item())) <= 1e-12 * float(a.double().sum().item())
    assert float(ob.item()) == 70000.0
