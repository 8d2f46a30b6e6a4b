"""Precision of each output against an FP64 reference (FP32 arithmetic everywhere, FP64
only in the global reductions and in the validation build).

Outputs: c and u (relative L2), rho (largest absolute error), the deposited mass m_b
(Sec. 4.2, relative), the total particle mass and the mass below the mid-height plane
(Sec. 4.2.3, Eq. flux; relative).

  * 128 x 256, the 1000-step workload: the FP64 build against the FP64 oracle, and the
    FP32 build against the oracle at steps 250, 500, 1000;
  * 2048 x 4096: the FP32 build against the FP64 build on the same GPU (itself held to
    the oracle at 1e-12 by the parity tests) at steps 100, 500, 1000, well before the
    interface instability saturates.

The measured table is printed, and written as JSON to $LW_PRECISION_OUT when that is set.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2106_07694_gb300 import workloads
from tests.helpers import rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROWS = []


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()
    yield
    out = os.environ.get("LW_PRECISION_OUT")
    if out and ROWS:
        with open(out, "w") as fh:
            json.dump(ROWS, fh, indent=1)


def _kw(wl):
    return dict(tau=wl.tau, gravity=wl.gravity, density_contrast=wl.density_contrast,
                settling_velocity=wl.settling_velocity, diffusivity=wl.diffusivity)


def _errors(case, step, got, ref):
    """got/ref: (rho, u, c, deposit, total mass, mass below mid-height) as numpy / floats."""
    r = dict(case=case, step=step,
             c=rel_l2(got[2], ref[2]), u=rel_l2(got[1], ref[1]),
             rho_abs=float(np.max(np.abs(got[0] - ref[0]))),
             deposit=abs(got[3] - ref[3]) / abs(ref[3]),
             total_mass=abs(got[4] - ref[4]) / abs(ref[4]),
             mass_below_mid=abs(got[5] - ref[5]) / abs(ref[5]))
    ROWS.append(r)
    print(json.dumps(r))
    return r


def _gpu_state(s, ny):
    rho, u, c = (to_np(t) for t in s.fields())
    return rho, u, c, s.deposit, s.total_mass, s.mass_below(ny // 2)


def _oracle_state(o, ny):
    rho, u, c = o.fields()
    return rho, u, c, o.deposit, o.total_mass, o.mass_below(ny // 2)


def test_precision_128x256_against_the_oracle():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    wl = workloads.SMALL_2D
    kw = _kw(wl)
    ny = wl.shape[1]
    c0 = wl.initial_c()
    g64 = Simulation(wl.shape, fp64=True, **kw)
    g64.init(c0)
    o = oracle.OracleSim(wl.shape, **kw)
    o.init(c0)
    g64.step(wl.steps)
    o.step(wl.steps)
    e = _errors("128x256 FP64 build vs oracle", wl.steps, _gpu_state(g64, ny), _oracle_state(o, ny))
    assert e["c"] <= 1e-12 and e["deposit"] <= 1e-12 and e["total_mass"] <= 1e-13
    assert e["mass_below_mid"] <= 1e-12 and e["rho_abs"] <= 1e-12  # rho ~ 1: 1e-12 relative

    c32 = c0.astype(np.float32).astype(np.float64)
    g32 = Simulation(wl.shape, fp64=False, **kw)
    g32.init(c32)
    o32 = oracle.OracleSim(wl.shape, **kw)
    o32.init(c32)
    done = 0
    for step in (250, 500, 1000):
        g32.step(step - done)
        o32.step(step - done)
        done = step
        e = _errors("128x256 FP32 build vs oracle", step, _gpu_state(g32, ny), _oracle_state(o32, ny))
        assert e["c"] <= 1e-5 and e["deposit"] <= 1e-5 and e["total_mass"] <= 1e-6
        assert e["mass_below_mid"] <= 1e-5 and e["rho_abs"] <= 1e-6 and e["u"] <= 5e-5


def test_precision_2048x4096_fp32_against_the_fp64_build():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    wl = workloads.MAIN_2D
    kw = _kw(wl)
    ny = wl.shape[1]
    c0 = wl.initial_c().astype(np.float32).astype(np.float64)
    g32 = Simulation(wl.shape, fp64=False, **kw)
    g64 = Simulation(wl.shape, fp64=True, **kw)
    for s in (g32, g64):
        s.init(c0)
    done = 0
    for step in (100, 500, 1000):
        for s in (g32, g64):
            s.step(step - done)
        done = step
        got, ref = _gpu_state(g32, ny), _gpu_state(g64, ny)
        e = _errors("2048x4096 FP32 build vs FP64 build", step, got, ref)
        assert e["c"] <= 1e-5 and e["deposit"] <= 1e-5 and e["total_mass"] <= 1e-6
        assert e["mass_below_mid"] <= 1e-5 and e["rho_abs"] <= 1e-6
        # u is still small here (1e-6 .. 1e-4: the flow has barely started) and carries the
        # largest relative error of the outputs (measured 2.3e-6 at step 100, 1.0e-5 at 500)
        assert e["u"] <= 5e-5
    del g64
    torch.cuda.empty_cache()
