"""FP32 against the FP64 oracle along the pre-saturation window of the 128 x 256 workload
(A = 1e-5, Vs = 1e-3, kappa = 1e-3, tau = 0.6, seed 0).

The window ends when the dominant mode of the front height H(x) (the lowest height where
c = 1/2, Sec. 4.1) reaches 40 % of its wavelength (Sec. 4.1: the linear regime used for
the growth rates; Eqs. Fourier, PSD).  The mode amplitude is read as 2 |H~(k)| / nx, the
amplitude of the sinusoid, against the wavelength nx / k.

The interface is unstable from the start and amplifies every perturbation, FP32 rounding
included, so no FP32 state can track FP64 element-wise to the end of the window: an FP64
twin of the oracle whose initial c differs by half an FP32 unit in the last place per
node already drifts 1.3e-5 (relative L2 of c) away from it there.  The test holds:
  * c within 1e-5 relative L2 at every 1000 steps up to step 8000 (mode amplitude below
    0.1 % of its wavelength);
  * from there to the end of the window (step 34000), c within the larger of 2.5e-5 and
    500 x the twin's drift at the same step: the FP32 error first grows by the rounding of
    each step (1.1e-5 .. 2.0e-5 up to step 15000, 1450 .. 430 x the still tiny twin drift)
    and then at the rate of the instability itself, at 240 - 370 x the twin's drift;
  * the deposited mass within 3e-6 throughout (measured 1.5e-6 at most).
"""
import numpy as np
import pytest

import oracle
from oracle import lsa
from paper_2106_07694_gb300 import workloads
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


def mode_ratio(c):
    """Largest ratio of a front-height mode's amplitude to its wavelength."""
    h = lsa.front_height(c)
    nx = h.size
    H = np.fft.rfft(h - h.mean())
    k = np.arange(1, H.size)
    return float(np.max((2 * np.abs(H[1:]) / nx) / (nx / k)))


def test_fp32_tracks_the_oracle_through_the_pre_saturation_window():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    shape = (128, 256)
    kw = dict(tau=0.6, gravity=1e-5, density_contrast=1.0, settling_velocity=1e-3, diffusivity=1e-3)
    c0 = workloads.SMALL_2D.initial_c().astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(5)
    ulp = np.spacing(np.abs(c0).astype(np.float32)).astype(np.float64)
    c0_twin = c0 + (rng.random(c0.shape) - 0.5) * ulp
    g = Simulation(shape, fp64=False, **kw)
    g.init(c0)
    o = oracle.OracleSim(shape, **kw)
    o.init(c0)
    tw = oracle.OracleSim(shape, **kw)
    tw.init(c0_twin)
    every, step, ratio, worst = 1000, 0, 0.0, 0.0
    while ratio < 0.4:
        for s in (g, o, tw):
            s.step(every)
        step += every
        cg = g.fields()[2].double().numpy()
        co, ct = o.fields()[2], tw.fields()[2]
        ratio = mode_ratio(co)
        err, twin = rel_l2(cg, co), rel_l2(ct, co)
        assert abs(g.deposit - o.deposit) <= 3e-6 * abs(o.deposit), step
        if step <= 8000:
            assert ratio < 1e-3 and err <= 1e-5, (step, ratio, err)
        else:
            assert err <= max(2.5e-5, 500 * twin), (step, ratio, err, twin)
            worst = max(worst, err / twin)
        assert step <= 40000, "the window did not close"
    assert step >= 30000  # the default point saturates near 34000 steps
    print(f"window closed at step {step}; FP32 error / twin drift after step 8000: at most {worst:.0f}")
