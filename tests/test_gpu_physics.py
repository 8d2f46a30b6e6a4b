"""The GPU FP32 path reproduces the LSA growth rate of a seeded interface mode (Sec. 3,
Sec. 4.1) within 10 %, like the oracle does (tests/test_physics_lsa.py)."""
import numpy as np
import pytest

from oracle import lsa
from tests.test_physics_lsa import PHYS_LSA, mode_growth, seeded_interface

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_07694_gb300 import build
    build.build()


@pytest.mark.parametrize("mode", [1, 2])
def test_gpu_fp32_growth_rate_matches_lsa(mode):
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    nx, ny = 64, 128
    c0 = seeded_interface(nx, ny, mode)
    g = Simulation((nx, ny), fp64=False, u_cap=0.5, **PHYS_LSA)
    g.init(c0)

    def at(t):
        g.step(t - g.steps)
        return g.steps, g.fields()[2].double().numpy()
    sigma_sim = mode_growth(at, 25 if mode > 1 else 50, 40 if mode > 1 else 26, nx, mode)
    h = Simulation((nx, ny), fp64=False, u_cap=0.5, **PHYS_LSA)
    h.init(c0)
    h.step(300)
    y = np.arange(ny) + 0.5
    yc, delta = lsa.fit_erf(y, h.fields()[2].double().numpy().mean(axis=1))
    nu = (PHYS_LSA["tau"] - 0.5) / 3.0
    sigma_lsa = lsa.growth_rate(2 * np.pi * mode / nx, ny, nu, PHYS_LSA["gravity"], PHYS_LSA["diffusivity"],
                                PHYS_LSA["settling_velocity"], lambda yy: lsa.erf_profile(yy, yc, delta), m=256)
    assert abs(sigma_sim - sigma_lsa) < 0.10 * sigma_lsa, (sigma_sim, sigma_lsa)


def test_gpu_fp32_growth_rate_with_sugar_matches_lsa():
    from paper_2106_07694_gb300.lbm_wenoc import Simulation
    from tests.test_physics_lsa import SUGAR_LSA, sugar_layer, sugar_lsa_rate
    nx, ny, mode = 64, 128, 1
    c0 = seeded_interface(nx, ny, mode)
    S0 = sugar_layer(nx, ny)
    g = Simulation((nx, ny), fp64=False, u_cap=0.5, **SUGAR_LSA)
    g.init(c0)
    g.set_sugar(S0)

    def at(t):
        g.step(t - g.steps)
        return g.steps, g.fields()[2].double().numpy()
    sigma_sim = mode_growth(at, 50, 40, nx, mode)
    h = Simulation((nx, ny), fp64=False, u_cap=0.5, **SUGAR_LSA)
    h.init(c0)
    h.set_sugar(S0)
    h.step(300)
    sigma_lsa = sugar_lsa_rate(h.fields()[2].double().numpy().mean(axis=1), h.sugar().double().numpy().mean(axis=1),
                               ny, nx, mode, SUGAR_LSA)
    assert abs(sigma_sim - sigma_lsa) < 0.10 * sigma_lsa, (sigma_sim, sigma_lsa)
