"""Seeded synthetic inputs and the named workloads.

This module holds none of the method's arithmetic: it only draws random numbers
and lays out the initial concentration field, so that the CUDA path and the
CPU oracle can be fed identical inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014): the state
advances by 0x9E3779B97F4A7C15, the output is the state passed through the
published 64-bit finaliser, and a double in [0, 1) is the top 53 bits times
2^-53.  Draws are taken in node order (x fastest, the vertical axis slowest).
"""
from dataclasses import dataclass, field, replace

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """The doubles r_k in [0, 1), k = offset .. offset+count-1, of the SplitMix64 stream of `seed`."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def interface_field(shape, interface_frac=0.75, width=2.0, amplitude=1e-3, seed=0,
                    upper=1.0, lower=0.0):
    """Initial concentration: a tanh step between `lower` (below) and `upper` (above).

    shape = (nx, ny) or (nx, ny, nz); returns a float64 array indexed [z][y][x].
    The vertical coordinate of node v is v + 1/2 (the floor wall sits at 0, the
    lid at N), the step is centred at interface_frac * N with tanh length scale
    `width`, and each node gets an independent U(-amplitude, amplitude) draw.
    """
    grid = tuple(reversed([int(s) for s in shape]))
    nv = grid[0]
    yv = np.arange(nv, dtype=np.float64) + 0.5
    prof = lower + (upper - lower) * 0.5 * (1.0 + np.tanh((yv - interface_frac * nv) / width))
    c = np.broadcast_to(prof.reshape((nv,) + (1,) * (len(grid) - 1)), grid).copy()
    n = c.size
    if amplitude:
        xi = (2.0 * splitmix64_uniform(seed, n) - 1.0) * amplitude
        c += xi.reshape(grid)
    return c


@dataclass(frozen=True)
class Workload:
    """One named configuration of the coupled solver (lattice units)."""
    name: str
    shape: tuple              # (nx, ny) or (nx, ny, nz); vertical axis last
    dtype: str                # "f32" or "f64"
    steps: int
    tau: float = 0.6
    gravity: float = 1e-5     # A = gravity * density_contrast; force = -A c along the vertical
    density_contrast: float = 1.0
    settling_velocity: float = 1e-3
    diffusivity: float = 1e-3
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return int(np.prod(self.shape))

    def initial_c(self) -> np.ndarray:
        return interface_field(self.shape, interface_frac=self.extra.get("interface_frac", 0.75), seed=self.seed)

    def initial_S(self) -> np.ndarray:
        """Sugar layer (S = 1) below the interface, S = 0 above, no noise (Eqs. ini1, ini)."""
        return 1.0 - interface_field(self.shape, interface_frac=self.extra.get("interface_frac", 0.75),
                                     amplitude=0.0, seed=self.seed)

    @property
    def sugar(self) -> dict:
        """Keyword parameters of the sugar scalar ({} when the workload has none)."""
        return dict(self.extra.get("sugar", {}))

    @property
    def scheme(self) -> dict:
        """Keyword parameters of a transport-scheme variant ({} for flux-split WENO5)."""
        return dict(self.extra.get("scheme", {}))

    @property
    def class_vs(self) -> tuple:
        """Settling velocities of the particle classes (() for one class)."""
        return tuple(self.extra.get("class_vs", ()))

    def initial_classes(self) -> list:
        """Initial class fields: the interface field shared equally between the classes."""
        c0 = self.initial_c()
        k = len(self.class_vs)
        return [c0 / k for _ in range(k)]

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# 2D D2Q9, 128 x 256, FP64: the small case the oracle finishes in seconds.
SMALL_2D = Workload("d2q9_128x256_f64", (128, 256), "f64", 1000)
# 2D D2Q9, 2048 x 4096, FP32 populations stored as f - w_i, FP32 WENO5.
MAIN_2D = Workload("d2q9_2048x4096_f32", (2048, 4096), "f32", 20000)
# 3D D3Q19, 256 x 256 x 512, FP32.
MAIN_3D = Workload("d3q19_256x256x512_f32", (256, 256, 512), "f32", 10000, gravity=2e-5)

# Gradient of the deposited mass: 2D D2Q9, 512 x 1024, FP32, 2000 steps, state kept
# every 100 steps; Lax-Friedrichs alpha fixed at Vs + 0.1 (the default u_cap).
ADJOINT_2D = Workload("d2q9_512x1024_f32_adjoint", (512, 1024), "f32", 2000,
                      extra=dict(segment=100, lf_alpha=1e-3 + 0.1))

# The paper's two-layer state (Eqs. ini1, ini) on the 2048 x 4096 lattice: particles over a
# sugar solution, statically stable.  Physical values mapped to lattice units: particle
# contrast R = rho_p/rho_0 - 1 = 1.519 (glass beads), phi0 = 1.19e-3 (3 g/l, Table 1), with
# g R phi0 = 1e-5 as in the plain workload (g = 5.53e-3, density_contrast = R phi0); sugar
# S* = 0.0084 (rho_f = 1008.4 kg/m3), so the sugar layer outweighs the particles 4.6x;
# Vs(S) = Vs (1 - S*/R S) from Eq. stokes_vel; D_s = nu / 2000 (sugar in water).
SUGAR_2D = Workload("d2q9_2048x4096_f32_sugar", (2048, 4096), "f32", 20000, gravity=5.53e-3,
                    density_contrast=1.808e-3,
                    extra=dict(interface_frac=0.5,
                               sugar=dict(sugar=True, sugar_contrast=8.4e-3, sugar_diffusivity=1.7e-5,
                                          phi0=1.19e-3, vs_sugar=5.53e-3)))

# Variants of the 2048 x 4096 case: the paper's third-order WENO (two stencils, weights 2/3
# and 1/3), the sign-upwind choice of the WENO5 stencil in place of the Lax-Friedrichs split,
# and three particle classes (settling velocities spanning the sweep grid's range, each
# class a third of the interface field, phi_tot = sum of the classes).
WENO3_2D = MAIN_2D.with_(name="d2q9_2048x4096_f32_weno3", extra=dict(scheme=dict(weno3=True)))
SIGN_SPLIT_2D = MAIN_2D.with_(name="d2q9_2048x4096_f32_signsplit", extra=dict(scheme=dict(sign_split=True)))
CLASSES_2D = MAIN_2D.with_(name="d2q9_2048x4096_f32_3classes", extra=dict(class_vs=(5e-4, 1e-3, 2e-3)))

# Sweep grid of the 2048 x 4096 case: buoyancy amplitude x settling velocity.
MAIN_2D_SWEEP = [(a, vs) for a in (1e-5, 2e-5, 5e-5) for vs in (5e-4, 1e-3, 2e-3)]


def batch_sweep(count=64, seed=0):
    """Sizes and parameters of the batched sweep: nx = 64*U{4..16}, ny = 2 nx,
    A log-uniform in [2e-6, 1e-4], Vs log-uniform in [2e-4, 4e-3]."""
    r = splitmix64_uniform(seed, 3 * count).reshape(count, 3)
    out = []
    for k in range(count):
        nx = 64 * (4 + min(12, int(r[k, 0] * 13)))
        a = float(np.exp(np.log(2e-6) + r[k, 1] * (np.log(1e-4) - np.log(2e-6))))
        vs = float(np.exp(np.log(2e-4) + r[k, 2] * (np.log(4e-3) - np.log(2e-4))))
        out.append(Workload(f"batch{k}", (nx, 2 * nx), "f32", 5000, gravity=a, settling_velocity=vs,
                            seed=seed * 1000 + k))
    return out
