"""FP64 CPU oracle of the coupled LBM + WENO5 step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2106_07694_gb300``) and never imports it.

The arithmetic lives in ``lbm_wenoc_oracle.c`` (one routine per step a1..a9 of
the method; see its header for the passages each follows; its last section is
the reverse sweep for the gradient of the deposited mass).  This module only
marshals numpy arrays.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ORC_PERIODIC_VERTICAL = 1
ORC_FROZEN_VELOCITY = 2
ORC_SUGAR = 4
ORC_WENO3 = 8
ORC_SIGN_SPLIT = 16


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("tau", ctypes.c_double),
        ("gravity", ctypes.c_double),
        ("density_contrast", ctypes.c_double),
        ("settling_velocity", ctypes.c_double),
        ("diffusivity", ctypes.c_double),
        ("lf_alpha", ctypes.c_double),
        ("u_cap", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("flags", ctypes.c_uint32),
        ("sugar_contrast", ctypes.c_double),
        ("sugar_diffusivity", ctypes.c_double),
        ("phi0", ctypes.c_double),
        ("vs_sugar", ctypes.c_double),
        ("n_classes", ctypes.c_int32),
        ("class_vs", ctypes.c_double * 8),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Params)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_init.argtypes = [ctypes.c_void_p, dp, dp]
        L.orc_init.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_step.restype = ctypes.c_int
        L.orc_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_population_moments.argtypes = [ctypes.c_void_p, dp]
        L.orc_deposit.argtypes = [ctypes.c_void_p]
        L.orc_deposit.restype = ctypes.c_double
        L.orc_total_mass.argtypes = [ctypes.c_void_p]
        L.orc_total_mass.restype = ctypes.c_double
        L.orc_mass_below.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_mass_below.restype = ctypes.c_double
        L.orc_alpha.argtypes = [ctypes.c_void_p]
        L.orc_alpha.restype = ctypes.c_double
        L.orc_steps.argtypes = [ctypes.c_void_p]
        L.orc_steps.restype = ctypes.c_int64
        L.orc_transport_rate.argtypes = [ctypes.c_void_p, dp, dp, dp]
        L.orc_weno5_left.argtypes = [dp, ctypes.c_double]
        L.orc_weno5_left.restype = ctypes.c_double
        L.orc_weno3_left.argtypes = [dp, ctypes.c_double]
        L.orc_weno3_left.restype = ctypes.c_double
        L.orc_lattice.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), dp]
        L.orc_lattice.restype = ctypes.c_int
        L.orc_deposit_gradient.argtypes = [ctypes.POINTER(_Params), dp, ctypes.c_int64, dp, dp, dp]
        L.orc_deposit_gradient.restype = ctypes.c_int
        L.orc_set_sugar.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_class.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        L.orc_set_class.restype = ctypes.c_int
        L.orc_class.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        L.orc_class.restype = ctypes.c_int
        L.orc_class_deposit.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_class_deposit.restype = ctypes.c_double
        L.orc_set_sugar.restype = ctypes.c_int
        L.orc_sugar.argtypes = [ctypes.c_void_p, dp]
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def weno5_left(v, eps):
    """One WENO5-JS face value from the five upwind-side values v[0..4] = h_{i-2..i+2}."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.shape == (5,)
    return lib().orc_weno5_left(_dptr(v), float(eps))


def _params(shape, tau=0.6, gravity=0.0, density_contrast=1.0, settling_velocity=0.0, diffusivity=0.0,
            lf_alpha=0.0, u_cap=0.0, body_force=(0.0, 0.0, 0.0), periodic_vertical=False, frozen_velocity=False,
            sugar=False, sugar_contrast=0.0, sugar_diffusivity=0.0, phi0=0.0, vs_sugar=0.0, weno3=False,
            sign_split=False, class_vs=()):
    p = _Params()
    p.dim = len(shape)
    p.nx, p.ny = int(shape[0]), int(shape[1])
    p.nz = int(shape[2]) if p.dim == 3 else 1
    p.tau, p.gravity, p.density_contrast = tau, gravity, density_contrast
    p.settling_velocity, p.diffusivity = settling_velocity, diffusivity
    p.lf_alpha, p.u_cap = lf_alpha, u_cap
    for d in range(3):
        p.body_force[d] = float(body_force[d]) if d < len(body_force) else 0.0
    p.flags = (ORC_PERIODIC_VERTICAL if periodic_vertical else 0) | \
              (ORC_FROZEN_VELOCITY if frozen_velocity else 0) | (ORC_SUGAR if sugar else 0) | \
              (ORC_WENO3 if weno3 else 0) | (ORC_SIGN_SPLIT if sign_split else 0)
    p.sugar_contrast, p.sugar_diffusivity, p.phi0, p.vs_sugar = sugar_contrast, sugar_diffusivity, phi0, vs_sugar
    p.n_classes = len(class_vs)
    for k, v in enumerate(class_vs):
        p.class_vs[k] = float(v)
    return p


def deposit_gradient(shape, c0, nsteps, **params):
    """Reverse sweep of the oracle: (J, dJ/dc0, dJ/dVs) for the deposited mass after
    nsteps steps from c0 (2D, walls, lf_alpha > 0 held fixed)."""
    p = _params(shape, **params)
    grid = (int(shape[1]), int(shape[0]))
    c0 = np.ascontiguousarray(c0, dtype=np.float64).reshape(grid)
    g = np.empty(grid)
    dvs = ctypes.c_double()
    J = ctypes.c_double()
    rc = lib().orc_deposit_gradient(ctypes.byref(p), _dptr(c0), int(nsteps), _dptr(g), ctypes.byref(dvs),
                                    ctypes.byref(J))
    if rc != 0:
        raise ValueError(f"orc_deposit_gradient failed: {rc}")
    return J.value, g, dvs.value


def weno3_left(v, eps):
    """One third-order WENO face value from the upwind-side values v[0..2] = h_{i-1..i+1}."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.shape == (3,)
    return lib().orc_weno3_left(_dptr(v), float(eps))


class OracleSim:
    """A simulation held by the C oracle.

    shape: (nx, ny) in 2D or (nx, ny, nz) in 3D; arrays are indexed [z][y][x]
    (numpy shape (ny, nx) or (nz, ny, nx)); the vertical axis is the slowest one.
    """

    def __init__(self, shape, tau=0.6, gravity=0.0, density_contrast=1.0,
                 settling_velocity=0.0, diffusivity=0.0, lf_alpha=0.0, u_cap=0.0,
                 body_force=(0.0, 0.0, 0.0), periodic_vertical=False, frozen_velocity=False,
                 sugar=False, sugar_contrast=0.0, sugar_diffusivity=0.0, phi0=0.0, vs_sugar=0.0, weno3=False,
                 sign_split=False, class_vs=()):
        dim = len(shape)
        p = _params(shape, tau, gravity, density_contrast, settling_velocity, diffusivity, lf_alpha, u_cap,
                    body_force, periodic_vertical, frozen_velocity, sugar, sugar_contrast, sugar_diffusivity,
                    phi0, vs_sugar, weno3, sign_split, class_vs)
        self._p = p
        self.dim = dim
        self.grid = tuple(reversed([int(s) for s in shape]))  # numpy shape, vertical first
        self.n = int(np.prod(self.grid))
        h = lib().orc_create(ctypes.byref(p))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    @property
    def alpha(self):
        return lib().orc_alpha(self._h)

    def init(self, c0, u0=None):
        c0 = np.ascontiguousarray(c0, dtype=np.float64).reshape(self.grid)
        self._c0_keep = c0
        up = None
        if u0 is not None:
            u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape((self.dim,) + self.grid)
            self._u0_keep = u0
            up = _dptr(u0)
        rc = lib().orc_init(self._h, _dptr(c0), up)
        if rc != 0:
            raise RuntimeError(f"orc_init failed: {rc}")

    def set_sugar(self, S0):
        """Sugar field (sugar=True handles), after init."""
        S0 = np.ascontiguousarray(S0, dtype=np.float64).reshape(self.grid)
        self._S_keep = S0
        if lib().orc_set_sugar(self._h, _dptr(S0)) != 0:
            raise RuntimeError("orc_set_sugar failed")

    def sugar(self):
        S = np.empty(self.grid)
        lib().orc_sugar(self._h, _dptr(S))
        return S

    def set_class(self, k, ck):
        """Particle class k (polydisperse handles), after init (class 0 = c0 there)."""
        ck = np.ascontiguousarray(ck, dtype=np.float64).reshape(self.grid)
        self._cls_keep = getattr(self, "_cls_keep", {})
        self._cls_keep[k] = ck
        if lib().orc_set_class(self._h, int(k), _dptr(ck)) != 0:
            raise RuntimeError("orc_set_class failed")

    def class_field(self, k):
        out = np.empty(self.grid)
        if lib().orc_class(self._h, int(k), _dptr(out)) != 0:
            raise RuntimeError("orc_class failed")
        return out

    def class_deposit(self, k):
        return lib().orc_class_deposit(self._h, int(k))

    def step(self, n=1):
        return lib().orc_step(self._h, int(n))

    def fields(self):
        rho = np.empty(self.grid)
        u = np.empty((self.dim,) + self.grid)
        c = np.empty(self.grid)
        lib().orc_fields(self._h, _dptr(rho), _dptr(u), _dptr(c))
        return rho, u, c

    def population_moments(self):
        out = np.empty(4)
        lib().orc_population_moments(self._h, _dptr(out))
        return out

    @property
    def deposit(self):
        return lib().orc_deposit(self._h)

    @property
    def total_mass(self):
        return lib().orc_total_mass(self._h)

    def mass_below(self, level):
        """Mass below the plane under vertical level `level`, deposit included (Sec. 4.2.3,
        Eq. flux)."""
        return lib().orc_mass_below(self._h, int(level))

    @property
    def steps(self):
        return lib().orc_steps(self._h)

    def transport_rate(self, c, u):
        """L(c) for a given c and transport velocity u (shape (dim,)+grid)."""
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(self.grid)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape((self.dim,) + self.grid)
        L = np.empty(self.grid)
        lib().orc_transport_rate(self._h, _dptr(c), _dptr(u), _dptr(L))
        return L

    def lattice(self):
        ci = (ctypes.c_int * 57)()
        wi = np.empty(19)
        q = lib().orc_lattice(self._h, ci, _dptr(wi))
        return np.array(ci[: 3 * q]).reshape(q, 3), wi[:q].copy()
