"""Python binding of the lbm_wenoc C ABI (include/lbm_wenoc.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
liblbm_wenoc.so.  There is no CPU fallback -- if the library is not built, or no
CUDA device is present, the calls raise.

The functions carry the C names; ``Simulation`` is a convenience wrapper that
allocates the workspace with PyTorch on the current device and passes torch's
current stream.
"""
import ctypes
import os

import numpy as np

LW_OK = 0
LW_EINVAL = -1
LW_ENOMEM = -2
LW_ECUDA = -3
LW_EUNSTABLE = -4
LW_ETIMEOUT = -5
LW_ESTATE = -6

LW_FP64 = 0x1
LW_PERIODIC_VERTICAL = 0x2
LW_FROZEN_VELOCITY = 0x4
LW_NO_GRAPH = 0x8
LW_FUSED_RK3 = 0x10
LW_SUGAR = 0x20
LW_WENO3 = 0x40
LW_SIGN_SPLIT = 0x80
LW_ONE_COLUMN = 0x100

_ERRORS = {LW_EINVAL: "LW_EINVAL", LW_ENOMEM: "LW_ENOMEM", LW_ECUDA: "LW_ECUDA",
           LW_EUNSTABLE: "LW_EUNSTABLE", LW_ETIMEOUT: "LW_ETIMEOUT", LW_ESTATE: "LW_ESTATE"}

EXPORTED = [
    "lbm_wenoc_workspace_bytes", "lbm_wenoc_create", "lbm_wenoc_init", "lbm_wenoc_step",
    "lbm_wenoc_deposited_mass", "lbm_wenoc_total_mass", "lbm_wenoc_mass_below", "lbm_wenoc_fields",
    "lbm_wenoc_status",
    "lbm_wenoc_steps", "lbm_wenoc_profile_enable", "lbm_wenoc_profile_read",
    "lbm_wenoc_launch_count", "lbm_wenoc_set_segment_rows", "lbm_wenoc_total_mass_noalloc",
    "lbm_wenoc_destroy", "lbm_wenoc_batch_workspace_bytes", "lbm_wenoc_batch_create",
    "lbm_wenoc_batch_instance", "lbm_wenoc_batch_step", "lbm_wenoc_batch_autotune",
    "lbm_wenoc_batch_launch_count", "lbm_wenoc_batch_destroy", "lbm_wenoc_batch_set_persistent",
    "lbm_wenoc_batch_set_wait_limit", "lbm_wenoc_batch_status",
    "lbm_wenoc_gradient_workspace_bytes", "lbm_wenoc_deposit_gradient", "lbm_wenoc_set_sugar",
    "lbm_wenoc_sugar", "lbm_wenoc_set_class", "lbm_wenoc_class", "lbm_wenoc_class_deposit",
    "lbm_wenoc_state_bytes", "lbm_wenoc_save_state", "lbm_wenoc_load_state",
]


class LbmWenocError(RuntimeError):
    def __init__(self, call, code):
        super().__init__(f"{call} returned {_ERRORS.get(code, code)}")
        self.code = code


class lbm_wenoc_params(ctypes.Structure):
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


class lbm_wenoc_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "liblbm_wenoc.so")


def load():
    """Load liblbm_wenoc.so (built by paper_2106_07694_gb300.build.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    P = ctypes.POINTER(lbm_wenoc_params)
    L.lbm_wenoc_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    L.lbm_wenoc_create.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    L.lbm_wenoc_init.argtypes = [vp, vp, vp]
    L.lbm_wenoc_step.argtypes = [vp, i64]
    L.lbm_wenoc_deposited_mass.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.lbm_wenoc_total_mass.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.lbm_wenoc_mass_below.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    L.lbm_wenoc_fields.argtypes = [vp, vp, vp, vp]
    L.lbm_wenoc_status.argtypes = [vp]
    L.lbm_wenoc_state_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.lbm_wenoc_save_state.argtypes = [vp, vp, ctypes.c_size_t]
    L.lbm_wenoc_load_state.argtypes = [vp, vp, ctypes.c_size_t]
    L.lbm_wenoc_steps.argtypes = [vp]
    L.lbm_wenoc_steps.restype = i64
    L.lbm_wenoc_profile_enable.argtypes = [vp, ctypes.c_int]
    L.lbm_wenoc_profile_read.argtypes = [vp, ctypes.POINTER(lbm_wenoc_kernel_stat), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.lbm_wenoc_launch_count.argtypes = [vp]
    L.lbm_wenoc_launch_count.restype = i64
    L.lbm_wenoc_set_segment_rows.argtypes = [vp, ctypes.c_int32]
    L.lbm_wenoc_total_mass_noalloc.argtypes = [vp, i64, ctypes.c_int32, vp, vp]
    L.lbm_wenoc_destroy.argtypes = [vp]
    L.lbm_wenoc_destroy.restype = None
    L.lbm_wenoc_batch_workspace_bytes.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
    L.lbm_wenoc_batch_create.argtypes = [P, ctypes.c_int32, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
    L.lbm_wenoc_batch_instance.argtypes = [vp, ctypes.c_int32]
    L.lbm_wenoc_batch_instance.restype = vp
    L.lbm_wenoc_batch_step.argtypes = [vp, i64]
    L.lbm_wenoc_batch_autotune.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    L.lbm_wenoc_batch_launch_count.argtypes = [vp]
    L.lbm_wenoc_batch_launch_count.restype = i64
    L.lbm_wenoc_batch_destroy.argtypes = [vp]
    L.lbm_wenoc_batch_set_persistent.argtypes = [vp, ctypes.c_int32]
    L.lbm_wenoc_batch_set_wait_limit.argtypes = [vp, i64, ctypes.c_int32]
    L.lbm_wenoc_batch_status.argtypes = [vp]
    L.lbm_wenoc_batch_destroy.restype = None
    L.lbm_wenoc_gradient_workspace_bytes.argtypes = [P, i64, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]
    dp = ctypes.POINTER(ctypes.c_double)
    L.lbm_wenoc_deposit_gradient.argtypes = [vp, vp, i64, ctypes.c_int32, vp, ctypes.c_size_t, vp, dp, dp]
    L.lbm_wenoc_set_sugar.argtypes = [vp, vp]
    L.lbm_wenoc_sugar.argtypes = [vp, vp]
    L.lbm_wenoc_set_class.argtypes = [vp, ctypes.c_int32, vp]
    L.lbm_wenoc_class.argtypes = [vp, ctypes.c_int32, vp]
    L.lbm_wenoc_class_deposit.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    for name in EXPORTED:
        if name not in ("lbm_wenoc_steps", "lbm_wenoc_launch_count", "lbm_wenoc_destroy",
                        "lbm_wenoc_batch_instance", "lbm_wenoc_batch_launch_count", "lbm_wenoc_batch_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(call, rc):
    if rc != LW_OK:
        raise LbmWenocError(call, rc)
    return rc


def _ptr(x):
    """Address of a torch tensor, a numpy array or an int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# ---- the C entry points, same names --------------------------------------------------

def lbm_wenoc_workspace_bytes(params):
    n = ctypes.c_size_t(0)
    _check("lbm_wenoc_workspace_bytes", load().lbm_wenoc_workspace_bytes(ctypes.byref(params), ctypes.byref(n)))
    return n.value


def lbm_wenoc_create(params, workspace, nbytes, stream):
    h = ctypes.c_void_p()
    _check("lbm_wenoc_create", load().lbm_wenoc_create(ctypes.byref(params), _ptr(workspace), nbytes,
                                                       stream, ctypes.byref(h)))
    return h


def lbm_wenoc_init(h, c0, u0=None):
    return _check("lbm_wenoc_init", load().lbm_wenoc_init(h, _ptr(c0), _ptr(u0)))


def lbm_wenoc_step(h, nsteps):
    return _check("lbm_wenoc_step", load().lbm_wenoc_step(h, int(nsteps)))


def lbm_wenoc_deposited_mass(h):
    out = ctypes.c_double()
    _check("lbm_wenoc_deposited_mass", load().lbm_wenoc_deposited_mass(h, ctypes.byref(out)))
    return out.value


def lbm_wenoc_total_mass(h):
    out = ctypes.c_double()
    _check("lbm_wenoc_total_mass", load().lbm_wenoc_total_mass(h, ctypes.byref(out)))
    return out.value


def lbm_wenoc_mass_below(h, level):
    out = ctypes.c_double()
    _check("lbm_wenoc_mass_below", load().lbm_wenoc_mass_below(h, int(level), ctypes.byref(out)))
    return out.value


def lbm_wenoc_fields(h, rho=None, u=None, c=None):
    return _check("lbm_wenoc_fields", load().lbm_wenoc_fields(h, _ptr(rho), _ptr(u), _ptr(c)))


def lbm_wenoc_status(h):
    return load().lbm_wenoc_status(h)


def lbm_wenoc_state_bytes(h):
    out = ctypes.c_size_t()
    _check("lbm_wenoc_state_bytes", load().lbm_wenoc_state_bytes(h, ctypes.byref(out)))
    return out.value


def lbm_wenoc_save_state(h, dst, nbytes):
    return _check("lbm_wenoc_save_state", load().lbm_wenoc_save_state(h, _ptr(dst), int(nbytes)))


def lbm_wenoc_load_state(h, src, nbytes):
    return _check("lbm_wenoc_load_state", load().lbm_wenoc_load_state(h, _ptr(src), int(nbytes)))


def lbm_wenoc_steps(h):
    return load().lbm_wenoc_steps(h)


def lbm_wenoc_launch_count(h):
    return load().lbm_wenoc_launch_count(h)


def lbm_wenoc_profile_enable(h, enable=True):
    return _check("lbm_wenoc_profile_enable", load().lbm_wenoc_profile_enable(h, 1 if enable else 0))


def lbm_wenoc_profile_read(h, reset=False):
    stats = (lbm_wenoc_kernel_stat * 16)()
    count = ctypes.c_int(0)
    _check("lbm_wenoc_profile_read", load().lbm_wenoc_profile_read(h, stats, 16, ctypes.byref(count),
                                                                   1 if reset else 0))
    return {stats[i].name.decode(): (stats[i].launches, stats[i].total_ms) for i in range(count.value)}


def lbm_wenoc_set_segment_rows(h, rows):
    return _check("lbm_wenoc_set_segment_rows", load().lbm_wenoc_set_segment_rows(h, int(rows)))


def lbm_wenoc_total_mass_noalloc(c_dev, n, fp64, stream, out_dev):
    """Sum of n concentrations at c_dev into the double at out_dev, with no device
    allocation (scratch in a fixed static device array; see the C header)."""
    return _check("lbm_wenoc_total_mass_noalloc",
                  load().lbm_wenoc_total_mass_noalloc(_ptr(c_dev), int(n), 1 if fp64 else 0, stream, _ptr(out_dev)))


def lbm_wenoc_gradient_workspace_bytes(params, nsteps, segment):
    n = ctypes.c_size_t(0)
    _check("lbm_wenoc_gradient_workspace_bytes",
           load().lbm_wenoc_gradient_workspace_bytes(ctypes.byref(params), int(nsteps), int(segment),
                                                     ctypes.byref(n)))
    return n.value


def lbm_wenoc_deposit_gradient(h, c0, nsteps, segment, workspace, nbytes, grad_c0):
    """Deposited mass J after nsteps steps from c0 and its gradient: writes dJ/dc0 into
    grad_c0 and returns (J, dJ/dVs)."""
    dvs = ctypes.c_double()
    J = ctypes.c_double()
    _check("lbm_wenoc_deposit_gradient",
           load().lbm_wenoc_deposit_gradient(h, _ptr(c0), int(nsteps), int(segment), _ptr(workspace), nbytes,
                                             _ptr(grad_c0), ctypes.byref(dvs), ctypes.byref(J)))
    return J.value, dvs.value


def lbm_wenoc_set_sugar(h, S0):
    return _check("lbm_wenoc_set_sugar", load().lbm_wenoc_set_sugar(h, _ptr(S0)))


def lbm_wenoc_sugar(h, S_out):
    return _check("lbm_wenoc_sugar", load().lbm_wenoc_sugar(h, _ptr(S_out)))


def lbm_wenoc_set_class(h, k, ck):
    return _check("lbm_wenoc_set_class", load().lbm_wenoc_set_class(h, int(k), _ptr(ck)))


def lbm_wenoc_class(h, k, out):
    return _check("lbm_wenoc_class", load().lbm_wenoc_class(h, int(k), _ptr(out)))


def lbm_wenoc_class_deposit(h, k):
    out = ctypes.c_double()
    _check("lbm_wenoc_class_deposit", load().lbm_wenoc_class_deposit(h, int(k), ctypes.byref(out)))
    return out.value


def default_segment(nsteps):
    """Checkpoint spacing that minimises the stored states (checkpoints + one segment)."""
    return max(1, int(round(float(nsteps) ** 0.5)))


def lbm_wenoc_destroy(h):
    if h:
        load().lbm_wenoc_destroy(h)


# ---- convenience wrapper ---------------------------------------------------------------

def make_params(shape, tau=0.6, gravity=0.0, density_contrast=1.0, settling_velocity=0.0,
                diffusivity=0.0, lf_alpha=0.0, u_cap=0.0, body_force=(0.0, 0.0, 0.0), fp64=False,
                periodic_vertical=False, frozen_velocity=False, graphs=True, fused_rk3=False,
                sugar=False, sugar_contrast=0.0, sugar_diffusivity=0.0, phi0=0.0, vs_sugar=0.0,
                weno3=False, sign_split=False, class_vs=(), one_column=False):
    p = lbm_wenoc_params()
    p.dim = len(shape)
    p.nx, p.ny = int(shape[0]), int(shape[1])
    p.nz = int(shape[2]) if p.dim == 3 else 1
    p.tau, p.gravity, p.density_contrast = tau, gravity, density_contrast
    p.settling_velocity, p.diffusivity, p.lf_alpha, p.u_cap = settling_velocity, diffusivity, lf_alpha, u_cap
    for d in range(3):
        p.body_force[d] = float(body_force[d]) if d < len(body_force) else 0.0
    p.flags = ((LW_FP64 if fp64 else 0) | (LW_PERIODIC_VERTICAL if periodic_vertical else 0) |
               (LW_FROZEN_VELOCITY if frozen_velocity else 0) | (0 if graphs else LW_NO_GRAPH) |
               (LW_FUSED_RK3 if fused_rk3 else 0) | (LW_SUGAR if sugar else 0) | (LW_WENO3 if weno3 else 0) |
               (LW_SIGN_SPLIT if sign_split else 0) | (LW_ONE_COLUMN if one_column else 0))
    p.sugar_contrast, p.sugar_diffusivity, p.phi0, p.vs_sugar = sugar_contrast, sugar_diffusivity, phi0, vs_sugar
    p.n_classes = len(class_vs)
    for k, v in enumerate(class_vs):
        p.class_vs[k] = float(v)
    return p


class Simulation:
    """One handle plus its torch-allocated workspace on the current CUDA device.

    shape = (nx, ny) or (nx, ny, nz); fields are indexed [z][y][x] (vertical slowest).
    """

    def __init__(self, shape, stream=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lbm_wenoc needs a CUDA device; there is no CPU fallback")
        load()
        self.params = make_params(shape, **kw)
        self.dim = len(shape)
        self.grid = tuple(reversed([int(s) for s in shape]))
        self.fp64 = bool(self.params.flags & LW_FP64)
        self.dtype = torch.float64 if self.fp64 else torch.float32
        nbytes = lbm_wenoc_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = lbm_wenoc_create(self.params, self.workspace, nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            lbm_wenoc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _as_input(self, a, shape):
        import torch
        if isinstance(a, torch.Tensor):
            t = a.to(self.dtype).contiguous()
        else:
            t = torch.as_tensor(np.ascontiguousarray(a), dtype=self.dtype)
        assert tuple(t.shape) == shape or t.numel() == int(np.prod(shape)), (t.shape, shape)
        return t

    def init(self, c0, u0=None):
        c = self._as_input(c0, self.grid)
        u = None if u0 is None else self._as_input(u0, (self.dim,) + self.grid)
        self._keep = (c, u)  # host or device sources stay alive across the async copy
        lbm_wenoc_init(self.handle, c, u)

    def step(self, n=1):
        lbm_wenoc_step(self.handle, n)

    def fields(self, device="cpu"):
        import torch
        rho = torch.empty(self.grid, dtype=self.dtype, device=device)
        u = torch.empty((self.dim,) + self.grid, dtype=self.dtype, device=device)
        c = torch.empty(self.grid, dtype=self.dtype, device=device)
        lbm_wenoc_fields(self.handle, rho, u, c)
        return rho, u, c

    @property
    def deposit(self):
        return lbm_wenoc_deposited_mass(self.handle)

    @property
    def total_mass(self):
        return lbm_wenoc_total_mass(self.handle)

    def mass_below(self, level):
        """Particle mass below the horizontal plane under vertical level `level`, deposit
        included (Sec. 4.2.3, Eq. flux): J = (m(t) - m(t - dt)) / (A dt)."""
        return lbm_wenoc_mass_below(self.handle, level)

    @property
    def steps(self):
        return lbm_wenoc_steps(self.handle)

    def status(self):
        return lbm_wenoc_status(self.handle)

    def save_state(self, device="cuda"):
        """The handle's resumable state as a uint8 tensor (on `device`)."""
        import torch
        nbytes = lbm_wenoc_state_bytes(self.handle)
        out = torch.empty(nbytes, dtype=torch.uint8, device=device)
        lbm_wenoc_save_state(self.handle, out, nbytes)
        return out

    def load_state(self, state):
        """Continue from a state saved by a handle with the same parameters (a uint8 tensor
        from save_state, on any device, or a numpy byte array)."""
        nbytes = state.nbytes if isinstance(state, np.ndarray) else state.numel() * state.element_size()
        lbm_wenoc_load_state(self.handle, state, nbytes)

    def set_sugar(self, S0):
        """Sugar field of a sugar=True handle (after init)."""
        S = self._as_input(S0, self.grid)
        lbm_wenoc_set_sugar(self.handle, S)

    def sugar(self, device="cpu"):
        import torch
        S = torch.empty(self.grid, dtype=self.dtype, device=device)
        lbm_wenoc_sugar(self.handle, S)
        return S

    def set_class(self, k, ck):
        """Particle class k of a polydisperse handle (after init)."""
        lbm_wenoc_set_class(self.handle, k, self._as_input(ck, self.grid))

    def class_field(self, k, device="cpu"):
        import torch
        out = torch.empty(self.grid, dtype=self.dtype, device=device)
        lbm_wenoc_class(self.handle, k, out)
        return out

    def class_deposit(self, k):
        return lbm_wenoc_class_deposit(self.handle, k)

    def deposit_gradient(self, c0, nsteps, segment=None):
        """Run nsteps from c0 (fluid at rest) and return (J, dJ/dc0, dJ/dVs): J the
        deposited mass, dJ/dc0 a device tensor of the grid's shape.  The handle must be
        initialised again before further stepping."""
        import torch
        segment = default_segment(nsteps) if segment is None else int(segment)
        c = self._as_input(c0, self.grid)
        nbytes = lbm_wenoc_gradient_workspace_bytes(self.params, nsteps, segment)
        adj = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        grad = torch.empty(self.grid, dtype=self.dtype, device="cuda")
        self._keep = (c, None)
        J, dvs = lbm_wenoc_deposit_gradient(self.handle, c, nsteps, segment, adj, nbytes, grad)
        return J, grad, dvs


# ---- batched simulations ---------------------------------------------------------------

def lbm_wenoc_batch_workspace_bytes(params_list):
    arr = (lbm_wenoc_params * len(params_list))(*params_list)
    n = ctypes.c_size_t(0)
    _check("lbm_wenoc_batch_workspace_bytes",
           load().lbm_wenoc_batch_workspace_bytes(arr, len(params_list), ctypes.byref(n)))
    return n.value


def lbm_wenoc_batch_create(params_list, workspace, nbytes, stream):
    arr = (lbm_wenoc_params * len(params_list))(*params_list)
    h = ctypes.c_void_p()
    _check("lbm_wenoc_batch_create", load().lbm_wenoc_batch_create(arr, len(params_list), _ptr(workspace), nbytes,
                                                                   stream, ctypes.byref(h)))
    return h


def lbm_wenoc_batch_instance(b, i):
    return ctypes.c_void_p(load().lbm_wenoc_batch_instance(b, int(i)))


def lbm_wenoc_batch_step(b, nsteps):
    return _check("lbm_wenoc_batch_step", load().lbm_wenoc_batch_step(b, int(nsteps)))


def lbm_wenoc_batch_autotune(b, count, steps_per_trial=4):
    """Segment heights chosen for the `count` instances (a list)."""
    rows = (ctypes.c_int32 * count)()
    _check("lbm_wenoc_batch_autotune", load().lbm_wenoc_batch_autotune(b, int(steps_per_trial), rows))
    return list(rows)


def lbm_wenoc_batch_set_persistent(b, persistent=True):
    """True/1: one persistent launch per graph of steps; 2: grouped fluid launch + persistent
    stage launch per step; False/0: grouped launches."""
    mode = int(persistent) if not isinstance(persistent, bool) else (1 if persistent else 0)
    return _check("lbm_wenoc_batch_set_persistent", load().lbm_wenoc_batch_set_persistent(b, mode))


def lbm_wenoc_batch_set_wait_limit(b, cycles, skip_cta=-1):
    return _check("lbm_wenoc_batch_set_wait_limit", load().lbm_wenoc_batch_set_wait_limit(b, int(cycles),
                                                                                         int(skip_cta)))


def lbm_wenoc_batch_status(b):
    """LW_OK, LW_ETIMEOUT or an instance's status code (not raised)."""
    return load().lbm_wenoc_batch_status(b)


def lbm_wenoc_batch_launch_count(b):
    return load().lbm_wenoc_batch_launch_count(b)


def lbm_wenoc_batch_destroy(b):
    if b:
        load().lbm_wenoc_batch_destroy(b)


class _Instance:
    """View of one instance of a Batch (same methods as Simulation, no own workspace)."""

    def __init__(self, batch, i, shape, fp64=False):
        import torch
        self.handle = lbm_wenoc_batch_instance(batch.handle, i)
        self.dim = len(shape)
        self.grid = tuple(reversed([int(s) for s in shape]))
        self.fp64 = fp64
        self.dtype = torch.float32

    init = Simulation.init
    _as_input = Simulation._as_input
    fields = Simulation.fields
    deposit = Simulation.deposit
    total_mass = Simulation.total_mass
    steps = Simulation.steps
    status = Simulation.status


class Batch:
    """Many 2D FP32 simulations (shapes and parameters per instance) advanced together.

    specs: list of dicts with 'shape' and the keyword parameters of make_params."""

    def __init__(self, specs, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lbm_wenoc needs a CUDA device; there is no CPU fallback")
        load()
        self.params = [make_params(sp["shape"], **{k: v for k, v in sp.items() if k != "shape"}) for sp in specs]
        nbytes = lbm_wenoc_batch_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = lbm_wenoc_batch_create(self.params, self.workspace, nbytes, self.stream.cuda_stream)
        self.instances = [_Instance(self, i, sp["shape"]) for i, sp in enumerate(specs)]

    def autotune(self, steps_per_trial=4):
        return lbm_wenoc_batch_autotune(self.handle, len(self.instances), steps_per_trial)

    def set_persistent(self, persistent=True):
        lbm_wenoc_batch_set_persistent(self.handle, persistent)

    def status(self):
        return lbm_wenoc_batch_status(self.handle)

    def step(self, n=1):
        lbm_wenoc_batch_step(self.handle, n)

    def close(self):
        if getattr(self, "handle", None):
            lbm_wenoc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
