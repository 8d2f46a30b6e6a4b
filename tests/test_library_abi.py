"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports every
symbol the header declares, and its host-only parameter validation behaves.
No kernel is launched here (no GPU in this environment)."""
import ctypes
import os
import re

import pytest

from paper_2106_07694_gb300 import build as lbuild
from paper_2106_07694_gb300 import lbm_wenoc as lw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbuild.build()
    return lw.load()


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_wenoc_\w+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("lbm_wenoc_create", "lbm_wenoc_init", "lbm_wenoc_step",
                     "lbm_wenoc_deposited_mass", "lbm_wenoc_destroy"):
        assert required in names


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as C99 on its own (no C++ or CUDA types leak into it)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "lbm_wenoc.h"\nint main(void) { lbm_wenoc_params p = {0}; '
                   'size_t b = 0; return lbm_wenoc_workspace_bytes(&p, &b) == LW_OK; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_workspace_bytes_and_validation(lib):
    p = lw.make_params((128, 256), gravity=1e-5, settling_velocity=1e-3, diffusivity=1e-3, fp64=True)
    n = lw.lbm_wenoc_workspace_bytes(p)
    nodes = 128 * 256
    # populations + c + two stage fields + velocity, FP64
    assert n >= (9 + 3 + 2) * 8 * nodes
    assert n < (9 + 3 + 2) * 8 * nodes + 64 * 1024
    p32 = lw.make_params((2048, 4096))
    assert lw.lbm_wenoc_workspace_bytes(p32) >= (9 + 5) * 4 * 2048 * 4096
    p3 = lw.make_params((256, 256, 512))
    assert lw.lbm_wenoc_workspace_bytes(p3) >= (19 + 6) * 4 * 256 * 256 * 512
    for bad in (dict(tau=0.5), dict(tau=0.4), dict(settling_velocity=-1.0), dict(diffusivity=-1e-3)):
        with pytest.raises(lw.LbmWenocError) as e:
            lw.lbm_wenoc_workspace_bytes(lw.make_params((128, 256), **bad))
        assert e.value.code == lw.LW_EINVAL
    for shape in ((130, 256), (128, 2), (2, 128), (64, 64, 2)):
        with pytest.raises(lw.LbmWenocError):
            lw.lbm_wenoc_workspace_bytes(lw.make_params(shape))


def test_create_rejects_small_or_misaligned_workspace(lib):
    p = lw.make_params((128, 256))
    need = lw.lbm_wenoc_workspace_bytes(p)
    h = ctypes.c_void_p()
    rc = lib.lbm_wenoc_create(ctypes.byref(p), ctypes.c_void_p(4096 * 1024), need - 1, None, ctypes.byref(h))
    assert rc == lw.LW_ENOMEM and not h.value
    rc = lib.lbm_wenoc_create(ctypes.byref(p), ctypes.c_void_p(4096 * 1024 + 16), need, None, ctypes.byref(h))
    assert rc == lw.LW_EINVAL and not h.value
    rc = lib.lbm_wenoc_step(None, 1)
    assert rc == lw.LW_EINVAL


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(lw, "_lib", None)
    monkeypatch.setattr(lw, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        lw.load()


def test_state_and_batch_calls_reject_null_handles(lib):
    out = ctypes.c_size_t()
    assert lib.lbm_wenoc_state_bytes(None, ctypes.byref(out)) == lw.LW_EINVAL
    assert lib.lbm_wenoc_save_state(None, ctypes.c_void_p(4096), ctypes.c_size_t(1 << 20)) == lw.LW_EINVAL
    assert lib.lbm_wenoc_load_state(None, ctypes.c_void_p(4096), ctypes.c_size_t(1 << 20)) == lw.LW_EINVAL
    for mode in (0, 1, 2, 3, -1):
        assert lib.lbm_wenoc_batch_set_persistent(None, mode) == lw.LW_EINVAL
