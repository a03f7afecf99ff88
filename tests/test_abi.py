"""The C-ABI library builds for sm_103a, loads, exports every entry point
include/letkf.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import shutil

import numpy as np
import pytest

from paper_1408_7069_gb300 import letkf as L


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(L.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libletkf.so")
        from paper_1408_7069_gb300.build import build_library
        build_library()
    return L.lib()


def test_header_declares_the_boundary():
    names = L.header_symbols()
    for required in ("letkf_create", "letkf_destroy", "letkf_forecast", "letkf_analyze",
                     "letkf_run", "letkf_get_state", "letkf_set_state", "letkf_query",
                     "letkf_last_error", "letkf_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    for name in L.header_symbols():
        assert hasattr(built, name), name


def test_config_struct_layout_matches_c(tmp_path):
    """The ctypes mirror of letkf_config has the C compiler's layout: every
    field's offset and the size, printed by a C program built against
    include/letkf.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [n for n, _ in L.letkf_config._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"letkf.h\"\nint main(void) {\n"
                   + "".join(f'  printf("{n} %zu\\n", offsetof(letkf_config, {n}));\n'
                             for n in fields)
                   + '  printf("size %zu\\n", sizeof(letkf_config));\n  return 0;\n}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(L.HEADER))
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for n in fields:
        assert getattr(L.letkf_config, n).offset == int(out[n]), n
    assert ctypes.sizeof(L.letkf_config) == int(out["size"])


def _cfg(mask, **kw):
    c = L.letkf_config()
    c.nsub = mask.shape[0]
    c.subap_mask = mask.ctypes.data
    c.m, c.window, c.taper, c.rho, c.sigma2 = 8, 3, 0, 1.0, 0.01
    c.a_ar1, c.noise_std, c.precision = 0.99, 0.1, 0
    for k, v in kw.items():
        setattr(c, k, v)
    return c


@pytest.mark.parametrize("bad", [dict(m=1), dict(m=65), dict(m=33, precision=1), dict(window=0), dict(window=32),
                                 dict(taper=2), dict(rho=0.0), dict(sigma2=-1.0),
                                 dict(precision=3), dict(nsub=0), dict(rho=float("nan"))])
def test_create_rejects_bad_arguments(built, bad):
    mask = np.ones((4, 4), np.uint8)
    h = ctypes.c_void_p()
    st = built.letkf_create(ctypes.byref(_cfg(mask, **bad)), None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert L.letkf_last_error(None)


def test_create_rejects_empty_mask_and_null_pointers(built):
    mask = np.zeros((4, 4), np.uint8)
    h = ctypes.c_void_p()
    assert built.letkf_create(ctypes.byref(_cfg(mask)), None, ctypes.byref(h)) in (1, 2)
    assert built.letkf_create(None, None, ctypes.byref(h)) == 1
    assert built.letkf_create(ctypes.byref(_cfg(np.ones((4, 4), np.uint8))), None, None) == 1
    cfg = _cfg(np.ones((4, 4), np.uint8))
    cfg.subap_mask = None
    assert built.letkf_create(ctypes.byref(cfg), None, ctypes.byref(h)) == 1


def test_null_handle_calls_fail_cleanly(built):
    assert built.letkf_destroy(None) == 0
    assert built.letkf_query(None, None, None, None) == 1
    assert built.letkf_analyze(None, None, None, None) == 1
    assert built.letkf_forecast(None, None) == 1
    assert built.letkf_sync(None) == 1
    assert built.letkf_set_params(None, 0, 1.0, 1.0, 1.0) == 1
    assert built.letkf_set_frame(None, 0) == 1
    assert built.letkf_set_jacobi(None, 4e-6, 1e-3) == 1
    assert built.letkf_grad(None, 1, None, None, 0, None, None) == 1
