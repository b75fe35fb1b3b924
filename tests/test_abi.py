"""The C-ABI library builds, loads and exports every entry point include/rtcc.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtcc.h")
LIB = os.path.join(ROOT, "paper_2205_05175_gb300", "librtcc.so")


def declared_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rtcc_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2205_05175_gb300 import build
        build.build()
    from paper_2205_05175_gb300 import rtcc
    return rtcc


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["rtcc_create", "rtcc_destroy", "rtcc_ground_state", "rtcc_propagate", "rtcc_spectrum",
              "rtcc_rhs", "rtcc_dipole", "rtcc_get_state", "rtcc_set_state", "rtcc_state_size", "rtcc_last_error"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rtcc_[a-z_0-9]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    assert set(lib.EXPORTED) == set(declared_symbols())


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    import numpy as np
    f = np.eye(3)
    B = np.zeros((2, 3, 3))
    mu = np.zeros((3, 3, 3))
    with pytest.raises(lib.RtccError) as e:
        lib.Handle(f, B, mu, 0, 3)   # o = 0
    assert e.value.status == "INVALID_ARG"
    fa = f.copy()
    fa[0, 1] = 1.0
    with pytest.raises(lib.RtccError) as e:
        lib.Handle(fa, B, mu, 1, 2)
    assert e.value.status == "INVALID_ARG"
    assert "symmetric" in lib.rtcc_last_error()


def test_no_cpu_fallback_in_product_package():
    pkg = os.path.join(ROOT, "paper_2205_05175_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn


def test_frozen_core_count_is_checked_before_any_device_work(lib):
    import numpy as np
    o, v = 2, 2
    f = np.diag([-1.0, -0.5, 0.5, 1.0])
    B = np.zeros((2, 4, 4))
    mu = np.zeros((3, 4, 4))
    for nfc in (-1, o, o + 3):
        with pytest.raises(lib.RtccError) as e:
            lib.Handle(f, B, mu, o, v, nfc=nfc)
        assert e.value.status == "INVALID_ARG"
        assert "frozen-core" in lib.rtcc_last_error()


LAYOUT_C = r"""
#include <stdio.h>
#include "rtcc.h"
#define F(S, m) printf(#S " " #m " %zu %zu\n", offsetof(S, m), sizeof(((S*)0)->m))
int main(void) {
  F(rtcc_field_t, E0); F(rtcc_field_t, omega); F(rtcc_field_t, sigma); F(rtcc_field_t, t0);
  F(rtcc_field_t, pol); F(rtcc_field_t, carrier); F(rtcc_field_t, sign);
  F(rtcc_integrator_t, method); F(rtcc_integrator_t, h); F(rtcc_integrator_t, h1); F(rtcc_integrator_t, h2);
  F(rtcc_integrator_t, t_switch); F(rtcc_integrator_t, tol); F(rtcc_integrator_t, safety);
  F(rtcc_integrator_t, h_min); F(rtcc_integrator_t, h_max); F(rtcc_integrator_t, max_rejects);
  F(rtcc_integrator_t, nsteps); F(rtcc_integrator_t, t_end); F(rtcc_integrator_t, sweeps);
  F(rtcc_integrator_t, krylov);
  F(rtcc_profile_t, launches); F(rtcc_profile_t, ms); F(rtcc_profile_t, flops); F(rtcc_profile_t, bytes);
  printf("sizeof rtcc_field_t %zu\nsizeof rtcc_integrator_t %zu\nsizeof rtcc_profile_t %zu\n",
         sizeof(rtcc_field_t), sizeof(rtcc_integrator_t), sizeof(rtcc_profile_t));
  printf("enum %d %d %d %d %d %d %d %d %d %d %d\n", RTCC_RK4, RTCC_CK, RTCC_MIXED_RK4, RTCC_GL2, RTCC_GL2_NEWTON, RTCC_P64,
         RTCC_P32_TF32, RTCC_P32_3XTF32, RTCC_P32_BF16X3, RTCC_CARRIER_SIN, RTCC_CARRIER_COS);
  printf("status %d %d %d %d %d %d %d %d %d\n", RTCC_OK, RTCC_ERR_INVALID_ARG, RTCC_ERR_OOM, RTCC_ERR_CUDA,
         RTCC_ERR_NOCONV, RTCC_ERR_DIVERGED, RTCC_ERR_STEP_UNDERFLOW, RTCC_ERR_TIMEOUT, RTCC_ERR_UNSUPPORTED);
  return 0;
}
"""


def test_struct_layouts_and_enums_match_the_header(lib, tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's offsets and sizes, and the
    binding's constants the header's enum values (a field added on one side only fails here)."""
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text(LAYOUT_C)
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    mirrors = {"rtcc_field_t": lib.rtcc_field_t, "rtcc_integrator_t": lib.rtcc_integrator_t,
               "rtcc_profile_t": lib.rtcc_profile_t}
    seen = {k: [] for k in mirrors}
    for line in out:
        w = line.split()
        if w[0] == "sizeof":
            assert int(w[2]) == ctypes.sizeof(mirrors[w[1]]), line
        elif w[0] == "enum":
            assert [int(x) for x in w[1:]] == [lib.RK4, lib.CK, lib.MIXED_RK4, lib.GL2, lib.GL2_NEWTON, lib.P64, lib.P32_TF32,
                                               lib.P32_3XTF32, lib.P32_BF16X3, lib.CARRIER_SIN, lib.CARRIER_COS]
        elif w[0] == "status":
            names = ["OK", "INVALID_ARG", "OOM", "CUDA", "NOCONV", "DIVERGED", "STEP_UNDERFLOW", "TIMEOUT", "UNSUPPORTED"]
            assert {int(x): n for x, n in zip(w[1:], names)} == lib.STATUS
        else:
            S, m, off, size = w[0], w[1], int(w[2]), int(w[3])
            field = getattr(mirrors[S], m)
            assert (field.offset, field.size) == (off, size), line
            seen[S].append(m)
    for S, cls in mirrors.items():
        assert seen[S] == [f[0] for f in cls._fields_], S


def test_pade_spectrum_arguments_are_checked_before_any_device_work(lib):
    import numpy as np
    om = np.linspace(0.1, 1.0, 5)
    fld = lib.make_field()
    t = 0.1 * np.arange(11)
    t[5] += 0.01                                   # not uniform
    with pytest.raises(lib.RtccError) as e:
        lib.rtcc_spectrum_pade(t, np.zeros((11, 3)), fld, om, kappa=1.0)
    assert e.value.status == "INVALID_ARG" and "uniformly" in lib.rtcc_last_error()
    t = 0.1 * np.arange(1027)                      # M = 513, one above the largest order (512)
    with pytest.raises(lib.RtccError) as e:
        lib.rtcc_spectrum_pade(t, np.zeros((1027, 3)), fld, om, kappa=1.0)
    assert e.value.status == "INVALID_ARG" and "1025" in lib.rtcc_last_error()
    with pytest.raises(lib.RtccError) as e:
        lib.rtcc_spectrum_pade(t[:2], np.zeros((2, 3)), fld, om, kappa=1.0)
    assert e.value.status == "INVALID_ARG"


def test_binding_refuses_to_import_without_the_library(tmp_path):
    """No CPU fallback: a copy of the package without librtcc.so raises ImportError on import."""
    import shutil
    import sys
    pkg = tmp_path / "paper_2205_05175_gb300"
    pkg.mkdir()
    src = os.path.join(ROOT, "paper_2205_05175_gb300")
    for fn in os.listdir(src):
        if fn.endswith(".py"):
            shutil.copy(os.path.join(src, fn), pkg / fn)
    code = "import paper_2205_05175_gb300.rtcc"
    r = subprocess.run([sys.executable, "-c", code], cwd=str(tmp_path), capture_output=True, text=True,
                       env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0 and "ImportError" in r.stderr and "librtcc.so is missing" in r.stderr


def test_noalloc_binding_rejects_bad_tensors_before_the_device(lib):
    """rtcc_gemm_noalloc hands raw pointers to the library, so the binding refuses wrong dtypes,
    shapes and devices with ValueError (CPU tensors here: nothing reaches a GPU)."""
    import torch
    ok_a = torch.zeros((2, 5, 7), dtype=torch.float64)
    ok_b = torch.zeros((2, 3, 7), dtype=torch.float64)
    ok_c = torch.zeros((2, 5, 3), dtype=torch.float64)
    bad = [
        (ok_a, ok_b, torch.zeros((2, 5, 3), dtype=torch.complex64)),           # complex64 output
        (ok_a.float(), ok_b, ok_c),                                             # float32 input
        (ok_a.to(torch.complex64), ok_b, ok_c),                                 # complex64 input
        (ok_a, torch.zeros((2, 3, 6), dtype=torch.float64), ok_c),              # B's K differs
        (ok_a, torch.zeros((1, 3, 7), dtype=torch.float64), ok_c),              # B's batch differs
        (ok_a, ok_b, torch.zeros((2, 5, 4), dtype=torch.float64)),              # output shape
        (ok_a.to(torch.complex128), ok_b, ok_c),                                # complex input, real output
        (ok_a, ok_b, ok_c.to(torch.complex128)),                                # real inputs, complex output
        (ok_a.transpose(1, 2).contiguous().transpose(1, 2), ok_b, ok_c),        # not contiguous
        (ok_a, ok_b, ok_c),                                                     # right shapes, host memory
    ]
    for a, b, c in bad:
        with pytest.raises(ValueError):
            lib.rtcc_gemm_noalloc(3, a, b, c)
