"""The C-ABI library builds, loads and exports every entry point include/rtcc.h declares."""
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
