"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a, loads,
exports every entry point include/lsb.h declares, and carries the same velocity
sets as the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.lattice import D2Q9, D3Q19, D3Q27

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_05936_gb300 import build, lsb
    build.build()
    return lsb.load()


def test_header_symbols_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "lsb.h")).read()
    names = set(re.findall(r"\b(lsb_[a-z_]+)\s*\(", hdr))
    assert {"lsb_create_grid", "lsb_set_params", "lsb_step", "lsb_refine", "lsb_get_fields",
            "lsb_backward"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


@pytest.mark.parametrize("code,lat", [(0, D2Q9), (1, D3Q19), (2, D3Q27)], ids=["D2Q9", "D3Q19", "D3Q27"])
def test_lattice_tables_match_oracle(lib, code, lat):
    from paper_2601_05936_gb300 import lsb
    c, w, opp = lsb.lattice_table(code)
    assert c.shape[0] == lat.Q
    assert np.array_equal(c[:, :lat.D], lat.c)
    assert np.allclose(w, lat.w, rtol=1e-7)
    assert np.array_equal(opp, lat.opp)


def test_create_rejects_bad_input_without_gpu(lib):
    from paper_2601_05936_gb300 import lsb
    out = ctypes.c_void_p()
    st = lib.lsb_create_grid(0, None, None, None, None, ctypes.byref(out))
    assert st == 1 and not out.value
    assert b"n_cases" in lib.lsb_last_error(None)


def test_status_codes_match_header():
    from paper_2601_05936_gb300 import lsb
    hdr = open(os.path.join(ROOT, "include", "lsb.h")).read()
    for code, name in lsb.STATUS.items():
        assert re.search(rf"{name}\s*=\s*{code}\b", hdr), name


def test_autotune_rejects_bad_input_without_gpu(lib):
    best = (ctypes.c_int * 3)()
    st = lib.lsb_autotune(1, None, None, None, None, None, 0, 10, best, None)
    assert st == 1
    assert b"autotune" in lib.lsb_last_error(None)
