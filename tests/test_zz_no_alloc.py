"""lsb_get_fields_noalloc: the allocation-free field export.

For callers that cannot allocate device memory when they read results (their
device memory belongs to another allocator, or an allocation's latency and
implicit synchronisation are not acceptable in their loop), the library
offers a variant of lsb_get_fields that stages the exported field in a fixed
16 MiB array instead of a temporary cudaMalloc buffer.  These tests call it
through the C ABI and check its output against lsb_get_fields on two calls in
a row, and that a field too large for the fixed array is rejected.  The file
name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(g, field, level=None, case_idx=0):
    from paper_2601_05936_gb300 import lsb
    c = g.cases[case_idx]
    level = int(c.get("n_levels", 1)) - 1 if level is None else level
    code = lsb.FIELD[field]
    nbytes = g.lib.lsb_field_bytes(g.h, case_idx, code, level)
    out = np.empty(nbytes // 4, dtype=np.float32)
    st = g.lib.lsb_get_fields_noalloc(g.h, case_idx, code, level, out.ctypes.data, nbytes, 1)
    return st, out


def _grid(lattice, n, steps):
    from paper_2601_05936_gb300 import lsb
    D = 2 if lattice == "D2Q9" else 3
    base = (n,) * D
    x = np.arange(n) + 0.5
    mesh = np.meshgrid(*([x] * D), indexing="ij")[::-1]
    r = np.sqrt(sum((m - n / 2) ** 2 for m in mesh))
    case = dict(lattice=lattice, base=base, block=(32, 8) if D == 2 else (32, 4, 4),
                periodic=(False,) * D, rho_phys=(1.0, 0.1), nu=(0.1, 0.1), sigma=1e-3,
                gravity=(0.0,) * (D - 1) + (-1e-6,), x_ref=(n / 2,) * D, phi0=(n / 5 - r).reshape(-1))
    g = lsb.Grid(case)
    g.step(steps)
    return g


@pytest.mark.parametrize("lattice,n", [("D2Q9", 64), ("D3Q19", 32)])
def test_noalloc_export_matches_get_fields_twice(lattice, n):
    g = _grid(lattice, n, 5)
    for field in ("rho", "u", "f"):
        want = g.get(field).reshape(-1)
        for _ in range(2):  # two calls in a row share the staging array
            st, got = _noalloc(g, field)
            assert st == 0, g.lib.lsb_last_error(g.h)
            assert np.allclose(got, want, rtol=1e-6, atol=1e-7), field
    g.step(3)  # the state moves on; the staged copy must follow
    want = g.get("u").reshape(-1)
    st, got = _noalloc(g, "u")
    assert st == 0 and np.allclose(got, want, rtol=1e-6, atol=1e-7)
    g.close()


def test_noalloc_rejects_fields_larger_than_its_array():
    g = _grid("D3Q19", 64, 1)  # f: 19 x 64^3 floats = 19.9 MB > 16 MiB
    st, _ = _noalloc(g, "rho")
    assert st == 0
    code = 4
    nbytes = g.lib.lsb_field_bytes(g.h, 0, code, 0)
    buf = (ctypes.c_char * nbytes)()
    st = g.lib.lsb_get_fields_noalloc(g.h, 0, code, 0, ctypes.addressof(buf), nbytes, 1)
    assert st == 1
    assert b"staging array" in g.lib.lsb_last_error(g.h)
    g.close()


def test_noalloc_allocates_nothing_and_exports_to_device_memory():
    """After the first call (which resolves the fixed array's address and loads the export
    kernel), repeated calls leave the device's free memory unchanged; a device destination
    (a torch CUDA tensor, dst_on_host = 0) receives the same values as lsb_get_fields."""
    import torch
    from paper_2601_05936_gb300 import lsb
    g = _grid("D3Q19", 32, 4)
    code = lsb.FIELD["f"]
    nbytes = g.lib.lsb_field_bytes(g.h, 0, code, 0)
    dst = torch.zeros(nbytes // 4, dtype=torch.float32, device="cuda")
    host = np.empty(nbytes // 4, dtype=np.float32)
    assert g.lib.lsb_get_fields_noalloc(g.h, 0, code, 0, ctypes.c_void_p(dst.data_ptr()), nbytes, 0) == 0
    assert g.lib.lsb_get_fields_noalloc(g.h, 0, code, 0, host.ctypes.data, nbytes, 1) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        dst.zero_()
        st = g.lib.lsb_get_fields_noalloc(g.h, 0, code, 0, ctypes.c_void_p(dst.data_ptr()), nbytes, 0)
        assert st == 0, g.lib.lsb_last_error(g.h)
        assert g.lib.lsb_get_fields_noalloc(g.h, 0, code, 0, host.ctypes.data, nbytes, 1) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    want = g.get("f").reshape(-1)
    assert np.allclose(dst.cpu().numpy(), want, rtol=1e-6, atol=1e-7)
    assert np.array_equal(dst.cpu().numpy(), host)
    g.close()
