"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/bsp.h, and rejects bad arguments before touching CUDA."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_05303_gb300 import build, bsp

    build.build()
    return bsp.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bsp_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_1708_05303_gb300 import bsp

    decl = declared_symbols()
    assert "bsp_compute" in decl and "bsp_counts" in decl
    for name in decl:
        assert hasattr(lib, name), name
    assert set(bsp.EXPORTS) == decl


def test_version_and_strings(lib):
    from paper_1708_05303_gb300 import bsp

    assert bsp.bsp_version() >= 100
    assert lib.bsp_status_string(-1) == b"invalid argument"
    assert lib.bsp_status_string(0) == b"ok"


@pytest.mark.parametrize("kwargs", [
    dict(n=63, box=1000.0, edges=[1, 3], ells=(0,)),          # odd n
    dict(n=14, box=1000.0, edges=[1, 3], ells=(0,)),          # 7 is not a radix
    dict(n=64, box=-1.0, edges=[1, 3], ells=(0,)),            # box
    dict(n=64, box=1000.0, edges=[3, 1], ells=(0,)),          # edges not ascending
    dict(n=64, box=1000.0, edges=[0, 1], ells=(0,)),          # edge 0
    dict(n=64, box=1000.0, edges=[1, 60], ells=(0,)),         # beyond sqrt(3) n / 2
    dict(n=64, box=1000.0, edges=[1, 3], ells=(1,)),          # odd l
    dict(n=64, box=1000.0, edges=[1, 3], ells=(2, 0)),        # not ascending
    dict(n=64, box=1000.0, edges=[1, 3], ells=(0, 2, 4, 6)),  # too many / l = 6
    dict(n=1024, box=1000.0, edges=[1, 3], ells=(0,)),        # too large for this build
])
def test_bad_arguments_rejected_on_host(lib, kwargs):
    from paper_1708_05303_gb300 import bsp

    with pytest.raises(bsp.BspError) as ei:
        bsp.bsp_plan_create(kwargs["n"], kwargs["box"], kwargs["edges"], kwargs["ells"])
    assert ei.value.status == bsp.BSP_EINVAL


def test_null_arguments(lib):
    import ctypes

    from paper_1708_05303_gb300 import bsp

    assert lib.bsp_workspace_size(None, None) == bsp.BSP_EINVAL
    assert lib.bsp_counts(None, None, None) == bsp.BSP_EINVAL
    assert lib.bsp_compute(None, None, 0.0, None, None, None) == bsp.BSP_EINVAL
    n = ctypes.c_int()
    assert lib.bsp_plan_bins(None, ctypes.byref(n), None, None) == bsp.BSP_EINVAL
    lib.bsp_plan_destroy(None)


def test_null_arguments_of_the_spectra_entry_points(lib):
    # power, density, skew and integrated-bispectrum calls reject missing
    # handles and bad sizes on the host, before any CUDA call
    import ctypes

    from paper_1708_05303_gb300 import bsp

    nb = ctypes.c_size_t()
    assert lib.bsp_power_compute(None, None, 0.0, None, None, None, None) == bsp.BSP_EINVAL
    assert lib.bsp_skew_workspace_size(None, ctypes.byref(nb)) == bsp.BSP_EINVAL
    assert lib.bsp_skew_compute(None, None, None, 0, None, None, None) == bsp.BSP_EINVAL
    assert lib.bsp_ib_workspace_size(None, 8, ctypes.byref(nb)) == bsp.BSP_EINVAL
    assert lib.bsp_ib_compute(None, None, 8, None, 0, None, None, None) == bsp.BSP_EINVAL
    for n in (63, 14, 6):   # odd, a radix of 7, too small
        assert lib.bsp_density_workspace_size(n, ctypes.byref(nb)) == bsp.BSP_EINVAL
    assert lib.bsp_density_workspace_size(64, None) == bsp.BSP_EINVAL
    assert lib.bsp_density_workspace_size(64, ctypes.byref(nb)) == bsp.BSP_OK
    # two FP32 grids and two half spectra at least
    assert nb.value >= 2 * 64 ** 3 * 4 + 2 * 64 * 64 * 33 * 8
    assert lib.bsp_density_cic(64, 1000.0, 0, None, None, 0, None, None, None) == bsp.BSP_EINVAL


def test_static_triple_sums_reject_on_host(lib):
    # the allocation-free entry point checks sizes and indices before any CUDA
    # call, so fake (never dereferenced) device addresses are enough here
    import ctypes

    import numpy as np

    from paper_1708_05303_gb300 import bsp

    fake_fields, fake_T = 1 << 20, 1 << 21
    f = lib.bsp_triple_sums_static
    ok = np.zeros((4, 3), dtype=np.int32)
    assert f(fake_fields, 4096, 2, None, 4, fake_T, None) == bsp.BSP_EINVAL       # no triplets
    assert f(None, 4096, 2, ok.ctypes.data, 4, fake_T, None) == bsp.BSP_EINVAL     # no fields
    assert f(fake_fields + 4, 4096, 2, ok.ctypes.data, 4, fake_T, None) == bsp.BSP_EINVAL   # unaligned
    assert f(fake_fields, 4096, 2, ok.ctypes.data, 0, fake_T, None) == bsp.BSP_EINVAL       # empty
    bad = ok.copy()
    bad[3, 2] = 2                                                                  # index == nfields
    assert f(fake_fields, 4096, 2, bad.ctypes.data, 4, fake_T, None) == bsp.BSP_EINVAL
    bad[3, 2] = -1
    assert f(fake_fields, 4096, 2, bad.ctypes.data, 4, fake_T, None) == bsp.BSP_EINVAL
    big = np.zeros((131073, 3), dtype=np.int32)                                    # above the fixed scratch
    assert f(fake_fields, 4096, 2, big.ctypes.data, 131073, fake_T, None) == bsp.BSP_EINVAL
    del ctypes
