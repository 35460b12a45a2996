"""CPU-side checks of the C ABI library: it builds, loads, exports every
function declared in include/brillouin.h, and validates arguments before it
touches a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "brillouin.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bri_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1012_3615_gb300 import abi, build

    build.build()
    return abi.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_1012_3615_gb300 import abi

    names = _declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", abi.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(bri_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(abi.SIGNATURES) == set(names)


def test_create_validates_arguments_without_gpu(lib):
    from paper_1012_3615_gb300 import abi

    h = ctypes.c_void_p()
    assert lib.bri_create(None, ctypes.byref(h)) == abi.BRI_EINVAL
    bad = abi.bri_lattice((ctypes.c_int * 4)(4, 4, 2, 4), (ctypes.c_int * 4)(1, 1, 1, -1))
    assert lib.bri_create(ctypes.byref(bad), ctypes.byref(h)) == abi.BRI_EINVAL
    assert b"extents" in lib.bri_last_error(None)
    bad_bc = abi.bri_lattice((ctypes.c_int * 4)(4, 4, 4, 4), (ctypes.c_int * 4)(1, 1, 2, -1))
    assert lib.bri_create(ctypes.byref(bad_bc), ctypes.byref(h)) == abi.BRI_EINVAL
    # null contexts are rejected, not dereferenced
    assert lib.bri_apply(None, None, None, 1, 0.0, 0, 0, None) == abi.BRI_EINVAL
    assert lib.bri_destroy(None) == abi.BRI_OK
    assert lib.bri_kernel_launches(None) == 0


def test_python_binding_names_match_abi():
    from paper_1012_3615_gb300 import abi

    for n in _declared():
        assert n in abi.SIGNATURES


def test_noalloc_validates_pointers_without_gpu(lib):
    """bri_build_hops_noalloc rejects null and misaligned pointers before any
    CUDA call (the pointer values below are never dereferenced)."""
    from paper_1012_3615_gb300 import abi

    lat = abi.bri_lattice((ctypes.c_int * 4)(4, 4, 4, 4), (ctypes.c_int * 4)(1, 1, 1, -1))
    assert lib.bri_build_hops_noalloc(None, 256, 512, None) == abi.BRI_EINVAL
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), None, 512, None) == abi.BRI_EINVAL
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), 256, None, None) == abi.BRI_EINVAL
    assert b"null" in lib.bri_last_error(None)
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), 256, 520, None) == abi.BRI_EINVAL
    assert lib.bri_build_hops_noalloc(ctypes.byref(lat), 264, 512, None) == abi.BRI_EINVAL
    assert b"aligned" in lib.bri_last_error(None)


def test_new_entry_points_validate_without_gpu(lib):
    """The entry points added with the FP16 spinors, the pseudofermion action
    and the ALU peaks reject bad arguments before any CUDA call."""
    from paper_1012_3615_gb300 import abi

    # one right-hand side of the FP16-spinor storage: 48 V + 4 V rounded up to 16
    assert lib.bri_h16_field_bytes(81) == 48 * 81 + 336
    assert lib.bri_h16_field_bytes(256) == 48 * 256 + 1024
    assert lib.bri_h16_field_bytes(0) == 0
    assert lib.bri_convert_spinor(None, 256, abi.BRI_F16H, 512, abi.BRI_F32, 1, None) == abi.BRI_EINVAL
    assert lib.bri_inverse_action(None, None, None, None, 256, 0.0, 1e-10, 100, None, None) == abi.BRI_EINVAL
    v = ctypes.c_double()
    assert lib.bri_alu_peak(7, ctypes.byref(v)) == abi.BRI_EINVAL
    assert lib.bri_alu_peak(abi.BRI_F32, None) == abi.BRI_EINVAL
    assert b"prec" in lib.bri_last_error(None)
    assert lib.bri_debug_stall(None, 1) == abi.BRI_EINVAL
