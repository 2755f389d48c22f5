"""The C-ABI library builds, loads and exports every symbol include/disk.h
declares (no device calls: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(disk_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2512_04556_gb300 import _build
    _build.build()
    from paper_2512_04556_gb300 import disk
    return disk.lib()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 10
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_error_strings_and_version(lib):
    from paper_2512_04556_gb300 import disk
    assert disk.lib().disk_version() >= 10000
    assert disk.lib().disk_error_string(-2) == b"DISK_ERR_BAD_FILE"
    assert disk.lib().disk_error_string(12345) == b"DISK_ERR_UNKNOWN"


def test_validation_rejects_before_any_device_work(lib):
    """Argument checks run on the host and fail before touching the device."""
    import ctypes
    from paper_2512_04556_gb300 import disk
    h = ctypes.c_void_p()
    nn = (ctypes.c_int * 1)(4)
    nv = (ctypes.c_float * 4)(1.0, 2.0, 2.0, 3.0)           # not increasing
    th = (ctypes.c_float * (4 * 3))()
    rc = disk.lib().disk_basis_from_arrays(1, nn, nv, 1, 1, th, ctypes.byref(h))
    assert rc == -1 and b"increase" in disk.lib().disk_last_error_message()
    assert disk.lib().disk_basis_load(b"/nonexistent/basis.dkb", ctypes.byref(h)) == -2
    rc = disk.lib().disk_sv_filter(None, None, 0, None, 0, 8, 8, 3, 0, None, None)
    assert rc == -1
    sizes = (ctypes.c_int * 1)(9)
    rc = disk.lib().disk_fit_resume(None, sizes, 1, 2, 4, 0, 5, 5, 1e-3, 1e-4, 0, 0, 0.0, 0,
                                    None, None, None, None, None)
    assert rc == -1 and b"state" in disk.lib().disk_last_error_message()
    fake = ctypes.c_void_p(256)  # never dereferenced: the schedule check fails first
    for step0, steps, total in ((3, 3, 5), (-1, 2, 5), (0, -1, 5), (0, 2, 2000000)):
        rc = disk.lib().disk_fit_resume(fake, sizes, 1, 2, 4, step0, steps, total, 1e-3, 1e-4,
                                        0, 0, 0.0, 0, fake, fake, None, None, None)
        assert rc == -1 and b"step0" in disk.lib().disk_last_error_message()


def test_basis_file_rejects_corruption(tmp_path, lib):
    """The library's reader refuses truncated and bit-flipped files written by
    the independent writer (header and checksum are checked before any upload)."""
    import ctypes
    import numpy as np
    from oracle import basis_io
    from paper_2512_04556_gb300 import disk
    p = tmp_path / "b.dkb"
    basis_io.write(p, [[1.0, 2.0]], np.zeros((2, 1, 2, 3), np.float32))
    data = p.read_bytes()
    h = ctypes.c_void_p()
    (tmp_path / "t.dkb").write_bytes(data[:-3])
    assert disk.lib().disk_basis_load(str(tmp_path / "t.dkb").encode(), ctypes.byref(h)) == -2
    flipped = bytearray(data)
    flipped[40] ^= 0x10
    (tmp_path / "f.dkb").write_bytes(bytes(flipped))
    assert disk.lib().disk_basis_load(str(tmp_path / "f.dkb").encode(), ctypes.byref(h)) == -2
    assert b"checksum" in disk.lib().disk_last_error_message()
