"""The C-ABI library builds, loads and exports every symbol ``include/*.h``
declares; host-side argument validation returns the documented codes.  No
call here reaches a CUDA API, so these run without a GPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_2005_07403_gb300 import svd2 as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(svd2_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_batch_entry_points():
    names = declared_functions()
    for n in ("svd2_batch_d", "svd2_batch_z", "svd2_batch_s", "svd2_batch_c"):
        assert n in names


@pytest.mark.parametrize("name", declared_functions())
def test_library_exports_declared_symbol(name):
    assert hasattr(S.lib(), name), name


def _null4():
    return (ctypes.c_void_p * 4)()


def test_invalid_arguments_rejected_on_host():
    L = S.lib()
    z = _null4()
    # n < 0
    assert L.svd2_batch_d(-1, z, z, z, None, None, None, 0, None) == S.EINVAL
    # NULL arrays with n > 0
    assert L.svd2_batch_d(5, z, z, z, None, None, None, 0, None) == S.EINVAL
    assert L.svd2_batch_d(5, None, None, None, None, None, None, 0, None) == S.EINVAL
    # unknown flag bits
    assert L.svd2_batch_s(0, z, z, z, None, None, None, 0x80, None) == S.EINVAL
    # n == 0 is a no-op
    assert L.svd2_batch_z(0, None, None, None, None, None, None, 0, None) == S.OK
    assert L.svd2_batch_c(0, None, None, None, None, None, None, 0, None) == S.OK
    # values only: same rules
    assert L.svd2_values_d(-1, z, None, None, None, 0, None) == S.EINVAL
    assert L.svd2_values_s(5, None, None, None, None, 0, None) == S.EINVAL
    assert L.svd2_values_z(0, None, None, None, None, 0, None) == S.OK
    # interleaved: exactly one of U, V NULL, unknown flags, n < 0 (no pointer is dereferenced)
    fake = 256
    assert L.svd2_batch_interleaved_d(5, fake, fake, None, fake, fake, fake, 0, None) == S.EINVAL
    assert L.svd2_batch_interleaved_c(5, fake, None, fake, fake, fake, fake, 0, None) == S.EINVAL
    assert L.svd2_batch_interleaved_z(0, None, None, None, None, None, None, 0x80, None) == S.EINVAL
    assert L.svd2_batch_interleaved_s(-1, fake, fake, fake, fake, fake, fake, 0, None) == S.EINVAL
    assert L.svd2_batch_interleaved_s(0, None, None, None, None, None, None, 0, None) == S.OK
    # self-tests: unknown op, NULL or misaligned result (checked before any launch)
    assert L.svd2_arith_check(5, 8, fake, fake, fake, fake, None) == S.EINVAL
    assert L.svd2_arith_check(4, 8, fake, None, fake, fake, None) == S.EINVAL   # op 4 needs y
    assert L.svd2_arith_check(0, -1, fake, fake, fake, fake, None) == S.EINVAL
    assert L.svd2_fp32_selfcheck(4, 0, 8, fake, None) == S.EINVAL
    assert L.svd2_fp32_selfcheck(0, 0, 8, None, None) == S.EINVAL
    assert L.svd2_fp32_selfcheck(1, 0, 8, 260, None) == S.EINVAL
    assert L.svd2_fp32_selfcheck(2, 0, 0, fake, None) == S.OK


def test_launch_table_roundtrip_and_validation():
    L = S.lib()
    old = S.get_launch("s")
    try:
        S.set_launch("s", 128, 2, 2, 3)
        assert S.get_launch("s") == (128, 2, 2, 3)
        assert L.svd2_set_launch(2, 100, 1, 1, 0) == S.EINVAL     # not a multiple of 32
        assert L.svd2_set_launch(2, 1024, 1, 1, 0) == S.EINVAL    # above 512
        for op in (0, 1, 3, 4):                                     # 64-register kernels
            saved = S.get_launch({0: "d", 1: "z", 3: "c", 4: "s_tan64"}[op])
            assert L.svd2_set_launch(op, 1024, 1, 1, 0) == S.OK
            assert L.svd2_set_launch(op, 1056, 1, 1, 0) == S.EINVAL
            assert L.svd2_set_launch(op, *saved) == S.OK
        assert L.svd2_set_launch(2, 128, 3, 1, 0) == S.EINVAL     # mpt
        assert L.svd2_set_launch(9, 128, 1, 1, 0) == S.EINVAL     # op
    finally:
        S.set_launch("s", *old)


def test_version_string():
    assert "sm_103a" in S.version()
