"""The C-ABI library loads and exports every symbol include/*.h declares.
CPU only: no compute call is made here."""
import ctypes
import glob
import os
import re
import subprocess

import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(ec_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_header_declares_core_entry_points():
    names = declared_functions()
    for n in ("ec_plan_create", "ec_encode", "ec_decode", "ec_plan_destroy", "ec_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = xo.lib()
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"binding lacks {name}"


def test_exported_dynamic_symbols_cover_header():
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH],
                         stdout=subprocess.PIPE, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_functions() - exported
    assert not missing, missing


def test_version_and_error_string():
    assert "xorec" in xo.ec_version()
    assert isinstance(xo.ec_last_error(), str)


def test_noalloc_limits_are_checked_before_any_device_call():
    """ec_encode_noalloc rejects programs longer than its static array holds
    (EC_EINVAL) before it touches a device, and rejects bad block sizes the
    same way.  k + m above its block limit cannot reach it: plans already
    refuse k + m > 256 = EC_NOALLOC_MAX_BLOCKS."""
    import pytest
    plan = xo.ec_plan_create_ex(100, 4, opt_level=xo.EC_OPT_RAW)
    try:
        assert xo.ec_plan_info(plan)["code_words"] > 32768
        with pytest.raises(xo.XorecError) as e:
            xo.ec_encode_noalloc(plan, [16] * 100, [16] * 4, 128, 0)
        assert e.value.status == xo.EC_EINVAL
        assert "32768" in xo.ec_last_error()
    finally:
        xo.ec_plan_destroy(plan)
    plan = xo.ec_plan_create(4, 2)
    try:
        with pytest.raises(xo.XorecError) as e:
            xo.ec_encode_noalloc(plan, [16] * 4, [16] * 2, 100, 0)
        assert e.value.status == xo.EC_EINVAL
    finally:
        xo.ec_plan_destroy(plan)
    with pytest.raises(xo.XorecError) as e:
        xo.ec_plan_create(200, 57)
    assert e.value.status == xo.EC_EINVAL
