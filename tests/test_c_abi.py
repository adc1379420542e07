"""The C ABI used from C (tests/c/abi_host.c, compiled here with the
system C compiler): struct layouts match the Python binding's ctypes
mirrors, and host-only calls agree with the binding and the oracle.  CPU
only: no compute call is made."""
import ctypes
import os
import shutil
import subprocess

import pytest

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def output(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    xo.lib()                                   # builds the library if needed
    libdir = os.path.dirname(_abi.LIB_PATH)
    exe = str(tmp_path_factory.mktemp("cabi") / "abi_host")
    subprocess.run([cc, "-std=c11", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_host.c"), "-L", libdir, "-lxorec",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True)
    out = subprocess.run([exe], stdout=subprocess.PIPE, text=True, check=True).stdout
    return out.splitlines()


def _get(lines, key):
    return next(ln for ln in lines if ln.startswith(key)).split()


def test_struct_layouts_match_the_binding(output):
    mirrors = {"ec_plan_opts": _abi.PlanOpts, "ec_slp_stats": _abi.SlpStats,
               "ec_program_info": _abi.ProgramInfo, "ec_tune_result": _abi.TuneResult,
               "ec_job": _abi.Job, "ec_batch_info": _abi.BatchInfo,
               "ec_server_opts": _abi.ServerOpts, "ec_server_stats": _abi.ServerStats}
    for name, cls in mirrors.items():
        assert int(_get(output, f"sizeof {name} ")[2]) == ctypes.sizeof(cls), name
    assert int(_get(output, "offsetof ec_plan_opts.stream_temps")[2]) == \
        _abi.PlanOpts.stream_temps.offset
    assert int(_get(output, "offsetof ec_program_info.lop3")[2]) == _abi.ProgramInfo.lop3.offset
    assert int(_get(output, "offsetof ec_program_info.window_temps")[2]) == \
        _abi.ProgramInfo.window_temps.offset


def test_host_calls_agree_with_binding_and_oracle(output):
    m = [int(x) for x in _get(output, "matrix")[1:]]
    assert m == [int(x) for x in oracle.cauchy(10, 4).reshape(-1)]
    enc = _get(output, "encoder")
    plan = xo.ec_plan_create(10, 4)
    try:
        info = xo.ec_plan_info(plan)
        assert int(enc[2]) == 80 and int(enc[4]) == 32
        assert int(enc[6]) == info["raw"]["xors"] == 1234
        assert int(enc[8]) == info["fused"]["xors"] and int(enc[10]) == info["lop3"]
        assert int(enc[12]) == info["loads"] == 80
        dec = _get(output, "decoder")
        assert int(dec[4]) == 32 and int(dec[6]) == xo.ec_plan_info(plan, [0, 2, 5, 11])["raw"]["xors"]
    finally:
        xo.ec_plan_destroy(plan)
    assert _get(output, "program_check")[1] == "0"


def test_argument_errors_from_c(output):
    bad = _get(output, "bad_k")
    assert int(bad[1]) == xo.EC_EINVAL and bad[2] == "message"
    assert int(_get(output, "dup_erasure")[1]) == xo.EC_EINVAL
