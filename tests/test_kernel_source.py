"""The compiled tier's kernels compile for sm_103a without spilling: the
source each plan would compile (ec_plan_kernel_source) goes through NVRTC on
the host, with the library's options and ptxas's report.  Covers the
register-budgeted narrow programs (default and autotuned shapes) and the
two-level programs of wide codes, encoders and a decoder.  No GPU needed."""
import ctypes
import os
import re

import pytest

import paper_2108_02692_gb300 as xo

OPTS = [b"-arch=sm_103a", b"-std=c++17", b"-default-device", b"--extra-device-vectorization",
        b"--ptxas-options=-v"]


def _nvrtc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for name in ("libnvrtc.so", "libnvrtc.so.13", "libnvrtc.so.12"):
        for d in (os.path.join(home, "lib64"), os.path.join(home, "lib"), ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                continue
    pytest.skip("NVRTC not found")


def compile_report(src: str) -> str:
    lib = _nvrtc()
    prog = ctypes.c_void_p()
    assert lib.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"xorec_slp.cu", 0, None,
                                  None) == 0
    try:
        opts = (ctypes.c_char_p * len(OPTS))(*OPTS)
        rc = lib.nvrtcCompileProgram(prog, len(OPTS), opts)
        n = ctypes.c_size_t()
        lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
        log = ctypes.create_string_buffer(n.value)
        lib.nvrtcGetProgramLog(prog, log)
        text = log.value.decode(errors="replace")
        assert rc == 0, text
        return text
    finally:
        lib.nvrtcDestroyProgram(ctypes.byref(prog))


def check_no_spill(src: str):
    rep = compile_report(src)
    spills = [int(x) for x in re.findall(r"(\d+) bytes spill stores", rep)]
    regs = [int(x) for x in re.findall(r"Used (\d+) registers", rep)]
    assert spills and max(spills) == 0, rep
    m = re.search(r"__launch_bounds__\((\d+), (\d+)\)", src)
    threads, minb = int(m.group(1)), int(m.group(2))
    assert regs and max(regs) <= 65536 // (threads * minb), rep
    return max(regs)


@pytest.mark.parametrize("k,m,shape,erasures", [
    (10, 4, None, None),            # default shape, register budget 128
    (10, 4, (128, 160), None),      # the autotuner's RS(10,4) shape
    (10, 4, None, [1, 4, 9, 12]),
    (16, 4, None, None),            # two-level programs from here on
    (24, 8, None, None),
    (32, 4, None, [0, 5, 9, 33]),
    (48, 4, None, None),
])
def test_kernel_compiles_without_spills(k, m, shape, erasures):
    plan = xo.ec_plan_create(k, m)
    try:
        if shape:
            xo.ec_plan_set_launch(plan, *shape)
        src = xo.ec_plan_kernel_source(plan, erasures)
        info = xo.ec_plan_info(plan, erasures)
        # windowed programs (single group, more than 256 input strips) add a
        # producer warp to the threads that own a column
        windowed = "xk::run_window_pipeline(p, smem, SlpBody()" in src
        extra = 32 if windowed else 0
        assert windowed == (info["n_in"] > 256 and m == 4)
        assert f"__launch_bounds__({info['threads'] + extra}," in src
        assert ("xk_x3(" in src) == (info["window"] > 0)
        check_no_spill(src)
    finally:
        xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("k", [4, 8, 10, 11, 12])
def test_default_shape_never_spills(k):
    """Every narrow code at the default launch shape, encoder and a decoder:
    the register cap (128, or 168 from 11 data blocks up, where the preloaded
    input words and the pipeline's state exceed 128) holds the program."""
    for m in (1, 4, 8):
        plan = xo.ec_plan_create(k, m)
        try:
            for er in (None, list(range(m))):
                check_no_spill(xo.ec_plan_kernel_source(plan, er))
        finally:
            xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("budget", [96, 160, 200])
def test_explicit_register_budget_sets_the_cap(budget):
    """A plan asking for more than 128 registers per thread gets kernels
    whose register cap holds them (fewer CTAs per SM); smaller budgets keep
    the default cap.  Encoder and decoder compile without spills."""
    plan = xo.ec_plan_create_ex(10, 4, reg_budget=budget)
    try:
        for er in (None, [0, 3, 7, 11]):
            src = xo.ec_plan_kernel_source(plan, er)
            m = re.search(r"__launch_bounds__\((\d+), (\d+)\)", src)
            cap = 65536 // (int(m.group(1)) * int(m.group(2)))
            assert cap >= max(budget, 128)
            check_no_spill(src)
        with pytest.raises(xo.XorecError):
            xo.ec_plan_create_ex(10, 4, reg_budget=300)
    finally:
        xo.ec_plan_destroy(plan)


def live_values_of_emitted_code(src: str) -> int:
    """Most values a thread holds at once in the emitted straight-line body:
    a value (an input word loaded from the stage, or a statement's result)
    lives from the line that defines it to its last use; each statement is
    counted with its result."""
    body = src[src.index("struct SlpBody"):]
    body = body[:body.index("#undef I")]
    lines = [ln.strip() for ln in body.splitlines()]
    defs, last_use, stmts = {}, {}, []
    for i, ln in enumerate(lines):
        mm = re.match(r"const xk::u32 (\w+) = (.*);$", ln)
        if mm:
            name, rhs = mm.groups()
            defs[name] = i
            if not rhs.startswith("I("):
                stmts.append(i)
                for u in re.findall(r"\b([iv]\d+(?:_\d+)?)\b", rhs):
                    last_use[u] = i
            continue
        mm = re.match(r"O\(\d+, \d+, (\w+)\);$", ln)
        if mm:
            last_use[mm.group(1)] = i
    return max(sum(1 for n, d in defs.items() if d < L and last_use.get(n, -1) >= L) + 1
               for L in stmts)


@pytest.mark.parametrize("k,m", [(13, 4), (16, 4), (24, 8), (32, 4)])
@pytest.mark.parametrize("temps", [-1, 0], ids=["plain", "per-window"])
def test_two_level_register_model_matches_emitted_code(k, m, temps):
    """The planner's live-value count of a two-level program (the group size
    is chosen by it) equals the count read off the kernel it emits, where
    each input word is loaded once per group at its first use."""
    plan = xo.ec_plan_create_ex(k, m, stream_temps=temps)
    try:
        src = xo.ec_plan_kernel_source(plan)
        assert live_values_of_emitted_code(src) == xo.ec_plan_info(plan)["max_live"]
        info = xo.ec_plan_info(plan)
        assert len(re.findall(r"= I\(\d+\);", src)) == info["loads"]
    finally:
        xo.ec_plan_destroy(plan)


def live_values_preloaded(src: str) -> int:
    """Same count for a narrow body: every input word is in a register from
    the start of compute() to its last use."""
    body = src[src.index("void compute("):]
    body = body[:body.index("#undef I")]
    last_in, last_v, stmts = {}, {}, []
    for i, ln in enumerate(x.strip() for x in body.splitlines()):
        mm = re.match(r"const xk::u32 v(\d+) = (.*);$", ln) or re.match(r"O\(\d+, \d+, (.*)\)();$", ln)
        if not mm:
            continue
        if ln.startswith("const"):
            stmts.append((i, int(mm.group(1))))
            rhs = mm.group(2)
        else:
            rhs = mm.group(1)
        for c in re.findall(r"I\((\d+)\)", rhs):
            last_in[int(c)] = i
        for v in re.findall(r"\bv(\d+)\b", rhs):
            last_v[int(v)] = i
    defs = {v: i for i, v in stmts}
    return max(sum(1 for e in last_in.values() if e >= L) +
               sum(1 for w, d in defs.items() if d < L and last_v.get(w, -1) >= L) + 1
               for L, _ in stmts)


@pytest.mark.parametrize("k,m,er", [(10, 4, None), (10, 4, [0, 3, 7, 11]), (6, 3, None),
                                    (12, 4, None), (4, 2, [1, 4])])
def test_preloaded_register_model_matches_emitted_code(k, m, er):
    """The register-budgeted XorRePair picks its temporaries by the live
    values of the schedule with every input preloaded; the same count read
    off the emitted kernel agrees, and stays within the budget (128)."""
    plan = xo.ec_plan_create(k, m)
    try:
        src = xo.ec_plan_kernel_source(plan, er)
        live = live_values_preloaded(src)
        assert live == xo.ec_plan_info(plan, er)["max_live"] <= 128
    finally:
        xo.ec_plan_destroy(plan)


def test_kernel_source_buffer_protocol():
    plan = xo.ec_plan_create(4, 2)
    try:
        need = ctypes.c_size_t()
        lib = xo.lib()
        assert lib.ec_plan_kernel_source(plan, None, 0, None, 0, ctypes.byref(need)) == 0
        small = ctypes.create_string_buffer(16)
        assert lib.ec_plan_kernel_source(plan, None, 0, small, 16, None) == 0
        full = xo.ec_plan_kernel_source(plan)
        assert len(full) + 1 == need.value and small.value.decode() == full[:15]
        with pytest.raises(xo.XorecError):
            xo.ec_plan_kernel_source(plan, [0, 0])
    finally:
        xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("k,m,shape", [
    (10, 4, None),          # the decode benchmark's modules (default shape)
    (10, 4, (128, 160)),    # the autotuner's shapes on GB300 (batched mix)
    (12, 4, (128, 160)),
    (8, 4, (128, 112)),
    (6, 3, (128, 96)),
    (12, 4, None),
    (6, 3, None),
])
def test_batch_module_compiles_without_spills(k, m, shape):
    """A batch module of 48 decoders (ec_plan_module_source: the batched
    pipeline with its per-SM work queue, and a switch over the programs)
    compiles for sm_103a without spills at the plan's module shape: warp 0
    pops and prepares the next item only after the XOR program, when no
    input word is held in registers; decoders keep 8 registers below the
    module's cap; modules keep at least a 128-register cap."""
    import itertools
    import random
    plan = xo.ec_plan_create(k, m)
    try:
        if shape:
            xo.ec_plan_set_launch(plan, *shape)
        pats = [c for e in range(1, m + 1) for c in itertools.combinations(range(k + m), e)]
        sets = [list(c) for c in random.Random(k * 10 + m).sample(pats, 48)]
        src = xo.ec_plan_module_source(plan, sets)
        assert src.count("__device__ __forceinline__ void prog_") == 48
        assert "xorec_mod" in src and "%%smid" in src
        check_no_spill(src)
        check_no_spill(xo.ec_plan_module_source(plan))   # the encoder alone
    finally:
        xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("k,m", [(48, 4), (100, 4)])
def test_windowed_module_compiles_without_spills(k, m):
    """A batch module of wide single-group decoders (more than 256 input
    strips) takes the batched windowed pipeline: a producer warp beside the
    128 threads that own a column, a ring of windows instead of a stage of
    every strip; it compiles for sm_103a without spills."""
    import itertools
    import random
    plan = xo.ec_plan_create(k, m)
    try:
        pats = [c for e in range(1, m + 1) for c in itertools.combinations(range(k + m), e)]
        sets = [list(c) for c in random.Random(k).sample(pats, 8)]
        src = xo.ec_plan_module_source(plan, sets)
        assert "xk::run_batch_window_pipeline(p, smem, ModBody())" in src
        assert "__launch_bounds__(160, 3)" in src
        check_no_spill(src)
    finally:
        xo.ec_plan_destroy(plan)
