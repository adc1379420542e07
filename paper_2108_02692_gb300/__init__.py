"""XOR-based Reed-Solomon erasure coding on one GB300 (sm_103a).

Thin Python binding of the C ABI in include/xorec.h: every function here has
the name of the C entry point it calls and only converts arguments.  Device
buffers are passed as integer device pointers (e.g. ``tensor.data_ptr()``)
and streams as integer ``cudaStream_t`` handles
(``torch.cuda.current_stream().cuda_stream``); PyTorch only supplies memory
and streams.  All computation runs in libxorec.so; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi

EC_OK = _abi.EC_OK
EC_EINVAL = _abi.EC_EINVAL
EC_ENOMEM = _abi.EC_ENOMEM
EC_ESINGULAR = _abi.EC_ESINGULAR
EC_ETOOMANY = _abi.EC_ETOOMANY
EC_ECUDA = _abi.EC_ECUDA
EC_ETIMEOUT = _abi.EC_ETIMEOUT
EC_EBUSY = _abi.EC_EBUSY
EC_ENOTSUP = _abi.EC_ENOTSUP
EC_MATRIX_CAUCHY = _abi.EC_MATRIX_CAUCHY
EC_MATRIX_POWER = _abi.EC_MATRIX_POWER
EC_MATRIX_USER = _abi.EC_MATRIX_USER
EC_MATRIX_CAUCHY_MIN = _abi.EC_MATRIX_CAUCHY_MIN
EC_OPT_RAW = _abi.EC_OPT_RAW
EC_OPT_REPAIR = _abi.EC_OPT_REPAIR
EC_OPT_XORREPAIR = _abi.EC_OPT_XORREPAIR
EC_OPT_TRIPLE = _abi.EC_OPT_TRIPLE
EC_SCHED_DFS = _abi.EC_SCHED_DFS
EC_SCHED_GREEDY = _abi.EC_SCHED_GREEDY
EC_EXEC_AUTO = _abi.EC_EXEC_AUTO
EC_EXEC_INTERP = _abi.EC_EXEC_INTERP
EC_EXEC_COMPILED = _abi.EC_EXEC_COMPILED
EC_EXEC_DENSE = _abi.EC_EXEC_DENSE


class XorecError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"xorec status {status}: {msg}")
        self.status = status


def lib():
    return _abi.load()


def ec_last_error() -> str:
    return (lib().ec_last_error() or b"").decode()


def ec_version() -> str:
    return lib().ec_version().decode()


def _check(rc: int) -> None:
    if rc != 0:
        raise XorecError(rc, ec_last_error())


def _u8(arr):
    if arr is None:
        return None
    a = np.ascontiguousarray(arr, dtype=np.uint8)
    return a, a.ctypes.data_as(_abi.u8p)


def _vp_array(ptrs):
    arr = (ctypes.c_void_p * max(1, len(ptrs)))()
    for i, p in enumerate(ptrs):
        arr[i] = None if p is None else int(p)
    return arr


def _int_array(vals):
    return (ctypes.c_int * max(1, len(vals)))(*[int(v) for v in vals])


# ------------------------------------------------------------------- plans

def ec_plan_create(k: int, m: int, matrix=None) -> int:
    h = ctypes.c_void_p()
    keep = _u8(matrix)
    _check(lib().ec_plan_create(k, m, keep[1] if keep else None, ctypes.byref(h)))
    return h.value


def ec_plan_create_ex(k: int, m: int, matrix_kind: int = EC_MATRIX_CAUCHY, matrix=None,
                      opt_level: int = EC_OPT_XORREPAIR, sched: int = EC_SCHED_DFS,
                      greedy_cap: int = 128, executor: int = EC_EXEC_AUTO,
                      max_temps: int = -2, reg_budget: int = 0, stream_window: int = 0,
                      stream_temps: int = 0) -> int:
    h = ctypes.c_void_p()
    keep = _u8(matrix)
    opts = _abi.PlanOpts(opt_level, sched, greedy_cap, executor, max_temps, reg_budget,
                         stream_window, stream_temps)
    _check(lib().ec_plan_create_ex(k, m, matrix_kind, keep[1] if keep else None,
                                   ctypes.byref(opts), ctypes.byref(h)))
    return h.value


def ec_plan_destroy(plan: int) -> None:
    lib().ec_plan_destroy(plan)


def ec_plan_matrix(plan: int, k: int, m: int) -> np.ndarray:
    out = np.zeros((m, k), np.uint8)
    _check(lib().ec_plan_matrix(plan, out.ctypes.data_as(_abi.u8p)))
    return out


def _stats(s) -> dict:
    return {"xors": s.xors, "mem": s.mem, "nvar": s.nvar, "stmts": s.stmts}


def ec_plan_info(plan: int, erasures=None) -> dict:
    info = _abi.ProgramInfo()
    if erasures is None:
        _check(lib().ec_plan_info(plan, None, 0, ctypes.byref(info)))
    else:
        _check(lib().ec_plan_info(plan, _int_array(erasures), len(erasures), ctypes.byref(info)))
    return {"n_in": info.n_in, "n_out": info.n_out, "slots": info.slots, "stmts": info.stmts,
            "code_words": info.code_words, "sched_nvar": info.sched_nvar,
            "raw": _stats(info.raw), "compressed": _stats(info.compressed),
            "fused": _stats(info.fused), "compiled": bool(info.compiled), "regs": info.regs,
            "temps": info.temps, "max_live": info.max_live, "threads": info.threads,
            "lop3": info.lop3, "loads": info.loads, "window": info.window,
            "window_temps": info.window_temps}


def ec_plan_program(plan: int, erasures=None) -> np.ndarray:
    need = ctypes.c_size_t()
    er = _int_array(erasures) if erasures is not None else None
    ne = len(erasures) if erasures is not None else 0
    _check(lib().ec_plan_program(plan, er, ne, None, 0, ctypes.byref(need)))
    out = np.zeros(need.value, np.uint16)
    _check(lib().ec_plan_program(plan, er, ne,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)),
                                 need.value, None))
    return out


def ec_plan_dense_words(plan: int, erasures=None) -> np.ndarray:
    """The dense executor's control words: column masks, then row words."""
    need = ctypes.c_size_t()
    er = _int_array(erasures) if erasures is not None else None
    ne = len(erasures) if erasures is not None else 0
    _check(lib().ec_plan_dense_words(plan, er, ne, None, 0, ctypes.byref(need)))
    out = np.zeros(need.value, np.uint32)
    _check(lib().ec_plan_dense_words(plan, er, ne,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                     need.value, None))
    return out


def ec_plan_kernel_source(plan: int, erasures=None) -> str:
    """CUDA source of the compiled tier's kernel for the encoder or a decoder."""
    need = ctypes.c_size_t()
    er = _int_array(erasures) if erasures is not None else None
    ne = len(erasures) if erasures is not None else 0
    _check(lib().ec_plan_kernel_source(plan, er, ne, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().ec_plan_kernel_source(plan, er, ne, buf, need.value, None))
    return buf.value.decode()


def ec_plan_module_source(plan: int, sets=None) -> str:
    """CUDA source of the batch module compiled for the decoders of `sets`
    (erasure lists), or for the encoder when `sets` is empty."""
    sets = sets or []
    flat = _int_array([int(x) for st in sets for x in st]) if sets else None
    counts = _int_array([len(st) for st in sets]) if sets else None
    need = ctypes.c_size_t()
    _check(lib().ec_plan_module_source(plan, flat, counts, len(sets), None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().ec_plan_module_source(plan, flat, counts, len(sets), buf, need.value, None))
    return buf.value.decode()


def ec_plan_autotune(plan: int, block_bytes: int, n_stripes: int = 16, stream: int = 0) -> dict:
    r = _abi.TuneResult()
    _check(lib().ec_plan_autotune(plan, block_bytes, n_stripes, stream or None, ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in _abi.TuneResult._fields_}


def ec_program_check(code, n_in: int, n_out: int, n_slots: int) -> None:
    """Raise XorecError (EC_EINVAL) unless the instruction stream is well formed."""
    arr = np.ascontiguousarray(code, dtype=np.uint16)
    _check(lib().ec_program_check(arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), arr.size,
                                  n_in, n_out, n_slots))


def ec_debug_fail_alloc(n: int) -> None:
    _check(lib().ec_debug_fail_alloc(n))


def ec_debug_inject_timeout(n: int) -> None:
    _check(lib().ec_debug_inject_timeout(n))


def ec_plan_set_launch(plan: int, threads: int, reg_budget: int) -> None:
    _check(lib().ec_plan_set_launch(plan, threads, reg_budget))


def ec_plan_set_executor(plan: int, executor: int) -> None:
    _check(lib().ec_plan_set_executor(plan, executor))


# -------------------------------------------------------------- coding

def ec_encode(plan: int, data_ptrs, parity_ptrs, block_bytes: int, stream: int = 0) -> None:
    _check(lib().ec_encode(plan, _vp_array(data_ptrs), _vp_array(parity_ptrs), block_bytes,
                           stream or None))


def ec_encode_noalloc(plan: int, data_ptrs, parity_ptrs, block_bytes: int,
                      stream: int = 0) -> None:
    """ec_encode without any memory allocation (see include/xorec.h)."""
    _check(lib().ec_encode_noalloc(plan, _vp_array(data_ptrs), _vp_array(parity_ptrs),
                                   block_bytes, stream or None))


def ec_encode_strided(plan: int, data_ptr: int, data_stripe_stride: int, data_block_stride: int,
                      parity_ptr: int, par_stripe_stride: int, par_block_stride: int,
                      n_stripes: int, block_bytes: int, stream: int = 0) -> None:
    _check(lib().ec_encode_strided(plan, data_ptr, data_stripe_stride, data_block_stride,
                                   parity_ptr, par_stripe_stride, par_block_stride, n_stripes,
                                   block_bytes, stream or None))


def ec_encode_host_strided(plan: int, data_ptr: int, data_stripe_stride: int,
                           data_block_stride: int, parity_ptr: int, par_stripe_stride: int,
                           par_block_stride: int, n_stripes: int, block_bytes: int,
                           chunk_stripes: int = 0, stream: int = 0) -> None:
    """Encode stripes held in host memory (pinned for full speed)."""
    _check(lib().ec_encode_host_strided(plan, data_ptr, data_stripe_stride, data_block_stride,
                                        parity_ptr, par_stripe_stride, par_block_stride,
                                        n_stripes, block_bytes, chunk_stripes, stream or None))


def ec_decode(plan: int, erasures, block_ptrs, out_ptrs, block_bytes: int,
              stream: int = 0) -> None:
    _check(lib().ec_decode(plan, _int_array(erasures), len(erasures), _vp_array(block_ptrs),
                           _vp_array(out_ptrs), block_bytes, stream or None))


def ec_decode_prepare(plan: int, sets, n_threads: int = 0) -> None:
    flat = [int(x) for s in sets for x in s]
    counts = [len(s) for s in sets]
    _check(lib().ec_decode_prepare(plan, _int_array(flat), _int_array(counts), len(sets),
                                   n_threads))


EC_OP_ENCODE = _abi.EC_OP_ENCODE
EC_OP_DECODE = _abi.EC_OP_DECODE


def _jobs(jobs):
    """jobs: dicts with plan, op, blocks (pointer list), out (pointer list),
    block_bytes and, for decodes, erasures.  Returns the ctypes array and
    the objects that must stay alive while it is used."""
    arr = (_abi.Job * max(1, len(jobs)))()
    keep = []
    for i, j in enumerate(jobs):
        er = j.get("erasures") or []
        era = _int_array(er)
        bl = _vp_array(j["blocks"])
        ou = _vp_array(j["out"])
        keep += [era, bl, ou]
        arr[i] = _abi.Job(j["plan"], j.get("op", EC_OP_ENCODE),
                          ctypes.cast(era, _abi.intp), len(er),
                          ctypes.cast(bl, _abi.vpp), ctypes.cast(ou, _abi.vpp),
                          j["block_bytes"])
    return arr, keep


def ec_batch_create(jobs, executor: int = EC_EXEC_AUTO) -> int:
    arr, keep = _jobs(jobs)
    h = ctypes.c_void_p()
    _check(lib().ec_batch_create(arr, len(jobs), executor, ctypes.byref(h)))
    return h.value


def ec_batch_run(batch: int, stream: int = 0) -> None:
    _check(lib().ec_batch_run(batch, stream or None))


def ec_batch_status(batch: int, reset: bool = False) -> int:
    st = ctypes.c_int()
    _check(lib().ec_batch_status(batch, ctypes.byref(st), 1 if reset else 0))
    return st.value


def ec_batch_info_get(batch: int) -> dict:
    i = _abi.BatchInfo()
    _check(lib().ec_batch_info_get(batch, ctypes.byref(i)))
    return {f: getattr(i, f) for f, _ in _abi.BatchInfo._fields_}


def ec_batch_destroy(batch: int) -> None:
    lib().ec_batch_destroy(batch)


def ec_run_batch(jobs, stream: int = 0) -> None:
    arr, keep = _jobs(jobs)
    _check(lib().ec_run_batch(arr, len(jobs), stream or None))


def ec_plan_compile(plan: int, sets=None, n_threads: int = 0) -> None:
    sets = sets or []
    flat = [int(x) for s in sets for x in s]
    counts = [len(s) for s in sets]
    _check(lib().ec_plan_compile(plan, _int_array(flat), _int_array(counts), len(sets),
                                 n_threads))


def ec_server_create(hbm_budget: int = 0, max_batch: int = 0, slots: int = 0,
                     idle_spin_us: int = 0, background_compile: bool = True) -> int:
    h = ctypes.c_void_p()
    opts = _abi.ServerOpts(hbm_budget, max_batch, slots, idle_spin_us, 0 if background_compile else 1)
    _check(lib().ec_server_create(ctypes.byref(opts), ctypes.byref(h)))
    return h.value


def ec_server_warm(server: int, plan: int, max_erasures: int) -> None:
    _check(lib().ec_server_warm(server, plan, max_erasures))


def make_jobs(jobs):
    """ctypes job array (and the objects it references) for repeated use."""
    return _jobs(jobs)


def ec_server_submit_raw(server: int, job_struct) -> int:
    """Submit a prepared ctypes job; returns the ticket, 0 when the budget
    is full (EC_EBUSY)."""
    t = ctypes.c_uint64()
    rc = lib().ec_server_submit(server, ctypes.byref(job_struct), ctypes.byref(t))
    if rc == EC_EBUSY:
        return 0
    _check(rc)
    return t.value


def ec_server_submit(server: int, job) -> int:
    arr, keep = _jobs([job])
    return ec_server_submit_raw(server, arr[0])


def ec_server_cancel(server: int, ticket: int) -> bool:
    """True when the request was still queued and is now dropped; False when
    it is already on the GPU or done."""
    rc = lib().ec_server_cancel(server, ticket)
    if rc == EC_EBUSY:
        return False
    _check(rc)
    return True


def ec_server_poll(server: int, max_n: int = 4096):
    tickets = (ctypes.c_uint64 * max_n)()
    lat = (ctypes.c_double * max_n)()
    n = ctypes.c_int()
    _check(lib().ec_server_poll(server, tickets, lat, max_n, ctypes.byref(n)))
    return [(tickets[i], lat[i]) for i in range(n.value)]


def ec_server_poll_ex(server: int, max_n: int = 4096):
    """Completed requests since the last poll: (ticket, latency_us, status)
    with status EC_OK or the error the request failed with."""
    tickets = (ctypes.c_uint64 * max_n)()
    lat = (ctypes.c_double * max_n)()
    st = (ctypes.c_int * max_n)()
    n = ctypes.c_int()
    _check(lib().ec_server_poll_ex(server, tickets, lat, st, max_n, ctypes.byref(n)))
    return [(tickets[i], lat[i], st[i]) for i in range(n.value)]


def ec_server_stats_get(server: int) -> dict:
    s = _abi.ServerStats()
    _check(lib().ec_server_stats_get(server, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in _abi.ServerStats._fields_}


def ec_server_destroy(server: int) -> None:
    lib().ec_server_destroy(server)


def ec_device_status(reset: bool = False) -> int:
    st = ctypes.c_int()
    _check(lib().ec_device_status(ctypes.byref(st), 1 if reset else 0))
    return st.value


def ec_selftest_wait_timeout(stream: int = 0) -> None:
    _check(lib().ec_selftest_wait_timeout(stream or None))


def ec_synth_fill(ptr: int, n: int, seed: int, offset: int = 0, stream: int = 0) -> None:
    _check(lib().ec_synth_fill(ptr, n, seed, offset, stream or None))


# ------------------------------------------------------ straight-line programs

def ec_slp_parse(text: str) -> int:
    h = ctypes.c_void_p()
    _check(lib().ec_slp_parse(text.encode(), ctypes.byref(h)))
    return h.value


def ec_slp_from_matrix(A, form: int = 1) -> int:
    a, p = _u8(A)
    h = ctypes.c_void_p()
    _check(lib().ec_slp_from_matrix(a.shape[0], a.shape[1], p, form, ctypes.byref(h)))
    return h.value


def ec_slp_repair(slp: int, xor_cancel: bool = True) -> int:
    h = ctypes.c_void_p()
    _check(lib().ec_slp_repair(slp, 1 if xor_cancel else 0, ctypes.byref(h)))
    return h.value


def ec_slp_fuse(slp: int, cancel_pairs: bool = True) -> int:
    h = ctypes.c_void_p()
    _check(lib().ec_slp_fuse(slp, 1 if cancel_pairs else 0, ctypes.byref(h)))
    return h.value


def ec_slp_schedule(slp: int, kind: int = EC_SCHED_DFS, cap: int = 8) -> int:
    h = ctypes.c_void_p()
    _check(lib().ec_slp_schedule(slp, kind, cap, ctypes.byref(h)))
    return h.value


def ec_slp_stats_get(slp: int) -> dict:
    s = _abi.SlpStats()
    _check(lib().ec_slp_stats_get(slp, ctypes.byref(s)))
    return _stats(s)


def ec_slp_iocost(slp: int, cap: int) -> int:
    return int(lib().ec_slp_iocost(slp, cap))


def ec_slp_ccap(slp: int) -> int:
    return int(lib().ec_slp_ccap(slp))


def ec_slp_equivalent(a: int, b: int) -> bool:
    eq = ctypes.c_int()
    _check(lib().ec_slp_equivalent(a, b, ctypes.byref(eq)))
    return bool(eq.value)


def ec_slp_to_text(slp: int) -> str:
    need = ctypes.c_size_t()
    _check(lib().ec_slp_to_text(slp, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().ec_slp_to_text(slp, buf, need.value, None))
    return buf.value.decode()


def ec_slp_destroy(slp: int) -> None:
    lib().ec_slp_destroy(slp)
