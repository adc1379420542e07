"""ctypes declarations of the C ABI in include/xorec.h (argument marshalling
only).  The library is the in-tree build ``_build/libxorec.so``; importing
fails loudly when it is missing."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libxorec.so")

c_int = ctypes.c_int
c_long = ctypes.c_long
c_size = ctypes.c_size_t
c_u64 = ctypes.c_uint64
c_vp = ctypes.c_void_p
c_char_p = ctypes.c_char_p
u8p = ctypes.POINTER(ctypes.c_uint8)
intp = ctypes.POINTER(ctypes.c_int)
vpp = ctypes.POINTER(ctypes.c_void_p)

EC_OK = 0
EC_EINVAL = -1
EC_ENOMEM = -2
EC_ESINGULAR = -3
EC_ETOOMANY = -4
EC_ECUDA = -5
EC_ETIMEOUT = -6
EC_EBUSY = -7
EC_ENOTSUP = -8

EC_MATRIX_CAUCHY, EC_MATRIX_POWER, EC_MATRIX_USER, EC_MATRIX_CAUCHY_MIN = 0, 1, 2, 3
EC_OPT_RAW, EC_OPT_REPAIR, EC_OPT_XORREPAIR, EC_OPT_TRIPLE = 0, 1, 2, 3
EC_SCHED_DFS, EC_SCHED_GREEDY = 0, 1
EC_EXEC_AUTO, EC_EXEC_INTERP, EC_EXEC_COMPILED, EC_EXEC_DENSE = 0, 1, 2, 3


class PlanOpts(ctypes.Structure):
    _fields_ = [("opt_level", c_int), ("sched", c_int), ("greedy_cap", c_int),
                ("executor", c_int), ("max_temps", c_int), ("reg_budget", c_int),
                ("stream_window", c_int), ("stream_temps", c_int)]


class SlpStats(ctypes.Structure):
    _fields_ = [("xors", c_long), ("mem", c_long), ("nvar", c_int), ("stmts", c_int)]


class ProgramInfo(ctypes.Structure):
    _fields_ = [("n_in", c_int), ("n_out", c_int), ("slots", c_int), ("stmts", c_int),
                ("code_words", c_int), ("sched_nvar", c_int), ("raw", SlpStats),
                ("compressed", SlpStats), ("fused", SlpStats), ("compiled", c_int),
                ("regs", c_int), ("temps", c_int), ("max_live", c_int), ("threads", c_int), ("lop3", c_int),
                ("loads", c_int), ("window", c_int), ("window_temps", c_int)]


EC_OP_ENCODE, EC_OP_DECODE = 0, 1


class Job(ctypes.Structure):
    _fields_ = [("plan", c_vp), ("op", c_int), ("erasures", intp), ("n_erasures", c_int),
                ("blocks", vpp), ("out", vpp), ("block_bytes", c_size)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("stripes", ctypes.c_longlong), ("items", ctypes.c_longlong),
                ("bytes_in", ctypes.c_longlong), ("bytes_out", ctypes.c_longlong),
                ("programs", c_int), ("compiled_programs", c_int), ("launches", c_int),
                ("modules_built", c_int), ("prepare_ms", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", c_size), ("max_batch", c_int), ("slots", c_int),
                ("idle_spin_us", c_int), ("no_background_compile", c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_longlong) for n in
                ("submitted", "completed", "rejected", "failed", "batches", "max_batch_seen",
                 "bytes_in", "bytes_out", "admitted_bytes", "pending")] + [
        ("slots_busy", c_int), ("compiled_in_background", ctypes.c_longlong),
        ("cancelled", ctypes.c_longlong)]


class TuneResult(ctypes.Structure):
    _fields_ = [("threads", c_int), ("reg_budget", c_int), ("min_ctas_per_sm", c_int),
                ("candidates", c_int), ("ms", ctypes.c_double), ("gbps_in", ctypes.c_double)]


# name -> (restype, argtypes); every symbol declared in include/xorec.h
SIGNATURES = {
    "ec_plan_create": (c_int, [c_int, c_int, u8p, ctypes.POINTER(c_vp)]),
    "ec_plan_create_ex": (c_int, [c_int, c_int, c_int, u8p, ctypes.POINTER(PlanOpts),
                                  ctypes.POINTER(c_vp)]),
    "ec_plan_destroy": (None, [c_vp]),
    "ec_plan_matrix": (c_int, [c_vp, u8p]),
    "ec_plan_info": (c_int, [c_vp, intp, c_int, ctypes.POINTER(ProgramInfo)]),
    "ec_plan_module_source": (c_int, [c_vp, intp, intp, c_int, ctypes.c_char_p, c_size,
                                      ctypes.POINTER(c_size)]),
    "ec_plan_program": (c_int, [c_vp, intp, c_int, ctypes.POINTER(ctypes.c_uint16), c_size,
                                ctypes.POINTER(c_size)]),
    "ec_plan_dense_words": (c_int, [c_vp, intp, c_int, ctypes.POINTER(ctypes.c_uint32), c_size,
                                    ctypes.POINTER(c_size)]),
    "ec_plan_kernel_source": (c_int, [c_vp, intp, c_int, ctypes.c_char_p, c_size,
                                      ctypes.POINTER(c_size)]),
    "ec_encode": (c_int, [c_vp, vpp, vpp, c_size, c_vp]),
    "ec_encode_noalloc": (c_int, [c_vp, vpp, vpp, c_size, c_vp]),
    "ec_encode_strided": (c_int, [c_vp, c_vp, c_size, c_size, c_vp, c_size, c_size, c_int,
                                  c_size, c_vp]),
    "ec_encode_host_strided": (c_int, [c_vp, c_vp, c_size, c_size, c_vp, c_size, c_size, c_int,
                                       c_size, c_int, c_vp]),
    "ec_decode": (c_int, [c_vp, intp, c_int, vpp, vpp, c_size, c_vp]),
    "ec_decode_prepare": (c_int, [c_vp, intp, intp, c_int, c_int]),
    "ec_plan_compile": (c_int, [c_vp, intp, intp, c_int, c_int]),
    "ec_plan_autotune": (c_int, [c_vp, c_size, c_int, c_vp, ctypes.POINTER(TuneResult)]),
    "ec_plan_set_launch": (c_int, [c_vp, c_int, c_int]),
    "ec_program_check": (c_int, [ctypes.POINTER(ctypes.c_uint16), c_size, c_int, c_int, c_int]),
    "ec_debug_fail_alloc": (c_int, [c_int]),
    "ec_debug_inject_timeout": (c_int, [c_int]),
    "ec_plan_set_executor": (c_int, [c_vp, c_int]),
    "ec_batch_create": (c_int, [ctypes.POINTER(Job), c_int, c_int, ctypes.POINTER(c_vp)]),
    "ec_batch_run": (c_int, [c_vp, c_vp]),
    "ec_batch_info_get": (c_int, [c_vp, ctypes.POINTER(BatchInfo)]),
    "ec_batch_status": (c_int, [c_vp, intp, c_int]),
    "ec_batch_destroy": (None, [c_vp]),
    "ec_run_batch": (c_int, [ctypes.POINTER(Job), c_int, c_vp]),
    "ec_server_create": (c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(c_vp)]),
    "ec_server_warm": (c_int, [c_vp, c_vp, c_int]),
    "ec_server_submit": (c_int, [c_vp, ctypes.POINTER(Job), ctypes.POINTER(c_u64)]),
    "ec_server_cancel": (c_int, [c_vp, c_u64]),
    "ec_server_poll": (c_int, [c_vp, ctypes.POINTER(c_u64), ctypes.POINTER(ctypes.c_double),
                               c_int, intp]),
    "ec_server_poll_ex": (c_int, [c_vp, ctypes.POINTER(c_u64), ctypes.POINTER(ctypes.c_double),
                                  intp, c_int, intp]),
    "ec_server_stats_get": (c_int, [c_vp, ctypes.POINTER(ServerStats)]),
    "ec_server_destroy": (None, [c_vp]),
    "ec_device_status": (c_int, [intp, c_int]),
    "ec_last_error": (c_char_p, []),
    "ec_version": (c_char_p, []),
    "ec_selftest_wait_timeout": (c_int, [c_vp]),
    "ec_synth_fill": (c_int, [c_vp, c_size, c_u64, c_u64, c_vp]),
    "ec_slp_parse": (c_int, [c_char_p, ctypes.POINTER(c_vp)]),
    "ec_slp_from_matrix": (c_int, [c_int, c_int, u8p, c_int, ctypes.POINTER(c_vp)]),
    "ec_slp_repair": (c_int, [c_vp, c_int, ctypes.POINTER(c_vp)]),
    "ec_slp_fuse": (c_int, [c_vp, c_int, ctypes.POINTER(c_vp)]),
    "ec_slp_schedule": (c_int, [c_vp, c_int, c_int, ctypes.POINTER(c_vp)]),
    "ec_slp_stats_get": (c_int, [c_vp, ctypes.POINTER(SlpStats)]),
    "ec_slp_iocost": (c_long, [c_vp, c_int]),
    "ec_slp_ccap": (c_int, [c_vp]),
    "ec_slp_equivalent": (c_int, [c_vp, c_vp, intp]),
    "ec_slp_to_text": (c_int, [c_vp, c_char_p, c_size, ctypes.POINTER(c_size)]),
    "ec_slp_destroy": (None, [c_vp]),
}

_lib = None


def load():
    """Load libxorec.so (the CUDA path).  Raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libxorec.so not found at {LIB_PATH}; run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
