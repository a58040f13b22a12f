"""ctypes binding of the C ABI in include/xtn.h (argument marshalling only).

Every computation happens in libxtn.so's CUDA kernels.  Importing this module
does not need a GPU; calling a search does.  If the library has not been
built, ``lib()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libxtn.so")

XTN_OK = 0
XTN_ERR_INVALID_ARG = -1
XTN_ERR_BAD_RESIDUE = -2
XTN_ERR_SEQ_TOO_LONG = -3
XTN_ERR_OOM = -4
XTN_ERR_BUFFER_TOO_SMALL = -5
XTN_ERR_CUDA = -6
XTN_ERR_DEVICE_TIMEOUT = -7
XTN_ERR_TOO_LARGE = -8
XTN_ERR_CAPACITY = -9
XTN_TUNE_SORT_RECORDS = 0
XTN_TUNE_SORT_PAIRS = 1
XTN_TUNE_RECORD_HISTOGRAM = 2
XTN_TUNE_GROUPING = 3
XTN_TUNE_FILTER_SEGMENT = 4
XTN_NOALLOC_MAX_SEQS = 1 << 18
XTN_NOALLOC_MAX_ROWS = 1 << 22
XTN_MAX_LEN = 25
XTN_MAX_D = 3

# Every function the header declares: name -> (restype, argtypes).
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
SIGNATURES = {
    "xtn_status_string": (ctypes.c_char_p, [_I]),
    "xtn_version": (_I, []),
    "xtn_search_self": (_I, [_P, _P, _I64, _I, _P, _I64, _P, _I64, _P, _P]),
    "xtn_search_self_hamming": (_I, [_P, _P, _I64, _I, _P, _I64, _P, _I64, _P, _P]),
    "xtn_search_between": (_I, [_P, _P, _I64, _I, _P, _I64, _I, _P, _I64, _P, _P]),
    "xtn_search_paired": (_I, [_P, _P, _P, _P, _I64, _I, _P, _I64, _P, _P]),
    "xtn_search_self_streaming": (_I, [_P, _P, _I64, _I, _P, _I64, _I, _I, _I64, _P, _I64, _P,
                                       _P, _P]),
    "xtn_index_build": (_I, [_P, _P, _I64, _I, _P, _P]),
    "xtn_index_free": (_I, [_P]),
    "xtn_index_info": (_I, [_P, _P, _P, _P, _P]),
    "xtn_search_query": (_I, [_P, _P, _P, _I64, _P, _I64, _P, _P]),
    "xtn_search_query_hamming": (_I, [_P, _P, _P, _I64, _P, _I64, _P, _P]),
    "xtn_search_query_scratch": (_I, [_P, _P, _I64, _P]),
    "xtn_tcrdist_filter": (_I, [_P, _P, _I64, _P, _I64, _I, _P, _P, _P]),
    "xtn_tcrdist_filter_noalloc": (_I, [_P, _P, _I64, _P, _I64, _I, _P, _P, _P]),
    "xtn_plan_create": (_I, [_P, _I64, _I, _P, _I64, _I64, _P]),
    "xtn_plan_run": (_I, [_P, _P, _P]),
    "xtn_plan_result": (_I, [_P, _P, _I64, _P, _P]),
    "xtn_plan_info": (_I, [_P, _P, _P, _P]),
    "xtn_plan_stats": (_I, [_P, _P, _P, _P, _P, _P]),
    "xtn_plan_free": (_I, [_P]),
    "xtn_tune_set": (_I, [_I, _I]),
    "xtn_tune_get": (_I, [_I]),
    "xtn_tune_count": (_I, [_I]),
    "xtn_scratch_trim": (_I, []),
    "xtn_set_wait_limit": (_I, [_I64]),
    "xtn_profile_enable": (_I, [_I]),
    "xtn_profile_only": (_I, [ctypes.c_char_p]),
    "xtn_profile_report": (_I, [ctypes.c_char_p, _I64]),
}

_lib = None
_lock = threading.Lock()


class XtnError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


def lib():
    """The loaded libxtn.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_2403_09010_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().xtn_status_string(status).decode()


def check(status: int, where: str) -> None:
    if status != XTN_OK:
        raise XtnError(status, where)
