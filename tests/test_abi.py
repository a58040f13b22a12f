"""The C-ABI library builds, loads without a GPU and exports every function
include/xtn.h declares; argument checks that need no device work behave."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2403_09010_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xtn.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xtn_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_09010_gb300 import buildlib
    buildlib.build()
    return native.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["xtn_search_self", "xtn_index_build", "xtn_search_query",
                     "xtn_tcrdist_filter", "xtn_index_free", "xtn_status_string"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    exported = subprocess.run(["nm", "-D", "--defined-only", native.LIB_PATH],
                              capture_output=True, text=True, check=True).stdout.split()
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(_declared()) == set(native.SIGNATURES)
    # nothing but the C ABI leaks out of the library
    public = [s for s in exported if s.startswith("xtn")]
    assert sorted(public) == _declared()


def test_status_strings(lib):
    for code in range(-8, 1):
        assert native.status_string(code)
    assert native.status_string(native.XTN_ERR_BUFFER_TOO_SMALL) == "output buffer too small"
    assert lib.xtn_version() >= 10000


def test_argument_checks_before_device_work(lib):
    n_out = ctypes.c_int64(7)
    off = (ctypes.c_int64 * 2)(0, 3)
    seq = ctypes.c_char_p(b"CAS")
    # n_out missing, bad d, negative n, negative cap: rejected on the host
    assert lib.xtn_search_self(seq, off, 1, 1, None, 0, None, 0, None, None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_self(seq, off, 1, 4, None, 0, None, 0, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert n_out.value == 0
    assert lib.xtn_search_self(seq, off, -1, 1, None, 0, None, 0, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_self(seq, off, 1, 1, None, 0, None, -1, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    # batched mode needs at least one repertoire
    assert lib.xtn_search_self(seq, off, 1, 1, off, 0, None, 0, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    # empty input: nothing to do, no device needed
    assert lib.xtn_search_self(seq, off, 0, 2, None, 0, None, 0, ctypes.byref(n_out), None) == native.XTN_OK
    assert n_out.value == 0
    assert lib.xtn_index_build(seq, off, 0, 1, None, None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_query(None, seq, off, 1, None, 0, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_query_hamming(None, seq, off, 1, None, 0, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_index_free(None) == native.XTN_OK
    assert lib.xtn_index_info(None, None, None, None, None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_tcrdist_filter(seq, off, 1, None, 0, 24, None, ctypes.byref(n_out), None) == native.XTN_OK
    # pairs between repertoires: repertoires required, metric 0 or 1
    rep = (ctypes.c_int64 * 2)(0, 1)
    assert lib.xtn_search_between(seq, off, 1, 1, None, 0, 0, None, 0, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_between(seq, off, 1, 1, rep, 1, 2, None, 0, ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_between(seq, off, 0, 1, rep, 1, 1, None, 0, ctypes.byref(n_out), None) == native.XTN_OK
    # search in passes: metric 0 or 1, between needs repertoires
    assert lib.xtn_search_self_streaming(seq, off, 1, 1, None, 0, 2, 0, 0, None, 0, ctypes.byref(n_out), None, None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_self_streaming(seq, off, 1, 1, None, 0, 0, 1, 0, None, 0, ctypes.byref(n_out), None, None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_self_streaming(seq, off, 0, 1, None, 0, 0, 0, 0, None, 0, ctypes.byref(n_out), None, None) == native.XTN_OK


def test_tuning_knobs(lib):
    R, P, H = native.XTN_TUNE_SORT_RECORDS, native.XTN_TUNE_SORT_PAIRS, native.XTN_TUNE_RECORD_HISTOGRAM
    assert lib.xtn_tune_count(H) == 2
    assert lib.xtn_tune_count(R) == lib.xtn_tune_count(P) > 0
    assert lib.xtn_tune_count(99) == native.XTN_ERR_INVALID_ARG
    for knob in (R, P, H):
        old = lib.xtn_tune_get(knob)
        assert 0 <= old < lib.xtn_tune_count(knob)
        assert lib.xtn_tune_set(knob, lib.xtn_tune_count(knob)) == native.XTN_ERR_INVALID_ARG
        assert lib.xtn_tune_set(knob, -1) == native.XTN_ERR_INVALID_ARG
        assert lib.xtn_tune_get(knob) == old
        last = lib.xtn_tune_count(knob) - 1
        assert lib.xtn_tune_set(knob, last) == native.XTN_OK and lib.xtn_tune_get(knob) == last
        assert lib.xtn_tune_set(knob, old) == native.XTN_OK
    assert lib.xtn_tune_set(99, 0) == native.XTN_ERR_INVALID_ARG


def test_tuning_applied_restores_knobs(lib):
    from paper_2403_09010_gb300 import xtn
    knobs = [k for _, k in xtn._TUNING_KNOBS]
    before = [lib.xtn_tune_get(k) for k in knobs]
    want = {"grouping": 1, "record_hist": 1, "records_cfg": 0, "pairs_cfg": 1}
    with xtn.tuning_applied(want):
        assert [lib.xtn_tune_get(k) for k in knobs] == [1, 1, 0, 1]
    assert [lib.xtn_tune_get(k) for k in knobs] == before
    with xtn.tuning_applied({"pairs_cfg": 2}):   # keys left out stay as they are
        assert [lib.xtn_tune_get(k) for k in knobs] == before[:3] + [2]
    assert [lib.xtn_tune_get(k) for k in knobs] == before


def test_wait_limit_range(lib):
    # a host-side setting: negative and above-default limits are refused
    assert lib.xtn_set_wait_limit(-1) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_set_wait_limit((1 << 20) + 1) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_set_wait_limit(5) == native.XTN_OK
    assert lib.xtn_set_wait_limit(0) == native.XTN_OK


def test_profile_only_names(lib):
    # a host-side setting: names of 64 characters or more are refused; NULL
    # and "" time every launch again
    assert lib.xtn_profile_only(b"k_onesweep_records") == native.XTN_OK
    assert lib.xtn_profile_only(b"x" * 64) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_profile_only(b"x" * 63) == native.XTN_OK
    assert lib.xtn_profile_only(None) == native.XTN_OK
    assert lib.xtn_profile_only(b"") == native.XTN_OK


def test_paired_argument_checks(lib):
    n_out = ctypes.c_int64(7)
    off = (ctypes.c_int64 * 2)(0, 3)
    seq = ctypes.c_char_p(b"CAS")
    # a missing second chain, d above 2, missing n_out: refused on the host
    assert lib.xtn_search_paired(seq, off, seq, None, 1, 1, None, 0,
                                 ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert n_out.value == 0
    assert lib.xtn_search_paired(seq, off, seq, off, 1, 3, None, 0,
                                 ctypes.byref(n_out), None) == native.XTN_ERR_INVALID_ARG
    assert lib.xtn_search_paired(seq, off, seq, off, 1, 1, None, 0, None,
                                 None) == native.XTN_ERR_INVALID_ARG
