"""CPU oracle for symmetric-deletion Levenshtein neighbour search.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers. The product
package never imports this module and shares no code with it.

The arithmetic lives in ``xtn_oracle.cpp`` (plain C++, strings, full DP,
``std::unordered_map``); this file compiles it with g++ and wraps it with
ctypes. Every function returns numpy arrays of uint32 rows:

* ``symdel_self``      (i, j, dist), i < j          -- Appendix, SymDel steps 0-4
* ``symdel_batched``   (rep, i, j, dist)            -- the same per repertoire
* ``symdel_cross``     (i, j, dist)                 -- pairs between repertoires
* ``symdel_self_sharded`` (i, j, dist)              -- symdel_self on several threads
* ``symdel_query``     (q, r, dist)                 -- steps 1-2 on the reference,
                                                       step 3 with the queries
* ``bruteforce_self`` / ``bruteforce_query``        -- exhaustive search (pin);
                                                       ``threads=`` splits the
                                                       references over threads
* ``hamming``; ``metric="hamming"`` of ``symdel_self`` / ``symdel_batched`` /
  ``bruteforce_self``  -- the Hamming variant (the last step filters by
  Hamming distance; unequal lengths are never neighbours)
* ``neighbors_of``     (j, dist) for one i          -- plain definition, sampled checks
* ``tcrdist_filter`` / ``tcrdist_allpairs``          -- TCRdist post-filter (Results)
* ``symdel_paired`` / ``bruteforce_paired``         -- paired chains joined by a
                                                       token no edit may touch
                                                       (Discussion)
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xtn_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2). Returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", _SRC, "-o",
                        tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def built_from(path: str):
    """Within the block, every function of this module calls the library at
    `path`, a build of a copy of xtn_oracle.cpp (tests plant mistakes in such
    copies to check that the pins catch them)."""
    global _lib
    saved = _load()
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _configure(lib):
    for name in ("xo_symdel_self", "xo_symdel_self_hamming", "xo_bruteforce_self"):
        getattr(lib, name).argtypes = [_P, _P, _I64, ctypes.c_int]
        getattr(lib, name).restype = _P
    lib.xo_bruteforce_self_metric.argtypes = [_P, _P, _I64, ctypes.c_int, ctypes.c_int]
    lib.xo_bruteforce_self_metric.restype = _P
    lib.xo_symdel_self_sharded.argtypes = [_P, _P, _I64, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int]
    lib.xo_symdel_self_sharded.restype = _P
    lib.xo_symdel_batched.argtypes = [_P, _P, _P, _I64, ctypes.c_int, ctypes.c_int]
    lib.xo_symdel_batched.restype = _P
    lib.xo_symdel_cross.argtypes = [_P, _P, _P, _I64, ctypes.c_int, ctypes.c_int]
    lib.xo_symdel_cross.restype = _P
    lib.xo_hamming.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    lib.xo_hamming.restype = ctypes.c_int
    for name in ("xo_symdel_query", "xo_bruteforce_query"):
        getattr(lib, name).argtypes = [_P, _P, _I64, _P, _P, _I64, ctypes.c_int]
        getattr(lib, name).restype = _P
    for name in ("xo_symdel_query_metric", "xo_bruteforce_query_metric"):
        getattr(lib, name).argtypes = [_P, _P, _I64, _P, _P, _I64, ctypes.c_int, ctypes.c_int]
        getattr(lib, name).restype = _P
    lib.xo_bruteforce_query_threaded.argtypes = [_P, _P, _I64, _P, _P, _I64, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int]
    lib.xo_bruteforce_query_threaded.restype = _P
    lib.xo_neighbors_of.argtypes = [_P, _P, _I64, _I64, ctypes.c_int]
    lib.xo_neighbors_of.restype = _P
    lib.xo_tcrdist_filter.argtypes = [_P, _P, _P, _I64, ctypes.c_int]
    lib.xo_tcrdist_filter.restype = _P
    lib.xo_tcrdist_allpairs.argtypes = [_P, _P, _I64, ctypes.c_int, ctypes.c_int]
    lib.xo_tcrdist_allpairs.restype = _P
    lib.xo_result_rows.argtypes = [_P]
    lib.xo_result_rows.restype = _I64
    lib.xo_result_width.argtypes = [_P]
    lib.xo_result_width.restype = ctypes.c_int
    lib.xo_result_copy.argtypes = [_P, _P]
    lib.xo_result_free.argtypes = [_P]
    lib.xo_levenshtein.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    lib.xo_levenshtein.restype = ctypes.c_int
    lib.xo_tcrdist.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    lib.xo_tcrdist.restype = ctypes.c_int
    lib.xo_count_variants.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
    lib.xo_count_variants.restype = _I64
    for name in ("xo_symdel_paired", "xo_bruteforce_paired"):
        getattr(lib, name).argtypes = [_P, _P, _I64, ctypes.c_int]
        getattr(lib, name).restype = _P
    lib.xo_lev_token.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int]
    lib.xo_lev_token.restype = ctypes.c_int
    lib.xo_count_variants_token.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
    lib.xo_count_variants_token.restype = _I64
    lib.xo_blosum62.argtypes = [ctypes.c_char, ctypes.c_char]
    lib.xo_blosum62.restype = ctypes.c_int
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _prep(seqs, offsets):
    s = np.ascontiguousarray(seqs, dtype=np.uint8)
    if s.size == 0:
        s = np.zeros(1, np.uint8)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    return s, o


def _take(h) -> np.ndarray:
    lib = _load()
    rows, width = lib.xo_result_rows(h), lib.xo_result_width(h)
    out = np.empty((rows, width), dtype=np.uint32)
    if rows:
        lib.xo_result_copy(h, _ptr(out))
    lib.xo_result_free(h)
    return out


_METRICS = {"levenshtein": 0, "hamming": 1}


def symdel_self(seqs, offsets, d: int, metric: str = "levenshtein") -> np.ndarray:
    s, o = _prep(seqs, offsets)
    if metric not in _METRICS:
        raise ValueError(f"unknown metric {metric!r}")
    fn = _load().xo_symdel_self_hamming if metric == "hamming" else _load().xo_symdel_self
    return _take(fn(_ptr(s), _ptr(o), o.size - 1, d))


def symdel_batched(seqs, offsets, rep_offsets, d: int, metric: str = "levenshtein") -> np.ndarray:
    s, o = _prep(seqs, offsets)
    r = np.ascontiguousarray(rep_offsets, dtype=np.int64)
    return _take(_load().xo_symdel_batched(_ptr(s), _ptr(o), _ptr(r), r.size - 1, d,
                                           _METRICS[metric]))


def symdel_self_sharded(seqs, offsets, d: int, metric: str = "levenshtein",
                        threads: int = 0) -> np.ndarray:
    """symdel_self with the variant keys partitioned over threads (0: all of
    the host's hardware threads); the same rows."""
    s, o = _prep(seqs, offsets)
    return _take(_load().xo_symdel_self_sharded(_ptr(s), _ptr(o), o.size - 1, d,
                                                _METRICS[metric], int(threads)))


def symdel_cross(seqs, offsets, rep_offsets, d: int, metric: str = "levenshtein") -> np.ndarray:
    """Pairs (i, j, dist) whose sequences lie in different repertoires."""
    s, o = _prep(seqs, offsets)
    r = np.ascontiguousarray(rep_offsets, dtype=np.int64)
    return _take(_load().xo_symdel_cross(_ptr(s), _ptr(o), _ptr(r), r.size - 1, d,
                                         _METRICS[metric]))


def symdel_query(ref_seqs, ref_offsets, q_seqs, q_offsets, d: int,
                 metric: str = "levenshtein") -> np.ndarray:
    rs, ro = _prep(ref_seqs, ref_offsets)
    qs, qo = _prep(q_seqs, q_offsets)
    return _take(_load().xo_symdel_query_metric(_ptr(rs), _ptr(ro), ro.size - 1, _ptr(qs),
                                                _ptr(qo), qo.size - 1, d, _METRICS[metric]))


def bruteforce_self(seqs, offsets, d: int, metric: str = "levenshtein") -> np.ndarray:
    s, o = _prep(seqs, offsets)
    return _take(_load().xo_bruteforce_self_metric(_ptr(s), _ptr(o), o.size - 1, d,
                                                   _METRICS[metric]))


def bruteforce_query(ref_seqs, ref_offsets, q_seqs, q_offsets, d: int,
                     metric: str = "levenshtein", threads: int = 1) -> np.ndarray:
    """Every (q, r, dist) with dist <= d by comparing each query with each
    reference; threads != 1 splits the references over that many threads
    (0: all hardware threads), with the same rows."""
    rs, ro = _prep(ref_seqs, ref_offsets)
    qs, qo = _prep(q_seqs, q_offsets)
    if threads != 1:
        return _take(_load().xo_bruteforce_query_threaded(
            _ptr(rs), _ptr(ro), ro.size - 1, _ptr(qs), _ptr(qo), qo.size - 1, d,
            _METRICS[metric], int(threads)))
    return _take(_load().xo_bruteforce_query_metric(_ptr(rs), _ptr(ro), ro.size - 1, _ptr(qs),
                                                    _ptr(qo), qo.size - 1, d,
                                                    _METRICS[metric]))


def neighbors_of(seqs, offsets, i: int, d: int) -> np.ndarray:
    s, o = _prep(seqs, offsets)
    return _take(_load().xo_neighbors_of(_ptr(s), _ptr(o), o.size - 1, int(i), d))


def tcrdist_filter(seqs, offsets, triples, max_score: int) -> np.ndarray:
    s, o = _prep(seqs, offsets)
    t = np.ascontiguousarray(triples, dtype=np.uint32).reshape(-1, 3)
    if t.size == 0:
        return np.zeros((0, 3), np.uint32)
    return _take(_load().xo_tcrdist_filter(_ptr(s), _ptr(o), _ptr(t), t.shape[0], max_score))


def tcrdist_allpairs(seqs, offsets, lev_max: int, max_score: int) -> np.ndarray:
    s, o = _prep(seqs, offsets)
    return _take(_load().xo_tcrdist_allpairs(_ptr(s), _ptr(o), o.size - 1, lev_max, max_score))


# ------------------------------------------------------------ paired chains
TOKEN = "|"


def join_chains(a_seqs, a_offsets, b_seqs, b_offsets):
    """Receptors as one string each, alpha + TOKEN + beta (packed)."""
    a = np.asarray(a_seqs, np.uint8)
    b = np.asarray(b_seqs, np.uint8)
    ao = np.asarray(a_offsets, np.int64)
    bo = np.asarray(b_offsets, np.int64)
    parts = []
    for i in range(ao.size - 1):
        parts.append(a[ao[i]:ao[i + 1]].tobytes() + TOKEN.encode() + b[bo[i]:bo[i + 1]].tobytes())
    lens = np.array([len(p) for p in parts], np.int64)
    off = np.zeros(lens.size + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    return np.frombuffer(b"".join(parts), np.uint8).copy(), off


def symdel_paired(a_seqs, a_offsets, b_seqs, b_offsets, d: int) -> np.ndarray:
    """Paired-chain SymDel search: rows (i, j, dist), dist = the edit distance
    of alpha + TOKEN + beta with the token never edited."""
    s, o = _prep(*join_chains(a_seqs, a_offsets, b_seqs, b_offsets))
    return _take(_load().xo_symdel_paired(_ptr(s), _ptr(o), o.size - 1, d))


def bruteforce_paired(a_seqs, a_offsets, b_seqs, b_offsets, d: int) -> np.ndarray:
    s, o = _prep(*join_chains(a_seqs, a_offsets, b_seqs, b_offsets))
    return _take(_load().xo_bruteforce_paired(_ptr(s), _ptr(o), o.size - 1, d))


def lev_token(a: str, b: str) -> int:
    """Edit distance with the joining token never deleted, inserted or
    substituted (FORBIDDEN = 2^20 or more when no admissible alignment)."""
    ab, bb = a.encode(), b.encode()
    return _load().xo_lev_token(ab, len(ab), bb, len(bb))


def count_variants_token(s: str, d: int) -> int:
    b = s.encode()
    return _load().xo_count_variants_token(b, len(b), d)


def hamming(a: str, b: str) -> int:
    """Differing positions of two equal-length strings; -1 when the lengths
    differ (never Hamming neighbours)."""
    ab, bb = a.encode(), b.encode()
    return _load().xo_hamming(ab, len(ab), bb, len(bb))


def levenshtein(a: str, b: str) -> int:
    ab, bb = a.encode(), b.encode()
    return _load().xo_levenshtein(ab, len(ab), bb, len(bb))


def tcrdist(a: str, b: str) -> int:
    ab, bb = a.encode(), b.encode()
    return _load().xo_tcrdist(ab, len(ab), bb, len(bb))


def count_variants(s: str, d: int) -> int:
    b = s.encode()
    return _load().xo_count_variants(b, len(b), d)


def blosum62(a: str, b: str) -> int:
    return _load().xo_blosum62(a.encode(), b.encode())
