"""Seeded synthetic CDR3-beta-like amino-acid sequences.

This module only draws inputs. It holds none of the search method's
arithmetic (no deletion variants, no distances, no keys) and is the one piece
of code that both the CUDA path's callers (tests, benchmark) and the CPU
oracle's tests use.

Why synthetic: the paper benchmarks on real TCR-beta CDR3 repertoires
(Results, "Computational complexity of algorithmic approaches"), which are not
available here. The generator mimics their shape instead:

* length ~ N(14.5, 2^2) rounded to an integer, redrawn until it lies in
  [8, 22] (a truncated discretised normal);
* positions 0, 1, 2 are C, A, S with probability 0.9 each (else a draw from
  the frequency vector) and the last residue is F with probability 0.9;
* every other residue is i.i.d. from ``FREQ``, a fixed, non-uniform 20-letter
  frequency vector chosen for this generator (not estimated from any data);
* a fraction of sequences is *derived*: a copy of a uniformly chosen earlier
  fresh sequence with 1 or 2 (equally likely) random edits.  Each edit is a
  substitution, insertion or deletion with equal probability at a uniform
  position; a substitution always changes the residue; an insertion that
  would exceed 24 residues or a deletion that would go below 6 becomes a
  substitution;
* a fraction of sequences is an exact copy of a uniformly chosen earlier
  fresh sequence.

Sequences are returned packed: one ``uint8`` array holding the ASCII letters of
all sequences back to back, plus ``int64`` offsets of length n+1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

AA = "ACDEFGHIKLMNPQRSTVWY"
AA_BYTES = np.frombuffer(AA.encode(), dtype=np.uint8)

# Builder-chosen residue frequencies for non-flank positions (order of AA).
FREQ = np.array([
    0.07, 0.01, 0.06, 0.07, 0.03,   # A C D E F
    0.12, 0.02, 0.02, 0.02, 0.06,   # G H I K L
    0.01, 0.05, 0.05, 0.06, 0.05,   # M N P Q R
    0.10, 0.07, 0.03, 0.02, 0.08,   # S T V W Y
])
assert abs(FREQ.sum() - 1.0) < 1e-12

WIDTH = 24          # longest sequence the generator can produce (after edits)
LEN_MIN, LEN_MAX = 8, 22
LEN_MEAN, LEN_SD = 14.5, 2.0
FLANK_P = 0.9
MIN_AFTER_DELETE = 6
_CHUNK = 1 << 20


@dataclasses.dataclass(frozen=True)
class Workload:
    """Parameters of one synthetic self-search workload."""
    name: str
    n: int
    d: int
    seed: int
    derived_frac: float
    dup_frac: float


# The five workloads (plain d=1, plain d=2, batched, served, TCRdist prefilter).
SELF_SMALL = Workload("selfsearch_n1e4_d1", 10_000, 1, 1, 0.20, 0.0)
SELF_1M = Workload("selfsearch_n1e6_d2", 1_000_000, 2, 2, 0.15, 0.01)
TCRDIST_1M = Workload("tcrdist_n1e6_d2", 1_000_000, 2, 5, 0.15, 0.01)


def _draw_residues(rng: np.random.Generator, shape) -> np.ndarray:
    idx = rng.choice(20, size=shape, p=FREQ)
    return AA_BYTES[idx]


def _draw_lengths(rng: np.random.Generator, n: int, mean: float = LEN_MEAN, sd: float = LEN_SD,
                  lo: int = LEN_MIN, hi: int = LEN_MAX) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    todo = np.arange(n)
    while todo.size:
        v = np.rint(rng.normal(mean, sd, size=todo.size)).astype(np.int64)
        ok = (v >= lo) & (v <= hi)
        out[todo[ok]] = v[ok]
        todo = todo[~ok]
    return out


def _fresh(rng: np.random.Generator, n: int, prefix: bytes = b"CAS", lengths=None):
    """n fresh sequences as a (n, WIDTH) ASCII matrix (0-padded) and lengths.
    `lengths` = (mean, sd, lo, hi) of the length law (default: the CDR3-beta
    law above); `prefix` = the conserved first residues."""
    mats, lens = [], []
    for start in range(0, n, _CHUNK):
        m = min(_CHUNK, n - start)
        L = _draw_lengths(rng, m) if lengths is None else _draw_lengths(rng, m, *lengths)
        M = _draw_residues(rng, (m, WIDTH))
        for pos, ch in enumerate(prefix):
            keep = rng.random(m) < FLANK_P
            M[keep, pos] = ch
        last = rng.random(m) < FLANK_P
        M[np.arange(m)[last], L[last] - 1] = ord("F")
        M[np.arange(WIDTH)[None, :] >= L[:, None]] = 0
        mats.append(M)
        lens.append(L)
    if not mats:
        return np.zeros((0, WIDTH), np.uint8), np.zeros(0, np.int64)
    return np.concatenate(mats), np.concatenate(lens)


def mutate(rng: np.random.Generator, M: np.ndarray, L: np.ndarray,
           n_edits: np.ndarray) -> None:
    """Apply n_edits[r] (0, 1 or 2) random edits to row r of M in place."""
    cols = np.arange(WIDTH)[None, :]
    for e in range(int(n_edits.max(initial=0))):
        rows = np.flatnonzero(n_edits > e)
        if rows.size == 0:
            continue
        kind = rng.integers(0, 3, size=rows.size)          # 0 sub, 1 ins, 2 del
        Lr = L[rows]
        kind[(kind == 1) & (Lr >= WIDTH)] = 0
        kind[(kind == 2) & (Lr <= MIN_AFTER_DELETE)] = 0
        u = rng.random(rows.size)
        new_res = _draw_residues(rng, rows.size)
        shift = rng.integers(0, 19, size=rows.size)
        # substitution: another residue, uniform over the 19 others
        sub = rows[kind == 0]
        if sub.size:
            p = np.floor(u[kind == 0] * L[sub]).astype(np.int64)
            cur = M[sub, p]
            cur_idx = np.searchsorted(AA_BYTES, cur)   # AA is sorted
            M[sub, p] = AA_BYTES[(cur_idx + 1 + shift[kind == 0]) % 20]
        ins = rows[kind == 1]
        if ins.size:
            p = np.floor(u[kind == 1] * (L[ins] + 1)).astype(np.int64)
            src = np.where(cols > p[:, None], cols - 1, cols)
            Mi = np.take_along_axis(M[ins], src, axis=1)
            Mi[cols == p[:, None]] = new_res[kind == 1]
            M[ins] = Mi
            L[ins] += 1
        dele = rows[kind == 2]
        if dele.size:
            p = np.floor(u[kind == 2] * L[dele]).astype(np.int64)
            src = np.where(cols >= p[:, None], cols + 1, cols)
            Mp = np.concatenate([M[dele], np.zeros((dele.size, 1), np.uint8)], axis=1)
            M[dele] = np.take_along_axis(Mp, src, axis=1)
            L[dele] -= 1


def _pack(M: np.ndarray, L: np.ndarray):
    mask = np.arange(WIDTH)[None, :] < L[:, None]
    seqs = np.ascontiguousarray(M[mask])
    offsets = np.zeros(L.size + 1, dtype=np.int64)
    np.cumsum(L, out=offsets[1:])
    return seqs, offsets


def generate(n: int, seed: int, derived_frac: float = 0.2, dup_frac: float = 0.0):
    """n sequences; returns (seqs uint8[total], offsets int64[n+1])."""
    M, L = generate_matrix(n, seed, derived_frac, dup_frac)
    return _pack(M, L)


def generate_matrix(n: int, seed: int, derived_frac: float = 0.2, dup_frac: float = 0.0):
    rng = np.random.default_rng(seed)
    M, L = _fresh(rng, n)
    if n == 0:
        return M, L
    kind = rng.choice(3, size=n, p=[1.0 - derived_frac - dup_frac, derived_frac, dup_frac])
    kind[0] = 0
    fresh_idx = np.flatnonzero(kind == 0)
    other = np.flatnonzero(kind != 0)
    if other.size:
        n_before = np.searchsorted(fresh_idx, other)          # >= 1 (slot 0 fresh)
        src = fresh_idx[np.floor(rng.random(other.size) * n_before).astype(np.int64)]
        M[other] = M[src]
        L[other] = L[src]
        der = other[kind[other] == 1]
        n_edits = np.zeros(n, dtype=np.int64)
        n_edits[der] = 1 + (rng.random(der.size) < 0.5)
        mutate(rng, M, L, n_edits)
    return M, L


def workload(w: Workload, n: int | None = None):
    """Sequences of a named workload; ``n`` (<= w.n) takes its first n."""
    seqs, off = generate(w.n, w.seed, w.derived_frac, w.dup_frac)
    if n is not None and n < w.n:
        seqs = seqs[: off[n]]
        off = off[: n + 1]
    return seqs, off


def from_strings(strs):
    """Pack a list of str/bytes into (seqs, offsets)."""
    bs = [s.encode() if isinstance(s, str) else bytes(s) for s in strs]
    offsets = np.zeros(len(bs) + 1, dtype=np.int64)
    np.cumsum([len(b) for b in bs], out=offsets[1:])
    seqs = np.frombuffer(b"".join(bs), dtype=np.uint8).copy()
    return seqs, offsets


def to_strings(seqs, offsets):
    raw = bytes(np.asarray(seqs, dtype=np.uint8))
    off = np.asarray(offsets)
    return [raw[off[i]:off[i + 1]].decode() for i in range(off.size - 1)]


# ---------------------------------------------------------------- batched ---
BATCH_REPS, BATCH_MIN, BATCH_MAX, BATCH_SEED, BATCH_D = 256, 1_000, 200_000, 3, 2


def batched(n_rep: int = BATCH_REPS, seed: int = BATCH_SEED, size_min: int = BATCH_MIN,
            size_max: int = BATCH_MAX):
    """Repertoires with log-uniform sizes on [size_min, size_max].

    Returns (seqs, offsets, rep_offsets) where rep_offsets[r]..rep_offsets[r+1]
    are the sequence indices of repertoire r in the concatenation.
    """
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(size_min), math.log(size_max), n_rep)))
    sizes = sizes.astype(np.int64)
    parts_s, parts_o = [], []
    for r in range(n_rep):
        s, o = generate(int(sizes[r]), seed * 1_000_003 + r, 0.15, 0.01)
        parts_s.append(s)
        parts_o.append(o)
    return concat(parts_s, parts_o) + (np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64),)


def concat(parts_s, parts_o):
    seqs = np.concatenate(parts_s) if parts_s else np.zeros(0, np.uint8)
    lens = np.concatenate([np.diff(o) for o in parts_o]) if parts_o else np.zeros(0, np.int64)
    off = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return seqs, off


# ----------------------------------------------------------------- served ---
SERVE_REF_N, SERVE_REQUESTS, SERVE_MAX_REQ, SERVE_RATE, SERVE_SEED = 10_000_000, 2_000, 10_000, 200.0, 4


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    seqs: np.ndarray
    offsets: np.ndarray


def served(ref_n: int = SERVE_REF_N, n_req: int = SERVE_REQUESTS, max_req: int = SERVE_MAX_REQ,
           rate: float = SERVE_RATE, seed: int = SERVE_SEED):
    """A reference set plus a stream of query requests.

    Request sizes are round(exp(U(0, ln max_req))); half the queries of a
    request are 1-2-edit mutants of uniformly chosen reference entries, the
    rest fresh draws; arrivals form a Poisson process of the given rate.
    Returns (ref_seqs, ref_offsets, [Request]).
    """
    M, L = generate_matrix(ref_n, seed, 0.15, 0.01)
    ref_seqs, ref_off = _pack(M, L)
    rng = np.random.default_rng(seed + 7_777)
    sizes = np.rint(np.exp(rng.uniform(0.0, math.log(max_req), n_req))).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    reqs = []
    for r in range(n_req):
        m = int(sizes[r])
        n_mut = m // 2
        src = rng.integers(0, ref_n, n_mut)
        Mm, Lm = M[src].copy(), L[src].copy()
        mutate(rng, Mm, Lm, 1 + (rng.random(n_mut) < 0.5).astype(np.int64))
        Mf, Lf = _fresh(rng, m - n_mut)
        Mq = np.concatenate([Mm, Mf])
        Lq = np.concatenate([Lm, Lf])
        perm = rng.permutation(m)
        s, o = _pack(Mq[perm], Lq[perm])
        reqs.append(Request(r, float(arrivals[r]), s, o))
    return ref_seqs, ref_off, reqs


# ---------------------------------------------------------- paired chains ---
# CDR3-alpha-like first chains: length ~ N(13.5, 2^2) on [7, 21], conserved
# 'CAV' start and final F with probability 0.9 each (builder-chosen, like
# FREQ); the second chain follows the CDR3-beta law above.
ALPHA_LENGTHS = (13.5, 2.0, 7, 21)
ALPHA_PREFIX = b"CAV"


def paired(n: int, seed: int, derived_frac: float = 0.15, dup_frac: float = 0.01):
    """n receptors (alpha chain, beta chain).  A derived receptor copies both
    chains of an earlier fresh one and gets 1 or 2 edits in all, each in the
    alpha or the beta chain with equal probability; a duplicate copies both
    chains.  Returns (a_seqs, a_offsets, b_seqs, b_offsets)."""
    rng = np.random.default_rng(seed)
    Ma, La = _fresh(rng, n, ALPHA_PREFIX, ALPHA_LENGTHS)
    Mb, Lb = _fresh(rng, n)
    if n:
        kind = rng.choice(3, size=n, p=[1.0 - derived_frac - dup_frac, derived_frac, dup_frac])
        kind[0] = 0
        fresh_idx = np.flatnonzero(kind == 0)
        other = np.flatnonzero(kind != 0)
        if other.size:
            n_before = np.searchsorted(fresh_idx, other)
            src = fresh_idx[np.floor(rng.random(other.size) * n_before).astype(np.int64)]
            Ma[other], La[other] = Ma[src], La[src]
            Mb[other], Lb[other] = Mb[src], Lb[src]
            der = other[kind[other] == 1]
            total = 1 + (rng.random(der.size) < 0.5)
            in_a = rng.binomial(total, 0.5)
            edits_a = np.zeros(n, dtype=np.int64)
            edits_b = np.zeros(n, dtype=np.int64)
            edits_a[der] = in_a
            edits_b[der] = total - in_a
            mutate(rng, Ma, La, edits_a)
            mutate(rng, Mb, Lb, edits_b)
    return _pack(Ma, La) + _pack(Mb, Lb)
