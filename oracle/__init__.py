"""CPU oracle for junction detection -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never does, and shares no code with it.

Thin ctypes wrappers over ``twopaco_oracle.cpp``; see that file for what each
function computes and the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np

from . import build as _build

_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def use_library(path):
    """Test hook: make the wrappers call another build of the oracle (one with a
    planted mistake); None goes back to the normal build. Returns the previous one."""
    global _lib
    prev = _lib
    _lib = _load(path) if isinstance(path, str) else path
    return prev


def _load(path: str) -> ctypes.CDLL:
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    U64 = ctypes.c_uint64
    I = ctypes.c_int
    L.oracle_junctions.argtypes = [P, P, U64, I, I, I, P, P]
    L.oracle_junctions_parallel.argtypes = [P, P, U64, I, I, I, I, P]
    L.oracle_junctions_parallel.restype = I
    L.oracle_alg1_exact.argtypes = [P, P, U64, I, I, I, P]
    L.oracle_pass1.argtypes = [P, P, U64, I, I, I, U64, I, U64, U64, U64, P, P]
    L.oracle_partition_cuts.argtypes = [P, U64, I, P]
    L.oracle_edges.argtypes = [P, P, U64, I, I, I, P, P, P, P, P, P, P, P, P, P]
    L.oracle_edges.restype = ctypes.c_longlong
    for f in (L.oracle_junctions, L.oracle_alg1_exact, L.oracle_pass1,
              L.oracle_partition_cuts):
        f.restype = I
    return L


class OracleError(RuntimeError):
    pass


def _check(rc: int) -> None:
    if rc == -1:
        raise OracleError("invalid argument")
    if rc == -2:
        raise OracleError("byte outside ACGTacgt (and Nn unless split_n)")
    if rc != 0:
        raise OracleError(f"oracle error {rc}")


def _prep(seqs) -> Tuple[np.ndarray, np.ndarray]:
    if isinstance(seqs, tuple) and len(seqs) == 2 and isinstance(seqs[1], np.ndarray) \
            and seqs[1].dtype == np.uint64:
        buf, off = seqs
    else:
        arrs = [np.frombuffer(s.encode(), np.uint8) if isinstance(s, str)
                else np.asarray(s, dtype=np.uint8) for s in seqs]
        lens = np.array([a.size for a in arrs], dtype=np.uint64)
        off = np.zeros(len(arrs) + 1, dtype=np.uint64)
        np.cumsum(lens, out=off[1:])
        buf = np.concatenate(arrs) if arrs else np.zeros(0, np.uint8)
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    if buf.size == 0:
        buf = np.zeros(1, np.uint8)  # valid pointer for an empty input
    return buf, np.ascontiguousarray(off, dtype=np.uint64)


def _split(flags: np.ndarray, off: np.ndarray) -> List[np.ndarray]:
    return [np.flatnonzero(flags[int(off[t]):int(off[t + 1])]).astype(np.uint64)
            for t in range(off.size - 1)]


def junction_flags(seqs, k: int, both_strands: bool = True,
                   split_n: bool = False) -> Tuple[np.ndarray, np.ndarray, int]:
    """(flags per global byte, offsets, number of distinct k-mers) by definition."""
    buf, off = _prep(seqs)
    m = int(off[-1])
    flags = np.zeros(max(m, 1), np.uint8)
    nd = ctypes.c_uint64(0)
    _check(lib().oracle_junctions(buf.ctypes.data, off.ctypes.data, off.size - 1, k,
                                  int(both_strands), int(split_n), flags.ctypes.data,
                                  ctypes.byref(nd)))
    return flags[:m], off, int(nd.value)


def junctions(seqs, k: int, both_strands: bool = True, split_n: bool = False,
              threads: int = 1) -> List[np.ndarray]:
    """Sorted junction positions of every string, by definition of J(S, k).

    With ``split_n`` every N ends its string there (the N-free pieces are the
    strings of the definition); positions stay offsets into the input strings.
    With ``threads`` > 1 the definition runs split over that many threads
    (each owns the k-mers of one hash class and scans all input).
    """
    if threads <= 1:
        flags, off, _ = junction_flags(seqs, k, both_strands, split_n)
        return _split(flags, off)
    buf, off = _prep(seqs)
    m = int(off[-1])
    flags = np.zeros(max(m, 1), np.uint8)
    _check(lib().oracle_junctions_parallel(buf.ctypes.data, off.ctypes.data, off.size - 1, k,
                                           int(both_strands), int(split_n), int(threads),
                                           flags.ctypes.data))
    return _split(flags[:m], off)


def alg1_exact(seqs, k: int, both_strands: bool = True, marks=None,
               split_n: bool = False) -> List[np.ndarray]:
    """Algorithm 1 with an exact (k+1)-mer set; all positions marked unless given."""
    buf, off = _prep(seqs)
    m = int(off[-1])
    if marks is None:
        marks = np.zeros(max(m, 1), np.uint8)
        for t in range(off.size - 1):
            a, b = int(off[t]), int(off[t + 1])
            if b - a >= k:
                marks[a:b - k + 1] = 1
    marks = np.ascontiguousarray(marks, dtype=np.uint8).copy()
    if marks.size == 0:
        marks = np.zeros(1, np.uint8)
    _check(lib().oracle_alg1_exact(buf.ctypes.data, off.ctypes.data, off.size - 1, k,
                                   int(both_strands), int(split_n), marks.ctypes.data))
    return _split(marks[:m], off)


def pass1_marks(seqs, k: int, filter_bits: int, hashes: int, both_strands: bool = True,
                q: int = 1, bin_lo: int = 0, bin_hi: int = 1,
                split_n: bool = False) -> Tuple[np.ndarray, np.ndarray, int, int]:
    """First pass with the split-block filter: (marks per byte, offsets, active, kept)."""
    buf, off = _prep(seqs)
    m = int(off[-1])
    marks = np.zeros(max(m, 1), np.uint8)
    cnt = np.zeros(2, np.uint64)
    _check(lib().oracle_pass1(buf.ctypes.data, off.ctypes.data, off.size - 1, k,
                              int(both_strands), int(split_n), filter_bits, hashes, q, bin_lo, bin_hi,
                              marks.ctypes.data, cnt.ctypes.data))
    return marks[:m], off, int(cnt[0]), int(cnt[1])


def partition_cuts(counts: Sequence[int], rounds: int) -> np.ndarray:
    """Greedy class boundaries over q counters for ``rounds`` classes."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    cuts = np.zeros(rounds + 1, np.uint64)
    _check(lib().oracle_partition_cuts(c.ctypes.data, c.size, rounds, cuts.ctypes.data))
    return cuts


def edges(seqs, k: int, both_strands: bool = True, split_n: bool = False, flags=None):
    """Compacted-graph edges by consecutive junction positions, as a dict of arrays.

    Keys: from_hi, from_lo, to_hi, to_lo (normalized k-mers), from_rc, to_rc,
    start, length (per edge, string order then position order) and
    per_string (edge count of every string). With ``flags`` (one byte per
    input byte) the edges join consecutive flagged positions instead of
    consecutive junctions (a partially compacted graph).
    """
    if flags is None:
        flags, off, _ = junction_flags(seqs, k, both_strands, split_n)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    buf, off = _prep(seqs)
    nj = max(int(flags.sum()), 1)
    out = {name: np.zeros(nj, np.uint64) for name in ("from_hi", "from_lo", "to_hi", "to_lo",
                                                         "start", "length")}
    out["from_rc"] = np.zeros(nj, np.uint8)
    out["to_rc"] = np.zeros(nj, np.uint8)
    per = np.zeros(max(off.size - 1, 1), np.uint64)
    fl = np.ascontiguousarray(flags if flags.size else np.zeros(1, np.uint8))
    e = lib().oracle_edges(buf.ctypes.data, off.ctypes.data, off.size - 1, k, int(both_strands),
                           int(split_n), fl.ctypes.data, out["from_hi"].ctypes.data, out["from_lo"].ctypes.data,
                           out["to_hi"].ctypes.data, out["to_lo"].ctypes.data,
                           out["from_rc"].ctypes.data, out["to_rc"].ctypes.data,
                           out["start"].ctypes.data, out["length"].ctypes.data, per.ctypes.data)
    _check(0 if e >= 0 else int(e))
    res = {name: a[:e] for name, a in out.items()}
    res["per_string"] = per[:off.size - 1]
    return res
