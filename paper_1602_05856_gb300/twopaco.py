"""Python binding of the C ABI in ``include/twopaco.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
part of the computation: the junction detection runs in the CUDA kernels of
``libtwopaco.so``. If the library is not built this module raises on first
use -- there is no CPU path.

``DeviceBuild`` adds the device-resident workflow on top of the same calls,
with PyTorch used only to own device memory and to name the CUDA stream.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtwopaco.so")

OK, EINVAL, EBADBASE, ENOMEM, ETIMEOUT, ECUDA, EOVERFLOW, ESCRATCH = 0, -1, -2, -3, -4, -5, -6, -7
NOALLOC_SCRATCH_BYTES = 32 << 20
STATE_CANDIDATES, STATE_JUNCTIONS, STATE_BINS, STATE_CUTS = 0, 1, 2, 3


class TwopacoError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib().twopaco_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


class _Options(ctypes.Structure):
    _fields_ = [("hashes", ctypes.c_int), ("both_strands", ctypes.c_int),
                ("partition_bins", ctypes.c_uint32), ("table_slots", ctypes.c_uint64),
                ("candidate_records", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p),
                ("split_at_n", ctypes.c_int), ("run_capacity", ctypes.c_uint64),
                ("wide_layout", ctypes.c_int), ("partial", ctypes.c_int),
                ("per_string_launches", ctypes.c_int), ("bucket_inserts", ctypes.c_int),
                ("launch_blocks_per_sm", ctypes.c_int), ("ordered_first_pass", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("positions", ctypes.c_uint64), ("pass1_marks", ctypes.c_uint64),
                ("pass2_marks", ctypes.c_uint64), ("table_slots", ctypes.c_uint64),
                ("bad_base_index", ctypes.c_uint64), ("overflow", ctypes.c_uint32),
                ("timeout", ctypes.c_uint32), ("ordered_rounds", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class _Edge(ctypes.Structure):
    _fields_ = [("from_hi", ctypes.c_uint64), ("from_lo", ctypes.c_uint64), ("to_hi", ctypes.c_uint64),
                ("to_lo", ctypes.c_uint64), ("start", ctypes.c_uint64), ("length", ctypes.c_uint64),
                ("from_rc", ctypes.c_uint32), ("to_rc", ctypes.c_uint32)]


EDGE_DTYPE = np.dtype([("from_hi", np.uint64), ("from_lo", np.uint64), ("to_hi", np.uint64),
                       ("to_lo", np.uint64), ("start", np.uint64), ("length", np.uint64),
                       ("from_rc", np.uint32), ("to_rc", np.uint32)])


class _EdgeList(ctypes.Structure):
    _fields_ = [("n_seqs", ctypes.c_uint64), ("offsets", ctypes.POINTER(ctypes.c_uint64)),
                ("edges", ctypes.POINTER(_Edge))]


class _Result(ctypes.Structure):
    _fields_ = [("n_seqs", ctypes.c_uint64), ("offsets", ctypes.POINTER(ctypes.c_uint64)),
                ("positions", ctypes.POINTER(ctypes.c_uint64)), ("stats", _Stats)]


_LIB: Optional[ctypes.CDLL] = None


def _lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_1602_05856_gb300.build.build() (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.twopaco_strerror.argtypes = [I]
        L.twopaco_strerror.restype = ctypes.c_char_p
        L.twopaco_default_options.argtypes = [ctypes.POINTER(_Options)]
        L.twopaco_default_options.restype = None
        L.twopaco_build_ex.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(U64), U64, I,
                                       U64, I, ctypes.POINTER(_Options),
                                       ctypes.POINTER(ctypes.POINTER(_Result))]
        L.twopaco_build_ex.restype = I
        L.twopaco_build.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(U64), U64, I,
                                    U64, I, ctypes.POINTER(ctypes.POINTER(_Result))]
        L.twopaco_build.restype = I
        L.twopaco_result_free.argtypes = [ctypes.POINTER(_Result)]
        L.twopaco_result_free.restype = None
        L.twopaco_workspace_size.argtypes = [U64, U64, I, U64, I, ctypes.POINTER(_Options),
                                             ctypes.POINTER(U64)]
        L.twopaco_workspace_size.restype = I
        L.twopaco_run_device.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options), P, U64,
                                         P, P, U64]
        L.twopaco_run_device.restype = I
        L.twopaco_run_rounds.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options), P, U64,
                                         I, I, P, P, U64]
        L.twopaco_run_rounds.restype = I
        L.twopaco_run_streamed.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options), P, U64,
                                           P, U64, P, P, U64]
        L.twopaco_run_streamed.restype = I
        L.twopaco_shard_begin.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options), P, U64, I]
        L.twopaco_shard_begin.restype = I
        L.twopaco_shard_rounds.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options), P, U64,
                                           I, I, P]
        L.twopaco_shard_rounds.restype = I
        L.twopaco_state_device.argtypes = [U64, U64, I, U64, I, ctypes.POINTER(_Options), P, I,
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(U64)]
        L.twopaco_state_device.restype = I
        L.twopaco_selftest_bounded_wait.argtypes = [P]
        L.twopaco_selftest_bounded_wait.restype = I
        L.twopaco_checkpoint_bytes.argtypes = [U64, U64, I, U64, I, ctypes.POINTER(_Options),
                                               ctypes.POINTER(U64)]
        L.twopaco_checkpoint_bytes.restype = I
        L.twopaco_checkpoint_save.argtypes = [P, I, P, U64, P]
        L.twopaco_checkpoint_save.restype = I
        L.twopaco_checkpoint_load.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options), P,
                                              U64, P, U64, ctypes.POINTER(I)]
        L.twopaco_checkpoint_load.restype = I
        L.twopaco_run_device_noalloc.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options),
                                                 P, P, U64, ctypes.POINTER(_Stats)]
        L.twopaco_run_device_noalloc.restype = I
        L.twopaco_read_stats.argtypes = [P, P, ctypes.POINTER(_Stats)]
        L.twopaco_read_stats.restype = I
        L.twopaco_read_state.argtypes = [P, I, P, U64, P]
        L.twopaco_read_state.restype = I
        L.twopaco_kernel_launches.argtypes = []
        L.twopaco_kernel_launches.restype = ctypes.c_ulonglong
        L.twopaco_context_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
        L.twopaco_context_create.restype = I
        L.twopaco_context_destroy.argtypes = [P]
        L.twopaco_context_destroy.restype = None
        L.twopaco_build_ctx.argtypes = [P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(U64), U64,
                                        I, U64, I, ctypes.POINTER(_Options), ctypes.POINTER(_Result)]
        L.twopaco_build_ctx.restype = I
        L.twopaco_edges_ctx.argtypes = [P, ctypes.POINTER(_EdgeList)]
        L.twopaco_edges_ctx.restype = I
        L.twopaco_edges_device.argtypes = [P, P, U64, P, P, P, P, U64, P]
        L.twopaco_edges_device.restype = I
        L.twopaco_plan_create.argtypes = [P, P, U64, U64, I, U64, I, ctypes.POINTER(_Options), P, U64,
                                          P, P, U64, ctypes.POINTER(ctypes.c_void_p)]
        L.twopaco_plan_create.restype = I
        L.twopaco_plan_launch.argtypes = [P, P]
        L.twopaco_plan_launch.restype = I
        L.twopaco_plan_destroy.argtypes = [P]
        L.twopaco_plan_destroy.restype = None
        L.twopaco_profile_enable.argtypes = [I]
        L.twopaco_profile_enable.restype = I
        L.twopaco_profile_kernels.argtypes = [ctypes.POINTER(ctypes.c_char_p),
                                              ctypes.POINTER(ctypes.c_ulonglong),
                                              ctypes.POINTER(ctypes.c_double), I]
        L.twopaco_profile_kernels.restype = I
        _LIB = L
    return _LIB


def load() -> ctypes.CDLL:
    """Load ``libtwopaco.so`` (raises if it is not built)."""
    return _lib()


@dataclass
class Options:
    hashes: int = 4
    both_strands: bool = True
    partition_bins: int = 65536
    table_slots: int = 0
    cuda_stream: int = 0  # cudaStream_t as an integer; 0 = default stream
    candidate_records: int = 0
    split_at_n: bool = False  # an N (either case) ends its string there
    run_capacity: int = 0     # split_at_n: room for piece boundaries; 0 = automatic
    wide_layout: int = 0      # 1/2: the large-input workspace layout at any size (testing)
    partial: bool = False     # omit pass 2: the partially compacted graph's positions
    per_string_launches: bool = False  # every loop launched once per string (a baseline)
    bucket_inserts: int = 0   # first-pass ORs through region buckets: 0 auto (> 64 MiB), 1 always, 2 never
    launch_blocks_per_sm: int = 0  # launch shape of the pass kernels: resident blocks per SM (0: all)
    ordered_first_pass: int = 0    # first pass in filter-region order: 0 auto (>= 1 GiB), 1 always, 2 never

    def _c(self) -> _Options:
        return _Options(int(self.hashes), int(bool(self.both_strands)), int(self.partition_bins),
                        int(self.table_slots), int(self.candidate_records),
                        ctypes.c_void_p(int(self.cuda_stream) or None), int(bool(self.split_at_n)),
                        int(self.run_capacity), int(self.wide_layout), int(bool(self.partial)),
                        int(bool(self.per_string_launches)), int(self.bucket_inserts),
                        int(self.launch_blocks_per_sm), int(self.ordered_first_pass))


def _stats_dict(s: _Stats) -> Dict[str, int]:
    return {f: int(getattr(s, f)) for f, _ in _Stats._fields_}


def _as_bytes(s) -> np.ndarray:
    if isinstance(s, str):
        return np.frombuffer(s.encode("ascii"), np.uint8)
    if isinstance(s, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(s), np.uint8)
    return np.ascontiguousarray(s, dtype=np.uint8)


def twopaco_strerror(code: int) -> str:
    return _lib().twopaco_strerror(int(code)).decode()


def twopaco_kernel_launches() -> int:
    return int(_lib().twopaco_kernel_launches())


def twopaco_profile_enable(on: bool) -> None:
    _lib().twopaco_profile_enable(int(bool(on)))


def twopaco_profile_kernels() -> Dict[str, Dict[str, float]]:
    """{kernel name: {"launches": n, "ms": summed device time}} since profiling was enabled."""
    cap = 64
    names = (ctypes.c_char_p * cap)()
    cnt = (ctypes.c_ulonglong * cap)()
    ms = (ctypes.c_double * cap)()
    n = _lib().twopaco_profile_kernels(names, cnt, ms, cap)
    if n < 0:
        raise TwopacoError(n, "twopaco_profile_kernels")
    return {names[i].decode(): {"launches": int(cnt[i]), "ms": float(ms[i])} for i in range(min(n, cap))}


def twopaco_build_ex(seqs: Sequence, k: int, filter_bits: int, rounds: int = 1,
                     options: Optional[Options] = None):
    """Host-to-host build: (list of junction-position arrays, stats dict)."""
    L = _lib()
    arrs = [_as_bytes(s) for s in seqs]
    n = len(arrs)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data if a.size else None for a in arrs])
    lens = (ctypes.c_uint64 * max(n, 1))(*[a.size for a in arrs])
    out = ctypes.POINTER(_Result)()
    opt = (options or Options())._c()
    rc = L.twopaco_build_ex(ptrs, lens, n, int(k), int(filter_bits), int(rounds),
                            ctypes.byref(opt), ctypes.byref(out))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_build_ex")
    try:
        r = out.contents
        off = np.ctypeslib.as_array(r.offsets, shape=(n + 1,)).copy()
        total = int(off[-1])
        pos = (np.ctypeslib.as_array(r.positions, shape=(total,)).copy() if total
               else np.zeros(0, np.uint64))
        stats = _stats_dict(r.stats)
    finally:
        L.twopaco_result_free(out)
    return [pos[off[t]:off[t + 1]] for t in range(n)], stats


class Context:
    """A reusable build context (``twopaco_context_create``): device and pinned
    buffers survive across ``build`` calls, so repeated builds allocate nothing."""

    def __init__(self):
        h = ctypes.c_void_p()
        rc = _lib().twopaco_context_create(ctypes.byref(h))
        if rc != OK:
            raise TwopacoError(rc, "twopaco_context_create")
        self._h = h

    def close(self) -> None:
        if self._h:
            _lib().twopaco_context_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build(self, seqs: Sequence, k: int, filter_bits: int, rounds: int = 1,
              options: Optional[Options] = None, copy: bool = True):
        """twopaco_build_ctx: (list of junction-position arrays, stats). With
        copy=False the arrays are views of the context's pinned buffers, valid
        until the next call."""
        arrs = [_as_bytes(s) for s in seqs]
        n = len(arrs)
        ptrs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data if a.size else None for a in arrs])
        lens = (ctypes.c_uint64 * max(n, 1))(*[a.size for a in arrs])
        res = _Result()
        opt = (options or Options())._c()
        rc = _lib().twopaco_build_ctx(self._h, ptrs, lens, n, int(k), int(filter_bits), int(rounds),
                                      ctypes.byref(opt), ctypes.byref(res))
        if rc != OK:
            raise TwopacoError(rc, "twopaco_build_ctx")
        off = np.ctypeslib.as_array(res.offsets, shape=(n + 1,))
        total = int(off[-1])
        pos = (np.ctypeslib.as_array(res.positions, shape=(total,)) if total
               else np.zeros(0, np.uint64))
        if copy:
            off, pos = off.copy(), pos.copy()
        return [pos[off[t]:off[t + 1]] for t in range(n)], _stats_dict(res.stats)

    def edges(self):
        """twopaco_edges_ctx: (edge offsets per string, structured array of EDGE_DTYPE)."""
        lst = _EdgeList()
        rc = _lib().twopaco_edges_ctx(self._h, ctypes.byref(lst))
        if rc != OK:
            raise TwopacoError(rc, "twopaco_edges_ctx")
        n = int(lst.n_seqs)
        off = np.ctypeslib.as_array(lst.offsets, shape=(n + 1,)).copy()
        ne = int(off[-1])
        if ne:
            raw = ctypes.cast(lst.edges, ctypes.POINTER(ctypes.c_uint8 * (ne * EDGE_DTYPE.itemsize))).contents
            arr = np.frombuffer(bytes(raw), dtype=EDGE_DTYPE).copy()
        else:
            arr = np.zeros(0, EDGE_DTYPE)
        return off, arr


def twopaco_build(seqs: Sequence, k: int, filter_bits: int, rounds: int = 1):
    return twopaco_build_ex(seqs, k, filter_bits, rounds, None)


def twopaco_workspace_size(total_bases: int, n_seqs: int, k: int, filter_bits: int, rounds: int = 1,
                           options: Optional[Options] = None) -> int:
    b = ctypes.c_uint64(0)
    opt = (options or Options())._c()
    rc = _lib().twopaco_workspace_size(int(total_bases), int(n_seqs), int(k), int(filter_bits),
                                       int(rounds), ctypes.byref(opt), ctypes.byref(b))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_workspace_size")
    return int(b.value)


def twopaco_run_device(d_bases: int, d_offsets: int, n_seqs: int, total_bases: int, k: int,
                       filter_bits: int, rounds: int, options: Optional[Options], d_workspace: int,
                       workspace_bytes: int, d_out_offsets: int, d_out_positions: int,
                       out_capacity: int) -> None:
    opt = (options or Options())._c()
    rc = _lib().twopaco_run_device(d_bases or None, d_offsets or None, int(n_seqs), int(total_bases),
                                   int(k), int(filter_bits), int(rounds), ctypes.byref(opt),
                                   d_workspace or None, int(workspace_bytes), d_out_offsets or None,
                                   d_out_positions or None, int(out_capacity))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_run_device")


def twopaco_run_rounds(d_bases: int, d_offsets: int, n_seqs: int, total_bases: int, k: int,
                       filter_bits: int, rounds: int, options: Optional[Options], d_workspace: int,
                       workspace_bytes: int, round_begin: int, round_end: int, d_out_offsets: int,
                       d_out_positions: int, out_capacity: int) -> None:
    opt = (options or Options())._c()
    rc = _lib().twopaco_run_rounds(d_bases or None, d_offsets or None, int(n_seqs), int(total_bases),
                                   int(k), int(filter_bits), int(rounds), ctypes.byref(opt),
                                   d_workspace or None, int(workspace_bytes), int(round_begin),
                                   int(round_end), d_out_offsets or None, d_out_positions or None,
                                   int(out_capacity))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_run_rounds")


def twopaco_run_streamed(h_bases: int, d_offsets: int, n_seqs: int, total_bases: int, k: int,
                         filter_bits: int, rounds: int, options: Optional[Options], d_workspace: int,
                         workspace_bytes: int, d_staging: int, staging_bytes: int, d_out_offsets: int,
                         d_out_positions: int, out_capacity: int) -> None:
    """A run whose input bytes (host address h_bases) are streamed in through d_staging."""
    opt = (options or Options())._c()
    rc = _lib().twopaco_run_streamed(h_bases or None, d_offsets or None, int(n_seqs), int(total_bases),
                                     int(k), int(filter_bits), int(rounds), ctypes.byref(opt),
                                     d_workspace or None, int(workspace_bytes), d_staging or None,
                                     int(staging_bytes), d_out_offsets or None, d_out_positions or None,
                                     int(out_capacity))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_run_streamed")


def twopaco_shard_begin(d_bases: int, d_offsets: int, n_seqs: int, total_bases: int, k: int,
                        filter_bits: int, rounds: int, options: Optional[Options], d_workspace: int,
                        workspace_bytes: int, compute_cut: bool) -> None:
    opt = (options or Options())._c()
    rc = _lib().twopaco_shard_begin(d_bases or None, d_offsets or None, int(n_seqs), int(total_bases),
                                    int(k), int(filter_bits), int(rounds), ctypes.byref(opt),
                                    d_workspace or None, int(workspace_bytes), int(bool(compute_cut)))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_shard_begin")


def twopaco_shard_rounds(d_bases: int, d_offsets: int, n_seqs: int, total_bases: int, k: int,
                         filter_bits: int, rounds: int, options: Optional[Options], d_workspace: int,
                         workspace_bytes: int, shard: int, n_shards: int, d_class_cut: int = 0) -> None:
    opt = (options or Options())._c()
    rc = _lib().twopaco_shard_rounds(d_bases or None, d_offsets or None, int(n_seqs), int(total_bases),
                                     int(k), int(filter_bits), int(rounds), ctypes.byref(opt),
                                     d_workspace or None, int(workspace_bytes), int(shard), int(n_shards),
                                     d_class_cut or None)
    if rc != OK:
        raise TwopacoError(rc, "twopaco_shard_rounds")


def twopaco_state_device(total_bases: int, n_seqs: int, k: int, filter_bits: int, rounds: int,
                         options: Optional[Options], d_workspace: int, which: int):
    """(device address, bytes) of one piece of a workspace's state."""
    opt = (options or Options())._c()
    ptr, nb = ctypes.c_void_p(), ctypes.c_uint64(0)
    rc = _lib().twopaco_state_device(int(total_bases), int(n_seqs), int(k), int(filter_bits), int(rounds),
                                     ctypes.byref(opt), d_workspace or None, int(which), ctypes.byref(ptr),
                                     ctypes.byref(nb))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_state_device")
    return int(ptr.value or 0), int(nb.value)


class _DeviceWords:
    """A device buffer of 32-bit words described by __cuda_array_interface__, so that
    torch.as_tensor can view it in place (no copy)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes // 4,), "typestr": "<i4",
                                         "data": (ptr, False), "version": 3, "strides": None}


def twopaco_selftest_bounded_wait(cuda_stream: int = 0) -> int:
    """Run one bounded device wait that must give up; returns the library's code
    (ETIMEOUT expected)."""
    return int(_lib().twopaco_selftest_bounded_wait(cuda_stream or None))


def twopaco_checkpoint_bytes(total_bases: int, n_seqs: int, k: int, filter_bits: int, rounds: int,
                             options: Optional[Options] = None) -> int:
    out = ctypes.c_uint64(0)
    opt = (options or Options())._c()
    rc = _lib().twopaco_checkpoint_bytes(int(total_bases), int(n_seqs), int(k), int(filter_bits),
                                         int(rounds), ctypes.byref(opt), ctypes.byref(out))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_checkpoint_bytes")
    return int(out.value)


def twopaco_checkpoint_save(d_workspace: int, next_round: int, nbytes: int,
                            cuda_stream: int = 0) -> bytes:
    buf = ctypes.create_string_buffer(max(int(nbytes), 1))
    rc = _lib().twopaco_checkpoint_save(d_workspace or None, int(next_round), buf, int(nbytes),
                                        cuda_stream or None)
    if rc != OK:
        raise TwopacoError(rc, "twopaco_checkpoint_save")
    return buf.raw[:int(nbytes)]


def twopaco_checkpoint_load(d_bases: int, d_offsets: int, n_seqs: int, total_bases: int, k: int,
                            filter_bits: int, rounds: int, options: Optional[Options],
                            d_workspace: int, workspace_bytes: int, blob: bytes) -> int:
    opt = (options or Options())._c()
    nxt = ctypes.c_int(0)
    rc = _lib().twopaco_checkpoint_load(d_bases or None, d_offsets or None, int(n_seqs),
                                        int(total_bases), int(k), int(filter_bits), int(rounds),
                                        ctypes.byref(opt), d_workspace or None, int(workspace_bytes),
                                        blob, len(blob), ctypes.byref(nxt))
    if rc != OK:
        raise TwopacoError(rc, "twopaco_checkpoint_load")
    return int(nxt.value)


def twopaco_run_device_noalloc(d_bases: int, d_offsets: int, n_seqs: int, total_bases: int, k: int,
                               filter_bits: int, rounds: int, options: Optional[Options],
                               d_out_offsets: int, d_out_positions: int, out_capacity: int,
                               check: bool = True) -> Dict[str, int]:
    """The run that allocates nothing (its workspace is the library's static
    scratch buffer); waits for the run and returns its stats."""
    opt = (options or Options())._c()
    st = _Stats()
    rc = _lib().twopaco_run_device_noalloc(d_bases or None, d_offsets or None, int(n_seqs),
                                           int(total_bases), int(k), int(filter_bits), int(rounds),
                                           ctypes.byref(opt), d_out_offsets or None,
                                           d_out_positions or None, int(out_capacity),
                                           ctypes.byref(st))
    if check and rc != OK:
        raise TwopacoError(rc, "twopaco_run_device_noalloc")
    d = _stats_dict(st)
    d["rc"] = int(rc)
    return d


def twopaco_edges_device(d_workspace: int, d_offsets: int, n_seqs: int, d_out_offsets: int,
                         d_out_positions: int, d_edge_offsets: int, d_edges: int, edge_capacity: int,
                         cuda_stream: int = 0) -> None:
    rc = _lib().twopaco_edges_device(d_workspace or None, d_offsets or None, int(n_seqs),
                                     d_out_offsets or None, d_out_positions or None,
                                     d_edge_offsets or None, d_edges or None, int(edge_capacity),
                                     cuda_stream or None)
    if rc != OK:
        raise TwopacoError(rc, "twopaco_edges_device")


def twopaco_read_stats(d_workspace: int, cuda_stream: int = 0, check: bool = True) -> Dict[str, int]:
    s = _Stats()
    rc = _lib().twopaco_read_stats(d_workspace or None, cuda_stream or None, ctypes.byref(s))
    if check and rc != OK:
        raise TwopacoError(rc, "twopaco_read_stats")
    d = _stats_dict(s)
    d["rc"] = int(rc)
    return d


def twopaco_read_state(d_workspace: int, which: int, count: int, cuda_stream: int = 0) -> np.ndarray:
    out = np.zeros(max(int(count), 1), np.uint32)
    rc = _lib().twopaco_read_state(d_workspace or None, int(which), out.ctypes.data, int(count) * 4,
                                   cuda_stream or None)
    if rc != OK:
        raise TwopacoError(rc, "twopaco_read_state")
    return out[:int(count)]


class DeviceBuild:
    """Device-resident runs over one input, with buffers owned by PyTorch.

    ``bases`` (uint8) and ``offsets`` (n + 1 entries) may be host arrays or
    CUDA tensors; they are made resident once. ``run()`` launches one full
    build on ``stream`` (default: the current stream) without synchronising.
    With ``resident=False`` the bases stay where they are (host memory) and
    only ``run_streamed`` runs. ``capacity`` bounds the output positions
    (default: one per k-mer position, which can never overflow).
    """

    def __init__(self, bases, offsets, k: int, filter_bits: int, rounds: int = 1,
                 options: Optional[Options] = None, device: str = "cuda",
                 capacity: Optional[int] = None, resident: bool = True):
        import torch
        self.torch = torch
        self.k, self.filter_bits, self.rounds = int(k), int(filter_bits), int(rounds)
        self.options = options or Options()
        dev = torch.device(device)
        if resident:
            self.bases = torch.as_tensor(np.asarray(bases, dtype=np.uint8) if not torch.is_tensor(bases)
                                         else bases, device=dev).contiguous()
        else:
            self.bases = None
        off = offsets.cpu().numpy() if torch.is_tensor(offsets) else np.asarray(offsets)
        off = off.astype(np.uint64)
        self.n_seqs = off.size - 1
        self.total_bases = int(off[-1])
        self.positions_upper = int(sum(max(0, int(off[t + 1] - off[t]) - self.k + 1)
                                       for t in range(self.n_seqs)))
        self.offsets = torch.as_tensor(off.view(np.int64), device=dev).contiguous()
        self.ws_bytes = twopaco_workspace_size(self.total_bases, self.n_seqs, self.k,
                                               self.filter_bits, self.rounds, self.options)
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        self.out_offsets = torch.zeros(self.n_seqs + 1, dtype=torch.int64, device=dev)
        self.capacity = max(self.positions_upper if capacity is None else int(capacity), 1)
        self.out_positions = torch.empty(self.capacity, dtype=torch.int64, device=dev)

    def _bases_ptr(self, reads: bool = True) -> int:
        """Device address of the bases. A build that is not resident has none: only
        calls that do not read the bases (writing the output again) take the host
        address its last streamed run read; the others raise."""
        if not self.total_bases:
            return 0
        if self.bases is not None:
            return self.bases.data_ptr()
        if reads or not getattr(self, "_host_ptr", 0):
            raise ValueError("the bases of this build are not resident on the device")
        return self._host_ptr

    def _stream(self, stream) -> int:
        if stream is None:
            stream = self.torch.cuda.current_stream()
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)

    def run(self, stream=None) -> None:
        if getattr(self, "_plan", None):
            rc = _lib().twopaco_plan_launch(self._plan, self._stream(stream) or None)
            if rc != OK:
                raise TwopacoError(rc, "twopaco_plan_launch")
            return
        opt = dataclasses.replace(self.options, cuda_stream=self._stream(stream))
        twopaco_run_device(self._bases_ptr(), self.offsets.data_ptr(),
                           self.n_seqs, self.total_bases, self.k, self.filter_bits, self.rounds, opt,
                           self.ws_ptr, self.ws_bytes, self.out_offsets.data_ptr(),
                           self.out_positions.data_ptr(), self.capacity)

    def run_streamed(self, host_bases, staging, stream=None) -> None:
        """One full build with the bases read from host memory (twopaco_run_streamed):
        host_bases a page-locked CPU uint8 tensor (or any host array) of total_bases
        bytes, staging a 256-byte aligned CUDA uint8 tensor split into two halves."""
        import torch
        hp = host_bases.data_ptr() if torch.is_tensor(host_bases) else np.asarray(host_bases).ctypes.data
        self._host_ptr = hp
        if staging.data_ptr() % 256:
            raise ValueError("the staging buffer must be 256-byte aligned")
        opt = dataclasses.replace(self.options, cuda_stream=self._stream(stream))
        twopaco_run_streamed(hp if self.total_bases else 0, self.offsets.data_ptr(), self.n_seqs,
                             self.total_bases, self.k, self.filter_bits, self.rounds, opt, self.ws_ptr,
                             self.ws_bytes, staging.data_ptr(), staging.numel(), self.out_offsets.data_ptr(),
                             self.out_positions.data_ptr(), self.capacity)

    def run_rounds(self, round_begin: int, round_end: int, stream=None) -> None:
        """Rounds [round_begin, round_end) of the run (twopaco_run_rounds)."""
        opt = dataclasses.replace(self.options, cuda_stream=self._stream(stream))
        twopaco_run_rounds(self._bases_ptr(reads=round_begin < self.rounds), self.offsets.data_ptr(),
                           self.n_seqs, self.total_bases, self.k, self.filter_bits, self.rounds, opt,
                           self.ws_ptr, self.ws_bytes, round_begin, round_end,
                           self.out_offsets.data_ptr(), self.out_positions.data_ptr(), self.capacity)

    def checkpoint(self, next_round: int, stream=None) -> bytes:
        """The state after the rounds before next_round, as bytes (twopaco_checkpoint_save)."""
        n = twopaco_checkpoint_bytes(self.total_bases, self.n_seqs, self.k, self.filter_bits,
                                     self.rounds, self.options)
        return twopaco_checkpoint_save(self.ws_ptr, next_round, n, self._stream(stream))

    def restore(self, blob: bytes, stream=None) -> int:
        """Load a checkpoint of this input into this workspace; returns the round to continue with."""
        opt = dataclasses.replace(self.options, cuda_stream=self._stream(stream))
        return twopaco_checkpoint_load(self._bases_ptr(),
                                       self.offsets.data_ptr(), self.n_seqs, self.total_bases, self.k,
                                       self.filter_bits, self.rounds, opt, self.ws_ptr, self.ws_bytes,
                                       blob)

    def shard_begin(self, compute_cut: bool, stream=None) -> None:
        """Pack the input and (compute_cut) cut the classes: twopaco_shard_begin."""
        opt = dataclasses.replace(self.options, cuda_stream=self._stream(stream))
        twopaco_shard_begin(self._bases_ptr(), self.offsets.data_ptr(),
                            self.n_seqs, self.total_bases, self.k, self.filter_bits, self.rounds, opt,
                            self.ws_ptr, self.ws_bytes, compute_cut)

    def shard_rounds(self, shard: int, n_shards: int, class_cut=None, stream=None) -> None:
        """This shard's rounds (twopaco_shard_rounds); class_cut: a CUDA tensor of
        rounds + 1 32-bit words, or None to keep the workspace's cut."""
        opt = dataclasses.replace(self.options, cuda_stream=self._stream(stream))
        twopaco_shard_rounds(self._bases_ptr(), self.offsets.data_ptr(),
                             self.n_seqs, self.total_bases, self.k, self.filter_bits, self.rounds, opt,
                             self.ws_ptr, self.ws_bytes, shard, n_shards,
                             class_cut.data_ptr() if class_cut is not None else 0)

    def state_tensor(self, which: int):
        """An int32 CUDA tensor viewing one piece of the workspace's state in place
        (twopaco_state_device): writes through it change the workspace."""
        ptr, nb = twopaco_state_device(self.total_bases, self.n_seqs, self.k, self.filter_bits,
                                       self.rounds, self.options, self.ws_ptr, which)
        if nb == 0:
            return self.torch.zeros(0, dtype=self.torch.int32, device=self.workspace.device)
        return self.torch.as_tensor(_DeviceWords(ptr, nb), device=self.workspace.device)

    def write_output(self, stream=None) -> None:
        """Write the output from the C_final the workspace holds
        (twopaco_run_rounds(..., rounds, rounds, ...))."""
        self.run_rounds(self.rounds, self.rounds, stream)

    def capture(self) -> None:
        """Capture this run as a CUDA graph (twopaco_plan_create); run() then replays it."""
        self.release_plan()
        h = ctypes.c_void_p()
        opt = self.options._c()
        rc = _lib().twopaco_plan_create(self._bases_ptr() or None,
                                        self.offsets.data_ptr(), self.n_seqs, self.total_bases,
                                        self.k, self.filter_bits, self.rounds, ctypes.byref(opt),
                                        self.ws_ptr, self.ws_bytes, self.out_offsets.data_ptr(),
                                        self.out_positions.data_ptr(), self.capacity, ctypes.byref(h))
        if rc != OK:
            raise TwopacoError(rc, "twopaco_plan_create")
        self._plan = h

    def release_plan(self) -> None:
        if getattr(self, "_plan", None):
            _lib().twopaco_plan_destroy(self._plan)
            self._plan = None

    def stats(self, stream=None, check: bool = True) -> Dict[str, int]:
        return twopaco_read_stats(self.ws_ptr, self._stream(stream), check)

    def state(self, which: int, count: int, stream=None) -> np.ndarray:
        return twopaco_read_state(self.ws_ptr, which, count, self._stream(stream))

    def result(self, stream=None) -> List[np.ndarray]:
        self.stats(stream)
        off = self.out_offsets.cpu().numpy().view(np.uint64)
        pos = self.out_positions[: int(off[-1])].cpu().numpy().view(np.uint64)
        return [pos[off[t]:off[t + 1]] for t in range(self.n_seqs)]
