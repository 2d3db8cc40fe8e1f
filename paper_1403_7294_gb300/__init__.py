"""GB300 Aho-Corasick DNA scan: Python binding of libac.so (include/ac.h).

The binding only marshals arguments: every step of a scan (packing, the
walk, emission, counts) runs in the library's CUDA kernels. PyTorch provides
device memory and streams. If libac.so has not been built, every compute
call raises; there is no CPU fallback.

    import paper_1403_7294_gb300 as acg
    dfa = acg.build([b"ACGT", b"GATTACA"])
    res = acg.scan(dfa, torch_uint8_ascii_text_on_cuda)
    res.pos, res.pattern_id, res.counts
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Sequence

import numpy as np
import torch

from . import _native as N
from ._native import AcError

__all__ = [
    "Dfa", "ScanResult", "build", "pack", "scan", "scan_failureless", "scan_batch", "BatchPlan", "Stream", "PartSet",
    "build_partitioned", "autotune", "autotune_batch", "Server", "fault_inject", "mem_usage",
    "AcError", "lib",
]


def lib() -> ctypes.CDLL:
    return N.load()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _as_bytes(p) -> bytes:
    if isinstance(p, bytes):
        return p
    if isinstance(p, str):
        return p.encode("ascii")
    if isinstance(p, torch.Tensor):
        return p.cpu().numpy().astype(np.uint8).tobytes()
    return np.asarray(p, dtype=np.uint8).tobytes()


# -------------------------------------------------------------------- dfa


class Dfa:
    """A built machine (ac_build). Immutable; freed with close() or on GC."""

    def __init__(self, patterns: Sequence, fold_case: bool = False, host_only: bool = False, stride2: bool = True,
                 stride2_states: int = 0, failureless: bool = False, stride3: bool = True, stride3_states: int = 0):
        L = lib()
        self._bufs = [_as_bytes(p) for p in patterns]
        n = len(self._bufs)
        ptrs = (ctypes.c_char_p * max(n, 1))(*self._bufs)
        lens = np.array([len(b) for b in self._bufs], dtype=np.uint32)
        opts = N.BuildOpts((N.AC_BUILD_FOLD_CASE if fold_case else 0) | (N.AC_BUILD_HOST_ONLY if host_only else 0)
                           | (0 if stride2 else N.AC_BUILD_NO_STRIDE2) | (N.AC_BUILD_FAILURELESS if failureless else 0)
                           | (0 if stride3 else N.AC_BUILD_NO_STRIDE3), stride2_states, stride3_states)
        h = ctypes.c_void_p()
        N.check(L.ac_build(ctypes.cast(ptrs, ctypes.c_void_p), lens.ctypes.data, n, ctypes.byref(opts),
                           ctypes.byref(h)), "ac_build")
        self.h = h
        self.n_patterns = n
        self._bufs = None  # keywords were copied into the machine
        info = N.DfaInfo()
        N.check(L.ac_dfa_info(self.h, ctypes.byref(info)), "ac_dfa_info")
        self.info = {k: getattr(info, k) for k, _ in N.DfaInfo._fields_}

    @property
    def n_states(self) -> int:
        return self.info["n_states"]

    @property
    def max_len(self) -> int:
        return self.info["max_len"]

    def tables(self) -> dict[str, np.ndarray]:
        """Copies of the host tables (see ac_dfa_tables)."""
        t = N.DfaTables()
        N.check(lib().ac_dfa_tables(self.h, ctypes.byref(t)), "ac_dfa_tables")
        S, Pn, E = self.info["n_states"], self.info["n_patterns"], self.info["out_entries"]
        sizes = {"delta": 4 * S, "out_off": S + 1, "out_pid": E, "pat_len": Pn, "pat_state": Pn, "depth": S, "fail": S,
                 "delta2": self.info["table2_bytes"] // 4, "delta3": self.info["table3_bytes"] // 4}
        if t.gotos:  # failure-less form
            sizes.update({"gotos": 4 * S, "own_off": S + 1, "own_pid": Pn})
        return {k: np.ctypeslib.as_array(getattr(t, k), shape=(v,)).copy() if v else np.zeros(0, np.uint32)
                for k, v in sizes.items()}

    def close(self):
        if getattr(self, "h", None):
            lib().ac_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build(patterns: Sequence, fold_case: bool = False, host_only: bool = False, stride2: bool = True,
          stride2_states: int = 0, failureless: bool = False, stride3: bool = True, stride3_states: int = 0) -> Dfa:
    return Dfa(patterns, fold_case=fold_case, host_only=host_only, stride2=stride2, stride2_states=stride2_states,
               failureless=failureless, stride3=stride3, stride3_states=stride3_states)


# ------------------------------------------------------------------- texts


def _text_desc(text, encoding: int | None, n_bases: int | None):
    """(ac_text, keepalive) for a torch tensor / numpy array / bytes."""
    keep = text
    if isinstance(text, (bytes, bytearray, str)):
        arr = np.frombuffer(_as_bytes(text), dtype=np.uint8)
        keep = arr
        ptr, on_dev, enc = arr.ctypes.data, 0, N.AC_TEXT_ASCII if encoding is None else encoding
        n = arr.size if n_bases is None else n_bases
    elif isinstance(text, np.ndarray):
        arr = np.ascontiguousarray(text)
        keep = arr
        ptr, on_dev = arr.ctypes.data, 0
        enc = encoding if encoding is not None else (N.AC_TEXT_ASCII if arr.dtype == np.uint8 else N.AC_TEXT_PACKED2)
        n = n_bases if n_bases is not None else (arr.size if enc == N.AC_TEXT_ASCII else None)
    elif isinstance(text, torch.Tensor):
        if not text.is_contiguous():
            raise ValueError("text tensor must be contiguous")
        ptr, on_dev = text.data_ptr(), int(text.is_cuda)
        enc = encoding if encoding is not None else (N.AC_TEXT_ASCII if text.dtype == torch.uint8 else N.AC_TEXT_PACKED2)
        n = n_bases if n_bases is not None else (text.numel() if enc == N.AC_TEXT_ASCII else None)
    else:
        raise TypeError(f"unsupported text type {type(text)}")
    if n is None:
        raise ValueError("packed text needs n_bases")
    return N.Text(ptr if n else None, n, enc, on_dev), keep


def pack(ascii_text: torch.Tensor, fold_case: bool = False, stream=None) -> torch.Tensor:
    """ASCII uint8 CUDA tensor -> packed int32 tensor of ceil(n/16) words (ac_pack)."""
    if not (isinstance(ascii_text, torch.Tensor) and ascii_text.is_cuda and ascii_text.dtype == torch.uint8):
        raise TypeError("pack() takes a uint8 CUDA tensor")
    n = ascii_text.numel()
    out = torch.empty(max(1, (n + 15) // 16), dtype=torch.int32, device=ascii_text.device)
    bad = ctypes.c_uint64(0)
    st = lib().ac_pack(ascii_text.data_ptr(), n, out.data_ptr(), N.AC_SCAN_FOLD_CASE if fold_case else 0,
                       ctypes.byref(bad), _stream_ptr(stream))
    if st == N.AC_ERR_ALPHABET:
        raise AcError(st, f"ac_pack: invalid base at offset {bad.value}")
    N.check(st, "ac_pack")
    return out


# ----------------------------------------------------------------- results


@dataclass
class ScanResult:
    pos: torch.Tensor         # int64 [n_matches] start positions
    pattern_id: torch.Tensor  # int64 [n_matches]
    text_id: torch.Tensor     # int64 [n_matches]
    counts: torch.Tensor | None  # int64 [P]
    n_matches: int
    stats: dict | None = None

    def canonical(self) -> np.ndarray:
        """Occurrences sorted by (text_id, pos, pattern_id) as an (k, 3) int64 array."""
        a = torch.stack([self.text_id, self.pos, self.pattern_id], 1).cpu().numpy()
        order = np.lexsort((a[:, 2], a[:, 1], a[:, 0]))
        return a[order]


def _split(raw: torch.Tensor, k: int):
    v = raw[:k]
    pos = v[:, 0]
    pid = v[:, 1] & 0xFFFFFFFF
    tid = (v[:, 1] >> 32) & 0xFFFFFFFF
    return pos, pid, tid


def _opts(range_=None, chunk=0, threads=0, interleave=0, hot_states=-1, fold_case=False, text_id=0, stride=0,
          chunks_per_lane=0):
    o = N.ScanOpts()
    o.range_begin, o.range_end = (range_ if range_ is not None else (0, 0))
    o.chunk, o.threads, o.interleave, o.hot_states = chunk, threads, interleave, hot_states
    o.stride = stride
    o.chunks_per_lane = chunks_per_lane
    o.flags = N.AC_SCAN_FOLD_CASE if fold_case else 0
    o.text_id = text_id
    return o


def _stats_dict(s: N.ScanStats) -> dict:
    return {k: getattr(s, k) for k, _ in N.ScanStats._fields_}


def _run(fn, dfa, texts_arg, n_texts, capacity, counts, device, opts, stream, want_stats, on_device=True, handle=None):
    """Calls ac_scan / ac_scan_batch / ac_stream_scan, growing the occurrence buffer once on overflow."""
    cap = capacity
    for attempt in range(2):
        if on_device:
            raw = torch.empty((max(cap, 1), 2), dtype=torch.int64, device=device)
            cnt = torch.empty(dfa.n_patterns, dtype=torch.int64, device=device) if counts else None
        else:
            raw = torch.empty((max(cap, 1), 2), dtype=torch.int64).pin_memory()
            cnt = torch.empty(dfa.n_patterns, dtype=torch.int64).pin_memory() if counts else None
        r = N.Result(raw.data_ptr(), cap, 0, cnt.data_ptr() if cnt is not None else None, int(on_device), 0, 0)
        stt = N.ScanStats()
        args = (handle if handle is not None else dfa.h, texts_arg) + ((n_texts,) if n_texts is not None else ())
        st = fn(*args, ctypes.byref(r), ctypes.byref(opts), stream, ctypes.byref(stt) if want_stats else None)
        if st == N.AC_ERR_OVERFLOW and attempt == 0:
            cap = int(r.n_matches)
            continue
        if st == N.AC_ERR_ALPHABET:
            raise AcError(st, f"invalid base at offset {r.bad_offset}")
        N.check(st, fn.__name__)
        k = int(r.n_matches)
        pos, pid, tid = _split(raw, k)
        return ScanResult(pos, pid, tid, cnt, k, _stats_dict(stt) if want_stats else None)
    raise AssertionError("unreachable")


def scan(dfa: Dfa, text, *, encoding: int | None = None, n_bases: int | None = None, capacity: int | None = None,
         counts: bool = True, range_=None, chunk: int = 0, threads: int = 0, interleave: int = 0,
         hot_states: int = -1, fold_case: bool = False, text_id: int = 0, stats: bool = False,
         stream=None, results_on_device: bool | None = None, stride: int = 0,
         chunks_per_lane: int = 0) -> ScanResult:
    """One text (ac_scan). text: uint8 ASCII or int32 packed (give n_bases), on CUDA or host."""
    desc, keep = _text_desc(text, encoding, n_bases)
    on_dev = bool(desc.on_device) if results_on_device is None else results_on_device
    device = text.device if isinstance(text, torch.Tensor) and text.is_cuda else torch.device("cuda")
    if capacity is None:
        capacity = max(1024, desc.n_bases // 64)
    o = _opts(range_, chunk, threads, interleave, hot_states, fold_case, text_id, stride, chunks_per_lane)
    res = _run(lib().ac_scan, dfa, ctypes.byref(desc), None, capacity, counts, device, o, _stream_ptr(stream),
               stats, on_dev)
    del keep
    return res


def scan_failureless(dfa: Dfa, text, *, encoding: int | None = None, n_bases: int | None = None,
                     capacity: int | None = None, counts: bool = True, range_=None, fold_case: bool = False,
                     text_id: int = 0, stats: bool = False, stream=None,
                     results_on_device: bool | None = None) -> ScanResult:
    """Failure-less matching, one thread per start position (ac_scan_failureless);
    the dfa must be built with failureless=True."""
    desc, keep = _text_desc(text, encoding, n_bases)
    on_dev = bool(desc.on_device) if results_on_device is None else results_on_device
    device = text.device if isinstance(text, torch.Tensor) and text.is_cuda else torch.device("cuda")
    if capacity is None:
        capacity = max(1024, desc.n_bases // 64)
    o = _opts(range_, 0, 0, 0, -1, fold_case, text_id)
    res = _run(lib().ac_scan_failureless, dfa, ctypes.byref(desc), None, capacity, counts, device, o,
               _stream_ptr(stream), stats, on_dev)
    del keep
    return res


def scan_batch(dfa: Dfa, texts: Sequence, *, encoding: int | None = None, n_bases: Sequence[int] | None = None,
               capacity: int | None = None, counts: bool = True, chunk: int = 0, threads: int = 0,
               interleave: int = 0, hot_states: int = -1, fold_case: bool = False, stats: bool = False,
               stream=None, results_on_device: bool | None = None, stride: int = 0) -> ScanResult:
    """Many independent texts in one persistent launch (ac_scan_batch)."""
    descs, keep = [], []
    for i, t in enumerate(texts):
        d, k = _text_desc(t, encoding, None if n_bases is None else int(n_bases[i]))
        descs.append(d)
        keep.append(k)
    arr = (N.Text * max(1, len(descs)))(*descs)
    on_dev = bool(descs[0].on_device) if (results_on_device is None and descs) else bool(results_on_device)
    total = sum(d.n_bases for d in descs)
    if capacity is None:
        capacity = max(1024, total // 64)
    o = _opts(None, chunk, threads, interleave, hot_states, fold_case, 0, stride)
    return _run(lib().ac_scan_batch, dfa, arr, len(descs), capacity, counts, torch.device("cuda"), o,
                _stream_ptr(stream), stats, on_dev)


class BatchPlan:
    """A graph-captured batched scan over fixed device-resident packed texts."""

    def __init__(self, dfa: Dfa, packed_texts: Sequence[torch.Tensor], n_bases: Sequence[int], capacity: int,
                 counts: bool = True, chunk: int = 0, threads: int = 0, interleave: int = 0,
                 hot_states: int = -1, stream=None, stride: int = 0):
        self.dfa = dfa
        self.texts = list(packed_texts)
        descs = [N.Text(t.data_ptr() if n else None, int(n), N.AC_TEXT_PACKED2, 1)
                 for t, n in zip(self.texts, n_bases)]
        arr = (N.Text * max(1, len(descs)))(*descs)
        dev = self.texts[0].device if self.texts else torch.device("cuda")
        self.capacity = capacity
        self.raw = torch.empty((max(capacity, 1), 2), dtype=torch.int64, device=dev)
        self.counts = torch.empty(dfa.n_patterns, dtype=torch.int64, device=dev) if counts else None
        r = N.Result(self.raw.data_ptr(), capacity, 0, self.counts.data_ptr() if counts else None, 1, 0, 0)
        o = _opts(None, chunk, threads, interleave, hot_states, False, 0, stride)
        h = ctypes.c_void_p()
        N.check(lib().ac_batch_plan_create(dfa.h, arr, len(descs), ctypes.byref(r), ctypes.byref(o),
                                           _stream_ptr(stream), ctypes.byref(h)), "ac_batch_plan_create")
        self.h = h

    def run(self, sync: bool = True, stream=None) -> int | None:
        r = N.Result()
        st = lib().ac_batch_plan_run(self.h, _stream_ptr(stream), 1 if sync else 0, ctypes.byref(r))
        if not sync:
            N.check(st, "ac_batch_plan_run")
            return None
        if st not in (N.AC_OK, N.AC_ERR_OVERFLOW):
            N.check(st, "ac_batch_plan_run")
        self.n_matches = int(r.n_matches)
        self.overflow = st == N.AC_ERR_OVERFLOW
        return self.n_matches

    def result(self) -> ScanResult:
        k = min(self.n_matches, self.capacity)
        pos, pid, tid = _split(self.raw, k)
        return ScanResult(pos, pid, tid, self.counts, self.n_matches)

    def close(self):
        if getattr(self, "h", None):
            lib().ac_batch_plan_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PartSet:
    """The paper's pattern-file split (Sec. IV.A, approach 2): one machine per
    consecutive chunk of keywords, each small enough for shared memory, all
    scanning the whole text in one launch (ac_build_partitioned /
    ac_scan_partitioned). Ids and counts are in the caller's numbering."""

    def __init__(self, patterns: Sequence, max_states: int = 0, fold_case: bool = False):
        bufs = [_as_bytes(p) for p in patterns]
        n = len(bufs)
        ptrs = (ctypes.c_char_p * max(n, 1))(*bufs)
        lens = np.array([len(b) for b in bufs], dtype=np.uint32)
        opts = N.BuildOpts(N.AC_BUILD_FOLD_CASE if fold_case else 0, 0, 0)
        h = ctypes.c_void_p()
        N.check(lib().ac_build_partitioned(ctypes.cast(ptrs, ctypes.c_void_p), lens.ctypes.data, n, max_states,
                                           ctypes.byref(opts), ctypes.byref(h)), "ac_build_partitioned")
        self.h = h
        self.n_patterns = n
        k, m = ctypes.c_uint32(), ctypes.c_uint32()
        N.check(lib().ac_part_set_info(self.h, ctypes.byref(k), ctypes.byref(m)), "ac_part_set_info")
        self.n_parts, self.max_states = k.value, m.value

    def scan(self, text, *, encoding: int | None = None, n_bases: int | None = None, capacity: int | None = None,
             counts: bool = True, range_=None, fold_case: bool = False, stats: bool = False, stream=None,
             results_on_device: bool | None = None) -> ScanResult:
        desc, keep = _text_desc(text, encoding, n_bases)
        on_dev = bool(desc.on_device) if results_on_device is None else results_on_device
        device = text.device if isinstance(text, torch.Tensor) and text.is_cuda else torch.device("cuda")
        if capacity is None:
            capacity = max(1024, desc.n_bases // 64)
        o = _opts(range_, 0, 0, 0, -1, fold_case)
        res = _run(lib().ac_scan_partitioned, self, ctypes.byref(desc), None, capacity, counts, device, o,
                   _stream_ptr(stream), stats, on_dev, handle=self.h)
        del keep
        return res

    def close(self):
        if getattr(self, "h", None):
            lib().ac_part_set_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_partitioned(patterns: Sequence, max_states: int = 0, fold_case: bool = False) -> PartSet:
    return PartSet(patterns, max_states=max_states, fold_case=fold_case)


class Stream:
    """One long text scanned in consecutive pieces (ac_stream_*): positions are
    global, and an occurrence spanning a piece boundary is reported once, by
    the piece that holds its end."""

    def __init__(self, dfa: Dfa):
        h = ctypes.c_void_p()
        N.check(lib().ac_stream_create(dfa.h, ctypes.byref(h)), "ac_stream_create")
        self.h = h
        self.dfa = dfa

    def scan(self, piece, *, encoding: int | None = None, n_bases: int | None = None, capacity: int | None = None,
             counts: bool = True, chunk: int = 0, threads: int = 0, interleave: int = 0, hot_states: int = -1,
             fold_case: bool = False, stats: bool = False, stream=None, results_on_device: bool | None = None,
             stride: int = 0) -> ScanResult:
        desc, keep = _text_desc(piece, encoding, n_bases)
        on_dev = bool(desc.on_device) if results_on_device is None else results_on_device
        device = piece.device if isinstance(piece, torch.Tensor) and piece.is_cuda else torch.device("cuda")
        if capacity is None:
            capacity = max(1024, desc.n_bases // 64)
        o = _opts(None, chunk, threads, interleave, hot_states, fold_case, 0, stride)
        res = _run(lib().ac_stream_scan, self.dfa, ctypes.byref(desc), None, capacity, counts, device, o,
                   _stream_ptr(stream), stats, on_dev, handle=self.h)
        del keep
        return res

    def reset(self):
        N.check(lib().ac_stream_reset(self.h), "ac_stream_reset")

    def close(self):
        if getattr(self, "h", None):
            lib().ac_stream_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(dfa: Dfa, packed_sample: torch.Tensor, n_bases: int, stream=None) -> dict:
    """Tunes the scan's launch shape on a device-resident packed text (ac_autotune)."""
    desc = N.Text(packed_sample.data_ptr(), int(n_bases), N.AC_TEXT_PACKED2, 1)
    o = N.ScanOpts()
    N.check(lib().ac_autotune(dfa.h, ctypes.byref(desc), ctypes.byref(o), _stream_ptr(stream)), "ac_autotune")
    return {"threads": o.threads, "interleave": o.interleave, "hot_states": o.hot_states, "stride": o.stride,
            "chunks_per_lane": o.chunks_per_lane, "chunk": o.chunk}


def autotune_batch(dfa: Dfa, packed_texts: Sequence[torch.Tensor], n_bases: Sequence[int], stream=None) -> int:
    """Tunes the work-item chunk of batched scans over device-resident packed texts
    (ac_autotune_batch); returns the chosen chunk (0: the built-in default)."""
    descs = [N.Text(t.data_ptr() if n else None, int(n), N.AC_TEXT_PACKED2, 1) for t, n in zip(packed_texts, n_bases)]
    arr = (N.Text * max(1, len(descs)))(*descs)
    o = N.ScanOpts()
    N.check(lib().ac_autotune_batch(dfa.h, arr, len(descs), ctypes.byref(o), _stream_ptr(stream)),
            "ac_autotune_batch")
    return int(o.chunk)


def fault_inject(spec: str | None) -> None:
    """Sets the host-side fault plan (ac_fault_inject): "oom@k", "cuda_err@k", both comma-separated, or
    None to clear it."""
    N.check(lib().ac_fault_inject(spec.encode() if spec else None), "ac_fault_inject")


def mem_usage() -> dict:
    """Device memory the library holds (ac_mem_usage)."""
    m = N.MemUsage()
    N.check(lib().ac_mem_usage(ctypes.byref(m)), "ac_mem_usage")
    return {k: getattr(m, k) for k, _ in N.MemUsage._fields_}


# ----------------------------------------------------------------- serving


class _Taken:
    """Owns one ac_serve_take result; gives it back when the last view goes."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        h, self.handle = self.handle, None
        if h:
            try:
                lib().ac_serve_release(h)
            except Exception:  # interpreter shutdown: the process gives the memory back
                pass


def _view(addr, n: int, owner) -> np.ndarray:
    """int64 numpy view of n values at addr, keeping owner alive while referenced."""
    if n == 0 or not addr:
        return np.zeros(n, dtype=np.int64)
    buf = (ctypes.c_int64 * n).from_address(addr)
    buf._owner = owner
    return np.ctypeslib.as_array(buf)


class Server:
    """Continuous-batching scan server (ac_serve_*)."""

    def __init__(self, device_budget_bytes: int = 0, n_streams: int = 0, max_batch: int = 0, max_queue: int = 0,
                 match_capacity_per_base_x1000: int = 0):
        o = N.ServeOpts(device_budget_bytes, n_streams, max_batch, max_queue, match_capacity_per_base_x1000)
        h = ctypes.c_void_p()
        N.check(lib().ac_serve_create(ctypes.byref(o), ctypes.byref(h)), "ac_serve_create")
        self.h = h
        self._dfas = []
        self._npat = {}

    def add_dfa(self, dfa: Dfa) -> int:
        slot = ctypes.c_uint32()
        N.check(lib().ac_serve_add_dfa(self.h, dfa.h, ctypes.byref(slot)), "ac_serve_add_dfa")
        self._dfas.append(dfa)
        self._npat[slot.value] = dfa.n_patterns
        return slot.value

    def submit(self, slot: int, text, encoding: int | None = None, n_bases: int | None = None) -> int:
        desc, keep = _text_desc(text, encoding, n_bases)
        if desc.on_device:
            raise ValueError("serving takes host texts")
        t = ctypes.c_uint64()
        st = lib().ac_serve_submit(self.h, slot, ctypes.byref(desc), ctypes.byref(t))
        del keep
        N.check(st, "ac_serve_submit")
        return t.value

    def try_submit(self, slot: int, text, encoding: int | None = None, n_bases: int | None = None):
        """Like submit but returns None when admission refuses (AC_ERR_BUSY)."""
        try:
            return self.submit(slot, text, encoding, n_bases)
        except AcError as e:
            if e.status == N.AC_ERR_BUSY:
                return None
            raise

    def wait(self, ticket: int, slot: int, capacity: int | None = None, timeout_us: int = -1):
        """Returns (matches (k,2) int64 numpy [pos, pid], counts int64[P], n_matches).

        capacity None: nothing is copied (ac_serve_take). The two arrays are
        views of the server's own copy of the results, which is given back
        (ac_serve_release) once neither array is referenced any more. An int:
        the results are copied (ac_serve_wait) into arrays of the caller's, that
        much room first and the exact size on overflow; the matches returned
        are then the first n_matches rows of the array allocated. Served
        occurrences carry text index 0, so column 1 is the keyword id as it
        stands."""
        if capacity is None:
            out = N.Served()
            N.check(lib().ac_serve_take(self.h, ticket, ctypes.byref(out), timeout_us), "ac_serve_take")
            held = _Taken(out.handle)
            k, pc = int(out.n_matches), int(out.n_counts)
            return _view(out.matches, 2 * k, held).reshape(k, 2), _view(out.counts, pc, held), k
        cap = int(capacity)
        for _ in range(2):
            raw = np.empty((max(cap, 1), 2), dtype=np.int64)
            cnt = np.empty(self._npat[slot], dtype=np.int64)
            r = N.Result(raw.ctypes.data if cap else None, cap, 0, cnt.ctypes.data, 0, 0, 0)
            st = lib().ac_serve_wait(self.h, ticket, ctypes.byref(r), timeout_us)
            if st == N.AC_ERR_OVERFLOW:  # the ticket stays valid: retry with the exact size
                cap = int(r.n_matches)
                continue
            N.check(st, "ac_serve_wait")
            k = int(r.n_matches)
            return raw[:k], cnt, k
        raise AssertionError("unreachable")

    def cancel(self, ticket: int) -> bool:
        """Withdraws a request (ac_serve_cancel): True when it was still queued, or finished and its
        results are dropped; False when its batch is running (the ticket stays valid)."""
        st = lib().ac_serve_cancel(self.h, ticket)
        if st == N.AC_ERR_BUSY:
            return False
        N.check(st, "ac_serve_cancel")
        return True

    def stats(self) -> dict:
        s = N.ServeStats()
        N.check(lib().ac_serve_stats(self.h, ctypes.byref(s)), "ac_serve_stats")
        return {k: getattr(s, k) for k, _ in N.ServeStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().ac_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
