"""CPU oracle for the Aho-Corasick scan (ctypes wrapper over ``ac_oracle.c``).

TEST INFRASTRUCTURE ONLY. The test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path
(``paper_1403_7294_gb300``) never does, and shares no code with it.

The oracle follows Sec. III.A of the paper: stage 1 builds goto / failure /
output, stage 2 reads the text once, following failure transitions and
re-reading the same character until a valid transition exists, and reports
every keyword in output(state) after each character (overlaps included,
Fig. 2). Occurrences are ``(start, pattern_id)``; start is 0-based.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ac_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")


def compile_oracle(out_path: str = _LIB_PATH, mutant: int = 0) -> str:
    """Compile ``ac_oracle.c`` into a shared library with gcc.

    ``mutant`` != 0 plants one known mistake (see ``ac_oracle.c``); it is
    used only by the test that shows the pins catch such mistakes.
    """
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", out_path, _SRC]
    if mutant:
        cmd.insert(1, f"-DORC_MUTANT={int(mutant)}")
    subprocess.run(cmd, check=True)
    return out_path


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    P = ctypes.c_void_p
    lib.orc_build.restype = P
    lib.orc_build.argtypes = [P, P, ctypes.c_uint32]
    lib.orc_free.argtypes = [P]
    lib.orc_free.restype = None
    lib.orc_num_states.argtypes = [P]
    lib.orc_num_states.restype = ctypes.c_int32
    lib.orc_goto.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
    lib.orc_goto.restype = ctypes.c_int32
    lib.orc_fail.argtypes = [P, ctypes.c_int32]
    lib.orc_fail.restype = ctypes.c_int32
    lib.orc_depth.argtypes = [P, ctypes.c_int32]
    lib.orc_depth.restype = ctypes.c_int32
    lib.orc_output.argtypes = [P, ctypes.c_int32, P, ctypes.c_int32]
    lib.orc_output.restype = ctypes.c_int32
    lib.orc_trace.argtypes = [P, P, ctypes.c_uint64, P, ctypes.c_int64]
    lib.orc_trace.restype = ctypes.c_int64
    lib.orc_scan.argtypes = [P, P, ctypes.c_uint64, P]
    lib.orc_scan.restype = P
    lib.orc_naive.argtypes = [P, P, ctypes.c_uint32, P, ctypes.c_uint64]
    lib.orc_naive.restype = P
    lib.orc_matches_size.argtypes = [P]
    lib.orc_matches_size.restype = ctypes.c_uint64
    lib.orc_matches_copy.argtypes = [P, P, P]
    lib.orc_matches_copy.restype = None
    lib.orc_matches_free.argtypes = [P]
    lib.orc_matches_free.restype = None
    return lib


_LIB: ctypes.CDLL | None = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (compiling first if needed) the oracle library."""
    global _LIB
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _LIB is None:
        if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            compile_oracle()
        _LIB = _bind(ctypes.CDLL(_LIB_PATH))
    return _LIB


def _as_bytes(x) -> bytes:
    if isinstance(x, bytes):
        return x
    if isinstance(x, str):
        return x.encode("latin-1")
    return np.ascontiguousarray(x, dtype=np.uint8).tobytes()


class _PatternArgs:
    """Keeps the keyword buffers alive while C holds pointers into them."""

    def __init__(self, patterns: Sequence):
        self.bufs = [_as_bytes(p) for p in patterns]
        n = len(self.bufs)
        self.ptrs = (ctypes.c_char_p * max(n, 1))(*self.bufs)
        self.lens = np.array([len(b) for b in self.bufs], dtype=np.uint32)
        self.n = n


def _take(lib, res) -> tuple[np.ndarray, np.ndarray]:
    if not res:
        raise MemoryError("oracle allocation failed")
    try:
        k = lib.orc_matches_size(res)
        pos = np.empty(k, dtype=np.uint64)
        pid = np.empty(k, dtype=np.uint32)
        lib.orc_matches_copy(res, pos.ctypes.data, pid.ctypes.data)
    finally:
        lib.orc_matches_free(res)
    return pos, pid


class Machine:
    """The paper's pattern matching machine (goto, fail, output)."""

    def __init__(self, patterns: Sequence, lib: ctypes.CDLL | None = None):
        self.lib = lib if lib is not None else load()
        self._args = _PatternArgs(patterns)
        self.n_patterns = self._args.n
        self.h = self.lib.orc_build(
            ctypes.cast(self._args.ptrs, ctypes.c_void_p), self._args.lens.ctypes.data, self._args.n
        )
        if not self.h:
            raise ValueError("orc_build failed (empty keyword, no keywords or out of memory)")

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_free(self.h)
            self.h = None

    __del__ = close

    # --- the three functions of stage 1
    @property
    def n_states(self) -> int:
        return self.lib.orc_num_states(self.h)

    def goto(self, s: int, c) -> int:
        c = ord(c) if isinstance(c, str) else int(c)
        return self.lib.orc_goto(self.h, s, c)

    def fail(self, s: int) -> int:
        return self.lib.orc_fail(self.h, s)

    def depth(self, s: int) -> int:
        return self.lib.orc_depth(self.h, s)

    def output(self, s: int) -> list[int]:
        buf = np.empty(4096, dtype=np.uint32)
        k = self.lib.orc_output(self.h, s, buf.ctypes.data, buf.size)
        if k > buf.size:
            buf = np.empty(k, dtype=np.uint32)
            self.lib.orc_output(self.h, s, buf.ctypes.data, buf.size)
        return [int(v) for v in buf[:k]]

    # --- stage 2
    def trace(self, text) -> list[int]:
        t = _as_bytes(text)
        cap = 4 * len(t) + 8
        buf = np.empty(cap, dtype=np.int32)
        k = self.lib.orc_trace(self.h, t, len(t), buf.ctypes.data, cap)
        return [int(v) for v in buf[: min(k, cap)]]

    def scan(self, text) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Returns (pos u64[k], pid u32[k], counts u64[P]) in scan order."""
        if isinstance(text, np.ndarray):
            t = np.ascontiguousarray(text, dtype=np.uint8)
            ptr, n = t.ctypes.data, t.size
        else:
            t = _as_bytes(text)
            ptr, n = t, len(t)
        counts = np.zeros(self.n_patterns, dtype=np.uint64)
        res = self.lib.orc_scan(self.h, ptr, n, counts.ctypes.data)
        pos, pid = _take(self.lib, res)
        return pos, pid, counts


def naive(patterns: Sequence, text, lib: ctypes.CDLL | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Brute force double loop; ordered by start, then pattern id."""
    lib = lib if lib is not None else load()
    a = _PatternArgs(patterns)
    if isinstance(text, np.ndarray):
        t = np.ascontiguousarray(text, dtype=np.uint8)
        ptr, n = t.ctypes.data, t.size
    else:
        t = _as_bytes(text)
        ptr, n = t, len(t)
    res = lib.orc_naive(ctypes.cast(a.ptrs, ctypes.c_void_p), a.lens.ctypes.data, a.n, ptr, n)
    return _take(lib, res)


def canonical(pos: np.ndarray, pid: np.ndarray, text_id: np.ndarray | None = None) -> np.ndarray:
    """Occurrences as a sorted structured array keyed (text_id, pos, pid)."""
    k = len(pos)
    out = np.empty(k, dtype=[("text_id", "<u4"), ("pos", "<u8"), ("pid", "<u4")])
    out["text_id"] = 0 if text_id is None else text_id
    out["pos"] = pos
    out["pid"] = pid
    out.sort(order=["text_id", "pos", "pid"])
    return out


# ------------------------------------------------ the two threaded forms (Sec. IV.A)


def _text_array(text) -> np.ndarray:
    if isinstance(text, np.ndarray):
        return np.ascontiguousarray(text, dtype=np.uint8)
    return np.frombuffer(_as_bytes(text), dtype=np.uint8)


def _run_threads(jobs, threads: int):
    from concurrent.futures import ThreadPoolExecutor

    if threads <= 1:
        return [j() for j in jobs]
    with ThreadPoolExecutor(max_workers=threads) as ex:  # each job is one C call (GIL released)
        return list(ex.map(lambda j: j(), jobs))


def scan_text_chunks(machine: Machine, text, threads: int, max_len: int):
    """Approach 1 of Sec. IV.A, made exact: the text's end positions are split
    into ``threads`` contiguous ranges; thread t scans its range preceded by
    the ``max_len - 1`` bases before it, from the root, and keeps only the
    occurrences that end inside its range (each occurrence has one end).
    All threads share the one machine (read only). Returns (pos, pid, counts)
    in range order."""
    t = _text_array(text)
    n = t.size
    k = max(1, int(threads))
    bounds = [n * i // k for i in range(k + 1)]

    def job(i):
        a, b = bounds[i], bounds[i + 1]
        lo = max(0, a - (max_len - 1))
        pos, pid, _ = machine.scan(t[lo:b])
        return pos + np.uint64(lo), pid

    parts = _run_threads([lambda i=i: job(i) for i in range(k)], k)
    pos = np.concatenate([p for p, _ in parts]) if parts else np.empty(0, np.uint64)
    pid = np.concatenate([q for _, q in parts]) if parts else np.empty(0, np.uint32)
    if pos.size:
        lens = machine._args.lens.astype(np.uint64)
        end = pos + lens[pid] - np.uint64(1)
        # range i keeps ends in [bounds[i], bounds[i+1]); ranges were scanned in order
        owner = np.searchsorted(np.asarray(bounds[1:], dtype=np.uint64), end, side="right")
        which = np.repeat(np.arange(k), [p.size for p, _ in parts])
        keep = owner == which
        pos, pid = pos[keep], pid[keep]
    counts = np.bincount(pid, minlength=machine.n_patterns).astype(np.uint64)
    return pos, pid, counts


def pattern_split(patterns: Sequence, parts: int) -> list[tuple[int, list]]:
    """Approach 2 of Sec. IV.A (Fig. 3): the keyword list cut into ``parts``
    consecutive pieces of near-equal size; each piece keeps the id of its
    first keyword so that local ids map back by an offset."""
    p = list(patterns)
    k = max(1, min(int(parts), len(p)))
    cut = [len(p) * i // k for i in range(k + 1)]
    return [(cut[i], p[cut[i] : cut[i + 1]]) for i in range(k)]


def scan_pattern_split(split, text, threads: int, machines: list | None = None):
    """Approach 2 of Sec. IV.A (Fig. 3): one machine per piece of the keyword
    list, every thread scanning the whole text with its own machine; the
    union of the pieces' occurrences with ids offset is the whole set's.
    ``machines`` (one per piece) skips the builds; otherwise each thread
    builds its own machine first, as in the paper. Returns (pos, pid,
    counts)."""
    t = _text_array(text)

    def job(i):
        off, pats = split[i]
        m = machines[i] if machines is not None else Machine(pats)
        pos, pid, c = m.scan(t)
        return pos, pid + np.uint32(off), off, c

    res = _run_threads([lambda i=i: job(i) for i in range(len(split))], threads)
    total = sum(len(p) for _, p in split)
    counts = np.zeros(total, dtype=np.uint64)
    for _, _, off, c in res:
        counts[off : off + c.size] = c
    pos = np.concatenate([r[0] for r in res]) if res else np.empty(0, np.uint64)
    pid = np.concatenate([r[1] for r in res]) if res else np.empty(0, np.uint32)
    return pos, pid, counts
