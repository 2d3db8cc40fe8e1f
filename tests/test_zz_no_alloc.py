"""ac_scan_noalloc: the scan entry point that allocates no device memory.

It is meant for callers that cannot allocate when they scan (their device
memory is already held by another allocator, or they run a loop that must
not enter an allocator); it uses the library's fixed scratch array instead
of pool memory. This file is collected last on purpose, so that a run that
stops at the first failure has run every other test before it. Each check
compares the call with ac_scan on the same inputs, and with the CPU oracle,
exactly (all results are integers), over two calls in a row: the scratch
array keeps the previous call's contents, so the second call shows that it
is cleared correctly. The launch-shape options are those of ac_scan, so one,
two and three bases per lookup are all checked.
"""
import ctypes
import random

import numpy as np
import pytest
import torch

import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from tests.gpu_helpers import oracle_canonical

pytestmark = pytest.mark.gpu


def _noalloc(dfa, packed, n, cap, opts=None):
    raw = torch.zeros((max(cap, 1), 2), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(dfa.n_patterns, dtype=torch.int64, device="cuda")
    desc = N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1)
    r = N.Result(raw.data_ptr(), cap, 0, cnt.data_ptr(), 1, 0, 0)
    st = acg.lib().ac_scan_noalloc(dfa.h, ctypes.byref(desc), ctypes.byref(r),
                                   ctypes.byref(opts) if opts is not None else None, None)
    k = int(r.n_matches)
    v = raw[: min(k, cap)]
    a = torch.stack([v[:, 0], v[:, 1] & 0xFFFFFFFF], 1).cpu().numpy()
    return st, a[np.lexsort((a[:, 1], a[:, 0]))], cnt.cpu().numpy(), k


def _case(seed, n, k):
    rng = random.Random(seed)
    text = bytes(rng.choice(b"ACGT") for _ in range(n)) + b"ACAC" * 300
    pats = [text[j : j + rng.randint(8, 20)] for j in rng.sample(range(n - 20), k)] + [b"ACACACACAC"]
    return text, pats


def test_noalloc_equals_ac_scan_on_two_calls_in_a_row():
    for seed, n in ((1, 1_000_000), (2, 300_000)):
        text, pats = _case(seed, n, 2000)
        d = acg.build(pats)
        packed = acg.pack(torch.tensor(np.frombuffer(text, np.uint8), device="cuda"))
        ref = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=len(text))
        want = ref.canonical()[:, 1:]
        want_counts = ref.counts.cpu().numpy()
        orc, orc_counts = oracle_canonical(pats, np.frombuffer(text, np.uint8))
        assert np.array_equal(want, orc[:, 1:]) and np.array_equal(want_counts, orc_counts)
        for _ in range(2):
            st, got, counts, k = _noalloc(d, packed, len(text), ref.n_matches + 8)
            assert st == N.AC_OK
            assert k == ref.n_matches
            assert np.array_equal(got, want)
            assert np.array_equal(counts, want_counts)


def test_noalloc_every_stride_against_the_oracle():
    text, pats = _case(4, 400_000, 1500)
    d = acg.build(pats)
    packed = acg.pack(torch.tensor(np.frombuffer(text, np.uint8), device="cuda"))
    orc, orc_counts = oracle_canonical(pats, np.frombuffer(text, np.uint8))
    for stride, threads, interleave in ((1, 0, 0), (2, 0, 0), (3, 0, 0), (3, 640, 1), (3, 512, 2)):
        o = N.ScanOpts()
        o.hot_states, o.stride, o.threads, o.interleave = -1, stride, threads, interleave
        for _ in range(2):
            st, got, counts, k = _noalloc(d, packed, len(text), len(orc) + 8, o)
            assert st == N.AC_OK, (stride, threads, interleave, st)
            assert k == len(orc) and np.array_equal(got, orc[:, 1:]), (stride, threads, interleave)
            assert np.array_equal(counts, orc_counts)
    # a stride whose table was not built is refused, as by ac_scan
    d1 = acg.build(pats, stride2=False, stride3=False)
    for stride in (2, 3):
        o = N.ScanOpts()
        o.hot_states, o.stride = -1, stride
        st, _, _, _ = _noalloc(d1, packed, len(text), 16, o)
        assert st == N.AC_ERR_INVALID_ARG


def test_noalloc_owned_range_and_overflow():
    text, pats = _case(3, 200_000, 500)
    d = acg.build(pats)
    packed = acg.pack(torch.tensor(np.frombuffer(text, np.uint8), device="cuda"))
    o = N.ScanOpts()
    o.range_begin, o.range_end, o.hot_states = 1000, 150_000, -1
    ref = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=len(text), range_=(1000, 150_000))
    st, got, counts, k = _noalloc(d, packed, len(text), ref.n_matches, o)
    assert st == N.AC_OK and np.array_equal(got, ref.canonical()[:, 1:])
    st, _, counts, k = _noalloc(d, packed, len(text), 3)  # too small: exact count, exact counts
    full = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=len(text))
    assert st == N.AC_ERR_OVERFLOW and k == full.n_matches
    assert np.array_equal(counts, full.counts.cpu().numpy())


def test_noalloc_rejects_what_it_cannot_do():
    d = acg.build([b"ACGT"])
    host = np.zeros(4, np.int32)
    r = N.Result(None, 0, 0, None, 1, 0, 0)
    t = N.Text(host.ctypes.data, 16, N.AC_TEXT_PACKED2, 0)  # host text
    assert acg.lib().ac_scan_noalloc(d.h, ctypes.byref(t), ctypes.byref(r), None, None) == N.AC_ERR_INVALID_ARG
    # a machine larger than the fixed scratch is refused with AC_ERR_TOO_LARGE
    rng = np.random.default_rng(7)
    codes = rng.integers(0, 4, size=(110_000, 30))
    big = [bytes(b"ACGT"[c] for c in row) for row in codes]
    D = acg.build(big)
    assert D.n_states > N.AC_NOALLOC_MAX_STATES
    dev = torch.zeros(4, dtype=torch.int32, device="cuda")
    t = N.Text(dev.data_ptr(), 16, N.AC_TEXT_PACKED2, 1)
    assert acg.lib().ac_scan_noalloc(D.h, ctypes.byref(t), ctypes.byref(r), None, None) == N.AC_ERR_TOO_LARGE
