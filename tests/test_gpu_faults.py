"""Failure handling without a GPU fault: host-side fault injection.

ac_fault_inject("oom@k") makes the library's k-th device allocation fail as if
the device were full, and "cuda_err@k" makes its k-th kernel launch report a
launch failure without launching anything; nothing faulty reaches the GPU.
Each entry point is swept over k = 1, 2, ... until the call runs clean. Every
failed call must return the documented status (AC_ERR_OOM / AC_ERR_CUDA),
hold no device memory afterwards (stream-ordered pool memory in use and the
library's own allocations back to where they were before the call), and leave
the device usable: the clean call at the end of every sweep, and a final scan,
equal the oracle. A serving request whose worker meets an injected failure
fails alone; the server goes on serving.
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
L = None


def lib():
    global L
    if L is None:
        L = acg.lib()
    return L


def _case(seed=5, n=200_000, k=600):
    rng = random.Random(seed)
    text = bytes(rng.choice(b"ACGT") for _ in range(n)) + b"ACAC" * 200
    pats = [text[j : j + rng.randint(6, 18)] for j in rng.sample(range(n - 20), k)] + [b"ACACACAC"]
    return text, pats


def _held():
    torch.cuda.synchronize()
    u = acg.mem_usage()
    return u["pool_used_bytes"], u["live_bytes"], u["live_allocations"]


def sweep(op, kind, expect, cleanup=None, max_k=80):
    """Runs op() under kind@k for k = 1.. until it returns AC_OK; returns (k of the clean run, its value)."""
    base = _held()
    for k in range(1, max_k + 1):
        acg.fault_inject(f"{kind}@{k}")
        try:
            st, val = op()
        finally:
            acg.fault_inject(None)
        if st == N.AC_OK:
            if cleanup:
                cleanup(val)
            assert _held() == base, f"{kind}@{k}: memory held after the clean call"
            return k, val
        assert st == expect, f"{kind}@{k}: status {st}, expected {expect}"
        assert _held() == base, f"{kind}@{k}: memory held after a failed call"
    raise AssertionError(f"{kind}: still failing after {max_k} injections")


def _result(cap, n_pat, on_device=True):
    if on_device:
        raw = torch.zeros((cap, 2), dtype=torch.int64, device="cuda")
        cnt = torch.zeros(n_pat, dtype=torch.int64, device="cuda")
    else:
        raw = torch.zeros((cap, 2), dtype=torch.int64).pin_memory()
        cnt = torch.zeros(n_pat, dtype=torch.int64).pin_memory()
    return raw, cnt, N.Result(raw.data_ptr(), cap, 0, cnt.data_ptr(), int(on_device), 0, 0)


def _canon(raw, k):
    a = raw[:k].cpu().numpy()
    a = np.stack([a[:, 0], a[:, 1] & 0xFFFFFFFF], 1)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def test_fault_plan_parsing():
    for spec in ("oom@1", "cuda_err@3", "oom@2,cuda_err@5", ""):
        acg.fault_inject(spec)
    acg.fault_inject(None)
    for bad in ("oom", "oom@0", "oom@x", "leak@1", "oom@1;cuda_err@2"):
        assert lib().ac_fault_inject(bad.encode()) == N.AC_ERR_INVALID_ARG


@pytest.mark.parametrize("kind,expect", [("oom", N.AC_ERR_OOM), ("cuda_err", N.AC_ERR_CUDA)])
def test_scan_entry_points_fail_cleanly(kind, expect):
    text, pats = _case()
    d = acg.build(pats)
    want, want_counts = oracle_canonical(pats, text)
    P, cap, n = len(pats), len(want) + 64, len(text)
    ascii_dev = torch.tensor(np.frombuffer(text, np.uint8), device="cuda")
    packed = acg.pack(ascii_dev)
    host_ascii = np.frombuffer(text, np.uint8).copy()

    def check(raw, cnt, r):
        assert int(r.n_matches) == len(want)
        assert np.array_equal(_canon(raw, len(want)), want[:, 1:])
        assert np.array_equal(cnt.cpu().numpy(), want_counts)

    forms = {
        "packed_dev": (N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1), True),
        "ascii_dev": (N.Text(ascii_dev.data_ptr(), n, N.AC_TEXT_ASCII, 1), True),
        "ascii_host": (N.Text(host_ascii.ctypes.data, n, N.AC_TEXT_ASCII, 0), False),
    }
    for name, (desc, on_dev) in forms.items():
        raw, cnt, r = _result(cap, P, on_dev)
        k, _ = sweep(lambda: (lib().ac_scan(d.h, ctypes.byref(desc), ctypes.byref(r), None, None, None), None),
                     kind, expect)
        assert k > 1, name  # at least one injection hit the call
        check(raw, cnt, r)
        if on_dev:  # failure-less matching over the same text
            df = acg.build(pats, failureless=True)
            raw, cnt, r = _result(cap, P, on_dev)
            k, _ = sweep(lambda: (lib().ac_scan_failureless(df.h, ctypes.byref(desc), ctypes.byref(r), None, None,
                                                            None), None), kind, expect)
            assert k > 1, name
            check(raw, cnt, r)
    # batch: device packed texts and host ASCII texts
    cuts = [0, 1, 70, 5000, 60_000, n]
    parts = [text[a:b] for a, b in zip(cuts[:-1], cuts[1:])]
    want_b = np.concatenate([oracle_canonical(pats, t, text_id=i)[0] for i, t in enumerate(parts)])
    want_b = want_b[np.lexsort((want_b[:, 2], want_b[:, 1], want_b[:, 0]))]
    dev_parts = [acg.pack(torch.tensor(np.frombuffer(t, np.uint8), device="cuda")) if t else
                 torch.zeros(4, dtype=torch.int32, device="cuda") for t in parts]
    host_parts = [np.frombuffer(t, np.uint8).copy() for t in parts]
    for on_dev in (True, False):
        descs = (N.Text * len(parts))(*[
            N.Text(dp.data_ptr() if t else None, len(t), N.AC_TEXT_PACKED2, 1) if on_dev else
            N.Text(hp.ctypes.data if t else None, len(t), N.AC_TEXT_ASCII, 0)
            for t, dp, hp in zip(parts, dev_parts, host_parts)])
        raw, cnt, r = _result(len(want_b) + 64, P, on_dev)
        k, _ = sweep(lambda: (lib().ac_scan_batch(d.h, descs, len(parts), ctypes.byref(r), None, None, None), None),
                     kind, expect)
        assert k > 1
        a = raw[: int(r.n_matches)].cpu().numpy()
        got = np.stack([(a[:, 1] >> 32) & 0xFFFFFFFF, a[:, 0], a[:, 1] & 0xFFFFFFFF], 1)
        assert np.array_equal(got[np.lexsort((got[:, 2], got[:, 1], got[:, 0]))], want_b)
    # pack
    out = torch.empty((n + 15) // 16, dtype=torch.int32, device="cuda")
    bad = ctypes.c_uint64()
    sweep(lambda: (lib().ac_pack(ascii_dev.data_ptr(), n, out.data_ptr(), 0, ctypes.byref(bad), None), None),
          kind, expect)
    assert torch.equal(out, packed[: out.numel()])


@pytest.mark.parametrize("kind,expect", [("oom", N.AC_ERR_OOM), ("cuda_err", N.AC_ERR_CUDA)])
def test_objects_fail_cleanly(kind, expect):
    """ac_build, streams, batch plans, partitioned sets: a failed create holds nothing; a failed
    stream scan leaves the stream unchanged, so the piece can be sent again."""
    text, pats = _case(6, 120_000, 400)
    want, want_counts = oracle_canonical(pats, text)
    bufs = [bytes(p) for p in pats]
    ptrs = (ctypes.c_char_p * len(bufs))(*bufs)
    lens = np.array([len(b) for b in bufs], np.uint32)

    def build():
        h = ctypes.c_void_p()
        st = lib().ac_build(ctypes.cast(ptrs, ctypes.c_void_p), lens.ctypes.data, len(bufs), None, ctypes.byref(h))
        return st, h

    if kind == "oom":
        k, h = sweep(build, kind, expect, cleanup=lambda h: lib().ac_free(h))
        assert k > 3  # one allocation per table
    d = acg.build(pats)
    n, P = len(text), len(pats)
    packed = acg.pack(torch.tensor(np.frombuffer(text, np.uint8), device="cuda"))

    # a stream fed in three pieces, each piece swept
    def make_stream():
        h = ctypes.c_void_p()
        return lib().ac_stream_create(d.h, ctypes.byref(h)), h

    if kind == "oom":
        sweep(make_stream, kind, expect, cleanup=lambda h: lib().ac_stream_free(h))
    s = acg.Stream(d)
    cuts = [0, 33_333, 33_340, n]
    rows, csum = [], np.zeros(P, np.int64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        piece = np.frombuffer(text[a:b], np.uint8).copy()
        desc = N.Text(piece.ctypes.data, b - a, N.AC_TEXT_ASCII, 0)
        raw, cnt, r = _result(len(want) + 64, P, True)
        sweep(lambda: (lib().ac_stream_scan(s.h, ctypes.byref(desc), ctypes.byref(r), None, None, None), None),
              kind, expect)
        rows.append(_canon(raw, int(r.n_matches)))
        csum += cnt.cpu().numpy()
    got = np.concatenate(rows)
    assert np.array_equal(got[np.lexsort((got[:, 1], got[:, 0]))], want[:, 1:])
    assert np.array_equal(csum, want_counts)
    s.close()
    # a batch plan over two device texts
    halves = [packed, acg.pack(torch.tensor(np.frombuffer(text[: n // 2], np.uint8), device="cuda"))]
    descs = (N.Text * 2)(N.Text(halves[0].data_ptr(), n, N.AC_TEXT_PACKED2, 1),
                         N.Text(halves[1].data_ptr(), n // 2, N.AC_TEXT_PACKED2, 1))
    raw, cnt, r = _result(4 * len(want) + 64, P, True)

    def make_plan():
        h = ctypes.c_void_p()
        return lib().ac_batch_plan_create(d.h, descs, 2, ctypes.byref(r), None, None, ctypes.byref(h)), h

    half = want[want[:, 1] + np.array([len(pats[p]) for p in want[:, 2]]) <= n // 2]

    def run_and_free(h):
        for _ in range(2):
            rr = N.Result()
            assert lib().ac_batch_plan_run(h, None, 1, ctypes.byref(rr)) == N.AC_OK
            assert int(rr.n_matches) == len(want) + len(half)
        lib().ac_batch_plan_free(h)

    k, _ = sweep(make_plan, kind, expect, cleanup=run_and_free)
    assert k > 1
    # partitioned keyword sets: the build and the scan
    if kind == "oom":
        def make_parts():
            h = ctypes.c_void_p()
            return lib().ac_build_partitioned(ctypes.cast(ptrs, ctypes.c_void_p), lens.ctypes.data, len(bufs), 2000,
                                              None, ctypes.byref(h)), h

        sweep(make_parts, kind, expect, cleanup=lambda h: lib().ac_part_set_free(h))
    ps = acg.build_partitioned(pats, max_states=2000)
    desc = N.Text(packed.data_ptr(), n, N.AC_TEXT_PACKED2, 1)
    raw, cnt, r = _result(len(want) + 64, P, True)
    sweep(lambda: (lib().ac_scan_partitioned(ps.h, ctypes.byref(desc), ctypes.byref(r), None, None, None), None),
          kind, expect)
    assert np.array_equal(_canon(raw, int(r.n_matches)), want[:, 1:])
    assert np.array_equal(cnt.cpu().numpy(), want_counts)
    ps.close()


def test_noalloc_allocates_nothing_and_fails_cleanly_on_a_launch_fault():
    text, pats = _case(7, 100_000, 300)
    d = acg.build(pats)
    want, want_counts = oracle_canonical(pats, text)
    packed = acg.pack(torch.tensor(np.frombuffer(text, np.uint8), device="cuda"))
    desc = N.Text(packed.data_ptr(), len(text), N.AC_TEXT_PACKED2, 1)
    raw, cnt, r = _result(len(want) + 64, len(pats), True)
    assert lib().ac_scan_noalloc(d.h, ctypes.byref(desc), ctypes.byref(r), None, None) == N.AC_OK  # first-call set-up
    acg.fault_inject("oom@1")
    st = lib().ac_scan_noalloc(d.h, ctypes.byref(desc), ctypes.byref(r), None, None)
    seen = acg.mem_usage()["allocations_seen"]
    acg.fault_inject(None)
    assert st == N.AC_OK and seen == 0  # no allocation was even attempted
    assert np.array_equal(_canon(raw, int(r.n_matches)), want[:, 1:])
    k, _ = sweep(lambda: (lib().ac_scan_noalloc(d.h, ctypes.byref(desc), ctypes.byref(r), None, None), None),
                 "cuda_err", N.AC_ERR_CUDA)
    assert k > 1
    assert np.array_equal(_canon(raw, int(r.n_matches)), want[:, 1:])
    assert np.array_equal(cnt.cpu().numpy(), want_counts)


@pytest.mark.parametrize("kind,expect", [("oom", N.AC_ERR_OOM), ("cuda_err", N.AC_ERR_CUDA)])
def test_serving_request_fails_alone(kind, expect):
    text, pats = _case(8, 150_000, 500)
    want, want_counts = oracle_canonical(pats, text)
    d = acg.build(pats)
    srv = acg.Server(n_streams=1, max_batch=8)
    slot = srv.add_dfa(d)
    host = np.frombuffer(text, np.uint8).copy()
    # warm the worker (its first batch sets up buffers) with a clean request
    m, c, k = srv.wait(srv.submit(slot, host), slot)
    assert k == len(want)
    base = _held()
    acg.fault_inject(f"{kind}@1")  # the worker's next allocation / launch fails
    t_bad = srv.submit(slot, host)
    with pytest.raises(acg.AcError) as e:
        srv.wait(t_bad, slot)
    acg.fault_inject(None)
    assert e.value.status == expect
    assert srv.stats()["failed"] == 1
    assert _held() == base
    for _ in range(2):  # the server goes on serving, exactly
        m, c, k = srv.wait(srv.submit(slot, host), slot)
        got = m[np.lexsort((m[:, 1], m[:, 0]))]
        assert np.array_equal(got, want[:, 1:]) and np.array_equal(c, want_counts)
    srv.close()


@pytest.mark.parametrize("kind,expect", [("oom", N.AC_ERR_OOM), ("cuda_err", N.AC_ERR_CUDA)])
def test_overlapped_host_scan_fails_cleanly(kind, expect):
    """The host-buffer path that overlaps copies and scans over pieces (texts of 512 Mbase or more):
    a failure in any piece releases everything; the clean run equals the device-resident scan."""
    n = (512 << 20) + 1_000_003
    g = torch.Generator(device="cuda").manual_seed(91)
    codes = torch.randint(0, 4, (n,), device="cuda", generator=g, dtype=torch.uint8)
    ascii_dev = torch.tensor(list(b"ACGT"), dtype=torch.uint8, device="cuda")[codes.long()]
    rng = random.Random(92)
    starts = rng.sample(range(n - 40), 300)
    pats = [bytes(ascii_dev[j : j + rng.randint(10, 16)].cpu().numpy()) for j in starts]
    d = acg.build(pats)
    ref = acg.scan(d, ascii_dev)
    want = ref.canonical()[:, 1:]
    host = ascii_dev.cpu().pin_memory()
    desc = N.Text(host.data_ptr(), n, N.AC_TEXT_ASCII, 0)
    raw, cnt, r = _result(ref.n_matches + 64, len(pats), False)
    k, _ = sweep(lambda: (lib().ac_scan(d.h, ctypes.byref(desc), ctypes.byref(r), None, None, None), None),
                 kind, expect)
    assert k > 3
    assert int(r.n_matches) == ref.n_matches
    assert np.array_equal(_canon(raw, ref.n_matches), want)
    assert np.array_equal(cnt.numpy(), ref.counts.cpu().numpy())
