"""GPU parity on the benchmark workloads at their full sizes, in the launch
configuration the benchmark times (the autotuned shape, as the benchmark
picks it).

  * 256 Mbase Markov chromosome, 10,000 keywords: every occurrence against
    the oracle's full scan, at one, two and three bases per lookup;
  * 3 Gbase Markov genome, 100,000 keywords: every occurrence and every
    per-keyword count against the oracle. The text is cut into 64 ranges of
    start positions; the oracle scans each range plus the L_max-1 bases after
    it (all host cores, one range per thread) and keeps the occurrences that
    start inside it, while the GPU's occurrences, sorted on the device by
    (start, keyword), are read back one range at a time. The same set comes
    out under launch shapes reading one, two and three bases per lookup;
  * 4,096 lognormal texts, 50,000 keywords: the graph-replayed batch and the
    per-text loop against the oracle on every text;
  * the 8 serving sets: every request alone and in the mix against the oracle,
    on a small genome, and 256 requests of the benchmark's own stream over its
    64 Mbase serving genome.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from paper_1403_7294_gb300 import synth
from tests.gpu_helpers import oracle_canonical

pytestmark = pytest.mark.gpu


def _keys(pos: torch.Tensor, pid: torch.Tensor) -> torch.Tensor:
    return pos * (1 << 20) + pid


def test_chromosome_full_parity():
    w = synth.plain_chromosome(device="cuda")
    d = acg.build(w.patterns)
    packed = acg.pack(w.text.ascii)
    n = w.text.ascii.numel()
    want, counts = oracle_canonical(w.patterns, w.text.ascii)
    for stride in (1, 2, 3):
        r = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=n, stride=stride)
        got = r.canonical()
        assert got.shape == want.shape and np.array_equal(got, want)
        assert r.counts.cpu().numpy().tolist() == counts.tolist()
    assert r.n_matches > 5000  # the substring half of the keywords occurs


PID_BITS = 17  # keyword ids of the genome workload are below 2^17


def _sorted_keys(pos: torch.Tensor, pid: torch.Tensor) -> torch.Tensor:
    """(start, keyword) pairs as one sorted int64 key per occurrence, on the device."""
    return torch.sort(pos * (1 << PID_BITS) + pid)[0]


def test_genome_full_parity_against_the_oracle():
    from concurrent.futures import ThreadPoolExecutor

    w = synth.plain_genome(device="cuda")
    n = w.text.ascii.numel()
    P = len(w.patterns)
    assert P < (1 << PID_BITS)
    d = acg.build(w.patterns)
    packed = acg.pack(w.text.ascii)
    lmax = max(len(p) for p in w.patterns)
    acg.autotune(d, packed, n)  # the benchmark's launch shape
    r = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=n, capacity=1 << 20)
    k = r.n_matches
    assert k > 1_000_000  # repeat-driven density
    assert int(r.counts.sum()) == k
    keys = _sorted_keys(r.pos, r.pattern_id)
    counts = r.counts.cpu().numpy()
    del r
    # the same set under other launch shapes: one base per lookup with two chains per lane and small
    # chunks, two bases per lookup, three bases per lookup in one 1024-thread block per SM
    for kw in ({"stride": 1, "interleave": 2, "chunk": 4096}, {"stride": 2, "interleave": 1, "hot_states": 0},
               {"stride": 3, "interleave": 1, "threads": 1024}):
        r2 = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=n, capacity=k + 16, **kw)
        assert r2.n_matches == k, kw
        assert torch.equal(keys, _sorted_keys(r2.pos, r2.pattern_id)), kw
        assert np.array_equal(r2.counts.cpu().numpy(), counts), kw
        del r2
    # every occurrence against the oracle, 64 ranges of start positions on all host cores
    text = w.text.ascii.cpu().numpy()
    del w.text.ascii, packed
    m = oracle.Machine(w.patterns)
    W = 64
    bounds = [n * i // W for i in range(W + 1)]

    def oracle_range(i):
        s0, s1 = bounds[i], bounds[i + 1]
        pos, pid, _ = m.scan(text[s0 : min(n, s1 + lmax - 1)])
        start = pos.astype(np.int64) + s0
        keep = start < s1  # every occurrence starting in [s0, s1) ends before s1 + lmax - 1
        pid = pid[keep].astype(np.int64)
        return np.sort((start[keep] << PID_BITS) | pid), np.bincount(pid, minlength=P)

    want_counts = np.zeros(P, np.int64)
    total = 0
    with ThreadPoolExecutor(max_workers=min(W, os.cpu_count() or 4)) as ex:
        for i, (want, c) in enumerate(ex.map(oracle_range, range(W))):
            lo = int(torch.searchsorted(keys, torch.tensor([bounds[i] << PID_BITS], device=keys.device)))
            hi = int(torch.searchsorted(keys, torch.tensor([bounds[i + 1] << PID_BITS], device=keys.device)))
            got = keys[lo:hi].cpu().numpy()
            assert got.shape == want.shape and np.array_equal(got, want), f"range {i} [{bounds[i]}, {bounds[i + 1]})"
            want_counts += c
            total += len(want)
    assert total == k
    assert np.array_equal(counts, want_counts)


def test_batched_full_parity():
    w = synth.batched(device="cuda")
    lens = [int(t.numel()) for t in w.texts]
    d = acg.build(w.patterns)
    packed = [acg.pack(t.contiguous()) for t in w.texts]
    rows, counts = [], np.zeros(len(w.patterns), np.int64)
    m = oracle.Machine(w.patterns)
    for i, t in enumerate(w.texts):
        pos, pid, c = m.scan(t.cpu().numpy())
        rows.append(np.stack([np.full(len(pos), i, np.int64), pos.astype(np.int64), pid.astype(np.int64)], 1))
        counts += c.astype(np.int64)
    want = np.concatenate(rows)
    want = want[np.lexsort((want[:, 2], want[:, 1], want[:, 0]))]
    plan = acg.BatchPlan(d, packed, lens, capacity=len(want) + 64)
    for _ in range(2):
        assert plan.run() == len(want)
        assert np.array_equal(plan.result().canonical(), want)
        assert plan.counts.cpu().numpy().tolist() == counts.tolist()
    plan.close()
    r = acg.scan_batch(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=lens)
    assert np.array_equal(r.canonical(), want)


def test_serving_sets_alone_vs_mix():
    """Every one of 48 requests: submitted together (batched with others of its machine while other
    batches run), then alone, then against the oracle."""
    from concurrent.futures import ThreadPoolExecutor

    genome = synth.markov_text(8 << 20, synth.BASE_SEED + 4, device="cuda")
    sets = synth.serve_sets(genome.ascii)
    g = genome.ascii.cpu().numpy()
    dfas = [acg.build(s) for s in sets]
    t_arr, lens, offs, which = synth.serve_requests(48, synth.BASE_SEED + 5, len(g), hi=2_000_000)
    srv = acg.Server(n_streams=4, max_batch=32)
    slots = [srv.add_dfa(x) for x in dfas]
    tks = [srv.submit(slots[s], g[o : o + n]) for s, o, n in zip(which, offs, lens)]
    mix = [srv.wait(t, slots[s], capacity=4096) for t, s in zip(tks, which)]
    st = srv.stats()
    assert st["completed"] == 48 and st["failed"] == 0
    machines = {s: oracle.Machine(sets[s]) for s in set(int(x) for x in which)}  # shared by the threads (read only)

    def want_of(i):
        s, o, n = int(which[i]), int(offs[i]), int(lens[i])
        pos, pid, c = machines[s].scan(g[o : o + n])
        a = np.stack([pos.astype(np.int64), pid.astype(np.int64)], 1)
        return a[np.lexsort((a[:, 1], a[:, 0]))], c.astype(np.int64)

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        wants = list(ex.map(want_of, range(48)))
    for i in range(48):
        s, o, n = int(which[i]), int(offs[i]), int(lens[i])
        alone = srv.wait(srv.submit(slots[s], g[o : o + n]), slots[s])
        a = alone[0][np.lexsort((alone[0][:, 1], alone[0][:, 0]))]
        b = mix[i][0][np.lexsort((mix[i][0][:, 1], mix[i][0][:, 0]))]
        want, counts = wants[i]
        assert np.array_equal(b, want) and np.array_equal(mix[i][1], counts), f"request {i} in the mix"
        assert np.array_equal(a, want) and np.array_equal(alone[1], counts), f"request {i} alone"
    srv.close()


def test_serving_at_benchmark_sizes_against_the_oracle():
    """The serving workload as the benchmark builds it: the 64 Mbase serving genome, the 8
    resident machines (1,000 to 100,000 keywords) and requests from the benchmark's own stream
    (1 kbase to 10 Mbase, the same seed), submitted at once so that batches of several requests
    form beside single ones; every request's occurrences and counts against the oracle."""
    from concurrent.futures import ThreadPoolExecutor

    genome = synth.markov_text(64 << 20, synth.BASE_SEED + 4, device="cuda")
    sets = synth.serve_sets(genome.ascii)
    g = genome.ascii.cpu().numpy()
    del genome
    dfas = [acg.build(s) for s in sets]
    n_req = 256
    _, lens, offs, which = synth.serve_requests(n_req, synth.BASE_SEED + 5, len(g))
    srv = acg.Server(device_budget_bytes=40 << 30, n_streams=4, max_batch=256)
    slots = [srv.add_dfa(d) for d in dfas]
    tickets = [srv.submit(slots[int(s)], g[int(o) : int(o) + int(n)]) for s, o, n in zip(which, offs, lens)]
    got = [srv.wait(t, slots[int(s)]) for t, s in zip(tickets, which)]
    st = srv.stats()
    assert st["completed"] == n_req and st["failed"] == 0
    assert st["batches_launched"] < n_req  # some requests were batched together
    machines = {s: oracle.Machine(sets[s]) for s in set(int(x) for x in which)}  # shared (read only)

    def want_of(i):
        s, o, n = int(which[i]), int(offs[i]), int(lens[i])
        pos, pid, c = machines[s].scan(g[o : o + n])
        a = np.stack([pos.astype(np.int64), pid.astype(np.int64)], 1)
        return a[np.lexsort((a[:, 1], a[:, 0]))], c.astype(np.int64)

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        for i, (want, counts) in enumerate(ex.map(want_of, range(n_req))):
            m, c, k = got[i]
            assert k == len(want), f"request {i}"
            assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want), f"request {i}"
            assert np.array_equal(c, counts), f"request {i}"
    srv.close()
