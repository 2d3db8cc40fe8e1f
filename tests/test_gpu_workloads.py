"""GPU parity on the benchmark workloads at their full sizes, in the launch
configuration the benchmark times (the library's default shape).

  * 256 Mbase Markov chromosome, 10,000 keywords: every occurrence against
    the oracle's full scan, at one, two and three bases per lookup;
  * 3 Gbase Markov genome, 100,000 keywords: occurrences in 24 sampled
    windows against the oracle run on each window (with the L_max-1 halo),
    plus properties that hold at any size (counts = histogram of the list,
    sum of counts = occurrences, the same set under launch shapes reading
    two and three bases per lookup);
  * 4,096 lognormal texts, 50,000 keywords: the graph-replayed batch and the
    per-text loop against the oracle on every text;
  * the 8 serving sets: requests alone and mixed against the oracle.
"""
import random

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


def test_genome_sampled_parity_and_invariants():
    w = synth.plain_genome(device="cuda")
    n = w.text.ascii.numel()
    d = acg.build(w.patterns)
    packed = acg.pack(w.text.ascii)
    lens = torch.tensor([len(p) for p in w.patterns], dtype=torch.int64, device="cuda")
    lmax = int(lens.max())
    r = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=n, capacity=1 << 20)
    k = r.n_matches
    assert k > 1_000_000  # repeat-driven density
    # any-size properties
    assert int(r.counts.sum()) == k
    hist = torch.bincount(r.pattern_id, minlength=len(w.patterns))
    assert torch.equal(hist, r.counts)
    # the same set under a second launch shape (two bases per lookup, small chunks, nothing in shared memory)
    r2 = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=n, capacity=k + 16, interleave=1, chunk=4096,
                  hot_states=0, stride=2)
    assert r2.n_matches == k
    a = torch.sort(_keys(r.pos, r.pattern_id))[0]
    b = torch.sort(_keys(r2.pos, r2.pattern_id))[0]
    assert torch.equal(a, b)
    del r2, b
    # and three bases per lookup, in one 1024-thread block per SM and in two 640-thread blocks
    for threads in (1024, 640):
        r3 = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=n, capacity=k + 16, interleave=1, stride=3,
                      threads=threads)
        assert r3.n_matches == k
        assert torch.equal(a, torch.sort(_keys(r3.pos, r3.pattern_id))[0])
        assert torch.equal(r.counts, r3.counts)
        del r3
    assert torch.equal(r.counts, acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=n, capacity=0,
                                          interleave=2, stride=1).counts)
    # sampled windows against the oracle
    end = r.pos + lens[r.pattern_id] - 1
    rng = random.Random(2024)
    m = oracle.Machine(w.patterns)
    lens_h = lens.cpu().numpy()
    starts = sorted(rng.sample(range(0, n - 2_000_000), 22)) + [0, n - 2_000_000]
    total = 0
    for s0 in starts:
        s1 = s0 + 2_000_000
        rb = max(0, s0 - (lmax - 1))
        win = w.text.ascii[rb:s1].cpu().numpy()
        pos, pid, _ = m.scan(win)
        e = pos.astype(np.int64) + lens_h[pid] - 1 + rb
        keep = e >= s0
        want = np.stack([pos[keep].astype(np.int64) + rb, pid[keep].astype(np.int64)], 1)
        want = want[np.lexsort((want[:, 1], want[:, 0]))]
        sel = (end >= s0) & (end < s1)
        got = torch.stack([r.pos[sel], r.pattern_id[sel]], 1).cpu().numpy()
        got = got[np.lexsort((got[:, 1], got[:, 0]))]
        assert np.array_equal(got, want), f"window {s0}"
        total += len(want)
    assert total > 0


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
    genome = synth.markov_text(8 << 20, synth.BASE_SEED + 4, device="cuda")
    sets = synth.serve_sets(genome.ascii)
    g = genome.ascii.cpu().numpy()
    dfas = [acg.build(s) for s in sets]
    t_arr, lens, offs, which = synth.serve_requests(48, synth.BASE_SEED + 5, len(g), hi=2_000_000)
    srv = acg.Server(n_streams=4, max_batch=32)
    slots = [srv.add_dfa(x) for x in dfas]
    tks = [srv.submit(slots[s], g[o : o + n]) for s, o, n in zip(which, offs, lens)]
    mix = [srv.wait(t, slots[s], capacity=4096) for t, s in zip(tks, which)]
    for i in range(0, 48, 6):  # a subset alone and against the oracle
        s, o, n = int(which[i]), int(offs[i]), int(lens[i])
        alone = srv.wait(srv.submit(slots[s], g[o : o + n]), slots[s])
        a = alone[0][np.lexsort((alone[0][:, 1], alone[0][:, 0]))]
        b = mix[i][0][np.lexsort((mix[i][0][:, 1], mix[i][0][:, 0]))]
        assert np.array_equal(a, b) and np.array_equal(alone[1], mix[i][1])
        want, counts = oracle_canonical(sets[s], g[o : o + n])
        assert np.array_equal(a, want[:, 1:]) and np.array_equal(alone[1], counts)
    srv.close()
