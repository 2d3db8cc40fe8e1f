"""CPU tests that the seeded generators produce the stated input recipe: the Markov text's
composition and tandem repeats, the keyword sets, the batch length law and the serving request
stream (the inputs stand in for the DNA workloads; the paper names no dataset)."""
import math

import numpy as np
import torch

from paper_1403_7294_gb300 import synth

ALPHA = np.frombuffer(b"ACGT", np.uint8)


def test_markov_chain_rows_and_stationary_gc():
    P = synth.markov_chain(synth.BASE_SEED + 1)
    assert P.shape == (16, 4) and np.allclose(P.sum(axis=1), 1.0) and (P > 0).all()
    # stationary distribution of the pair chain, by power iteration written out here
    T = np.zeros((16, 16))
    for ctx in range(16):
        for x in range(4):
            T[ctx, 4 * (ctx % 4) + x] += P[ctx, x]
    v = np.full(16, 1 / 16)
    for _ in range(3000):
        v = v @ T
    last = v.reshape(4, 4).sum(axis=0)  # distribution of the newest base
    assert abs((last[1] + last[2]) - 0.41) < 1e-3
    # CpG depletion: G after C is rarer than G after any other base
    g_after = [P[4 * a + b, 2] for a in range(4) for b in range(4)]
    after_c = [P[4 * a + 1, 2] for a in range(4)]
    others = [P[4 * a + b, 2] for a in range(4) for b in (0, 2, 3)]
    assert max(after_c) < min(others) and len(g_after) == 16


def test_markov_text_composition_and_tandem_repeats():
    n = 4_000_000
    t = synth.markov_text(n, synth.BASE_SEED + 11, device="cpu")
    a = t.ascii.numpy()
    assert a.shape == (n,) and np.isin(a, ALPHA).all()
    gc = np.isin(a, np.frombuffer(b"CG", np.uint8)).mean()
    assert 0.40 < gc < 0.43  # 0.41 outside repeats, repeat units are uniform
    st, ln, ul = t.strs.start.numpy(), t.strs.length.numpy(), t.strs.unit_len.numpy()
    assert abs(ln.sum() / n - 0.05) < 0.005
    assert (ln >= 20).all() and (ln <= 200).all() and (ul >= 1).all() and (ul <= 6).all()
    order = np.argsort(st)
    assert (st[order][1:] >= (st + ln)[order][:-1]).all()  # runs do not overlap
    for s, L, u in zip(st[:200], ln[:200], ul[:200]):
        run = a[s : s + L]
        assert (run[u:] == run[:-u]).all()  # each run repeats its unit
    c = (a[:-1] == ord("C")) & (a[1:] == ord("G"))
    expect = (a == ord("C")).mean() * (a == ord("G")).mean()
    assert c.mean() < 0.6 * expect  # CpG depleted


def test_generators_are_seeded():
    a = synth.markov_text(100_000, 5, device="cpu").ascii
    assert torch.equal(a, synth.markov_text(100_000, 5, device="cpu").ascii)
    assert not torch.equal(a, synth.markov_text(100_000, 6, device="cpu").ascii)
    assert synth.uniform_patterns(50, 8, 12, 3) == synth.uniform_patterns(50, 8, 12, 3)


def test_keyword_sets():
    u = synth.uniform_patterns(2000, 18, 30, 7, gc_clamp=(0.4, 0.6))
    assert len(u) == len(set(u)) == 2000
    for p in u:
        assert 18 <= len(p) <= 30 and set(p) <= set(b"ACGT")
        gc = sum(c in b"CG" for c in p) / len(p)
        assert 0.4 <= gc <= 0.6
    text = synth.markov_text(200_000, 9, device="cpu")
    s = synth.substring_patterns(text.ascii, 500, 20, 25, 10, avoid=text.strs)
    raw = bytes(text.ascii.numpy())
    assert len(s) == len(set(s)) == 500 and all(p in raw and 20 <= len(p) <= 25 for p in s)
    merged = synth.merge_dedupe([b"AC", b"GT"], [b"GT", b"AA"], [b"AC"])
    assert merged == [b"AC", b"GT", b"AA"]


def test_batch_lengths_law():
    lens = synth.batch_lengths(4096, synth.BASE_SEED + 3)
    assert int(lens.sum()) == 38_333_955  # the batch total the measurements quote
    assert lens.min() >= 100 and lens.max() <= 100_000
    big = synth.batch_lengths(200_000, 1)
    assert abs(np.median(big) - 2000) / 2000 < 0.03  # lognormal median e^mu
    assert 0.02 < (big == 100_000).mean() < 0.035 and 0.06 < (big == 100).mean() < 0.08


def test_serving_request_stream():
    t, lens, offs, sets = synth.serve_requests(200_000, 3, 64 << 20)
    rate = len(t) / t[-1]
    assert abs(rate - 2000) / 2000 < 0.02
    assert lens.min() >= 1_000 and lens.max() <= 10_000_000
    assert abs(np.log(lens).mean() - (math.log(1e3) + math.log(1e7)) / 2) < 0.02  # log-uniform
    assert (offs >= 0).all() and (offs + lens <= 64 << 20).all()
    assert set(np.unique(sets)) == set(range(8))
