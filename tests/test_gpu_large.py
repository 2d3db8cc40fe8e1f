"""GPU parity on a text longer than 2^32 bases (the largest size class).

Positions past 2^32 need the 64-bit position path end to end: chunk starts,
the end positions carried through the event queue, the start = end - len + 1
written by the drain, piece offsets of the host-buffer and streaming scans and
the batch's per-text items. The text is 2^32 + 200,000,037 i.i.d. bases, a
length that is a multiple of neither 16 nor 64. The keywords are 200 uniform
ones plus substrings taken from the text at known places past 2^32 (one starts
exactly at 2^32, one straddles it, one ends on the last base). Checks:

  * the oracle on 2 Mbase windows (with the L_max-1 halo) around 2^32, at the
    end and at two random places past 2^32, against the scan's occurrences
    ending in each window;
  * every planted keyword is reported at the place it was taken from;
  * counts are the histogram of the list and sum to the number of occurrences;
  * the same occurrence set at one, two and three bases per lookup, from ASCII
    input, from two owned ranges split just past 2^32, from pinned host
    buffers (the overlapped path), as text 1 of a two-text batch and from a
    stream fed in 1 Gbase pieces.
"""
import random

import numpy as np
import pytest
import torch

import oracle
import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from paper_1403_7294_gb300 import synth

pytestmark = pytest.mark.gpu

TWO32 = 1 << 32
N_BASES = TWO32 + 200_000_037
SLICE = 1 << 29  # bases generated per call of the uniform generator


def _keys(pos, pid):
    return torch.sort(pos * (1 << 20) + pid)[0]


@pytest.fixture(scope="module")
def big():
    ascii_ = torch.empty(N_BASES, dtype=torch.uint8, device="cuda")
    for i, a in enumerate(range(0, N_BASES, SLICE)):
        b = min(N_BASES, a + SLICE)
        ascii_[a:b] = synth.uniform_text(b - a, synth.BASE_SEED + 900 + i, device="cuda")
    rng = random.Random(4242)
    pats = synth.uniform_patterns(200, 10, 14, synth.BASE_SEED + 950)
    starts = [TWO32, TWO32 - 9, N_BASES - 24, TWO32 + 1]
    starts += rng.sample(range(TWO32 + 2, N_BASES - 30), 36)
    planted = []
    for s in starts:
        ln = 24 if s == N_BASES - 24 else rng.randint(18, 24)
        p = bytes(ascii_[s : s + ln].cpu().numpy())
        if p not in pats:
            planted.append((len(pats), s))
            pats.append(p)
    d = acg.build(pats)
    packed = acg.pack(ascii_)
    r = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=N_BASES)
    yield ascii_, packed, pats, planted, d, r
    d.close()


def test_windows_against_oracle(big):
    ascii_, packed, pats, planted, d, r = big
    lens = torch.tensor([len(p) for p in pats], dtype=torch.int64, device="cuda")
    lmax = int(lens.max())
    end = r.pos + lens[r.pattern_id] - 1
    m = oracle.Machine(pats)
    lens_h = lens.cpu().numpy()
    win = 1 << 21
    rng = random.Random(77)
    starts = [TWO32 - win // 2, N_BASES - win] + rng.sample(range(TWO32, N_BASES - win), 2)
    total = 0
    for s0 in starts:
        s1 = s0 + win
        rb = s0 - (lmax - 1)
        pos, pid, _ = m.scan(ascii_[rb:s1].cpu().numpy())
        e = pos.astype(np.int64) + lens_h[pid] - 1 + rb
        keep = e >= s0
        want = np.stack([pos[keep].astype(np.int64) + rb, pid[keep].astype(np.int64)], 1)
        want = want[np.lexsort((want[:, 1], want[:, 0]))]
        sel = (end >= s0) & (end < s1)
        got = torch.stack([r.pos[sel], r.pattern_id[sel]], 1).cpu().numpy()
        got = got[np.lexsort((got[:, 1], got[:, 0]))]
        assert np.array_equal(got, want), f"window at {s0}"
        total += len(want)
    assert total > 0


def test_planted_and_counts(big):
    ascii_, packed, pats, planted, d, r = big
    assert len(planted) >= 38
    have = set(zip(r.pos.cpu().tolist(), r.pattern_id.cpu().tolist()))
    for k, s in planted:
        assert (s, k) in have, (k, s)
    assert int(r.pos.max()) >= N_BASES - 24  # the keyword planted on the last bases
    assert int(r.counts.sum()) == r.n_matches
    assert torch.equal(torch.bincount(r.pattern_id, minlength=len(pats)), r.counts)


@pytest.mark.parametrize("stride", [1, 2, 3])
def test_strides_and_ascii_agree(big, stride):
    ascii_, packed, pats, planted, d, r = big
    want = _keys(r.pos, r.pattern_id)
    g = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=N_BASES, stride=stride)
    assert torch.equal(_keys(g.pos, g.pattern_id), want)
    assert torch.equal(g.counts, r.counts)
    a = acg.scan(d, ascii_, stride=stride)
    assert torch.equal(_keys(a.pos, a.pattern_id), want)


def test_owned_ranges_split_past_2_32(big):
    ascii_, packed, pats, planted, d, r = big
    cut = TWO32 + 7
    lo = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=N_BASES, range_=(0, cut))
    hi = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=N_BASES, range_=(cut, N_BASES))
    assert lo.n_matches + hi.n_matches == r.n_matches
    assert torch.equal(_keys(torch.cat([lo.pos, hi.pos]), torch.cat([lo.pattern_id, hi.pattern_id])),
                       _keys(r.pos, r.pattern_id))
    assert torch.equal(lo.counts + hi.counts, r.counts)


def test_host_buffers(big):
    ascii_, packed, pats, planted, d, r = big
    host = packed.cpu().pin_memory()
    h = acg.scan(d, host, encoding=N.AC_TEXT_PACKED2, n_bases=N_BASES)
    assert not h.pos.is_cuda
    assert torch.equal(_keys(h.pos, h.pattern_id), _keys(r.pos, r.pattern_id).cpu())
    assert torch.equal(h.counts, r.counts.cpu())


def test_batch_and_stream(big):
    ascii_, packed, pats, planted, d, r = big
    small = acg.pack(ascii_[:100_000])
    b = acg.scan_batch(d, [small, packed], encoding=N.AC_TEXT_PACKED2, n_bases=[100_000, N_BASES])
    one = b.text_id == 1
    assert torch.equal(_keys(b.pos[one], b.pattern_id[one]), _keys(r.pos, r.pattern_id))
    s = acg.Stream(d)
    step = 1_000_000_000  # bases per piece; a multiple of 64, so every piece starts 16-byte aligned
    pos, pid = [], []
    for a in range(0, N_BASES, step):
        n = min(step, N_BASES - a)
        g = s.scan(packed[a // 16 : (a + n + 15) // 16], encoding=N.AC_TEXT_PACKED2, n_bases=n)
        pos.append(g.pos)
        pid.append(g.pattern_id)
    s.close()
    assert torch.equal(_keys(torch.cat(pos), torch.cat(pid)), _keys(r.pos, r.pattern_id))
