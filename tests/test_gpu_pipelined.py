"""GPU tests of the host-buffer scan that overlaps its copies with the scan.

A text of more than 512 Mbase held in pinned host memory, with the results
also in host memory, is scanned in pieces: the copy-in of the next piece and
the copy-out of the previous piece's occurrences run while a piece is
scanned. The Aho-Corasick walk itself (Sec. III.A) is unchanged, so the
occurrence set and the counts must equal:

  * those of the device-resident scan of the same text (itself checked
    against the oracle elsewhere), for ASCII and 2-bit packed host input,
    for a sub-range, without counts and through an overflow retry;
  * the one-shot host path (taken when statistics are asked for);
  * the oracle, on windows straddling the piece boundaries and at the end.
An invalid byte in any piece is reported at its absolute offset.
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

PIECE = 256 << 20  # owned bases per piece of the overlapped host path
FIRST = 8 << 20  # its first piece is short
N_BASES = (640 << 20) + 12_345  # a short piece, two full pieces and a ragged fourth
BOUNDS = [FIRST, FIRST + PIECE, FIRST + 2 * PIECE]  # where pieces meet


@pytest.fixture(scope="module")
def work():
    t = synth.markov_text(N_BASES, synth.BASE_SEED + 21, device="cuda")
    pats = synth.merge_dedupe(
        synth.substring_patterns(t.ascii, 2000, 8, 24, synth.BASE_SEED + 22),
        synth.uniform_patterns(500, 10, 14, synth.BASE_SEED + 23),
    )
    d = acg.build(pats)
    host = t.ascii.cpu().pin_memory()
    want = acg.scan(d, t.ascii)
    yield pats, d, t.ascii, host, want
    del t


def _same(got, want):
    assert got.n_matches == want.n_matches
    assert np.array_equal(got.canonical(), want.canonical())
    if want.counts is not None:
        assert np.array_equal(got.counts.cpu().numpy(), want.counts.cpu().numpy())


def test_host_ascii_equals_device(work):
    pats, d, dev, host, want = work
    assert want.n_matches > 100_000
    got = acg.scan(d, host)
    assert not got.pos.is_cuda
    _same(got, want)


def test_host_packed_equals_device(work):
    pats, d, dev, host, want = work
    packed = acg.pack(dev).cpu().pin_memory()
    _same(acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=N_BASES), want)


def test_host_two_blocks_per_sm_shape(work):
    pats, d, dev, host, want = work
    _same(acg.scan(d, host, stride=3, threads=640), want)


def test_one_shot_host_path_agrees(work):
    pats, d, dev, host, want = work
    _same(acg.scan(d, host, stats=True), want)


def test_overflow_retry(work):
    pats, d, dev, host, want = work
    _same(acg.scan(d, host, capacity=1000), want)


def test_sub_range_without_counts(work):
    pats, d, dev, host, want = work
    rng = (12_345_677, N_BASES - 1_000_003)
    ref = acg.scan(d, dev, range_=rng, counts=False)
    got = acg.scan(d, host, range_=rng, counts=False)
    assert got.counts is None
    _same(got, ref)
    assert 0 < ref.n_matches < want.n_matches


def test_piece_boundaries_against_oracle(work):
    pats, d, dev, host, want = work
    got = acg.scan(d, host)
    lens = np.array([len(p) for p in pats], np.int64)
    lmax = int(lens.max())
    pos, pid = got.pos.numpy(), got.pattern_id.numpy()
    end = pos + lens[pid] - 1
    m = oracle.Machine(pats)
    win = 1 << 20
    starts = [b - win // 2 for b in BOUNDS] + [b - win for b in BOUNDS] + [N_BASES - win, 0]
    starts += random.Random(7).sample(range(0, N_BASES - win), 3)
    for s0 in starts:
        s1 = s0 + win
        rb = max(0, s0 - (lmax - 1))
        p, k, _ = m.scan(host[rb:s1].numpy())
        e = p.astype(np.int64) + lens[k] - 1 + rb
        keep = e >= s0
        w = np.stack([p[keep].astype(np.int64) + rb, k[keep].astype(np.int64)], 1)
        w = w[np.lexsort((w[:, 1], w[:, 0]))]
        sel = (end >= s0) & (end < s1)
        g = np.stack([pos[sel], pid[sel]], 1)
        g = g[np.lexsort((g[:, 1], g[:, 0]))]
        assert np.array_equal(g, w), f"window at {s0}"


@pytest.mark.parametrize("where", [[300_000_000, N_BASES - 5], [N_BASES - 5], [FIRST], [FIRST + PIECE], [5]])
def test_bad_byte_absolute_offset(work, where):
    pats, d, dev, host, want = work
    old = [int(host[i]) for i in where]
    try:
        for i in where:
            host[i] = ord("N")
        with pytest.raises(acg.AcError) as e:
            acg.scan(d, host)
        assert e.value.status == N.AC_ERR_ALPHABET and f"offset {min(where)}" in str(e.value)
    finally:
        for i, v in zip(where, old):
            host[i] = v
