"""GPU parity of the streaming scan (ac_stream_*): a text cut into pieces of
any length (1, 15, 16, 17, 63, 64, L_max-1, ... bases), ASCII or packed, host
or device, gives exactly the occurrences and counts of one scan of the whole
text and of the oracle, with global positions; reset starts a new text."""
import random

import numpy as np
import pytest
import torch

import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from tests.gpu_helpers import oracle_canonical

pytestmark = pytest.mark.gpu


def _text_and_patterns(seed, n):
    rng = random.Random(seed)
    text = bytes(rng.choice(b"ACGT") for _ in range(n)) + b"ACACACACAC" * 50
    pats = [text[j : j + rng.randint(3, 24)] for j in rng.sample(range(len(text) - 30), 300)]
    pats += [bytes(rng.choice(b"ACGT") for _ in range(rng.randint(3, 12))) for _ in range(100)]
    return text, pats, rng


def _pieces(rng, n, lmax):
    cuts, p = [], 0
    sizes = [1, 2, 15, 16, 17, 63, 64, 65, lmax - 1, lmax, lmax + 1, 997, 4096, 10_000]
    while p < n:
        k = min(n - p, rng.choice(sizes))
        cuts.append((p, p + k))
        p += k
    return cuts


@pytest.mark.parametrize("form", ["ascii_dev", "ascii_host", "packed_dev", "packed_host"])
@pytest.mark.parametrize("stride,threads", [(1, 0), (2, 0), (3, 0), (3, 640)])
def test_stream_equals_one_scan(form, stride, threads):
    text, pats, rng = _text_and_patterns(31, 60_000)
    d = acg.build(pats)
    lmax = max(len(p) for p in pats)
    want, counts = oracle_canonical(pats, text)
    s = acg.Stream(d)
    rows, csum = [], np.zeros(len(pats), np.int64)
    for a, b in _pieces(rng, len(text), lmax):
        piece = text[a:b]
        if form == "ascii_dev":
            arg, kw = torch.tensor(list(piece), dtype=torch.uint8, device="cuda"), {}
        elif form == "ascii_host":
            arg, kw = piece, {}
        else:
            packed = acg.pack(torch.tensor(list(piece), dtype=torch.uint8, device="cuda"))
            arg = packed if form == "packed_dev" else packed.cpu().numpy()
            kw = {"encoding": N.AC_TEXT_PACKED2, "n_bases": b - a}
        r = s.scan(arg, capacity=2, stride=stride, threads=threads, **kw)  # tiny capacity: the stream retries the piece
        rows.append(r.canonical())
        csum += r.counts.cpu().numpy()
    got = np.concatenate(rows)
    got = got[np.lexsort((got[:, 2], got[:, 1], got[:, 0]))]
    assert np.array_equal(got, want)
    assert csum.tolist() == counts.tolist()
    s.close()


def test_stream_reset_and_alphabet_error_keep_state():
    text, pats, rng = _text_and_patterns(32, 5_000)
    d = acg.build(pats)
    s = acg.Stream(d)
    first = s.scan(text[:2500]).canonical()
    with pytest.raises(acg.AcError) as e:
        s.scan(b"ACGTN")  # rejected: the stream does not advance
    assert e.value.status == N.AC_ERR_ALPHABET
    second = s.scan(text[2500:]).canonical()
    got = np.concatenate([first, second])
    got = got[np.lexsort((got[:, 2], got[:, 1], got[:, 0]))]
    want, _ = oracle_canonical(pats, text)
    assert np.array_equal(got, want)
    s.reset()  # a new text starts at position 0
    again = s.scan(text).canonical()
    assert np.array_equal(again, want)
    s.close()


@pytest.mark.parametrize("lmax", list(range(2, 35)))
def test_stream_every_carry_offset(lmax):
    """The carried L_max-1 bases put the next piece at every offset within a
    packed word (the splice's word-shift path and its edge words)."""
    rng = random.Random(700 + lmax)
    text = bytes(rng.choice(b"ACGT") for _ in range(3_000)) + b"ACGTACGTAC" * 20
    pats = [text[j : j + rng.randint(1, lmax)] for j in rng.sample(range(len(text) - 40), 60)]
    pats.append(text[100 : 100 + lmax])
    d = acg.build(pats)
    want, counts = oracle_canonical(pats, text)
    s = acg.Stream(d)
    rows, csum = [], np.zeros(len(pats), np.int64)
    for a, b in _pieces(rng, len(text), lmax):
        packed = acg.pack(torch.tensor(list(text[a:b]), dtype=torch.uint8, device="cuda"))
        r = s.scan(packed, encoding=N.AC_TEXT_PACKED2, n_bases=b - a)
        rows.append(r.canonical())
        csum += r.counts.cpu().numpy()
    got = np.concatenate(rows)
    got = got[np.lexsort((got[:, 2], got[:, 1], got[:, 0]))]
    assert np.array_equal(got, want)
    assert csum.tolist() == counts.tolist()
    s.close()
