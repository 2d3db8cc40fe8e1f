"""GPU parity of failure-less matching (the PFAC scheme of Sec. II; one thread
per start position over the trie edges only): the same occurrences and counts
as the failure-folded walk and the oracle, with owned ranges and host/device
buffers."""
import random

import numpy as np
import pytest
import torch

import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from tests.gpu_helpers import assert_same, oracle_canonical

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(6))
def test_failureless_equals_oracle(seed):
    rng = random.Random(61 + seed)
    n = rng.choice([1, 63, 5000, 120_000])
    text = bytes(rng.choice(b"ACGT") for _ in range(n)) + b"AAAAAAAAAACACACACA" * (seed + 1)
    pats = [text[j : j + rng.randint(1, 22)] for j in rng.sample(range(len(text) - 1), min(300, len(text) - 1))]
    pats += [bytes(rng.choice(b"ACGT") for _ in range(rng.randint(2, 10))) for _ in range(50)]
    pats += [b"A" * 5, b"A" * 3, pats[0]]  # nested and duplicate keywords
    d = acg.build(pats, failureless=True)
    want, counts = oracle_canonical(pats, text)
    t = torch.tensor(list(text), dtype=torch.uint8, device="cuda")
    assert_same(acg.scan_failureless(d, t, capacity=4), want, counts)
    assert_same(acg.scan_failureless(d, text), want, counts)  # host buffers
    r = acg.scan(d, t)
    assert_same(r, want, counts)


def test_failureless_owned_ranges():
    rng = random.Random(7)
    text = bytes(rng.choice(b"ACGT") for _ in range(50_000))
    pats = [text[j : j + rng.randint(5, 15)] for j in rng.sample(range(49_000), 200)]
    d = acg.build(pats, failureless=True)
    t = acg.pack(torch.tensor(list(text), dtype=torch.uint8, device="cuda"))
    full = acg.scan_failureless(d, t, encoding=N.AC_TEXT_PACKED2, n_bases=len(text)).canonical()
    parts = [acg.scan_failureless(d, t, encoding=N.AC_TEXT_PACKED2, n_bases=len(text), range_=(a, b)).canonical()
             for a, b in ((0, 777), (777, 30_001), (30_001, 50_000))]
    cat = np.concatenate(parts)
    assert np.array_equal(cat[np.lexsort((cat[:, 2], cat[:, 1], cat[:, 0]))], full)


def test_failureless_needs_the_flag():
    d = acg.build([b"ACGT"])
    with pytest.raises(acg.AcError) as e:
        acg.scan_failureless(d, b"ACGTACGT")
    assert e.value.status == N.AC_ERR_INVALID_ARG
