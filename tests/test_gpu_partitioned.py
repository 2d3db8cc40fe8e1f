"""GPU parity of the pattern-file split (the paper's approach 2, Sec. IV.A,
Fig. 3): machines over consecutive keyword chunks, each in shared memory,
scanning the whole text in one launch, give exactly the single machine's
occurrences and counts (ids in the caller's numbering) and the oracle's."""
import random

import numpy as np
import pytest
import torch

import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from tests.gpu_helpers import assert_same, oracle_canonical

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("max_states", [0, 40, 300, 5000])
def test_partitioned_equals_single_machine_and_oracle(max_states):
    rng = random.Random(41 + max_states)
    text = bytes(rng.choice(b"ACGT") for _ in range(200_000)) + b"ACACACACGTGT" * 40
    pats = [text[j : j + rng.randint(4, 20)] for j in rng.sample(range(len(text) - 30), 600)]
    pats += [bytes(rng.choice(b"ACGT") for _ in range(rng.randint(4, 14))) for _ in range(200)]
    pats += [pats[3], b"ACACAC"]  # a duplicate and a periodic keyword
    ps = acg.build_partitioned(pats, max_states=max_states)
    assert ps.n_parts >= 1 and (max_states == 0 or ps.max_states <= max_states)
    if max_states == 40:
        assert ps.n_parts > 50
    want, counts = oracle_canonical(pats, text)
    t = torch.tensor(list(text), dtype=torch.uint8, device="cuda")
    for arg, kw in ((t, {}), (acg.pack(t), {"encoding": N.AC_TEXT_PACKED2, "n_bases": len(text)}), (text, {})):
        r = ps.scan(arg, capacity=8, **kw)
        assert_same(r, want, counts)
    ps.close()


def test_partitioned_rejects_keyword_longer_than_a_machine():
    with pytest.raises(acg.AcError) as e:
        acg.build_partitioned([b"ACGTACGTACGT"], max_states=5)
    assert e.value.status == N.AC_ERR_TOO_LARGE
