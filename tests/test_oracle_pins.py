"""Pins of the CPU oracle against what the paper and the definitions fix.

Every check here is independent of the oracle's own code: the paper's worked
example (Sec. III.A, Fig. 1/2, stored under tests/golden/), brute force written
with Python's str.find, the definitions of the failure and output functions
evaluated on strings, closed forms, and invariants (the paper's two thread
decompositions of Sec. IV.A must give the single machine's result).
A mutation test at the end compiles the oracle with known mistakes planted and
shows that this battery catches each of them.
"""
import os
import random
import tempfile

import numpy as np
import pytest

import oracle
from tests.conftest import load_golden

# ----------------------------------------------------------------- helpers


def brute(patterns, text):
    """Every (start, pid) with text[start:start+len] == pattern, by str.find."""
    out = set()
    for pid, p in enumerate(patterns):
        j = text.find(p)
        while j != -1:
            out.add((j, pid))
            j = text.find(p, j + 1)
    return out


def as_set(pos, pid):
    return set(zip(pos.tolist(), pid.tolist()))


def state_strings(m):
    """string(s) for every state, recovered by walking goto from the root."""
    strings = {0: ""}
    stack = [0]
    while stack:
        s = stack.pop()
        for c in range(256):
            t = m.goto(s, c)
            if t >= 0:
                strings[t] = strings[s] + chr(c)
                stack.append(t)
    return strings


# ----------------------------------------------------- P1: worked example


@pytest.mark.parametrize("fixture", ["worked_example.txt", "worked_example_dna.txt"])
def test_worked_example(fixture):
    g = load_golden(fixture)
    kws = g["keywords"][0]
    text = g["text"][0][0]
    m = oracle.Machine(kws)
    assert m.n_states == 10  # root + 9 states of Fig. 1
    for s, c, t in g["goto"]:
        assert m.goto(int(s), c) == int(t), (s, c, t)
    for s, f in g["fail"]:
        assert m.fail(int(s)) == int(f)
    for s, kw in g["final"]:
        assert m.output(int(s)) == [kws.index(kw)]
    assert m.trace(text) == [int(v) for v in g["trajectory"][0]]
    pos, pid, counts = m.scan(text)
    want = {(int(p), kws.index(kw)) for p, kw in g["match"]}
    assert as_set(pos, pid) == want
    assert counts.tolist() == [sum(1 for _, q in want if q == i) for i in range(len(kws))]


def test_worked_example_caller_order():
    # Fig. 1's caption lists HIS, SHE, HERS; ids follow the caller's order.
    m = oracle.Machine(["HIS", "SHE", "HERS"])
    pos, pid, counts = m.scan("SHERS")
    assert as_set(pos, pid) == {(0, 1), (1, 2)}
    assert counts.tolist() == [0, 1, 1]


# ------------------------------------- definitions of fail() and output()


def random_dna_patterns(rng, k, lo, hi):
    return ["".join(rng.choice("ACGT") for _ in range(rng.randint(lo, hi))) for _ in range(k)]


@pytest.mark.parametrize("seed", range(20))
def test_fail_and_output_definitions(seed):
    rng = random.Random(1000 + seed)
    pats = random_dna_patterns(rng, rng.randint(1, 30), 1, 7)
    if seed % 3 == 0:
        pats += [pats[0], pats[0][:1]]  # duplicate and prefix
    m = oracle.Machine(pats)
    strings = state_strings(m)
    assert len(strings) == m.n_states
    by_string = {v: k for k, v in strings.items()}
    prefixes = {p[:i] for p in pats for i in range(len(p) + 1)}
    assert set(by_string) == prefixes
    for s, w in strings.items():
        assert m.depth(s) == len(w)
        if s == 0:
            continue
        # fail(s): the state of the longest proper suffix of string(s) in the trie
        best = max((w[i:] for i in range(1, len(w) + 1) if w[i:] in prefixes), key=len)
        assert m.fail(s) == by_string[best], (w, best)
        # output(s): every keyword that is a suffix of string(s)
        want = sorted(pid for pid, p in enumerate(pats) if w.endswith(p))
        assert sorted(m.output(s)) == want, (w,)


# ------------------------------------------------------- P2: brute force


def fuzz_case(rng):
    n = rng.choice([0, 1, 2, 5, 17, 64, 200, 700, 2000])
    alpha = rng.choice(["ACGT", "AC", "A", "ACGTN", "HISER"])
    if rng.random() < 0.3:  # periodic text
        unit = "".join(rng.choice(alpha) for _ in range(rng.randint(1, 4)))
        text = (unit * (n // max(len(unit), 1) + 1))[:n]
    else:
        text = "".join(rng.choice(alpha) for _ in range(n))
    k = rng.randint(1, 50)
    pats = []
    for _ in range(k):
        r = rng.random()
        if r < 0.35 and n > 0:
            L = rng.randint(1, 8)
            j = rng.randint(0, max(0, n - 1))
            p = text[j : j + L]
            pats.append(p if p else "A")
        elif r < 0.45 and pats:
            q = rng.choice(pats)
            pats.append(q[: rng.randint(1, len(q))] if rng.random() < 0.5 else q[-rng.randint(1, len(q)) :])
        elif r < 0.5 and pats:
            pats.append(rng.choice(pats))  # duplicate
        elif r < 0.55:
            pats.append("".join(rng.choice(alpha) for _ in range(n + rng.randint(1, 3))))  # longer than text
        else:
            pats.append("".join(rng.choice(alpha) for _ in range(rng.randint(1, 8))))
    return pats, text


def test_oracle_vs_bruteforce_fuzz():
    rng = random.Random(14037294)
    total = 0
    for _ in range(1500):
        pats, text = fuzz_case(rng)
        m = oracle.Machine(pats)
        pos, pid, counts = m.scan(text)
        want = brute(pats, text)
        got = as_set(pos, pid)
        assert len(got) == len(pos), "duplicate occurrence reported"
        assert got == want, (pats, text)
        hist = np.bincount(pid.astype(np.int64), minlength=len(pats))
        assert counts.tolist() == hist.tolist()
        total += len(pos)
    assert total > 10000  # the fuzz actually exercises matches


def test_naive_vs_bruteforce():
    rng = random.Random(7)
    for _ in range(200):
        pats, text = fuzz_case(rng)
        pos, pid = oracle.naive(pats, text)
        assert as_set(pos, pid) == brute(pats, text)


def test_scan_order_is_end_position_order():
    rng = random.Random(3)
    pats, text = random_dna_patterns(rng, 20, 1, 5), "".join(rng.choice("ACGT") for _ in range(500))
    m = oracle.Machine(pats)
    lens = np.array([len(p) for p in pats], dtype=np.uint64)
    pos, pid, _ = m.scan(text)
    end = pos + lens[pid] - 1
    assert np.all(np.diff(end.astype(np.int64)) >= 0)


# ------------------------------------------------------ P4: closed forms


@pytest.mark.parametrize("n,k", [(1, 1), (10, 3), (100, 20), (57, 57), (5, 9)])
def test_closed_form_homopolymer(n, k):
    m = oracle.Machine(["A" * k])
    pos, pid, counts = m.scan("A" * n)
    assert pos.tolist() == list(range(max(0, n - k + 1)))
    assert counts[0] == max(0, n - k + 1)


@pytest.mark.parametrize("m_,j", [(1, 1), (50, 3), (50, 50), (8, 9)])
def test_closed_form_dinucleotide(m_, j):
    m = oracle.Machine(["AC" * j, "CA" * j])
    pos, pid, counts = m.scan("AC" * m_)
    assert counts[0] == max(0, m_ - j + 1)
    assert counts[1] == max(0, m_ - j)  # CA^j needs one more base at the front
    assert sorted(pos[pid == 0].tolist()) == [2 * i for i in range(max(0, m_ - j + 1))]


def test_single_pattern_is_repeated_find():
    rng = random.Random(11)
    text = "".join(rng.choice("ACGT") for _ in range(20000))
    for _ in range(20):
        p = "".join(rng.choice("ACGT") for _ in range(rng.randint(1, 6)))
        want, j = [], text.find(p)
        while j != -1:
            want.append(j)
            j = text.find(p, j + 1)
        pos, _, _ = oracle.Machine([p]).scan(text)
        assert pos.tolist() == want


def test_planted_occurrences():
    rng = random.Random(5)
    text = list("".join(rng.choice("ACGT") for _ in range(10000)))
    pat = "GATTACAGATTACA"
    spots = sorted(rng.sample(range(0, 10000 - len(pat)), 30))
    spots = [s for i, s in enumerate(spots) if i == 0 or s - spots[i - 1] >= len(pat)]
    for s in spots:
        text[s : s + len(pat)] = pat
    pos, _, _ = oracle.Machine([pat]).scan("".join(text))
    assert set(spots) <= set(pos.tolist())


def test_empty_and_short_text():
    m = oracle.Machine(["ACGT", "A"])
    pos, pid, counts = m.scan("")
    assert len(pos) == 0 and counts.tolist() == [0, 0]
    pos, pid, counts = m.scan("ACG")
    assert as_set(pos, pid) == {(0, 1)}


def test_rejects_empty_keyword():
    with pytest.raises(ValueError):
        oracle.Machine(["ACG", ""])
    with pytest.raises(ValueError):
        oracle.Machine([])


# ------------------------------------------------------- P3: invariants


def test_pattern_partition_union_equals_one_machine():
    """The paper's thread approach 2 (Sec. IV.A, Fig. 3): one machine per
    chunk of the pattern file, each over the whole input; the union (ids
    offset by the chunk start) equals the single machine's result."""
    rng = random.Random(21)
    text = "".join(rng.choice("ACGT") for _ in range(30000))
    pats = random_dna_patterns(rng, 300, 3, 9) + [text[i : i + 7] for i in range(0, 3000, 100)]
    pos, pid, counts = oracle.Machine(pats).scan(text)
    one = as_set(pos, pid)
    for k in (2, 3, 7):
        cut = sorted(rng.sample(range(1, len(pats)), k - 1))
        bounds = [0] + cut + [len(pats)]
        union, csum = set(), np.zeros(len(pats), dtype=np.uint64)
        for a, b in zip(bounds[:-1], bounds[1:]):
            p2, q2, c2 = oracle.Machine(pats[a:b]).scan(text)
            union |= {(x, y + a) for x, y in zip(p2.tolist(), q2.tolist())}
            csum[a:b] += c2
        assert union == one
        assert csum.tolist() == counts.tolist()


def test_text_chunks_with_halo_equal_one_pass():
    """Thread approach 1 (Sec. IV.A): chunks of the text; a chunk that owns
    end positions [a, b) scans from max(0, a - (Lmax - 1)) and keeps only
    occurrences ending in [a, b). Every occurrence is kept exactly once."""
    rng = random.Random(22)
    text = "".join(rng.choice("ACGT") for _ in range(5000))
    pats = random_dna_patterns(rng, 60, 1, 9) + ["ACGTACGTA"]
    lens = np.array([len(p) for p in pats], dtype=np.uint64)
    lmax = int(lens.max())
    m = oracle.Machine(pats)
    pos, pid, _ = m.scan(text)
    full = sorted(zip(pos.tolist(), pid.tolist()))
    for C in (1, 2, lmax - 1, lmax, 97, 4096, len(text)):
        got = []
        for a in range(0, len(text), C):
            b = min(a + C, len(text))
            s0 = max(0, a - (lmax - 1))
            p2, q2, _ = m.scan(text[s0:b])
            end = p2 + lens[q2] - 1 + s0
            keep = end >= a
            got += list(zip((p2[keep] + s0).tolist(), q2[keep].tolist()))
        assert sorted(got) == full, C


def test_threaded_forms_equal_bruteforce():
    """The oracle's two threaded forms of Sec. IV.A (approach 1: text ranges
    with an L_max-1 halo, ownership by end; approach 2: the keyword list split
    into pieces, one machine each) against brute force, with more threads
    than bases, than keywords, and ranges shorter than L_max."""
    rng = random.Random(24)
    for case in range(120):
        pats, text = fuzz_case(rng)
        want = brute(pats, text)
        hist = np.zeros(len(pats), np.int64)
        for _, q in want:
            hist[q] += 1
        m = oracle.Machine(pats)
        lmax = max(len(p) for p in pats)
        for T in (1, 2, 5, 33):
            p1, q1, c1 = oracle.scan_text_chunks(m, text, T, lmax)
            assert len(p1) == len(want) and as_set(p1, q1) == want, (case, T)
            assert c1.tolist() == hist.tolist()
            p2, q2, c2 = oracle.scan_pattern_split(oracle.pattern_split(pats, T), text, T)
            assert len(p2) == len(want) and as_set(p2, q2) == want, (case, T)
            assert c2.tolist() == hist.tolist()


def test_pattern_split_pieces():
    pats = [f"A{i}" for i in range(10)]
    for k in (1, 3, 10, 25):
        split = oracle.pattern_split(pats, k)
        assert len(split) == min(k, 10)
        assert [p for _, piece in split for p in piece] == pats
        assert all(off == sum(len(x) for _, x in split[:i]) for i, (off, _) in enumerate(split))
        sizes = [len(x) for _, x in split]
        assert max(sizes) - min(sizes) <= 1


def test_counts_sum_to_occurrences():
    rng = random.Random(23)
    text = "".join(rng.choice("AC") for _ in range(20000))  # repeat-rich
    pats = random_dna_patterns(rng, 100, 1, 6)
    pats = [p.replace("G", "A").replace("T", "C") for p in pats]
    pos, pid, counts = oracle.Machine(pats).scan(text)
    assert int(counts.sum()) == len(pos)


# --------------------------------------------- the pins catch each mistake


def _battery(lib):
    """Run a compact version of the pins above against one oracle build.
    Returns the name of the first failing pin, or None."""
    g = load_golden("worked_example.txt")
    kws, text = g["keywords"][0], g["text"][0][0]
    m = oracle.Machine(kws, lib=lib)
    if m.fail(9) != 4:
        return "worked example fail(9)"
    if m.trace(text) != [int(v) for v in g["trajectory"][0]]:
        return "worked example trajectory"
    pos, pid, counts = m.scan(text)
    if as_set(pos, pid) != {(0, 2), (1, 1)}:
        return "worked example matches"
    rng = random.Random(99)
    for _ in range(300):
        pats, text = fuzz_case(rng)
        m = oracle.Machine(pats, lib=lib)
        pos, pid, counts = m.scan(text)
        if as_set(pos, pid) != brute(pats, text):
            return "brute force"
        if counts.tolist() != np.bincount(pid.astype(np.int64), minlength=len(pats)).tolist():
            return "counts"
    return None


MUTANTS = {
    1: "output(s) without output(fail(s))",
    2: "start position off by one",
    3: "character not re-read after a failure hop",
    4: "single failure hop when building fail()",
    5: "root edges ignored when the failure chain reaches the root",
    6: "inherited keywords not counted",
}


def test_battery_passes_on_the_real_oracle():
    assert _battery(oracle.load()) is None


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant):
    with tempfile.TemporaryDirectory() as d:
        path = oracle.compile_oracle(os.path.join(d, f"liboracle_m{mutant}.so"), mutant=mutant)
        lib = oracle.load(path)
        assert _battery(lib) is not None, f"pins missed mutant {mutant}: {MUTANTS[mutant]}"
