"""GPU parity of the single-text scan (ac_scan, ac_pack) against the oracle.

Bit-exact comparison after the canonical sort (the occurrence set is unique,
only its order is free), plus exact per-keyword counts. Covers the worked
example, seeded fuzz over every launch shape the kernels offer (chunk sizes
1, 2, L_max-1, L_max, 97, 4096, n; shared-memory states 0, 1, all; interleave
1, 2, 4, 8), owned ranges, host and device buffers, overflow, alphabet
errors and the 1 Mbase uniform workload in full."""
import random
import re

import numpy as np
import pytest
import torch

import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from paper_1403_7294_gb300 import synth
from tests.conftest import load_golden
from tests.gpu_helpers import assert_same, oracle_canonical, unpack_codes

pytestmark = pytest.mark.gpu

DEV = "cuda"


def rand_dna(rng, n):
    return bytes(rng.choice(b"ACGT") for _ in range(n))


def to_dev(b: bytes) -> torch.Tensor:
    return torch.tensor(list(b), dtype=torch.uint8, device=DEV) if b else torch.empty(0, dtype=torch.uint8, device=DEV)


def test_pack_round_trip_and_alphabet():
    """Packing is the definition (A, C, G, T -> 0, 1, 2, 3, base j at bits 2j) for 16-byte
    aligned texts (64 bases at a time, then word by word) and texts at every misalignment;
    case folding; and the reported offset is the first byte that is not a base."""
    rng = random.Random(1)
    base = to_dev(rand_dna(rng, 300_000))
    for n in (1, 15, 16, 17, 63, 64, 65, 127, 128, 129, 1000, 4097, 100_003):
        for shift in (0, 1, 4, 15):  # data_ptr offset: 0 keeps the 16-byte alignment
            t = base[shift : shift + n]
            packed = acg.pack(t)
            codes = unpack_codes(packed, n).cpu().numpy()
            assert codes.tolist() == [b"ACGT".index(c) for c in bytes(t.cpu().numpy())], (n, shift)
    low = to_dev(b"acgtACGT")
    assert unpack_codes(acg.pack(low, fold_case=True), 8).tolist() == [0, 1, 2, 3, 0, 1, 2, 3]
    mixed = bytes(rng.choice(b"ACGTacgt") for _ in range(1000))
    assert unpack_codes(acg.pack(to_dev(mixed), fold_case=True), 1000).tolist() == [
        b"ACGT".index(bytes([c]).upper()) for c in mixed]
    with pytest.raises(acg.AcError) as e:
        acg.pack(to_dev(b"ACGTNACGT"))
    assert e.value.status == N.AC_ERR_ALPHABET and "offset 4" in str(e.value)
    for n, where, fold in ((1000, [5, 700], False), (1000, [64, 63 + 64], False), (4096, [4095], False),
                           (100_003, [99_999, 100_002], False), (1000, [333], True), (200, [0, 199], False)):
        t = bytearray(rand_dna(rng, n))
        if fold:
            t = bytearray(bytes(t).lower())
        for k, i in enumerate(where):
            t[i] = (b"Nn" if fold else b"NaU")[k % (2 if fold else 3)]
        for shift in (0, 3):
            dev = to_dev(b"A" * shift + bytes(t))[shift:]
            with pytest.raises(acg.AcError) as e:
                acg.pack(dev, fold_case=fold)
            assert e.value.status == N.AC_ERR_ALPHABET and f"offset {min(where)}" in str(e.value), (n, where, shift)


def test_worked_example_dna():
    g = load_golden("worked_example_dna.txt")
    kws = [w.encode() for w in g["keywords"][0]]
    text = g["text"][0][0].encode()
    d = acg.build(kws)
    want = sorted((int(p), [w.decode() for w in kws].index(k)) for p, k in g["match"])
    for t in (to_dev(text), text):  # device and host ASCII
        r = acg.scan(d, t)
        assert sorted(zip(r.pos.tolist(), r.pattern_id.tolist())) == want


def _cases(seed, k):
    rng = random.Random(seed)
    for _ in range(k):
        n = rng.choice([0, 1, 31, 64, 65, 200, 1000, 5000, 20000])
        if rng.random() < 0.25:
            unit = rand_dna(rng, rng.randint(1, 4))
            text = (unit * (n // len(unit) + 1))[:n]
        else:
            text = rand_dna(rng, n)
        pats = [rand_dna(rng, rng.randint(1, 12)) for _ in range(rng.randint(1, 40))]
        if n > 20:
            for _ in range(rng.randint(0, 10)):
                j = rng.randint(0, n - 1)
                p = text[j : j + rng.randint(1, 15)]
                if p:
                    pats.append(p)
        if rng.random() < 0.3:
            pats.append(pats[0])  # duplicate keyword
        yield pats, text


SHAPES = ["default", "c1", "c2", "cLm1", "cL", "c97", "c4096", "cn", "hot0", "hot1", "i1", "i2", "i8",
          "s2", "s2i2", "s2i4", "s2hot0", "s2c1", "s2c97", "s1", "s2rows3", "s2rows40i2",
          "s3", "s3i2", "s3hot0", "s3hot1", "s3c1", "s3c97", "s3rows3", "s3rows40i2",
          "s3t640", "s3t256", "s3t640hot1", "s3rows3t640"]  # tN: N-thread blocks (two or more per SM)


@pytest.mark.parametrize("shape", SHAPES)
def test_fuzz_vs_oracle(shape):
    for pats, text in _cases(77, 25):
        lmax = max(len(p) for p in pats)
        kw, build_kw = {}, {}
        if shape.startswith("c"):
            kw["chunk"] = {"c1": 1, "c2": 2, "cLm1": max(1, lmax - 1), "cL": lmax, "c97": 97, "c4096": 4096,
                           "cn": max(1, len(text))}[shape]
        elif shape == "hot0":
            kw["hot_states"] = 0
        elif shape == "hot1":
            kw["hot_states"] = 1
        elif shape.startswith("i"):
            kw["interleave"] = int(shape[1:])
        elif shape.startswith("s"):  # two or three bases per lookup (s1: one, forced)
            m = re.fullmatch(r"s(\d)(?:rows(\d+))?(?:t(\d+))?(?:i(\d+))?(?:hot(\d+))?(?:c(\d+))?", shape)
            stride, rows, threads, il, hot, chunk = m.groups()
            kw["stride"] = int(stride)
            if rows:  # multi-base rows only for the shallowest states
                if kw["stride"] == 3:  # R three-base rows, 2R two-base rows, one-base lookups beyond
                    build_kw["stride3_states"] = int(rows)
                    build_kw["stride2_states"] = 2 * int(rows)
                else:
                    build_kw["stride2_states"] = int(rows)
            for key, v in (("threads", threads), ("interleave", il), ("hot_states", hot), ("chunk", chunk)):
                if v:
                    kw[key] = int(v)
        d = acg.build(pats, **build_kw)
        want, counts = oracle_canonical(pats, text)
        r = acg.scan(d, to_dev(text), capacity=4, **kw)  # tiny capacity: exercises the overflow retry
        assert_same(r, want, counts)


@pytest.mark.parametrize("stride", [1, 2, 3])
def test_owned_ranges_concatenate_to_the_whole(stride):
    rng = random.Random(5)
    text = rand_dna(rng, 30000)
    pats = [text[j : j + rng.randint(3, 10)] for j in rng.sample(range(29000), 50)] + [b"ACGTACGT"]
    d = acg.build(pats)
    t = acg.pack(to_dev(text))
    full = acg.scan(d, t, encoding=N.AC_TEXT_PACKED2, n_bases=len(text)).canonical()
    parts, counts = [], np.zeros(len(pats), np.int64)
    cuts = [0, 1, 17, 4096, 10000, 29999, 30000]
    for a, b in zip(cuts[:-1], cuts[1:]):
        r = acg.scan(d, t, encoding=N.AC_TEXT_PACKED2, n_bases=len(text), range_=(a, b), stride=stride)
        c = r.canonical()
        ends = c[:, 1] + np.array([len(pats[p]) for p in c[:, 2]]) - 1
        assert np.all((ends >= a) & (ends < b))
        parts.append(c)
        counts += r.counts.cpu().numpy()
    cat = np.concatenate(parts)
    cat = cat[np.lexsort((cat[:, 2], cat[:, 1], cat[:, 0]))]
    assert np.array_equal(cat, full)
    assert counts.tolist() == np.bincount(full[:, 2], minlength=len(pats)).tolist()


def test_host_and_device_buffers_agree():
    rng = random.Random(6)
    text = rand_dna(rng, 100000)
    pats = [text[j : j + 12] for j in range(0, 100000, 997)]
    d = acg.build(pats)
    want, counts = oracle_canonical(pats, text)
    assert_same(acg.scan(d, to_dev(text)), want, counts)  # device ASCII
    assert_same(acg.scan(d, text), want, counts)  # host ASCII, host results
    packed_dev = acg.pack(to_dev(text))
    assert_same(acg.scan(d, packed_dev, encoding=N.AC_TEXT_PACKED2, n_bases=len(text)), want, counts)
    packed_host = packed_dev.cpu().numpy()
    assert_same(acg.scan(d, packed_host, encoding=N.AC_TEXT_PACKED2, n_bases=len(text)), want, counts)


def test_edge_cases():
    d = acg.build([b"ACGTACGT", b"A"])
    r = acg.scan(d, torch.empty(0, dtype=torch.uint8, device=DEV))
    assert r.n_matches == 0 and r.counts.sum().item() == 0
    r = acg.scan(d, to_dev(b"ACGTACG"))  # shorter than the long keyword
    assert sorted(r.pos.tolist()) == [0, 4] and r.counts.tolist() == [0, 2]
    with pytest.raises(acg.AcError) as e:
        acg.scan(d, to_dev(b"ACGTTTN"))
    assert e.value.status == N.AC_ERR_ALPHABET and "offset 6" in str(e.value)
    r = acg.scan(d, to_dev(b"acgtacgt"), fold_case=True)
    assert r.counts.tolist() == [1, 2]


def test_overflow_reports_exact_count():
    import ctypes

    d = acg.build([b"A"])
    t = to_dev(b"A" * 5000)
    raw = torch.empty((10, 2), dtype=torch.int64, device=DEV)
    cnt = torch.empty(1, dtype=torch.int64, device=DEV)
    desc = N.Text(t.data_ptr(), 5000, N.AC_TEXT_ASCII, 1)
    r = N.Result(raw.data_ptr(), 10, 0, cnt.data_ptr(), 1, 0, 0)
    st = acg.lib().ac_scan(d.h, ctypes.byref(desc), ctypes.byref(r), None, None, None)
    assert st == N.AC_ERR_OVERFLOW and r.n_matches == 5000 and cnt.item() == 5000
    got = sorted(raw[:, 0].tolist())
    assert len(set(got)) == 10 and all(0 <= g < 5000 for g in got)


def test_invalid_arguments():
    import ctypes

    d = acg.build([b"ACG"])
    t = to_dev(b"ACGT" * 100)
    packed = acg.pack(t)
    mis = N.Text(packed.data_ptr() + 4, 16, N.AC_TEXT_PACKED2, 1)  # not 16-byte aligned
    r = N.Result()
    assert acg.lib().ac_scan(d.h, ctypes.byref(mis), ctypes.byref(r), None, None, None) == N.AC_ERR_INVALID_ARG
    o = N.ScanOpts()
    o.range_begin, o.range_end, o.hot_states = 10, 5, -1
    ok = N.Text(t.data_ptr(), 400, N.AC_TEXT_ASCII, 1)
    assert acg.lib().ac_scan(d.h, ctypes.byref(ok), ctypes.byref(r), ctypes.byref(o), None, None) == N.AC_ERR_INVALID_ARG
    o.range_begin, o.range_end, o.interleave = 0, 0, 3
    assert acg.lib().ac_scan(d.h, ctypes.byref(ok), ctypes.byref(r), ctypes.byref(o), None, None) == N.AC_ERR_INVALID_ARG


def test_plain_1mbase_uniform_full():
    """The 1 Mbase i.i.d. workload with 100 keywords of length 8-20, ASCII on the device."""
    w = synth.plain_small(device="cpu")
    d = acg.build(w.patterns)
    want, counts = oracle_canonical(w.patterns, w.text.ascii)
    r = acg.scan(d, w.text.ascii.to(DEV), stats=True)
    assert_same(r, want, counts)
    assert r.stats["scan_ms"] > 0


def test_tuned_shape_serves_nearby_text_sizes():
    """A shape tuned for one text size is used for a text of another size
    (same machine size, nearest tuned text size), and stays exact."""
    rng = random.Random(10)
    text = rand_dna(rng, 3 << 20)
    pats = [text[j : j + rng.randint(9, 15)] for j in rng.sample(range((3 << 20) - 20), 3000)]
    d = acg.build(pats)
    packed = acg.pack(to_dev(text))
    best = acg.autotune(d, packed, len(text))
    part = text[: 600_000]
    want, counts = oracle_canonical(pats, part)
    r = acg.scan(d, to_dev(part), stats=True)
    assert_same(r, want, counts)
    assert (r.stats["stride"], r.stats["threads"], r.stats["interleave"]) == (
        best["stride"], best["threads"], best["interleave"])


def test_autotune_then_exact():
    rng = random.Random(9)
    text = rand_dna(rng, 1 << 20)
    pats = [text[j : j + 16] for j in rng.sample(range((1 << 20) - 20), 500)]
    d = acg.build(pats)
    packed = acg.pack(to_dev(text))
    best = acg.autotune(d, packed, len(text))
    assert best["interleave"] in (1, 2, 4, 8) and best["threads"] in (256, 512, 640, 768, 1024)
    assert best["stride"] in (1, 2, 3)
    want, counts = oracle_canonical(pats, text)
    r = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=len(text), threads=best["threads"],
                 interleave=best["interleave"], hot_states=best["hot_states"])
    assert_same(r, want, counts)


@pytest.mark.parametrize("stride,threads", [(1, 0), (2, 0), (3, 0), (3, 640)])
def test_every_tuner_chunk_candidate_is_exact(stride, threads):
    """The tuner's chunk axis: 1, 2, 4 and 8 chunks per resident lane (shorter chunks, more halo
    re-reads) give the oracle's occurrences and counts on the fuzz set."""
    for pats, text in _cases(78, 12):
        d = acg.build(pats)
        want, counts = oracle_canonical(pats, text)
        for cpl in (1, 2, 4, 8):
            r = acg.scan(d, to_dev(text), capacity=4, stride=stride, threads=threads, chunks_per_lane=cpl,
                         stats=True)
            assert_same(r, want, counts)
            assert r.stats["chunks_per_lane"] == cpl


def test_autotune_picks_a_chunk_and_stays_exact():
    rng = random.Random(19)
    text = rand_dna(rng, 4 << 20) + b"ACGT" * 5000
    pats = [text[j : j + rng.randint(12, 24)] for j in rng.sample(range((4 << 20) - 30), 4000)]
    d = acg.build(pats)
    packed = acg.pack(to_dev(text))
    best = acg.autotune(d, packed, len(text))
    assert best["chunks_per_lane"] in (1, 2, 4, 8) and best["chunk"] > 0
    want, counts = oracle_canonical(pats, text)
    r = acg.scan(d, packed, encoding=N.AC_TEXT_PACKED2, n_bases=len(text), stats=True)  # the tuned shape
    assert_same(r, want, counts)
    assert (r.stats["chunks_per_lane"], r.stats["chunk"]) == (best["chunks_per_lane"], best["chunk"])


def test_misaligned_device_results_are_refused():
    """Occurrences are written as whole 16-byte records, so a device result buffer that is not
    16-byte aligned is refused before anything runs (no write is attempted)."""
    import ctypes

    d = acg.build([b"ACGT"])
    text = acg.pack(to_dev(b"ACGT" * 100))
    raw = torch.zeros(256, dtype=torch.int64, device=DEV)
    desc = N.Text(text.data_ptr(), 400, N.AC_TEXT_PACKED2, 1)
    for off in (8, 4):
        r = N.Result(raw.data_ptr() + off, 64, 0, None, 1, 0, 0)
        L = acg.lib()
        assert L.ac_scan(d.h, ctypes.byref(desc), ctypes.byref(r), None, None, None) == N.AC_ERR_INVALID_ARG
        assert L.ac_scan_noalloc(d.h, ctypes.byref(desc), ctypes.byref(r), None, None) == N.AC_ERR_INVALID_ARG
        descs = (N.Text * 1)(desc)
        assert L.ac_scan_batch(d.h, descs, 1, ctypes.byref(r), None, None, None) == N.AC_ERR_INVALID_ARG
    r = N.Result(raw.data_ptr(), 128, 0, None, 1, 0, 0)  # aligned: fine
    assert acg.lib().ac_scan(d.h, ctypes.byref(desc), ctypes.byref(r), None, None, None) == N.AC_OK
    assert r.n_matches == 100
