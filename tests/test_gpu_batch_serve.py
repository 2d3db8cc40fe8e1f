"""GPU parity of the batched scan (ac_scan_batch, batch plans) and of serving.

Batch = the concatenation of per-text scans = the oracle on every text.
Serving: every request's result is the same alone and in a concurrent mix,
and equals the oracle (tolerance 0: all results are exact integers)."""
import random
import threading
import time

import numpy as np
import pytest
import torch

import paper_1403_7294_gb300 as acg
from paper_1403_7294_gb300 import _native as N
from tests.gpu_helpers import oracle_canonical

pytestmark = pytest.mark.gpu
DEV = "cuda"


def rand_dna(rng, n):
    return bytes(rng.choice(b"ACGT") for _ in range(n))


def batch_case(seed, n_texts=150):
    rng = random.Random(seed)
    lens = [rng.choice([0, 1, 5, 63, 64, 65, 300, 2000, 9000]) for _ in range(n_texts)]
    texts = [rand_dna(rng, n) for n in lens]
    src = b"".join(texts)
    pats = [rand_dna(rng, rng.randint(4, 14)) for _ in range(200)]
    pats += [src[j : j + rng.randint(4, 14)] for j in rng.sample(range(max(1, len(src) - 20)), 200)]
    return texts, pats


def oracle_batch(pats, texts):
    rows, counts = [], np.zeros(len(pats), np.int64)
    for i, t in enumerate(texts):
        a, c = oracle_canonical(pats, t, text_id=i)
        rows.append(a)
        counts += c
    a = np.concatenate(rows) if rows else np.zeros((0, 3), np.int64)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))], counts


def packed_dev(texts):
    out = []
    for t in texts:
        if t:
            out.append(acg.pack(torch.tensor(list(t), dtype=torch.uint8, device=DEV)))
        else:
            out.append(torch.zeros(4, dtype=torch.int32, device=DEV))
    return out


@pytest.mark.parametrize("form", ["packed_dev", "ascii_dev", "ascii_host", "packed_host"])
@pytest.mark.parametrize("interleave,stride,threads",
                         [(1, 1, 0), (4, 1, 0), (1, 2, 0), (2, 2, 0), (1, 3, 0), (2, 3, 0), (1, 3, 640), (1, 3, 256)])
def test_batch_vs_oracle(form, interleave, stride, threads):
    texts, pats = batch_case(11)
    d = acg.build(pats)
    want, counts = oracle_batch(pats, texts)
    lens = [len(t) for t in texts]
    if form == "packed_dev":
        arg, enc = packed_dev(texts), N.AC_TEXT_PACKED2
    elif form == "packed_host":
        arg, enc = [p.cpu().numpy() for p in packed_dev(texts)], N.AC_TEXT_PACKED2
    elif form == "ascii_dev":
        arg = [torch.tensor(list(t), dtype=torch.uint8, device=DEV) if t else torch.empty(0, dtype=torch.uint8, device=DEV)
               for t in texts]
        enc = N.AC_TEXT_ASCII
    else:
        arg, enc = [np.frombuffer(t, np.uint8) if t else np.zeros(0, np.uint8) for t in texts], N.AC_TEXT_ASCII
    r = acg.scan_batch(d, arg, encoding=enc, n_bases=lens, capacity=16, interleave=interleave, stride=stride,
                       threads=threads)
    got = r.canonical()
    assert np.array_equal(got, want)
    assert r.counts.cpu().numpy().tolist() == counts.tolist()


def test_batch_equals_per_text_loop():
    texts, pats = batch_case(12, 60)
    d = acg.build(pats)
    pk = packed_dev(texts)
    lens = [len(t) for t in texts]
    b = acg.scan_batch(d, pk, encoding=N.AC_TEXT_PACKED2, n_bases=lens).canonical()
    loop = []
    for i, (p, n) in enumerate(zip(pk, lens)):
        loop.append(acg.scan(d, p, encoding=N.AC_TEXT_PACKED2, n_bases=n, text_id=i).canonical())
    loop = np.concatenate(loop)
    loop = loop[np.lexsort((loop[:, 2], loop[:, 1], loop[:, 0]))]
    assert np.array_equal(b, loop)


@pytest.mark.parametrize("chunk,stride,threads",
                         [(0, 1, 0), (64, 1, 0), (1000, 1, 0), (0, 2, 0), (64, 2, 0), (0, 3, 0), (1000, 3, 0), (0, 3, 640)])
def test_batch_plan_replays_exactly(chunk, stride, threads):
    texts, pats = batch_case(13, 100)
    d = acg.build(pats)
    want, counts = oracle_batch(pats, texts)
    pk = packed_dev(texts)
    plan = acg.BatchPlan(d, pk, [len(t) for t in texts], capacity=len(want) + 10, chunk=chunk, stride=stride,
                         threads=threads)
    for _ in range(3):  # replays reset their counters
        assert plan.run() == len(want)
        assert np.array_equal(plan.result().canonical(), want)
        assert plan.counts.cpu().numpy().tolist() == counts.tolist()
    plan.close()


def test_batch_plan_without_counts_replays_exactly():
    texts, pats = batch_case(17, 60)
    d = acg.build(pats)
    want, _ = oracle_batch(pats, texts)
    plan = acg.BatchPlan(d, packed_dev(texts), [len(t) for t in texts], capacity=len(want) + 10, counts=False)
    for _ in range(3):
        assert plan.run() == len(want)
        assert np.array_equal(plan.result().canonical(), want)
    plan.close()


def test_batch_plan_overflow_flag():
    texts = [b"A" * 1000, b"A" * 10]
    d = acg.build([b"A", b"AA"])
    plan = acg.BatchPlan(d, packed_dev(texts), [1000, 10], capacity=100)
    for _ in range(3):  # counts stay exact when replays overflow
        assert plan.run() == 1000 + 999 + 10 + 9 and plan.overflow
        assert plan.counts.cpu().tolist() == [1010, 1008]
    plan.close()


# ------------------------------------------------------------------ serving


def test_serve_alone_equals_mix_equals_oracle():
    rng = random.Random(21)
    genome = rand_dna(rng, 400_000)
    sets = []
    for k in range(3):
        pats = [genome[j : j + rng.randint(10, 20)] for j in rng.sample(range(399_000), 100 + 200 * k)]
        pats += [rand_dna(rng, 12) for _ in range(50)]
        sets.append(pats)
    dfas = [acg.build(p) for p in sets]
    reqs = []
    for _ in range(60):
        n = int(np.exp(rng.uniform(np.log(100), np.log(150_000))))
        off = rng.randint(0, len(genome) - n)
        reqs.append((rng.randint(0, 2), genome[off : off + n]))
    # alone: one request at a time
    srv = acg.Server(device_budget_bytes=1 << 30, n_streams=3, max_batch=16)
    slots = [srv.add_dfa(d) for d in dfas]
    alone = []
    for s, t in reqs:
        tk = srv.submit(slots[s], t)
        alone.append(srv.wait(tk, slots[s], capacity=8))
    # mix: submitted from 4 threads at once, waited in reverse order
    tickets = [None] * len(reqs)

    def submitter(idx):
        for i in idx:
            s, t = reqs[i]
            tickets[i] = srv.submit(slots[s], t)

    ths = [threading.Thread(target=submitter, args=(list(range(k, len(reqs), 4)),)) for k in range(4)]
    [t.start() for t in ths]
    [t.join() for t in ths]
    mix = [None] * len(reqs)
    for i in reversed(range(len(reqs))):
        mix[i] = srv.wait(tickets[i], slots[reqs[i][0]], capacity=1 << 12)
    st = srv.stats()
    srv.close()
    assert st["completed"] == 2 * len(reqs) and st["failed"] == 0
    assert st["batches_launched"] < 2 * len(reqs)  # requests were batched together
    for i, (s, t) in enumerate(reqs):
        a = alone[i][0][np.lexsort((alone[i][0][:, 1], alone[i][0][:, 0]))]
        m = mix[i][0][np.lexsort((mix[i][0][:, 1], mix[i][0][:, 0]))]
        assert np.array_equal(a, m)
        assert np.array_equal(alone[i][1], mix[i][1])
        want, counts = oracle_canonical(sets[s], t)
        assert np.array_equal(a, want[:, 1:])
        assert np.array_equal(alone[i][1], counts)


def test_serve_batch_overflow_reruns_exactly():
    """Requests far denser in occurrences than the server's output reservation:
    each overflowing batch runs once more with exactly the room it needs, and
    every request still gets its exact result."""
    rng = random.Random(22)
    pats = [b"AAAA", b"AAAAAA", b"ACAC", b"CACA", b"ACACACAC", b"GATTACA"]
    d = acg.build(pats)
    texts = []
    for i in range(24):
        n = rng.randint(2_000, 40_000)
        parts, L = [], 0
        while L < n:
            unit = rng.choice([b"A" * rng.randint(5, 60), b"AC" * rng.randint(3, 40), rand_dna(rng, rng.randint(5, 50))])
            parts.append(unit)
            L += len(unit)
        texts.append(b"".join(parts)[:n])
    srv = acg.Server(n_streams=2, max_batch=8, match_capacity_per_base_x1000=1)
    slot = srv.add_dfa(d)
    tickets = [srv.submit(slot, t) for t in texts]
    got = [srv.wait(tk, slot, capacity=1 << 16) for tk in tickets]
    st = srv.stats()
    srv.close()
    assert st["failed"] == 0 and st["overflow_batches"] > 0
    for t, (m, c, _) in zip(texts, got):
        want, counts = oracle_canonical(pats, t)
        assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:])
        assert np.array_equal(c, counts)


def test_serve_large_results_handed_over():
    """Requests with 1 MB or more of occurrences (65,536+) keep their results in a pinned
    block until they are waited for: results equal the oracle's whether waited at once,
    out of order, with a too-small first capacity, or (one of them) never, and blocks
    are reused across requests."""
    rng = random.Random(24)
    pats = [b"A", b"AA", b"AC", b"CA", b"ACGT"]
    d = acg.build(pats)
    srv = acg.Server(n_streams=2, max_batch=1)  # batches of one request
    slot = srv.add_dfa(d)
    texts = []
    for i in range(8):
        n = rng.randint(150_000, 400_000)
        texts.append(bytes(rng.choice(b"AAAAACGT") for _ in range(n)))
    texts.append(b"ACGT" * 10)  # a small result among them
    tickets = [srv.submit(slot, t) for t in texts]
    order = list(range(len(texts) - 1))
    rng.shuffle(order)
    for j, i in enumerate(order):
        m, c, k = srv.wait(tickets[i], slot, capacity=(1000 if j % 2 else None))
        want, counts = oracle_canonical(pats, texts[i])
        assert k == len(want) and k >= 65_536
        assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:])
        assert np.array_equal(c, counts)
    again = srv.submit(slot, texts[0])  # a block back from the pool
    m, c, k = srv.wait(again, slot)  # views of the server's copy, no copy made
    want, counts = oracle_canonical(pats, texts[0])
    assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:]) and np.array_equal(c, counts)
    with pytest.raises(acg.AcError) as e:
        srv.wait(again, slot)  # taken: the ticket is gone
    assert e.value.status == N.AC_ERR_NOT_FOUND
    srv.submit(slot, texts[1])  # left unclaimed: its block goes back when the server closes
    st = srv.stats()
    srv.close()
    assert st["failed"] == 0
    # a taken result stays valid after the server is gone; its block is given back with the arrays
    assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:]) and np.array_equal(c, counts)
    del m, c


@pytest.mark.parametrize("form", ["ascii", "packed"])
def test_serve_large_texts_pinned_at_submit(form):
    """Texts of 1 MB or more are held in pinned blocks from submit on and copied to the
    device from there, between runs of small staged texts of the same batch (odd lengths,
    ASCII or packed); every request gets the oracle's result."""
    rng = random.Random(25)
    src = rand_dna(rng, 3_000_000) * 2
    pats = [src[j : j + rng.randint(8, 16)] for j in rng.sample(range(2_999_000), 300)]
    d = acg.build(pats)
    srv = acg.Server(n_streams=2, max_batch=16)
    slot = srv.add_dfa(d)
    reqs = []
    for i in range(24):
        if i % 2 == 0:
            n = rng.randint(1, 5000)
        elif form == "ascii":
            n = rng.randint(1_100_000, 2_900_000)  # 1 byte a base
        else:
            n = rng.randint(4_300_000, 5_000_000)  # 16 bases a 4-byte word: over 1 MB of words
        off = rng.randint(0, len(src) - n)
        reqs.append(src[off : off + n])
    tickets = []
    for t in reqs:
        if form == "packed":
            pk = acg.pack(torch.from_numpy(np.frombuffer(t, np.uint8).copy()).to(DEV)).cpu().numpy()
            tickets.append(srv.submit(slot, pk, encoding=N.AC_TEXT_PACKED2, n_bases=len(t)))
        else:
            tickets.append(srv.submit(slot, t))
    for tk, t in zip(tickets, reqs):
        m, c, k = srv.wait(tk, slot)
        want, counts = oracle_canonical(pats, t)
        assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:])
        assert np.array_equal(c, counts)
    st = srv.stats()
    srv.close()
    assert st["failed"] == 0


def test_serve_admission_and_errors():
    d = acg.build([b"ACGT"])
    srv = acg.Server(device_budget_bytes=1 << 20, n_streams=1, max_batch=4, max_queue=2)
    slot = srv.add_dfa(d)
    big = b"A" * (1 << 20)  # alone exceeds the device budget
    assert srv.try_submit(slot, big) is None
    with pytest.raises(acg.AcError) as e:
        srv.submit(slot, b"ACGN")
    assert e.value.status == N.AC_ERR_ALPHABET
    with pytest.raises(acg.AcError) as e:
        srv.submit(99, b"ACGT")
    assert e.value.status == N.AC_ERR_NOT_FOUND
    tk = srv.submit(slot, b"ACGTACGT")
    m, c, k = srv.wait(tk, slot)
    assert k == 2 and c.tolist() == [2]
    st = srv.stats()
    assert st["rejected"] == 1
    srv.close()


def test_serve_submit_alphabet_check():
    """Submit rejects an ASCII text with any byte other than A, C, G, T, wherever it sits
    (64 bytes are checked per step, then the tail one by one), and queues good texts."""
    d = acg.build([b"ACGT"])
    srv = acg.Server(n_streams=1)
    slot = srv.add_dfa(d)
    rng = random.Random(23)
    for n in (1, 7, 8, 9, 15, 16, 17, 31, 40, 63, 64, 65, 127, 128, 129, 200):
        for pos in range(n):
            for v in (ord("a"), ord("N"), ord("B"), ord("U"), 0x00, 0xC1, 0xFF, ord("A") | 0x80):
                t = bytearray(rand_dna(rng, n))
                t[pos] = v
                with pytest.raises(acg.AcError) as e:
                    srv.submit(slot, bytes(t))
                assert e.value.status == N.AC_ERR_ALPHABET, (n, pos, v)
    big = bytearray(rand_dna(rng, (1 << 20) + 77))  # held in a pinned block from submit on
    for pos in (0, 63, 64, 4097, len(big) // 2, len(big) - 78, len(big) - 1):
        t = bytearray(big)
        t[pos] = ord("N")
        with pytest.raises(acg.AcError) as e:
            srv.submit(slot, bytes(t))
        assert e.value.status == N.AC_ERR_ALPHABET, pos
    # texts of 2 MB and more are copied in four parts of round_up(n / 4, 64) bytes: a bad byte at
    # either side of every part boundary, and a good text exact against the oracle
    huge = bytearray(rand_dna(rng, (4 << 20) + 333))
    part = ((len(huge) + 3) // 4 + 63) // 64 * 64
    for pos in (0, part - 1, part, 2 * part - 1, 2 * part, 3 * part - 1, 3 * part, len(huge) - 1):
        t = bytearray(huge)
        t[pos] = ord("a")
        with pytest.raises(acg.AcError) as e:
            srv.submit(slot, bytes(t))
        assert e.value.status == N.AC_ERR_ALPHABET, pos
    m, c, k = srv.wait(srv.submit(slot, bytes(huge)), slot)
    want, counts = oracle_canonical([b"ACGT"], bytes(huge))
    assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:]) and c.tolist() == counts.tolist()
    good = rand_dna(rng, 100_003)
    m, c, k = srv.wait(srv.submit(slot, good), slot)
    want, counts = oracle_canonical([b"ACGT"], good)
    assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:]) and c.tolist() == counts.tolist()
    assert srv.stats()["failed"] == 0
    srv.close()


def test_serve_wait_timeout_keeps_ticket():
    d = acg.build([b"ACGT"])
    srv = acg.Server(n_streams=1)
    slot = srv.add_dfa(d)
    tk = srv.submit(slot, b"ACGT" * 1000)
    import ctypes

    r = N.Result(None, 0, 0, None, 0, 0, 0)
    t0 = time.time()
    while True:
        st = acg.lib().ac_serve_wait(srv.h, tk, ctypes.byref(r), 0)
        if st != N.AC_ERR_TIMEOUT:
            break
        assert time.time() - t0 < 30
    assert st == N.AC_ERR_OVERFLOW and r.n_matches == 1000  # capacity 0: count reported, ticket kept
    m, c, k = srv.wait(tk, slot, capacity=1000)
    assert k == 1000
    srv.close()


def test_batch_chunk_candidates_and_tuner_are_exact():
    """Every work-item chunk the batch tuner tries (the halo rounded up to 64 bases, times 1 .. 32,
    and the built-in default) gives the oracle's result; the tuned chunk is then used by default."""
    texts, pats = batch_case(14, 120)
    d = acg.build(pats)
    want, counts = oracle_batch(pats, texts)
    pk = packed_dev(texts)
    lens = [len(t) for t in texts]
    unit = max(64, (max(len(p) for p in pats) - 1 + 63) // 64 * 64)
    for chunk in [0] + [unit * m for m in (1, 2, 4, 8, 16, 32)]:
        r = acg.scan_batch(d, pk, encoding=N.AC_TEXT_PACKED2, n_bases=lens, capacity=16, chunk=chunk, stats=True)
        assert np.array_equal(r.canonical(), want), chunk
        assert r.counts.cpu().numpy().tolist() == counts.tolist()
        if chunk:
            assert r.stats["chunk"] == chunk
    tuned = acg.autotune_batch(d, pk, lens)
    assert tuned in [unit * m for m in (1, 2, 4, 8, 16, 32)] or tuned >= 64
    r = acg.scan_batch(d, pk, encoding=N.AC_TEXT_PACKED2, n_bases=lens, stats=True)
    assert r.stats["chunk"] == tuned
    assert np.array_equal(r.canonical(), want)
    plan = acg.BatchPlan(d, pk, lens, capacity=len(want) + 10)  # plans take the tuned chunk too
    assert plan.run() == len(want)
    assert np.array_equal(plan.result().canonical(), want)
    plan.close()


def test_serve_cancel():
    """A request still queued behind a running batch is withdrawn and never scanned; a finished one
    that was not waited for has its results dropped; an unknown ticket is not found; a request whose
    batch is on the device cannot be withdrawn and stays waitable. The server goes on serving."""
    rng = random.Random(33)
    small = rand_dna(rng, 5000) + b"ACGTACGT"
    pats = [small[j : j + 10] for j in rng.sample(range(4900), 50)] + [b"ACGTACGT"]
    d_a, d_b = acg.build([b"ACGTACGTAC", b"GGGGG"]), acg.build(pats)
    srv = acg.Server(n_streams=1, max_batch=4)  # one worker: while it scans A, B waits in the queue
    sa, sb = srv.add_dfa(d_a), srv.add_dfa(d_b)  # different machines: A and B are never batched together
    big = np.frombuffer(rand_dna(rng, 1 << 20) * 128, np.uint8)  # 128 Mbase
    k_big = acg.scan(d_a, torch.tensor(big, device=DEV)).n_matches
    ta = srv.submit(sa, big)
    tb = srv.submit(sb, small)
    assert srv.cancel(tb)
    with pytest.raises(acg.AcError) as e:
        srv.wait(tb, sb)
    assert e.value.status == N.AC_ERR_NOT_FOUND
    assert srv.wait(ta, sa)[2] == k_big
    want, counts = oracle_canonical(pats, small)
    tc = srv.submit(sb, small)
    m, c, k = srv.wait(tc, sb)
    assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:]) and np.array_equal(c, counts)
    done_before = srv.stats()["completed"]
    td = srv.submit(sb, small)
    t0 = time.time()
    while srv.stats()["completed"] == done_before:  # finished, not waited for
        assert time.time() - t0 < 30
        time.sleep(0.001)
    assert srv.cancel(td)
    with pytest.raises(acg.AcError):
        srv.wait(td, sb)
    with pytest.raises(acg.AcError) as e:
        srv.cancel(987654321)
    assert e.value.status == N.AC_ERR_NOT_FOUND
    te = srv.submit(sa, big)
    t0 = time.time()
    while srv.stats()["batches_launched"] < 4:  # batches of A, C, D, then E's
        assert time.time() - t0 < 30
    if not srv.cancel(te):  # its batch is on the device: not withdrawn, and its result still comes
        assert srv.wait(te, sa)[2] == k_big
    st = srv.stats()
    assert st["cancelled"] == 1 and st["failed"] == 0
    srv.close()


def test_serve_split_batch_results_taken_without_copy():
    """Requests split out of one multi-request batch share one pinned block: each taken result
    (views, no copy) equals the oracle's, and stays valid while the batch's other results are
    released, and after the server is gone."""
    rng = random.Random(34)
    genome = rand_dna(rng, 300_000)
    pats = [genome[j : j + rng.randint(8, 14)] for j in rng.sample(range(299_000), 400)] + [b"ACGTAC"]
    d = acg.build(pats)
    srv = acg.Server(n_streams=1, max_batch=32)
    slot = srv.add_dfa(d)
    big = np.frombuffer(rand_dna(rng, 1 << 20) * 192, np.uint8)  # keeps the one worker busy meanwhile
    d_big = acg.build([b"ACGTACGTAC"])
    s_big = srv.add_dfa(d_big)
    t_big = srv.submit(s_big, big)
    texts = [genome[o : o + n] for o, n in ((rng.randint(0, 250_000), rng.randint(0, 40_000)) for _ in range(20))]
    tickets = [srv.submit(slot, t) for t in texts]  # queued together: one batch behind the big one
    got = [srv.wait(tk, slot) for tk in tickets]
    srv.wait(t_big, s_big)
    st = srv.stats()
    assert st["batches_launched"] < 1 + len(texts)  # the 20 requests were batched together
    wants = [oracle_canonical(pats, t) for t in texts]
    for i in rng.sample(range(len(texts)), len(texts)):  # release in random order, check the rest
        m, c, k = got[i]
        want, counts = wants[i]
        assert k == len(want)
        assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], want[:, 1:]) and np.array_equal(c, counts)
        got[i] = None
        del m, c
    keep = srv.wait(srv.submit(slot, texts[3]), slot)
    srv.close()
    m, c, k = keep
    assert np.array_equal(m[np.lexsort((m[:, 1], m[:, 0]))], wants[3][0][:, 1:]) and np.array_equal(c, wants[3][1])
