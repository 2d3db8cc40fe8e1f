"""Seeded synthetic DNA workloads (texts and pattern sets).

This module holds no matching arithmetic: it only draws random DNA. Both the
CUDA path and the CPU oracle take their inputs from it, so the two sides see
identical bytes. Everything is deterministic for a given (seed, device):
torch's CPU and CUDA generators give different streams, so a workload made on
``cuda`` differs from one made on ``cpu`` with the same seed.

Text models
  * uniform: i.i.d. bases with P(A)=P(T)=(1-gc)/2, P(C)=P(G)=gc/2;
  * markov:  an order-2 chain (context = the two previous bases) with base
             composition A=T=0.295, C=G=0.205, per-context multipliers drawn
             once from the seed in [0.7, 1.3], CpG depletion (P(G | C) x 0.25),
             then the G/C columns rescaled until the stationary GC content is
             0.41; on top, short tandem repeats (unit 1-6 bases, run 20-200
             bases, non-overlapping, one per stratum) cover 5% of the bases.

The chain is sampled block-parallel: ``lanes`` independent chains each emit a
contiguous segment, each started from the stationary pair distribution, so a
3 Gbase text takes a few hundred vectorised steps on the GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

ALPHABET = b"ACGT"
_ASCII = torch.tensor(list(ALPHABET), dtype=torch.uint8)

BASE_SEED = 14037294


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


# --------------------------------------------------------------- uniform


def uniform_text(n: int, seed: int, gc: float = 0.5, device="cpu") -> torch.Tensor:
    """i.i.d. ASCII bases (uint8 tensor of length n)."""
    g = _gen(seed, device)
    u = torch.rand(n, generator=g, device=device)
    at = (1.0 - gc) / 2.0
    # order A, C, G, T with cumulative thresholds
    code = (u >= at).to(torch.uint8) + (u >= at + gc / 2).to(torch.uint8) + (u >= 1.0 - at).to(torch.uint8)
    return _ASCII.to(device)[code.long()]


# ----------------------------------------------------------------- markov


def markov_chain(seed: int, gc_target: float = 0.41) -> np.ndarray:
    """16x4 matrix P[ctx, x] of the order-2 chain, ctx = 4*prev2 + prev1."""
    rng = np.random.default_rng(seed)
    base = np.array([0.295, 0.205, 0.205, 0.295])
    mult = rng.uniform(0.7, 1.3, size=(16, 4))
    raw = base[None, :] * mult
    raw[[4 * a + 1 for a in range(4)], 2] *= 0.25  # CpG depletion: G after C

    def stationary_gc(P):
        # pair chain on 16 states: (a,b) -> (b,x) with prob P[4a+b, x]
        T = np.zeros((16, 16))
        for ctx in range(16):
            b = ctx % 4
            for x in range(4):
                T[ctx, 4 * b + x] += P[ctx, x]
        v = np.full(16, 1 / 16)
        for _ in range(2000):
            v = v @ T
        last = np.array([v[[4 * a + x for a in range(4)]].sum() for x in range(4)])
        return last[1] + last[2], v

    def scaled(f):
        Q = raw.copy()
        Q[:, 1:3] *= f
        return Q / Q.sum(axis=1, keepdims=True)

    lo, hi = 0.2, 5.0
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        if stationary_gc(scaled(mid))[0] < gc_target:
            lo = mid
        else:
            hi = mid
    P = scaled(math.sqrt(lo * hi))
    return P


@dataclass
class StrRuns:
    start: torch.Tensor  # int64 [k]
    length: torch.Tensor  # int64 [k]
    unit_len: torch.Tensor  # int64 [k]


@dataclass
class Text:
    ascii: torch.Tensor  # uint8 [n]
    strs: StrRuns | None = None
    model: str = "uniform"
    meta: dict = field(default_factory=dict)


def markov_text(
    n: int,
    seed: int,
    device="cpu",
    gc_target: float = 0.41,
    str_fraction: float = 0.05,
    lanes: int | None = None,
) -> Text:
    P = markov_chain(seed, gc_target)
    cdf = torch.tensor(np.cumsum(P, axis=1)[:, :3], dtype=torch.float32, device=device)
    g = _gen(seed + 1, device)
    if lanes is None:
        lanes = 1 << 22 if n >= (1 << 28) else max(1, min(n, 4096))
    seg = (n + lanes - 1) // lanes
    # stationary pair distribution for the lane start contexts
    Tm = np.zeros((16, 16))
    for ctx in range(16):
        for x in range(4):
            Tm[ctx, 4 * (ctx % 4) + x] += P[ctx, x]
    v = np.full(16, 1 / 16)
    for _ in range(2000):
        v = v @ Tm
    start_cdf = torch.tensor(np.cumsum(v)[:-1], dtype=torch.float32, device=device)
    ctx = torch.searchsorted(start_cdf, torch.rand(lanes, generator=g, device=device)).long()
    out = torch.empty((seg, lanes), dtype=torch.uint8, device=device)
    for t in range(seg):
        u = torch.rand(lanes, generator=g, device=device)
        th = cdf[ctx]
        x = (u >= th[:, 0]).long() + (u >= th[:, 1]).long() + (u >= th[:, 2]).long()
        out[t] = x.to(torch.uint8)
        ctx = ((ctx * 4) + x) & 15
    codes = out.t().contiguous().view(-1)[:n]
    del out
    strs = None
    if str_fraction > 0 and n >= 4000:
        codes, strs = _plant_tandem_repeats(codes, seed + 2, str_fraction, device)
    ascii_ = _ASCII.to(device)[codes.long()] if n < (1 << 28) else _codes_to_ascii_inplace(codes)
    return Text(ascii_, strs, "markov", {"gc_target": gc_target, "str_fraction": str_fraction})


def _codes_to_ascii_inplace(codes: torch.Tensor) -> torch.Tensor:
    lut = _ASCII.to(codes.device)
    step = 1 << 28
    for a in range(0, codes.numel(), step):
        codes[a : a + step] = lut[codes[a : a + step].long()]
    return codes


def _plant_tandem_repeats(codes: torch.Tensor, seed: int, frac: float, device):
    n = codes.numel()
    mean_len = 110.0
    k = max(1, int(round(frac * n / mean_len)))
    stratum = n // k
    g = _gen(seed, device)
    length = torch.randint(20, 201, (k,), generator=g, device=device)
    unit_len = torch.randint(1, 7, (k,), generator=g, device=device)
    units = torch.randint(0, 4, (k, 6), generator=g, device=device, dtype=torch.int64)
    room = (stratum - length).clamp(min=1)
    off = (torch.rand(k, generator=g, device=device) * room.to(torch.float32)).long().clamp(max=room - 1)
    start = torch.arange(k, device=device, dtype=torch.int64) * stratum + off
    # expand runs into positions in slices to bound memory
    step = 1 << 20
    for a in range(0, k, step):
        b = min(k, a + step)
        L = length[a:b]
        run = torch.repeat_interleave(torch.arange(a, b, device=device), L)
        first = torch.cumsum(L, 0) - L
        j = torch.arange(run.numel(), device=device) - torch.repeat_interleave(first, L)
        pos = start[run] + j
        codes[pos] = units[run, j % unit_len[run]].to(codes.dtype)
    return codes, StrRuns(start, length, unit_len)


# --------------------------------------------------------------- patterns


def _dedupe_fill(want: int, draw, max_rounds: int = 50) -> list[bytes]:
    seen, out = set(), []
    for _ in range(max_rounds):
        for p in draw(want - len(out)):
            if p not in seen:
                seen.add(p)
                out.append(p)
                if len(out) == want:
                    return out
    return out


def uniform_patterns(k, lo, hi, seed, gc_clamp=None) -> list[bytes]:
    rng = np.random.default_rng(seed)

    def draw(m):
        res = []
        while len(res) < m:
            L = int(rng.integers(lo, hi + 1))
            c = rng.integers(0, 4, L)
            if gc_clamp is not None:
                gcf = np.isin(c, (1, 2)).mean()
                if not (gc_clamp[0] <= gcf <= gc_clamp[1]):
                    continue
            res.append(bytes(ALPHABET[i] for i in c))
        return res

    return _dedupe_fill(k, draw)


def substring_patterns(text: torch.Tensor, k, lo, hi, seed, avoid: StrRuns | None = None,
                       within: StrRuns | None = None) -> list[bytes]:
    """k distinct substrings of ``text`` with lengths U[lo, hi].

    ``avoid``: reject substrings that touch a tandem-repeat run;
    ``within``: take substrings from inside tandem-repeat runs only."""
    rng = np.random.default_rng(seed)
    n = text.numel()
    if within is not None:
        st, ln = within.start.cpu().numpy(), within.length.cpu().numpy()
    if avoid is not None:
        ast_, aln = avoid.start.cpu().numpy(), avoid.length.cpu().numpy()

    def draw(m):
        m2 = int(m * 1.3) + 8
        L = rng.integers(lo, hi + 1, m2)
        if within is not None:
            r = rng.integers(0, len(st), m2)
            ok = ln[r] >= L
            r, L = r[ok], L[ok]
            pos = st[r] + (rng.random(len(r)) * (ln[r] - L + 1)).astype(np.int64)
        else:
            pos = (rng.random(m2) * (n - L + 1)).astype(np.int64)
            if avoid is not None:
                idx = np.searchsorted(ast_, pos + L, side="left") - 1
                hit = (idx >= 0) & (ast_[np.clip(idx, 0, None)] + aln[np.clip(idx, 0, None)] > pos)
                pos, L = pos[~hit], L[~hit]
        if len(pos) == 0:
            return []
        idx = torch.from_numpy(pos)[:, None] + torch.arange(int(L.max()))[None, :]
        idx = idx.clamp(max=n - 1).to(text.device)
        rows = text[idx].cpu().numpy()
        return [rows[i, : L[i]].tobytes() for i in range(len(pos))]

    return _dedupe_fill(k, draw)


def merge_dedupe(*groups: list[bytes]) -> list[bytes]:
    seen, out = set(), []
    for grp in groups:
        for p in grp:
            if p not in seen:
                seen.add(p)
                out.append(p)
    return out


# -------------------------------------------------------------- workloads


@dataclass
class Workload:
    name: str
    text: Text | None
    patterns: list[bytes]
    texts: list[torch.Tensor] | None = None  # batched form
    meta: dict = field(default_factory=dict)


def plain_small(device="cpu", seed=BASE_SEED + 0, n=1_000_000, n_patterns=100) -> Workload:
    """1 Mbase i.i.d. uniform text, 100 patterns of length 8-20 (half text
    substrings, half uniform); ASCII input."""
    t = Text(uniform_text(n, seed, 0.5, device), None, "uniform")
    half = n_patterns // 2
    pats = merge_dedupe(substring_patterns(t.ascii, half, 8, 20, seed + 10),
                        uniform_patterns(n_patterns - half, 8, 20, seed + 11))
    return Workload(f"plain-{n}b-uniform-{len(pats)}pat", t, pats, meta={"encoding": "ascii"})


def plain_chromosome(device="cpu", seed=BASE_SEED + 1, n=268_435_456, n_patterns=10_000) -> Workload:
    """256 Mbase order-2 Markov text (41% GC, 5% tandem repeats), 10,000
    primer-like patterns of length 18-30 (half substrings, half uniform with
    GC clamped to 40-60%); 2-bit packed input."""
    t = markov_text(n, seed, device)
    half = n_patterns // 2
    pats = merge_dedupe(substring_patterns(t.ascii, half, 18, 30, seed + 10),
                        uniform_patterns(n_patterns - half, 18, 30, seed + 11, gc_clamp=(0.4, 0.6)))
    return Workload(f"plain-{n}b-markov-{len(pats)}pat", t, pats, meta={"encoding": "packed2"})


def plain_genome(device="cpu", seed=BASE_SEED + 2, n=3_000_000_000, n_patterns=100_000,
                 str_share=0.05) -> Workload:
    """3 Gbase Markov text, 100,000 patterns of length 20-25: 45% substrings
    of non-repeat regions, ``str_share`` substrings of tandem-repeat runs (the
    source of the repeat-driven match density), the rest uniform."""
    t = markov_text(n, seed, device)
    k_str = int(round(n_patterns * str_share))
    k_sub = int(round(n_patterns * 0.45))
    k_uni = n_patterns - k_str - k_sub
    pats = merge_dedupe(substring_patterns(t.ascii, k_sub, 20, 25, seed + 10, avoid=t.strs),
                        substring_patterns(t.ascii, k_str, 20, 25, seed + 12, within=t.strs),
                        uniform_patterns(k_uni, 20, 25, seed + 11))
    return Workload(f"plain-{n}b-markov-str-{len(pats)}pat", t, pats,
                    meta={"encoding": "packed2", "str_share": str_share})


def batch_lengths(n_texts: int, seed: int, mu=math.log(2000.0), sigma=2.013, lo=100, hi=100_000):
    rng = np.random.default_rng(seed)
    return np.clip(np.round(rng.lognormal(mu, sigma, n_texts)), lo, hi).astype(np.int64)


def batched(device="cpu", seed=BASE_SEED + 3, n_texts=4096, n_patterns=50_000) -> Workload:
    """4,096 texts with clipped lognormal lengths (100..100,000, median ~2
    kbase, total ~40 Mbase), i.i.d. bases at 40% GC; one set of 50,000
    patterns of length 15-25 (half substrings of the batch, half uniform)."""
    lens = batch_lengths(n_texts, seed)
    whole = uniform_text(int(lens.sum()), seed, 0.40, device)
    offs = np.concatenate([[0], np.cumsum(lens)])
    texts = [whole[offs[i] : offs[i + 1]] for i in range(n_texts)]
    half = n_patterns // 2
    pats = merge_dedupe(substring_patterns(whole, half, 15, 25, seed + 10),
                        uniform_patterns(n_patterns - half, 15, 25, seed + 11))
    return Workload(f"batch-{n_texts}texts-{int(lens.sum())}b-{len(pats)}pat", None, pats, texts=texts,
                    meta={"lengths": lens, "encoding": "packed2"})


SERVE_SET_SIZES = [int(round(1000 * 100 ** (k / 7))) for k in range(8)]


def serve_sets(genome: torch.Tensor, seed=BASE_SEED + 4, sizes=SERVE_SET_SIZES) -> list[list[bytes]]:
    """8 pattern sets of 1,000..100,000 patterns, length 12-30, half
    substrings of the serving genome, half uniform."""
    out = []
    for k, size in enumerate(sizes):
        half = size // 2
        out.append(merge_dedupe(substring_patterns(genome, half, 12, 30, seed + 100 * k),
                                uniform_patterns(size - half, 12, 30, seed + 100 * k + 1)))
    return out


def serve_requests(n_req: int, seed: int, genome_len: int, rate_hz=2000.0, lo=1_000, hi=10_000_000,
                   n_sets=8):
    """Poisson arrivals (exponential gaps), log-uniform lengths, uniform set
    choice, each text a window of the serving genome at a random offset."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_req)
    t_arr = np.cumsum(gaps)
    lens = np.exp(rng.uniform(math.log(lo), math.log(hi), n_req)).astype(np.int64)
    lens = np.minimum(lens, genome_len)
    offs = (rng.random(n_req) * (genome_len - lens + 1)).astype(np.int64)
    sets = rng.integers(0, n_sets, n_req)
    return t_arr, lens, offs, sets
