"""Shared helpers of the GPU parity tests (test infrastructure)."""
import numpy as np
import torch

import oracle


def oracle_canonical(patterns, text, text_id=0):
    """Oracle occurrences as a sorted (k, 3) int64 array [text_id, pos, pid] plus counts."""
    t = text.cpu().numpy() if isinstance(text, torch.Tensor) else text
    pos, pid, counts = oracle.Machine(patterns).scan(t)
    a = np.stack([np.full(len(pos), text_id, np.int64), pos.astype(np.int64), pid.astype(np.int64)], 1)
    order = np.lexsort((a[:, 2], a[:, 1], a[:, 0]))
    return a[order], counts.astype(np.int64)


def assert_same(gpu_res, want, want_counts=None):
    got = gpu_res.canonical()
    assert got.shape == want.shape, (got.shape, want.shape)
    if len(want):
        bad = np.nonzero(np.any(got != want, axis=1))[0]
        assert len(bad) == 0, f"first mismatch at row {bad[:5]}: gpu {got[bad[:5]]} oracle {want[bad[:5]]}"
    assert gpu_res.n_matches == len(want)
    if want_counts is not None and gpu_res.counts is not None:
        assert gpu_res.counts.cpu().numpy().tolist() == want_counts.tolist()


def unpack_codes(packed: torch.Tensor, n: int) -> torch.Tensor:
    """2-bit packed words -> codes 0..3 (uint8), for the pack round-trip test."""
    w = packed.to(torch.int64) & 0xFFFFFFFF
    shifts = torch.arange(0, 32, 2, device=packed.device, dtype=torch.int64)
    codes = ((w[:, None] >> shifts[None, :]) & 3).reshape(-1)
    return codes[:n].to(torch.uint8)
