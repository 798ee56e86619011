"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np
import torch

import paper_2310_19855_gb300 as gi
from paper_2310_19855_gb300.pipeline import Pipeline, view_of

# float32 path vs float64 oracle (tolerances)
REL = 1e-4
ABS = 1e-7


def require_gpu():
    gi.build()
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    torch.cuda.init()


def dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def close(got, want, rel=REL, atol=ABS):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return np.abs(got - want) <= rel * np.abs(want) + atol


def check_export_matches(ex: np.ndarray, oc, resolved: bool, value_rel=REL):
    """Bit-exact identities (and sums/counts before resolve); values within tolerance after."""
    assert np.array_equal(ex["identity"], oc.ids), (ex.size, oc.ids.size)
    if not resolved:
        assert np.array_equal(ex["sum"].astype(np.int64), oc.sums)
        assert np.array_equal(ex["count"].astype(np.int64), oc.count)
    else:
        assert np.all(ex["count"] == 0)
        assert np.array_equal(ex["stamp"].astype(np.int64) - 1, oc.stamp)
        ok = close(ex["value"], oc.value, rel=value_rel)
        assert ok.all(), (np.count_nonzero(~ok), np.abs(ex["value"] - oc.value).max())


def slot_identities(ex: np.ndarray, slots: np.ndarray, n_slots: int) -> np.ndarray:
    """Identity of the cell behind each slot id (0 for the miss / none codes)."""
    table = np.zeros(n_slots, np.uint64)
    table[ex["slot"]] = ex["identity"]
    out = np.zeros(slots.size, np.uint64)
    real = slots < n_slots
    out[real] = table[slots[real]]
    return out


def check_slot_ids(slots: np.ndarray, ex: np.ndarray, rec: np.ndarray, oracle_ident: np.ndarray, n_slots: int):
    ln = rec[9]
    miss = np.isposinf(ln)
    hit = oracle_ident != 0
    assert np.all(slots[miss] == gi.GI_SLOT_MISS)
    assert np.all(slots[~hit & ~miss] == gi.GI_SLOT_NONE)
    assert np.all(slots[hit] < n_slots)
    assert np.array_equal(slot_identities(ex, slots, n_slots)[hit], oracle_ident[hit])


__all__ = ["Pipeline", "view_of", "require_gpu", "dev", "u32", "close", "check_export_matches", "slot_identities",
           "check_slot_ids", "REL", "ABS"]
