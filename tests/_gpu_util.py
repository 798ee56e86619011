"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np
import torch

import paper_2310_19855_gb300 as gi
import workload as wl
from oracle import probes as OP
from oracle import sh as OSH
from oracle.cache import OracleCache
from oracle.frame import run_frame
from paper_2310_19855_gb300.pipeline import Pipeline, view_of

# float32 path vs float64 oracle: the float32 mean has at most 2 ulp of error and the EMA
# contracts an error by (1 - alpha) per frame
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


def sh_gpu(pl):
    return pl.probes.sh.cpu().numpy()[:, :27].reshape(-1, 9, 3).astype(np.float64)


# Interpolated irradiance: a pixel's flag (weighted, relaxed, none, sky) is a decision the float32
# kernel and the float64 oracle could take differently where every neighbour weight sits at zero;
# such flips may touch at most 1e-5 of the pixels (none observed on any workload).  Every pixel
# whose flag agrees -- including the decision-sensitive ones, with a neighbour's plane test within
# 1e-3 of its cut or a weight sum below 1e-2, whose weights are continuous there -- is compared at
# |dE| <= rel |E| + 1e-5 emag + 1e-7, emag the magnitude of the summed SH terms (float32
# cancellation in dark pixels).
MAX_FLIP_FRAC = 1e-5


def compare_frame(pl, fr, out, rel=1e-4):
    """Spawn, probe SH and interpolation of one frame against the oracle; returns (decision-sensitive
    pixels, flag flips)."""
    P = pl.probes.layout.num_probes
    # spawn: mask levels bit-exact, probe positions to float32 rounding
    mips_o = OP.build_mips(out["spawn"]["mask"])
    mips_g = pl.probes.mask_levels()
    assert len(mips_o) == len(mips_g)
    for a, b in zip(mips_o, mips_g):
        assert np.array_equal(a, b)
    pos_g = pl.probes.pos.cpu().numpy()
    nrm_g = pl.probes.nrm.cpu().numpy()
    v = out["spawn"]["valid"]
    assert np.array_equal(nrm_g[:, 3] == 1.0, v)
    scale = 1.0 + np.abs(fr.camera.pos).max() + np.abs(out["spawn"]["dist"]).max()
    assert np.abs(pos_g[v, :3] - out["spawn"]["pos"][v]).max() < 4e-7 * scale
    assert np.array_equal(nrm_g[v, :3], out["spawn"]["nrm"][v])
    # probe SH: relative to the probe's band-0 magnitude (individual coefficients can cancel)
    sg, so = sh_gpu(pl), out["sh"]
    mag = np.abs(so[:, 0:1, :]).max(axis=2, keepdims=True) + 1e-6
    err = np.abs(sg - so) / mag
    assert err.max() < rel, err.max()
    # irradiance at each probe normal
    Eg = OSH.irradiance(sg[v], out["spawn"]["nrm"][v])
    Eo = OSH.irradiance(so[v], out["spawn"]["nrm"][v])
    assert close(Eg, Eo, rel=rel, atol=1e-6).all()
    # interpolation: flags, then every pixel whose flag agrees
    irr = pl.irr.cpu().numpy()
    flag_g = irr[..., 3].astype(np.int64)
    flag_o = out["flag"]
    X = flag_o.size
    flips = flag_g != flag_o
    assert np.count_nonzero(flips) <= MAX_FLIP_FRAC * X, np.count_nonzero(flips)
    emag = out["diag"]["emag"][..., None]
    ok = (np.abs(irr[..., :3] - out["irr"]) <= rel * np.abs(out["irr"]) + 1e-5 * emag + 1e-7).all(axis=-1)
    bad = ~flips & ~ok
    assert np.count_nonzero(bad) == 0, (np.count_nonzero(bad), np.abs(irr[..., :3] - out["irr"])[bad].max())
    wsum, margin = out["diag"]["wsum"], out["diag"]["margin"]
    sensitive = (margin < 1e-3) | ((wsum > 0) & (wsum < 1e-2))
    return np.count_nonzero(sensitive), np.count_nonzero(flips)


def run_frames(config, frames, rel=1e-4, resolved_format=0):
    cfg = wl.CONFIGS[config]
    fr0 = frames[0]
    pl = Pipeline(fr0.camera.width, fr0.camera.height, fr0.rays_per_probe, cfg["log2_slots"],
                  resolved_format=resolved_format)
    oc = OracleCache(cfg["log2_slots"])
    stats = []
    try:
        for fr in frames:
            view = view_of(fr.camera, fr.frame)
            gb = dev(fr.gbuffer)
            rec = dev(fr.records)
            pl.frame(gb, rec, view)
            torch.cuda.synchronize()
            out = run_frame(oc, fr)
            stats.append(compare_frame(pl, fr, out, rel))
    finally:
        pl.close()
    return stats


__all__ = ["compare_frame", "run_frames", "sh_gpu", "Pipeline", "view_of", "require_gpu", "dev", "u32", "close", "check_export_matches", "slot_identities",
           "check_slot_ids", "REL", "ABS"]
