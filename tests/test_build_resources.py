"""The hot kernels compile for sm_103a without register spills, at the register budgets their
launch bounds set (ptxas resource usage, -Xptxas -v; no GPU needed)."""
import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_19855_gb300", "csrc")

# kernel (as its mangled name contains it) -> (source, most registers per thread)
HOT = {
    "8k_updateILi0ELb0E": ("gi_cache.cu", 32),  # the default form (no warp merge)
    "9k_resolveE": ("gi_cache.cu", 64),
    "16k_resolve_bitmapE": ("gi_cache.cu", 64),
    "14k_diag_atomicsILb1E": ("gi_diag.cu", 32),
    "11k_integrateILb1EE": ("gi_probes.cu", 128),  # 64 rays per probe
    "11k_integrateILb0EE": ("gi_probes.cu", 128),
    "13k_interpolateE": ("gi_probes.cu", 64),
    "10k_tile_keyILi0E": ("gi_tiles.cu", 32),
    "17k_tile_accumulate": ("gi_tiles.cu", 32),
    "14k_tile_resolve": ("gi_tiles.cu", 64),
}


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def _resources(nvcc, src, tmp):
    cmd = [nvcc, "-O3", "-std=c++17", "-gencode=arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
           "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-Xptxas", "-v", "-c", os.path.join(CSRC, src),
           "-o", os.path.join(tmp, src + ".o")]
    out = subprocess.run(cmd, capture_output=True, text=True, check=True).stderr
    res, name = {}, None
    for line in out.splitlines():
        m = re.search(r"Function properties for (\S+)", line)
        if m:
            name = m.group(1)
            res[name] = {"spill": 0, "regs": None}
            continue
        if name is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            res[name]["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            res[name]["regs"] = int(m.group(1))
    return res


def test_hot_kernels_do_not_spill(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    sources = sorted({src for src, _ in HOT.values()})
    with ThreadPoolExecutor(len(sources)) as ex:
        found = dict(zip(sources, ex.map(lambda s: _resources(nvcc, s, str(tmp_path)), sources)))
    for key, (src, max_regs) in HOT.items():
        names = [n for n in found[src] if key in n and "batched" not in n]
        assert names, f"{key} not compiled from {src}"
        for n in names:
            r = found[src][n]
            assert r["spill"] == 0, f"{n} spills {r['spill']} bytes"
            assert r["regs"] is not None and r["regs"] <= max_regs, f"{n} uses {r['regs']} registers"
