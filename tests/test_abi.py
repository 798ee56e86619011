"""libgi.so builds for sm_103a, loads without a GPU and exports every entry
point that include/gi.h declares; host-only entry points behave as the header
states (layout sizes, closed-form cell moments, argument validation before
any launch)."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2310_19855_gb300 as gi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gi.h")


@pytest.fixture(scope="module")
def lib():
    gi.build()
    return gi.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gi_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "gi_cache_update" in names and "gi_probes_interpolate" in names
    for name in names:
        assert hasattr(lib, name), name


STRUCTS = ["gi_cache_config", "gi_view", "gi_hits", "gi_gbuffer", "gi_probe_layout", "gi_probes",
           "gi_cache_stats_t", "gi_cell", "gi_tile", "gi_query", "gi_batch_tuning", "gi_batch_view", "gi_nrc_config",
           "gi_points", "gi_nrc_stats_t"]


def test_struct_layouts_match_the_c_header(tmp_path):
    # sizeof and every field offset as the C compiler lays them out, against the ctypes mirror
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gi.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in getattr(gi, name)._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split(" ") for line in out if line)
    for name in STRUCTS:
        cls = getattr(gi, name)
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def test_status_strings(lib):
    assert lib.gi_status_string(gi.GI_ERR_INVALID_ARG) == b"GI_ERR_INVALID_ARG"
    assert lib.gi_status_string(gi.GI_WARN_DROPPED) == b"GI_WARN_DROPPED"
    assert lib.gi_version() >= 100


def test_probe_layout(lib):
    lay = gi.gi_probes_layout(1920, 1080)
    assert (lay.tiles_x, lay.tiles_y, lay.num_probes) == (240, 135, 32400)
    dims = [(lay.mip_w[k], lay.mip_h[k]) for k in range(lay.mip_count)]
    assert dims == [(240, 135), (120, 68), (60, 34), (30, 17), (15, 9), (8, 5), (4, 3), (2, 2), (1, 1)]
    assert lay.mask_words == sum(w * h for w, h in dims)
    assert lay.mip_offset[3] == 240 * 135 + 120 * 68 + 60 * 34
    lay = gi.gi_probes_layout(3, 5)
    assert (lay.tiles_x, lay.tiles_y, lay.mip_count) == (1, 1, 1)


def test_cell_moments_match_oracle_quadrature(lib):
    from oracle import hemioct
    om, m1, m2 = hemioct.moments()
    m = gi.gi_cell_moments()
    assert np.abs(m[:, 0] - om).max() < 1e-13
    assert np.abs(m[:, 1:4] - m1).max() < 1e-13
    for col, (i, j) in zip(range(4, 10), [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        assert np.abs(m[:, col] - m2[:, i, j]).max() < 1e-13
    assert abs(m[:, 0].sum() - 2 * math.pi) < 1e-12


def test_invalid_arguments_are_rejected_on_the_host(lib):
    h = ctypes.c_void_p()
    bad = gi.gi_cache_config(40, 0.05, 4, 0.1, 8, 128, 0, 0, 0.8, 0)
    assert lib.gi_cache_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    assert b"configuration" in lib.gi_last_error()
    bad = gi.gi_cache_config(16, 0.05, 4, 0.1, 8, 300, 0, 0, 0.8, 0)  # probe runs must stay below 256
    assert lib.gi_cache_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    bad = gi.gi_cache_config(16, -1.0, 4, 0.1, 8, 128, 0, 0, 0.8, 0)
    assert lib.gi_cache_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    bad = gi.gi_cache_config(16, 0.05, 4, 0.1, 8, 128, 0, 0, 0.8, 3)  # unknown first-touch record
    assert lib.gi_cache_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    bad = gi.gi_cache_config(16, 0.05, 4, 0.1, 8, 128, 0, 0, 0.8, 0, 0, 16, 2)  # unknown merge form
    assert lib.gi_cache_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    # tile caches: at most 2^22 tiles, first touches always listed, min_samples >= 1, tiles in {0, 1}
    for bad in (gi.gi_cache_config(23, 0.05, 4, 0.1, 8, 128, 0, 0, 0.8, 0, 1, 16),
                gi.gi_cache_config(16, 0.05, 4, 0.1, 8, 128, 0, 0, 0.8, gi.GI_FIRST_TOUCH_BITMAP, 1, 16),
                gi.gi_cache_config(16, 0.05, 4, 0.1, 8, 128, 0, 0, 0.8, 0, 1, 0),
                gi.gi_cache_config(16, 0.05, 4, 0.1, 8, 128, 0, 0, 0.8, 0, 2, 16)):
        assert lib.gi_cache_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    cnt = ctypes.c_uint64()
    assert lib.gi_cache_export_tiles(None, None, 0, ctypes.byref(cnt), None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_cache_create(None, ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_cache_update(None, None, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_cache_resolve(None, 0, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_cache_stats(None, None, None) == gi.GI_ERR_INVALID_ARG
    lay = gi.gi_probe_layout()
    assert lib.gi_probes_layout(0, 10, ctypes.byref(lay)) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_probes_spawn(None, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_probes_interpolate(None, None, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_cell_moments(None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_cache_destroy(None) == gi.GI_OK
    assert lib.gi_probes_gather(None, None, None, None, 64, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_probes_filter(None, None, None, None, 0, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_probes_project(None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_diag_update_atomics(None, 0, 9, 0, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_diag_update_atomics(None, 0, 31, 0, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_diag_update_atomics(None, 0, 16, 3, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_diag_update_atomics(None, 16, 16, 0, None, None, None) == gi.GI_ERR_INVALID_ARG


def test_surrogate_arguments_are_rejected_on_the_host(lib):
    h = ctypes.c_void_p()
    good = gi.make_nrc_config((-1, 0, -1), (1, 2, 1))
    for field, value in (("log2_table", 30), ("batch", 64), ("lr", 0.0), ("beta2", 1.0), ("loss_eps", 0.0)):
        bad = gi.make_nrc_config((-1, 0, -1), (1, 2, 1))
        setattr(bad, field, value)
        assert lib.gi_nrc_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG, field
    bad = gi.make_nrc_config((-1, 0, -1), (1, 0, 1))  # empty box
    assert lib.gi_nrc_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    bad = gi.make_nrc_config((-1, 0, -1), (1, 2, 1), resolutions=(0,) + gi.default_resolutions()[1:])
    assert lib.gi_nrc_create(ctypes.byref(bad), ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    assert good.resolution[15] == 2048 and good.resolution[0] == 16
    assert lib.gi_nrc_create(None, ctypes.byref(h)) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_infer(None, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_backward(None, None, None, None, 0, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_adam(None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_train_frame(None, None, None, None, 0, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_query_frame(None, None, None, None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_probes_integrate_nrc(None, None, None, None, 64, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_stats(None, None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_batch_set_surrogate(None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_batch_set_view_surrogates(None, None) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_set_learning_rate(None, 1e-3) == gi.GI_ERR_INVALID_ARG
    assert lib.gi_nrc_destroy(None) == gi.GI_OK
