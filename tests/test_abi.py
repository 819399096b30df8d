"""The C-ABI library builds, loads without a GPU, exports every entry point
include/air.h declares, and the Python binding's structures match the C
layouts (sizes and field offsets from a gcc-compiled probe). No compute calls."""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

import paper_1010_5534_gb300 as air

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "air.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"AIR_API\s+[\w\s\*]*?\b(air_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    air.build()
    return air.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(air.EXPORTED) == names
    out = subprocess.run(["nm", "-D", "--defined-only", air.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (air_\w+)", out))
    assert set(names) <= exported


def test_version_and_error_string(lib):
    assert "sm_103a" in air.version()
    assert lib.air_last_error() == b""


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # argument checks run before any CUDA call
    h = C.c_void_p()
    assert lib.air_load_grid(None, None, C.byref(h)) == air.AIR_ERR_ARG
    assert b"NULL" in lib.air_last_error()
    assert lib.air_render_fixed(None, None, 4, -1, None) == air.AIR_ERR_ARG
    assert lib.air_render_adaptive(None, None, None, None) == air.AIR_ERR_ARG
    assert lib.air_profile_enable(None, 1) == air.AIR_ERR_ARG
    lib.air_free(None)


PROBE = r'''
#include <stdio.h>
#include <stddef.h>
#include "air.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("air_grid_desc %zu\n", sizeof(air_grid_desc));
  printf("air_view %zu\n", sizeof(air_view));
  printf("air_params %zu\n", sizeof(air_params));
  printf("air_image %zu\n", sizeof(air_image));
  F(air_grid_desc, kind) F(air_grid_desc, n) F(air_grid_desc, lo) F(air_grid_desc, hi)
  F(air_grid_desc, brick) F(air_grid_desc, max_level) F(air_grid_desc, n_bricks)
  F(air_grid_desc, brick_level) F(air_grid_desc, brick_origin) F(air_grid_desc, field_dtype)
  F(air_grid_desc, rho) F(air_grid_desc, temp) F(air_grid_desc, n_bands)
  F(air_grid_desc, emis_mode) F(air_grid_desc, lambda_table) F(air_grid_desc, n_tbins)
  F(air_grid_desc, logT_lo) F(air_grid_desc, logT_hi) F(air_grid_desc, kappa)
  F(air_view, dir) F(air_view, up) F(air_view, center) F(air_view, half_extent)
  F(air_params, base_res) F(air_params, max_level) F(air_params, xi_crit)
  F(air_params, xi_norm) F(air_params, refine_on) F(air_params, fp64_level)
  F(air_params, include_interior)
  F(air_image, mem) F(air_image, capacity) F(air_image, n_out) F(air_image, n_leaves)
  F(air_image, n_rays) F(air_image, n_steps) F(air_image, n_sweeps) F(air_image, level)
  F(air_image, i) F(air_image, j) F(air_image, is_leaf) F(air_image, coldens)
  F(air_image, intensity) F(air_image, p) F(air_image, band_flux)
  printf("air_batch_opts %zu\n", sizeof(air_batch_opts));
  F(air_batch_opts, bands_per_thread) F(air_batch_opts, use_graph)
  F(air_batch_opts, wait_timeout_ms) F(air_batch_opts, test_stall_barrier)
  printf("air_learned_opts %zu\n", sizeof(air_learned_opts));
  F(air_learned_opts, quantile)
  printf("air_learned_stats %zu\n", sizeof(air_learned_stats));
  F(air_learned_stats, proposed_rays) F(air_learned_stats, used_rays)
  F(air_learned_stats, wasted_rays) F(air_learned_stats, fallback_rays)
  F(air_learned_stats, waves) F(air_learned_stats, sweeps)
  F(air_learned_stats, under_predicted) F(air_learned_stats, over_predicted)
  printf("air_tuning %zu\n", sizeof(air_tuning));
  F(air_tuning, tile_w) F(air_tuning, bands_per_thread) F(air_tuning, batch_bands_per_thread)
  F(air_tuning, batch_blocks_per_sm) F(air_tuning, best_ms) F(air_tuning, trials)
  printf("AIR_MLP_NPARAMS %d\n", AIR_MLP_NPARAMS);
  return 0;
}
'''


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "probe.c"
    src.write_text(PROBE)
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in lines if l.strip())
    mapping = {"air_grid_desc": air.GridDesc, "air_view": air.View, "air_params": air.Params,
               "air_image": air.Image, "air_batch_opts": air.BatchOpts,
               "air_learned_opts": air.LearnedOpts, "air_learned_stats": air.LearnedStats,
               "air_tuning": air.Tuning}
    assert int(got["AIR_MLP_NPARAMS"]) == air.MLP_NPARAMS
    for cname, cls in mapping.items():
        assert C.sizeof(cls) == int(got[cname]), cname
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == int(got[f"{cname}.{f}"]), (cname, f)


def test_caller_output_arrays_are_checked_on_the_host():
    """Grid._image_of (the out= path of render_adaptive) builds the Image from
    caller-held arrays: capacity = the shortest per-node array, pointers set,
    and wrong dtypes, shapes or memory kinds rejected before any call."""
    import types

    import torch
    fake = types.SimpleNamespace(n_bands=2)
    n = 11
    out = dict(level=torch.zeros(n, dtype=torch.int32), i=torch.zeros(n + 3, dtype=torch.int32),
               coldens=torch.zeros(n, dtype=torch.float32),
               intensity=torch.zeros((2, n + 1), dtype=torch.float32),
               band_flux=torch.zeros(2, dtype=torch.float64))
    im = air.Grid._image_of(fake, out, "host")
    assert im.mem == air.AIR_HOST and im.capacity == n
    assert im.level == out["level"].data_ptr() and im.intensity == out["intensity"].data_ptr()
    assert not im.j and not im.p
    bad = [dict(out, level=torch.zeros(n, dtype=torch.int64)),
           dict(out, intensity=torch.zeros((3, n), dtype=torch.float32)),
           dict(out, band_flux=torch.zeros(1, dtype=torch.float64)),
           dict(out, coldens=torch.zeros((n, 2), dtype=torch.float32)[:, 0]),
           dict(out, bogus=torch.zeros(n))]
    for o in bad:
        with pytest.raises(ValueError):
            air.Grid._image_of(fake, o, "host")
    with pytest.raises(ValueError):
        air.Grid._image_of(fake, out, "device")   # host tensors for device outputs
