"""The C ABI without a GPU: the library loads, exports every call include/gsrf.h
declares, its struct layouts match the ctypes mirrors, and its host-side argument
checks and workspace sizing behave.  No kernel is launched here."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2502_01826_gb300 import _build, _lib as L
from paper_2502_01826_gb300.render import make_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsrf.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return L.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsrf_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(L.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _build.SO], capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(r"\bT %s\b" % name, out), name
    assert lib.gsrf_version().startswith(b"gsrf-gb300")


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "gsrf.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(gsrf_grid), sizeof(gsrf_gaussians), sizeof(gsrf_plan),
         sizeof(gsrf_layout), sizeof(gsrf_run_status));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", offsetof(gsrf_plan, f0_hz), offsetof(gsrf_plan, grid),
         offsetof(gsrf_plan, pair_capacity), offsetof(gsrf_run_status, stats), offsetof(gsrf_layout, view),
         offsetof(gsrf_plan, ray_block_w), offsetof(gsrf_plan, stage), offsetof(gsrf_plan, ckpt_every),
         offsetof(gsrf_plan, ckpt_slots), offsetof(gsrf_plan, variant), offsetof(gsrf_plan, fle_degree));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    assert sizes == [C.sizeof(L.gsrf_grid), C.sizeof(L.gsrf_gaussians), C.sizeof(L.gsrf_plan),
                     C.sizeof(L.gsrf_layout), C.sizeof(L.gsrf_run_status)]
    assert offs == [L.gsrf_plan.f0_hz.offset, L.gsrf_plan.grid.offset, L.gsrf_plan.pair_capacity.offset,
                    L.gsrf_run_status.stats.offset, L.gsrf_layout.view.offset, L.gsrf_plan.ray_block_w.offset,
                    L.gsrf_plan.stage.offset, L.gsrf_plan.ckpt_every.offset, L.gsrf_plan.ckpt_slots.offset,
                    L.gsrf_plan.variant.offset, L.gsrf_plan.fle_degree.offset]


def plan(n=1000, n_rx=4, n_az=360, n_el=90, cap=100000, **kw):
    return L.gsrf_plan(n, n_rx, kw.get("n_f", 1), kw.get("f0", 2.4e9), kw.get("df", 0.0),
                       make_grid(n_az, n_el, **kw.get("grid", {})), cap)


def test_workspace_size_grows_with_problem(lib):
    a, b = C.c_size_t(), C.c_size_t()
    assert lib.gsrf_workspace_size(C.byref(plan()), C.byref(a)) == L.GSRF_OK
    assert lib.gsrf_workspace_size(C.byref(plan(n=2000)), C.byref(b)) == L.GSRF_OK
    assert b.value > a.value > 0
    assert lib.gsrf_workspace_size(C.byref(plan(cap=200000)), C.byref(b)) == L.GSRF_OK
    # per pair of capacity: the 64-bit keys (inspection), the tile indices and two id buffers
    assert b.value >= a.value + 100000 * 20
    lay = L.gsrf_layout()
    assert lib.gsrf_workspace_layout(C.byref(plan()), C.byref(lay)) == L.GSRF_OK
    assert (lay.n_tiles_u, lay.n_tiles_v) == (23, 6)
    assert lay.status == 0 and lay.pair_keys % 256 == 0 and lay.tile_start % 256 == 0
    assert lib.gsrf_ray_state_bytes(C.byref(plan())) == 4 * 360 * 90 * 32


@pytest.mark.parametrize("bad", [
    dict(n=-1), dict(n_rx=0), dict(n_f=0), dict(n_f=65), dict(f0=0.0), dict(cap=-5),
    dict(n_az=0, grid=dict(daz_deg=1.0)), dict(grid=dict(daz_deg=0.0)), dict(grid=dict(alpha_max=1.0)),
    dict(grid=dict(eps_T=-1.0)), dict(grid=dict(az0_deg=400.0)),
])
def test_invalid_plans_rejected_synchronously(lib, bad):
    kw = dict(bad)
    p = plan(**{k: v for k, v in kw.items() if k in ("n", "n_rx", "n_az", "n_el", "cap")},
             **{k: v for k, v in kw.items() if k in ("n_f", "f0", "grid")})
    sz = C.c_size_t()
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_INVALID_ARG


def test_unsupported_configurations(lib):
    sz = C.c_size_t()
    for tw, th in ((12, 16), (16, 12), (64, 16), (8, 2)):  # tile sides outside 8|16|32 x 4|8|16|32
        p = plan(grid=dict(tile_w=tw, tile_h=th))
        assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_UNSUPPORTED, (tw, th)
    p = plan(n_az=2000)  # more than 64 azimuth tiles
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_UNSUPPORTED
    p = plan(grid=dict(tile_w=8, tile_h=16))
    p.ray_block_w = 16  # a 16 x 2 ray block does not tile an 8-wide tile
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_UNSUPPORTED
    p = plan(grid=dict(tile_w=32, tile_h=4))
    p.ray_block_w = 4  # a 4 x 8 ray block does not tile a 4-high tile
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_UNSUPPORTED


@pytest.mark.parametrize("tw,th,bw,stage", [(8, 16, 8, 16), (32, 8, 32, 32), (16, 16, 4, 0), (32, 32, 16, 16),
                                            (16, 4, 8, 32)])
def test_tile_shapes_ray_blocks_and_stages_accepted(lib, tw, th, bw, stage):
    sz = C.c_size_t()
    p = plan(grid=dict(tile_w=tw, tile_h=th))
    p.ray_block_w, p.stage = bw, stage
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_OK
    lay = L.gsrf_layout()
    assert lib.gsrf_workspace_layout(C.byref(p), C.byref(lay)) == L.GSRF_OK
    assert (lay.n_tiles_u, lay.n_tiles_v) == (-(-360 // tw), -(-90 // th))


@pytest.mark.parametrize("fields", [dict(ray_block_w=2), dict(ray_block_w=12), dict(ray_block_w=64),
                                    dict(stage=8), dict(stage=24), dict(stage=-1), dict(ckpt_every=48, ckpt_slots=4),
                                    dict(ckpt_every=-32, ckpt_slots=4), dict(ckpt_every=64, ckpt_slots=0),
                                    dict(ckpt_every=64, ckpt_slots=65), dict(variant=32), dict(variant=-1),
                                    dict(fle_degree=6), dict(fle_degree=-1)])
def test_bad_ray_block_stage_or_checkpoints_rejected(lib, fields):
    sz = C.c_size_t()
    p = plan()
    for k, v in fields.items():
        setattr(p, k, v)
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_INVALID_ARG


def test_ray_state_grows_with_checkpoints(lib):
    p = plan()
    base = lib.gsrf_ray_state_bytes(C.byref(p))
    p.ckpt_every, p.ckpt_slots = 256, 6
    assert lib.gsrf_ray_state_bytes(C.byref(p)) == base + 4 * 360 * 90 * 6 * 16


def test_calls_reject_bad_pointers_before_launch(lib):
    p = plan()
    g = L.gsrf_gaussians(1000, None, None, None, None, None, None)
    sz = C.c_size_t()
    lib.gsrf_workspace_size(C.byref(p), C.byref(sz))
    # null workspace, misaligned workspace, short workspace, null Gaussians
    assert lib.gsrf_project(C.byref(p), C.byref(g), C.c_void_p(256), C.c_void_p(256), None, sz.value,
                            None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_bin(C.byref(p), C.c_void_p(4096 + 8), sz.value, None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_bin(C.byref(p), C.c_void_p(4096), sz.value - 1, None) == L.GSRF_ERR_INVALID_ARG
    # the inspection call takes the same checks as the bin
    assert lib.gsrf_pair_keys(C.byref(p), None, sz.value, None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_pair_keys(C.byref(p), C.c_void_p(4096 + 8), sz.value, None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_pair_keys(C.byref(p), C.c_void_p(4096), sz.value - 1, None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_pair_keys(None, C.c_void_p(4096), sz.value, None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_project(C.byref(p), C.byref(g), C.c_void_p(256), C.c_void_p(256), C.c_void_p(4096),
                            sz.value, None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_received_signal(None, 1, 1, 1, 1, 0, None, None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_received_signal(C.c_void_p(256), 1, 1, 1, 1, 9, C.c_void_p(256), None) == \
        L.GSRF_ERR_INVALID_ARG


def test_autotune_sizing_and_argument_checks(lib):
    p = plan()
    a, b = C.c_size_t(), C.c_size_t()
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(a)) == L.GSRF_OK
    assert lib.gsrf_autotune_workspace_size(C.byref(p), C.byref(b)) == L.GSRF_OK
    assert b.value >= a.value
    for tw, th in ((32, 8), (8, 8), (32, 32)):  # every candidate tile shape fits the tuner's workspace
        q = plan(grid=dict(tile_w=tw, tile_h=th))
        assert lib.gsrf_workspace_size(C.byref(q), C.byref(a)) == L.GSRF_OK
        assert b.value >= a.value
    g = L.gsrf_gaussians(1000, None, None, None, None, None, None)
    best = L.gsrf_tune_result()
    res = (L.gsrf_tune_result * 4)()
    n = C.c_int32()
    dev = C.c_void_p(4096)
    # null workspace, zero repetitions, results wanted without a buffer, no best
    assert lib.gsrf_autotune(C.byref(p), C.byref(g), dev, dev, None, b.value, dev, None, 3, res, 4, C.byref(n),
                             C.byref(best), None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_autotune(C.byref(p), C.byref(g), dev, dev, dev, b.value, dev, None, 0, res, 4, C.byref(n),
                             C.byref(best), None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_autotune(C.byref(p), C.byref(g), dev, dev, dev, b.value, dev, None, 3, None, 4, C.byref(n),
                             C.byref(best), None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_autotune(C.byref(p), C.byref(g), dev, dev, dev, b.value, dev, None, 3, res, 4, C.byref(n),
                             None, None) == L.GSRF_ERR_INVALID_ARG
    bwd = L.gsrf_tune_backward(None, 4096, None, None, None, None, None, None)  # no ray state
    assert lib.gsrf_autotune(C.byref(p), C.byref(g), dev, dev, dev, b.value, dev, C.byref(bwd), 3, res, 4,
                             C.byref(n), C.byref(best), None) == L.GSRF_ERR_INVALID_ARG


def test_backward_refuses_variant_readings(lib):
    """The backward has the default reading, the normalised weight and the paper's circle
    culling (GPU tests); the radiance at the mean, the path through x_rep and the t_mid
    order are refused before any launch."""
    dev = C.c_void_p(1 << 20)
    g = L.gsrf_gaussians(1000, dev, dev, dev, dev, dev, None)
    for v in (L.VARIANT_RADIANCE_AT_MEAN, L.VARIANT_PATH_AT_REP, L.VARIANT_ORDER_T_MID,
              L.VARIANT_RADIANCE_AT_MEAN | L.VARIANT_NORMALISED_WEIGHT):
        p = plan()
        p.variant = v
        sz = C.c_size_t()
        assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_OK  # the forward takes it
        assert lib.gsrf_render_bwd(C.byref(p), C.byref(g), dev, sz.value, dev, dev, None, None, None, None,
                                   None, None, None) == L.GSRF_ERR_UNSUPPORTED


def test_other_fle_degrees_are_single_frequency(lib):
    """Degrees 1..5 size the coefficient and ray tables (and the backward's accumulators)
    by L; only L = 3 has several subcarriers, the batched render and the
    radiance-at-the-mean variant.  (The backward runs at every degree: GPU tests.)"""
    sizes = []
    for deg in (1, 2, 0, 4, 5):
        p = plan()
        p.fle_degree = deg
        sz = C.c_size_t()
        assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_OK
        sizes.append(sz.value)
    assert sizes == sorted(sizes) and len(set(sizes)) == 5
    for bad in (dict(n_f=4), dict(variant=L.VARIANT_RADIANCE_AT_MEAN)):
        p = plan(n_f=bad.get("n_f", 1))
        p.fle_degree = 5
        p.variant = bad.get("variant", 0)
        sz = C.c_size_t()
        assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_UNSUPPORTED


def test_path_variant_is_single_frequency_degree_three(lib):
    for kw in (dict(n_f=4), dict(fle_degree=2)):
        p = plan(n_f=kw.get("n_f", 1))
        p.variant = L.VARIANT_PATH_AT_REP
        p.fle_degree = kw.get("fle_degree", 0)
        sz = C.c_size_t()
        assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_UNSUPPORTED, kw


def test_tmid_order_variant_limits(lib):
    for kw in (dict(n_f=4), dict(fle_degree=2), dict(extra=L.VARIANT_PATH_AT_REP)):
        p = plan(n_f=kw.get("n_f", 1))
        p.variant = L.VARIANT_ORDER_T_MID | kw.get("extra", 0)
        p.fle_degree = kw.get("fle_degree", 0)
        sz = C.c_size_t()
        assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_ERR_UNSUPPORTED, kw
    a, b = C.c_size_t(), C.c_size_t()
    p = plan()
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(a)) == L.GSRF_OK
    p.variant = L.VARIANT_ORDER_T_MID
    assert lib.gsrf_workspace_size(C.byref(p), C.byref(b)) == L.GSRF_OK
    assert b.value >= a.value + 4 * 360 * 90 * 512 * 8  # the per-ray hit keys


def test_batch_and_tuned_backward_refuse_the_forward_only_readings(lib):
    """The batched render takes only the default degree and no per-pair path or t_mid
    order; the tuner times no backward for a reading the backward does not have.  Both
    refuse before touching the (fake, aligned) device pointers."""
    dev = C.c_void_p(1 << 20)
    for field, value in (("fle_degree", 2), ("variant", L.VARIANT_PATH_AT_REP), ("variant", L.VARIANT_ORDER_T_MID)):
        p = plan()
        setattr(p, field, value)
        sz, bsz = C.c_size_t(), C.c_size_t()
        assert lib.gsrf_workspace_size(C.byref(p), C.byref(sz)) == L.GSRF_OK
        plans = (L.gsrf_plan * 1)(p)
        assert lib.gsrf_batch_workspace_size(1, plans, C.byref(bsz)) == L.GSRF_OK
        wss = (C.c_void_p * 1)(dev)
        sizes = (C.c_size_t * 1)(sz.value)
        outs = (C.c_void_p * 1)(dev)
        assert lib.gsrf_render_batch(1, plans, wss, sizes, outs, dev, bsz.value, None, 0, None) == L.GSRF_ERR_UNSUPPORTED
    p = plan()
    p.variant = L.VARIANT_RADIANCE_AT_MEAN
    tsz = C.c_size_t()
    assert lib.gsrf_autotune_workspace_size(C.byref(p), C.byref(tsz)) == L.GSRF_OK
    g = L.gsrf_gaussians(1000, dev, dev, dev, dev, dev, None)
    bwd = L.gsrf_tune_backward(dev, dev, dev, dev, dev, dev, dev, None)
    best = L.gsrf_tune_result()
    n = C.c_int32()
    assert lib.gsrf_autotune(C.byref(p), C.byref(g), dev, dev, dev, tsz.value, dev, C.byref(bwd), 3, None, 0,
                             C.byref(n), C.byref(best), None) == L.GSRF_ERR_UNSUPPORTED


def test_stage_times_argument_checks(lib):
    # no CUDA call is reached: a workspace no stage was recorded on is refused first
    ms = (C.c_float * 8)()
    assert lib.gsrf_stage_times(None, ms) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_stage_times(C.c_void_p(4096), None) == L.GSRF_ERR_INVALID_ARG
    assert lib.gsrf_stage_times(C.c_void_p(4096), ms) == L.GSRF_ERR_INVALID_ARG
