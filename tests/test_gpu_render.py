"""GPU parity of the forward path (project -> bin -> render -> received signal)
against the FP64 oracle, through the C ABI.

Bars: splat keys, per-tile id lists and tile ranges bit-exact; per-ray complex signal
within 1e-4 relative L2, and per ray within 1e-4 of its sum of contribution magnitudes
plus its FP32 conditioning (see gpu_util); RSSI within 0.01 dB.  A ray on which FP32 and
FP64 may take one discrete decision differently must match the oracle with that
decision taken either way; rays with more are excluded (counted, at most 2%)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2502_01826_gb300 import _lib as L
from paper_2502_01826_gb300 import synthetic
from paper_2502_01826_gb300.render import Renderer, make_grid, received_signal, to_device

from gpu_util import (BANDS, TOL_DB, compare, gpu_render, oracle_grid, oracle_pair, require_gpu,
                      rssi_db)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    oracle.build()


def oracle_render(scene, rx, tx, f0, spec, rays=None, **kw):
    g = oracle_grid(spec, **kw)
    return oracle_pair(scene, rx, tx, f0, g, rays=rays)


def check_bins(R: Renderer, scene, rx_all, spec, **kw):
    """Keys, ids and tile ranges of every receiver equal the oracle's, bit for bit."""
    keys, ids, rb, ts = R.pairs()
    keys = keys.cpu().numpy().view(np.uint64)
    ids = ids.cpu().numpy().view(np.uint32)
    rb = rb.cpu().numpy()
    ts = ts.cpu().numpy()
    g = oracle_grid(spec, **kw)
    for r in range(rx_all.shape[0]):
        k_ref, i_ref, t_ref = oracle.bin_pairs(scene, rx_all[r], g)
        assert rb[r + 1] - rb[r] == len(k_ref)
        assert np.array_equal(keys[rb[r]:rb[r + 1]], k_ref), "keys differ for receiver %d" % r
        assert np.array_equal(ids[rb[r]:rb[r + 1]], i_ref), "ids differ for receiver %d" % r
        assert np.array_equal(ts[r].astype(np.int64), t_ref), "tile ranges differ for receiver %d" % r


# --------------------------------------------------------------------------- C1

def test_plain_forward_2k_matches_oracle():
    cfg = synthetic.config_plain()
    S, R, p, out = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"])
    ref = oracle_render(cfg["scene"], cfg["rx"][0], cfg["tx"], cfg["f0"], cfg["grid"])
    compare(S[0], ref)
    check_bins(R, cfg["scene"], cfg["rx"], cfg["grid"])
    # received signal through the library's reduction vs the oracle's coherent sum
    db = received_signal(out, L.SIG_RSSI_DB).cpu().numpy()[0, 0]
    assert abs(db - rssi_db(ref["S"][0])) <= TOL_DB
    # statistics: candidate tests and composited pairs
    st = R.status()
    assert st.code == 0
    assert abs(st.stats[0] - ref["ntest"].sum()) <= 0.01 * ref["ntest"].sum()
    assert abs(st.stats[1] - ref["nhit"].sum()) <= 0.01 * ref["nhit"].sum()


@pytest.mark.parametrize("eps_T", [0.0, 1e-2])
def test_plain_forward_termination_settings(eps_T):
    cfg = synthetic.config_plain()
    S, R, p, out = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"], eps_T=eps_T)
    ref = oracle_render(cfg["scene"], cfg["rx"][0], cfg["tx"], cfg["f0"], cfg["grid"], eps_T=eps_T)
    compare(S[0], ref)


# --------------------------------------------------------------------------- grids, receivers

@pytest.mark.parametrize("spec", [
    dict(n_az=30, n_el=7, az0_deg=10.0, daz_deg=9.0, el0_deg=-20.0, del_deg=7.0),  # ragged, offset
    dict(n_az=100, n_el=37, az0_deg=-45.0, daz_deg=1.7, el0_deg=-30.0, del_deg=2.5),
    dict(n_az=72, n_el=18),
    dict(n_az=180, n_el=45),
])
def test_grids_and_receivers(spec):
    scene = synthetic.tiny_scene(400, 101, box=(6.0, 5.0, 3.0), log_scale_mu=math.log(0.2))
    rng = np.random.default_rng(3)
    rx = (rng.uniform(0, 1, (3, 3)) * [6.0, 5.0, 3.0]).astype(np.float32)
    tx = np.array([0.5, 4.5, 2.5], np.float32)
    S, R, p, out = gpu_render(scene, rx, tx, 2.4e9, spec)
    check_bins(R, scene, rx, spec)
    for r in range(3):
        ref = oracle_render(scene, rx[r], tx, 2.4e9, spec)
        compare(S[r], ref)


def test_gaussians_around_the_receiver():
    """Gaussians enclosing the receiver, straddling the emitting sphere, inside it."""
    scene = synthetic.tiny_scene(300, 102, box=(3.0, 3.0, 2.0), log_scale_mu=math.log(0.4))
    rx = np.array([[1.5, 1.5, 1.0]], np.float32)
    scene["means"][:5] = rx[0] + np.array([[0, 0, 0], [0.3, 0, 0], [0, 0.9, 0.1], [1.0, 0, 0.2],
                                           [0, 0, 0.5]], np.float32)
    tx = np.array([0.2, 2.8, 0.3], np.float32)
    spec = dict(n_az=72, n_el=18)
    S, R, p, out = gpu_render(scene, rx, tx, 915e6, spec)
    check_bins(R, scene, rx, spec)
    ref = oracle_render(scene, rx[0], tx, 915e6, spec)
    compare(S[0], ref)


# --------------------------------------------------------------------------- edge cases

def test_empty_scene_gives_zero():
    scene = synthetic.tiny_scene(0, 1)
    S, R, p, out = gpu_render(scene, [[1, 1, 1]], [2, 2, 2], 2.4e9, dict(n_az=36, n_el=9), cap=0)
    assert np.all(S == 0)
    assert R.status().code == 0


def test_zero_opacity_gives_zero():
    scene = synthetic.tiny_scene(200, 103)
    scene["opacity_logit"][:] = -1e4
    S, R, p, out = gpu_render(scene, [[2, 2, 1]], [1, 1, 1], 2.4e9, dict(n_az=72, n_el=18))
    assert np.all(S == 0)


def test_single_gaussian():
    scene = synthetic.tiny_scene(1, 104)
    scene["means"][0] = [3.0, 2.0, 1.5]
    rx = np.array([[1.0, 1.0, 1.0]], np.float32)
    S, R, p, out = gpu_render(scene, rx, [0.5, 0.5, 0.5], 2.4e9, dict(n_az=360, n_el=90))
    ref = oracle_render(scene, rx[0], np.array([0.5, 0.5, 0.5], np.float32), 2.4e9, dict(n_az=360, n_el=90))
    assert np.count_nonzero(ref["S"][0]) > 20
    compare(S[0], ref)


def test_capacity_overflow_reports_required_pairs():
    cfg = synthetic.config_plain()
    g = oracle_grid(cfg["grid"])
    total = len(oracle.bin_pairs(cfg["scene"], cfg["rx"][0], g)[0])
    S, R, p, out = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"], cap=total - 1)
    st = R.status()
    assert st.code == L.GSRF_ERR_CAPACITY and st.required_pairs == total
    assert np.all(S == 0)
    S2, R2, _, _ = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"], cap=total)
    assert R2.status().code == 0 and np.count_nonzero(S2) > 0


def test_nonfinite_parameter_is_reported():
    scene = synthetic.tiny_scene(100, 105)
    scene["means"][37, 1] = np.nan
    scene["coeffs"][60, 3, 1] = np.inf
    S, R, p, out = gpu_render(scene, [[2, 2, 1]], [1, 1, 1], 2.4e9, dict(n_az=36, n_el=9), cap=100000)
    st = R.status()
    assert st.code == L.GSRF_ERR_NONFINITE and st.first_bad == 37


def test_render_is_deterministic():
    cfg = synthetic.config_plain()
    a = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"])[0]
    b = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"])[0]
    assert np.array_equal(a, b)


def test_received_signal_modes_match_fp64_sums():
    cfg = synthetic.config_plain()
    S, R, p, out = gpu_render(cfg["scene"], np.repeat(cfg["rx"], 3, 0) + np.float32([[0, 0, 0], [0.5, 0, 0],
                                                                                      [0, 0.5, 0.2]]),
                              cfg["tx"], cfg["f0"], cfg["grid"])
    Sd = S.astype(np.complex128)
    cs = received_signal(out, L.SIG_COMPLEX_SUM).cpu().numpy()
    assert np.allclose(cs[:, 0, 0] + 1j * cs[:, 0, 1], Sd.sum(1), rtol=1e-6, atol=1e-7)
    db = received_signal(out, L.SIG_RSSI_DB).cpu().numpy()[:, 0]
    assert np.allclose(db, 20 * np.log10(np.abs(Sd.sum(1))), atol=1e-4)
    pw = received_signal(out, L.SIG_POWER_SUM).cpu().numpy()[:, 0]
    assert np.allclose(pw, (np.abs(Sd) ** 2).sum(1), rtol=1e-6)
    mg = received_signal(out, L.SIG_SPECTRUM_MAG).cpu().numpy()
    assert np.allclose(mg.reshape(3, -1), np.abs(S), rtol=1e-6, atol=1e-9)


# --------------------------------------------------------------------------- full size

def test_ble_50k_64rx_full_size_sampled():
    """The benchmark's workload in its launch configuration: all 64 receivers in one
    call; bins of two receivers bit-exact, 400 sampled rays of four receivers and the
    RSSI of two receivers against the oracle."""
    cfg = synthetic.config_ble()
    S, R, p, out = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"])
    n_rays = S.shape[1]
    rng = np.random.default_rng(7)
    keys, ids, rb, ts = R.pairs()
    rb = rb.cpu().numpy()
    g = oracle_grid(cfg["grid"])
    for r in (0, 63):
        k_ref, i_ref, t_ref = oracle.bin_pairs(cfg["scene"], cfg["rx"][r], g)
        assert np.array_equal(keys[rb[r]:rb[r + 1]].cpu().numpy().view(np.uint64), k_ref)
        assert np.array_equal(ids[rb[r]:rb[r + 1]].cpu().numpy().view(np.uint32), i_ref)
        assert np.array_equal(ts[r].cpu().numpy().astype(np.int64), t_ref)
    for r in (1, 17, 40, 62):
        rays = np.sort(rng.choice(n_rays, 400, replace=False)).astype(np.int32)
        ref = oracle_pair(cfg["scene"], cfg["rx"][r], cfg["tx"], cfg["f0"], g, rays=rays)
        compare(S[r, rays], ref)
    db = received_signal(out, L.SIG_RSSI_DB).cpu().numpy()[:, 0]
    for r in (5, 33):
        ref = oracle.render(cfg["scene"], cfg["rx"][r], cfg["tx"], cfg["f0"], g)
        assert abs(db[r] - rssi_db(ref["S"][0])) <= TOL_DB


@pytest.mark.parametrize("spec", [
    dict(n_az=360, n_el=180, el0_deg=-90.0, del_deg=1.0),  # 1 degree, the full sphere
    dict(n_az=720, n_el=180),                              # 0.5 degree, the front hemisphere
    dict(n_az=72, n_el=36, el0_deg=-90.0, del_deg=5.0),    # 5 degrees, the full sphere
])
def test_angular_resolutions_full_size(spec):
    """The BLE scene (50,000 Gaussians) at the angular resolutions of the paper's study,
    through the poles on the full sphere: bins of one receiver bit-exact, 300 sampled rays
    of two receivers against the oracle."""
    cfg = synthetic.config_ble()
    rx = cfg["rx"][:4]
    S, R, p, out = gpu_render(cfg["scene"], rx, cfg["tx"], cfg["f0"], spec)
    assert R.status().code == 0
    g = oracle_grid(spec)
    keys, ids, rb, ts = R.pairs()
    rb = rb.cpu().numpy()
    k_ref, i_ref, t_ref = oracle.bin_pairs(cfg["scene"], rx[2], g)
    assert np.array_equal(keys[rb[2]:rb[3]].cpu().numpy().view(np.uint64), k_ref)
    assert np.array_equal(ids[rb[2]:rb[3]].cpu().numpy().view(np.uint32), i_ref)
    rng = np.random.default_rng(13)
    for r in (0, 3):
        rays = np.sort(rng.choice(S.shape[1], 300, replace=False)).astype(np.int32)
        ref = oracle_pair(cfg["scene"], rx[r], cfg["tx"], cfg["f0"], g, rays=rays)
        compare(S[r, rays], ref)


# --------------------------------------------------------------------------- stage timers

def test_stage_times_report_each_stage_of_the_last_call():
    """gsrf_stage_times: every stage that ran on the workspace has a positive time, the
    forward's stages add up to about the time CUDA events see around the same calls, and a
    stage never run on this workspace is absent."""
    cfg = synthetic.config_ble(n_rx=4)
    K = cfg["scene"]["means"].shape[0]
    p = to_device(cfg["scene"])
    rx = torch.tensor(cfg["rx"], device="cuda")
    tx = torch.tensor(cfg["tx"], device="cuda")
    R = Renderer(K, rx.shape[0], make_grid(**cfg["grid"]), cfg["f0"])
    R.ensure_capacity(p, rx, tx)
    out = torch.empty(R.out_shape(), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    R.forward(p, rx, tx, out)  # warm
    a.record(s)
    R.project(p, rx, tx)
    R.bin()
    R.render_fwd(p, out)
    b.record(s)
    t = R.stage_times()
    assert set(t) == {"project", "bin", "render_fwd"}, t
    assert all(v > 0.0 for v in t.values()), t
    total = a.elapsed_time(b)
    assert 0.7 * total <= sum(t.values()) <= 1.05 * total + 0.05, (t, total)
    state = R.ray_state()
    R.render_fwd(p, out, ray_state=state)
    grads = {k: torch.zeros_like(v) for k, v in p.items()}
    R.render_bwd(p, state, torch.ones_like(out), grads)
    t2 = R.stage_times()
    assert t2["render_bwd"] > 0.0 and t2["project"] == t["project"], t2


@pytest.mark.parametrize("K", [16_384, 16_385, 40_000])
def test_depth_sort_cluster_sizes_and_an_empty_receiver(K):
    """Depth sorts in clusters of 1, 2 and 3 CTAs (16,384 keys per CTA at most): a receiver
    inside the scene, one whose 40 x 12 window points away from it (no Gaussian covers a
    tile: an empty sort and no pairs) and one outside looking in.  Keys, ids and tile
    ranges equal the oracle's bit for bit, and the empty receiver renders zero."""
    scene = synthetic.tiny_scene(K, 104, box=(6.0, 5.0, 3.0), log_scale_mu=math.log(0.15))
    rx = np.array([[3.0, 2.5, 1.5], [-40.0, 2.5, 1.5], [9.0, -3.0, 1.0]], np.float32)
    spec = dict(n_az=40, n_el=12, az0_deg=150.0, daz_deg=1.0, el0_deg=-10.0, del_deg=2.0)
    S, R, p, out = gpu_render(scene, rx, [0.5, 4.5, 2.5], 2.4e9, spec)
    check_bins(R, scene, rx, spec)
    keys, ids, rb, ts = R.pairs()
    rb = rb.cpu().numpy()
    assert rb[2] - rb[1] == 0 and rb[1] - rb[0] > 0 and rb[3] - rb[2] > 0
    assert np.all(S[1] == 0)


def test_depth_sort_of_a_wide_depth_span():
    """Depths from 2 cm to 20 km, each Gaussian scaled with its distance so that all stay
    visible (about 20 binades: a key span above 2^27, so the cluster sort takes four 8-bit
    passes instead of 9-bit ones): keys, ids and tile ranges equal the oracle's bit for
    bit."""
    rng = np.random.default_rng(105)
    K = 20_000
    scene = synthetic.tiny_scene(K, 105, box=(6.0, 5.0, 3.0), log_scale_mu=math.log(0.05))
    rx = np.array([[0.0, 0.0, 0.0], [1.0, -2.0, 0.5]], np.float32)
    u = rng.normal(size=(K, 3))
    u[:, 2] = np.abs(u[:, 2])  # above the horizon of the 0..90 degree grid
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    dist = np.exp(rng.uniform(math.log(0.02), math.log(20000.0), K))
    scene["means"] = (u * dist[:, None]).astype(np.float32)
    scene["log_scales"] = (scene["log_scales"] + np.log(dist)[:, None]).astype(np.float32)
    spec = dict(n_az=72, n_el=18, r_rx=0.01)
    S, R, p, out = gpu_render(scene, rx, [5.0, 5.0, 2.0], 2.4e9, spec)
    check_bins(R, scene, rx, spec)


@pytest.mark.parametrize("K", [120_000, 150_000, 260_000])
def test_bins_bit_exact_at_large_scenes(K):
    """Scenes larger than the benchmark's (120k, 150k and 260k Gaussians, two receivers,
    360 x 90): keys, ids and tile ranges equal the oracle's bit for bit.  Up to 131,072
    Gaussians a receiver's depth sort runs in one cluster of up to 8 CTAs (8 at 120k);
    above, in the four global passes (dozens of sort chunks per receiver in every pass)."""
    cfg = synthetic.config_ble(K=K, n_rx=2)
    spec = dict(cfg["grid"])
    K_ = cfg["scene"]["means"].shape[0]
    R = Renderer(K_, 2, make_grid(**spec), cfg["f0"])
    p = to_device(cfg["scene"])
    R.ensure_capacity(p, torch.tensor(cfg["rx"], device="cuda"), torch.tensor(cfg["tx"], device="cuda"))
    check_bins(R, cfg["scene"], cfg["rx"], spec)
