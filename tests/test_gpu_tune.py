"""The autotuner (gsrf_autotune): its choice is the fastest of its own measurements,
every measured split is a valid one, and adopting the choice leaves the per-ray signal
bit-identical to the default split."""
import numpy as np
import pytest
import torch

from paper_2502_01826_gb300 import synthetic
from paper_2502_01826_gb300.render import Renderer, make_grid, to_device

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def test_autotune_picks_its_fastest_split_and_keeps_results():
    scene = {k: v for k, v in synthetic.scene(8000, 91).items() if not k.startswith("_")}
    rng = np.random.default_rng(7)
    rx = torch.tensor((rng.uniform(0, 1, (4, 3)) * [10.0, 8.0, 3.0]).astype(np.float32), device="cuda")
    tx = torch.tensor(np.array([1.0, 7.0, 2.5], np.float32), device="cuda")
    p = to_device(scene)
    R0 = Renderer(8000, 4, make_grid(360, 90), 2.4e9)
    R0.ensure_capacity(p, rx, tx)
    ref = R0.forward(p, rx, tx).cpu().numpy()

    R = Renderer(8000, 4, make_grid(360, 90), 2.4e9, pair_capacity=4 * R0.plan.pair_capacity)
    best, table = R.autotune(p, rx, tx, reps=2)
    assert len(table) >= 20
    tot = [t["project_bin_ms"] + t["render_ms"] for t in table]
    assert best["project_bin_ms"] + best["render_ms"] == min(tot)
    for t in table:
        assert t["tile_w"] % t["ray_block_w"] == 0 and t["tile_h"] % (32 // t["ray_block_w"]) == 0
        assert t["stage"] in (16, 32) and t["render_ms"] > 0.0
    assert (R.plan.grid.tile_w, R.plan.grid.tile_h, R.plan.ray_block_w, R.plan.stage) == \
        (best["tile_w"], best["tile_h"], best["ray_block_w"], best["stage"])
    out = R.forward(p, rx, tx).cpu().numpy()
    assert R.status().code == 0
    assert np.array_equal(out, ref)
    print("autotune best:", best)


def test_autotune_for_training_times_forward_and_backward():
    scene = {k: v for k, v in synthetic.scene(4000, 92).items() if not k.startswith("_")}
    rng = np.random.default_rng(8)
    rx = torch.tensor((rng.uniform(0, 1, (2, 3)) * [10.0, 8.0, 3.0]).astype(np.float32), device="cuda")
    tx = torch.tensor(np.array([2.0, 6.0, 1.5], np.float32), device="cuda")
    p = to_device(scene)
    R = Renderer(4000, 2, make_grid(180, 45), 2.4e9, pair_capacity=2_000_000, ckpt_every=64, ckpt_slots=8)
    fwd_best, fwd = R.autotune(p, rx, tx, reps=1)
    trn_best, trn = R.autotune(p, rx, tx, reps=1, training=True)
    assert len(trn) == len(fwd) >= 20
    tot = [t["project_bin_ms"] + t["render_ms"] for t in trn]
    assert trn_best["project_bin_ms"] + trn_best["render_ms"] == min(tot)
    # forward + backward costs more than the forward alone for the same split
    key = lambda t: (t["tile_w"], t["tile_h"], t["ray_block_w"], t["stage"])
    f = {key(t): t["render_ms"] for t in fwd}
    assert sum(t["render_ms"] > f[key(t)] for t in trn) >= 0.8 * len(trn)
