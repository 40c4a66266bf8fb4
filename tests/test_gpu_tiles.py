"""Tile shape, warp ray block and shared-memory stage size change how the work is cut,
never the result.

For each configuration: the splat keys, per-tile id lists and tile ranges equal the
oracle's binning with the same tile shape, bit for bit; the per-ray signal -- one and
several subcarriers -- is bit-identical to the default configuration (16 x 16 tiles,
8 x 4 rays per warp, 32 candidates per stage), which the other GPU tests hold to the
oracle: a ray composites the same Gaussians in the same depth order whatever list it
walks, and the warp-level rejections only skip candidates no ray of the warp can hit.
The backward's gradients are sums whose order follows the work split, so they are held
to 1e-5 relative to the default configuration's."""

import numpy as np
import pytest
import torch

import oracle
from paper_2502_01826_gb300 import synthetic
from paper_2502_01826_gb300.render import Renderer, make_grid, render, to_device

from gpu_util import oracle_grid, require_gpu

pytestmark = pytest.mark.gpu

SPLITS = [  # tile_w, tile_h, ray_block_w, stage
    (16, 16, 8, 32), (8, 16, 8, 16), (32, 8, 32, 32), (16, 16, 4, 32), (32, 32, 16, 16), (16, 4, 8, 32),
    (8, 8, 8, 16), (32, 16, 4, 32),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    oracle.build()


@pytest.fixture(scope="module")
def problem():
    scene = synthetic.scene(6000, 777)
    scene = {k: v for k, v in scene.items() if not k.startswith("_")}
    rng = np.random.default_rng(5)
    rx = (rng.uniform(0, 1, (3, 3)) * [10.0, 8.0, 3.0]).astype(np.float32)
    tx = np.array([9.0, 1.0, 2.0], np.float32)
    return scene, rx, tx


def run(scene, rx, tx, cfg, n_f=1, df=0.0, spec=dict(n_az=360, n_el=90)):
    tw, th, bw, stage = cfg
    grid = make_grid(**spec, tile_w=tw, tile_h=th)
    R = Renderer(scene["means"].shape[0], rx.shape[0], grid, 2.4e9, df_hz=df, n_f=n_f, ray_block_w=bw,
                 stage=stage)
    p = to_device(scene)
    rxd = torch.tensor(rx, device="cuda")
    txd = torch.tensor(tx, device="cuda")
    R.ensure_capacity(p, rxd, txd)
    out = R.forward(p, rxd, txd)
    torch.cuda.synchronize()
    assert R.status().code == 0
    return out.cpu().numpy(), R


@pytest.mark.parametrize("cfg", SPLITS)
def test_bins_match_oracle_and_rays_match_default(problem, cfg):
    scene, rx, tx = problem
    ref, _ = run(scene, rx, tx, SPLITS[0])
    out, R = run(scene, rx, tx, cfg)
    assert np.array_equal(out, ref), "per-ray signal differs from the default configuration"
    keys, ids, rb, ts = R.pairs()
    keys = keys.cpu().numpy().view(np.uint64)
    ids = ids.cpu().numpy().view(np.uint32)
    rb = rb.cpu().numpy()
    ts = ts.cpu().numpy()
    g = oracle_grid(dict(n_az=360, n_el=90), tile_w=cfg[0], tile_h=cfg[1])
    for r in range(rx.shape[0]):
        k_ref, i_ref, t_ref = oracle.bin_pairs(scene, rx[r], g)
        assert np.array_equal(keys[rb[r]:rb[r + 1]], k_ref)
        assert np.array_equal(ids[rb[r]:rb[r + 1]], i_ref)
        assert np.array_equal(ts[r].astype(np.int64), t_ref)


@pytest.mark.parametrize("cfg", [SPLITS[1], SPLITS[2], SPLITS[4]])
def test_subcarriers_match_default(problem, cfg):
    scene, rx, tx = problem
    spec = dict(n_az=180, n_el=45)
    ref, _ = run(scene, rx, tx, SPLITS[0], n_f=20, df=1.0e6, spec=spec)
    out, _ = run(scene, rx, tx, cfg, n_f=20, df=1.0e6, spec=spec)
    assert np.array_equal(out, ref)


def grads(scene, rx, tx, cfg, n_f=1, df=0.0):
    tw, th, bw, stage = cfg
    grid = make_grid(n_az=180, n_el=45, tile_w=tw, tile_h=th)
    R = Renderer(scene["means"].shape[0], rx.shape[0], grid, 2.4e9, df_hz=df, n_f=n_f, ray_block_w=bw,
                 stage=stage)
    p = {k: v.clone().requires_grad_(True) for k, v in to_device(scene).items()}
    rxd = torch.tensor(rx, device="cuda")
    txd = torch.tensor(tx, device="cuda")
    R.ensure_capacity({k: v.detach() for k, v in p.items()}, rxd, txd)
    S = render(R, p, rxd, txd)
    G = torch.sin(torch.arange(S.numel(), device="cuda", dtype=torch.float32) * 0.37).reshape(S.shape)
    (S * G).sum().backward()
    torch.cuda.synchronize()
    return {k: v.grad.double().cpu().numpy() for k, v in p.items()}


@pytest.mark.parametrize("cfg,n_f", [(SPLITS[2], 1), (SPLITS[3], 1), (SPLITS[1], 9)])
def test_backward_matches_default(problem, cfg, n_f):
    scene, rx, tx = problem
    small = {k: v[:2000] for k, v in scene.items()}
    ref = grads(small, rx, tx, SPLITS[0], n_f=n_f, df=2.0e6)
    got = grads(small, rx, tx, cfg, n_f=n_f, df=2.0e6)
    for k in ref:
        a, b = got[k].ravel(), ref[k].ravel()
        assert np.linalg.norm(a - b) <= 1e-5 * max(np.linalg.norm(b), 1e-30), k
