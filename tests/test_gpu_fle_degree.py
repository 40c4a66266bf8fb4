"""The Fourier-Legendre degree L of the radiance (Sec. 4.2; the paper studies L = 1..5):
the forward at each degree against the oracle at the same degree, and the default
(fle_degree = 0) bit-identical to an explicit L = 3."""
import numpy as np
import pytest

import oracle
from paper_2502_01826_gb300 import synthetic

from gpu_util import compare, gpu_render, oracle_pair, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    oracle.build()


def problem(K, seed, L, n_rx):
    scene = {k: v for k, v in synthetic.scene(K, seed, fle_degree=L).items() if not k.startswith("_")}
    rng = np.random.default_rng(seed)
    rx = (rng.uniform(0, 1, (n_rx, 3)) * [10.0, 8.0, 3.0]).astype(np.float32)
    tx = np.array([9.0, 1.0, 2.0], np.float32)
    return scene, rx, tx


@pytest.mark.parametrize("L", [1, 2, 4, 5])
@pytest.mark.parametrize("size", ["small", "dense"])
def test_degree_matches_oracle(L, size):
    K, n_rx, spec = (2048, 1, dict(n_az=36, n_el=9)) if size == "small" else (6000, 2, dict(n_az=180, n_el=45))
    scene, rx, tx = problem(K, 40 + L, L, n_rx)
    S, R, _, _ = gpu_render(scene, rx, tx, 2.4e9, spec, fle_degree=L)
    assert R.status().code == 0
    g = oracle.make_grid(**spec, fle_degree=L)
    for r in range(n_rx):
        compare(S[r], oracle_pair(scene, rx[r], tx, 2.4e9, g))


def test_default_degree_is_three():
    scene, rx, tx = problem(4000, 7, 3, 2)
    S0, _, _, _ = gpu_render(scene, rx, tx, 2.4e9, dict(n_az=180, n_el=45))
    S3, _, _, _ = gpu_render(scene, rx, tx, 2.4e9, dict(n_az=180, n_el=45), fle_degree=3)
    assert np.array_equal(S0, S3)


def test_degree_five_full_size_sampled():
    """L = 5 on the BLE workload's geometry (50,000 Gaussians, 360 x 90, four receivers):
    300 sampled rays of two receivers against the oracle."""
    cfg = synthetic.config_ble()
    scene = dict(cfg["scene"])
    scene["coeffs"] = np.random.default_rng(5).normal(0, 0.1, (scene["means"].shape[0], 36, 2)).astype(np.float32)
    rx = cfg["rx"][:4]
    S, R, _, _ = gpu_render(scene, rx, cfg["tx"], cfg["f0"], cfg["grid"], fle_degree=5)
    assert R.status().code == 0
    g = oracle.make_grid(**cfg["grid"], fle_degree=5)
    rng = np.random.default_rng(17)
    for r in (1, 3):
        rays = np.sort(rng.choice(S.shape[1], 300, replace=False)).astype(np.int32)
        compare(S[r][rays], oracle_pair(scene, rx[r], cfg["tx"], cfg["f0"], g, rays=rays))
