"""Variant readings (forward only): the radiance at the direction of the Gaussian's mean
instead of each ray's (GSRF_VARIANT_RADIANCE_AT_MEAN), the normalised density weight
(GSRF_VARIANT_NORMALISED_WEIGHT), the paper's splatting-circle culling
(GSRF_VARIANT_PAPER_CULLING), the per-pair path through the representative point
(GSRF_VARIANT_PATH_AT_REP) and each ray's hits in t_mid order (GSRF_VARIANT_ORDER_T_MID),
alone and together, held to the same bars against the
oracle rendering the same reading.  The circle is a discrete decision both sides take
in FP32 with the same operations, so it needs no band of its own."""
import numpy as np
import pytest

import oracle
from paper_2502_01826_gb300 import _lib as L
from paper_2502_01826_gb300 import synthetic

from gpu_util import compare, gpu_render, oracle_pair, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    oracle.build()


@pytest.mark.parametrize("variant", [L.VARIANT_RADIANCE_AT_MEAN, L.VARIANT_NORMALISED_WEIGHT,
                                     L.VARIANT_RADIANCE_AT_MEAN | L.VARIANT_NORMALISED_WEIGHT,
                                     L.VARIANT_PAPER_CULLING, L.VARIANT_PAPER_CULLING | L.VARIANT_RADIANCE_AT_MEAN,
                                     L.VARIANT_PATH_AT_REP, L.VARIANT_PATH_AT_REP | L.VARIANT_PAPER_CULLING,
                                     L.VARIANT_ORDER_T_MID, L.VARIANT_ORDER_T_MID | L.VARIANT_PAPER_CULLING])
@pytest.mark.parametrize("workload", ["plain", "dense"])
def test_variant_matches_oracle(variant, workload):
    if workload == "plain":
        cfg = synthetic.config_plain()
        scene, rx, tx, spec = cfg["scene"], cfg["rx"], cfg["tx"], cfg["grid"]
    else:
        scene = {k: v for k, v in synthetic.scene(6000, 778).items() if not k.startswith("_")}
        rng = np.random.default_rng(12)
        rx = (rng.uniform(0, 1, (2, 3)) * [10.0, 8.0, 3.0]).astype(np.float32)
        tx = np.array([9.0, 1.0, 2.0], np.float32)
        spec = dict(n_az=180, n_el=45)
    S, R, _, _ = gpu_render(scene, rx, tx, 2.4e9, spec, variant=variant)
    assert R.status().code == 0
    g = oracle.make_grid(**spec, variant=variant)
    for r in range(rx.shape[0]):
        ref = oracle_pair(scene, rx[r], tx, 2.4e9, g)
        compare(S[r], ref)


def test_paper_culling_full_size_sampled():
    """The paper's culling on the BLE workload in the benchmark's configuration (64
    receivers, 360 x 90): 300 sampled rays of two receivers against the oracle."""
    cfg = synthetic.config_ble()
    S, R, _, _ = gpu_render(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["grid"],
                            variant=L.VARIANT_PAPER_CULLING)
    assert R.status().code == 0
    g = oracle.make_grid(**cfg["grid"], variant=L.VARIANT_PAPER_CULLING)
    rng = np.random.default_rng(31)
    for r in (0, 47):
        rays = np.sort(rng.choice(g.n_az * g.n_el, 300, replace=False)).astype(np.int32)
        ref = oracle_pair(cfg["scene"], cfg["rx"][r], cfg["tx"], cfg["f0"], g, rays=rays)
        compare(S[r][rays], ref)


def test_tmid_order_full_size_sampled():
    """Hits in t_mid order on the BLE workload's geometry (50,000 Gaussians, 360 x 90, four
    receivers): dense rays keep their 512 nearest hits and terminate on them; 300 sampled
    rays of two receivers against the oracle."""
    cfg = synthetic.config_ble()
    rx = cfg["rx"][:4]
    S, R, _, _ = gpu_render(cfg["scene"], rx, cfg["tx"], cfg["f0"], cfg["grid"], variant=L.VARIANT_ORDER_T_MID)
    assert R.status().code == 0
    g = oracle.make_grid(**cfg["grid"], variant=L.VARIANT_ORDER_T_MID)
    rng = np.random.default_rng(37)
    for r in (0, 3):
        rays = np.sort(rng.choice(g.n_az * g.n_el, 300, replace=False)).astype(np.int32)
        compare(S[r][rays], oracle_pair(cfg["scene"], rx[r], cfg["tx"], cfg["f0"], g, rays=rays))
