"""GPU parity of the multi-frequency render (CSI-shaped: subcarriers f0 + s df) and of
the FP64 distance-to-phase step, against the FP64 oracle.

Per subcarrier the per-ray bars of gpu_util apply; the CSI value of a receiver (the
complex sum over rays per subcarrier) is held per (element, subcarrier) to 1e-4 of its
own magnitude plus 1e-2 of the element's rms over subcarriers; the stored path phase
must be within 1e-6 rad of the oracle's FP64 phase."""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_01826_gb300 import _lib as L
from paper_2502_01826_gb300 import synthetic
from paper_2502_01826_gb300.render import Renderer, make_grid, received_signal, to_device

from gpu_util import TOL_RAY, compare, oracle_choice, oracle_pair, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    oracle.build()


def render_mf(scene, rx, tx, f0, df, n_f, spec):
    K = scene["means"].shape[0]
    grid = make_grid(**spec)
    R = Renderer(K, rx.shape[0], grid, f0, df_hz=df, n_f=n_f)
    p = to_device(scene)
    rxd = torch.tensor(rx, device="cuda")
    txd = torch.tensor(tx, device="cuda")
    R.ensure_capacity(p, rxd, txd)
    out = R.forward(p, rxd, txd)
    torch.cuda.synchronize()
    return out, R


@pytest.mark.parametrize("n_f", [3, 8, 24, 40, 64])
def test_subcarriers_match_oracle(n_f):
    """Each subcarrier against the oracle, and the CSI sum per subcarrier.  The walk takes
    the smallest chunk of 8, 16, 32 or 64 subcarriers that holds n_f (24 and 40: ragged
    chunks of 32 and 64; 64: the CSI band in one walk, its phase recurrence 64 steps long)."""
    cfg = synthetic.config_csi(K=3000)
    rx = cfg["rx"][:4]  # one four-element array
    spec = cfg["grid"]
    df = cfg["df"] if n_f == 64 else 2.0e6
    f0 = cfg["f0"] if n_f == 64 else 5.2e9
    out, R = render_mf(cfg["scene"], rx, cfg["tx"], f0, df, n_f, spec)
    S = out.cpu().numpy()
    S = S[..., 0] + 1j * S[..., 1]  # [n_rx, n_f, n_el, n_az]
    g = oracle.make_grid(**spec)
    for r in (0, 3):
        ref = oracle_pair(cfg["scene"], rx[r], cfg["tx"], f0, g, df=df, n_f=n_f)
        for f in range(n_f):
            compare(S[r, f].reshape(-1), ref, f=f)
        # CSI: complex sum over rays per subcarrier, through the library's reduction
        cs = received_signal(out, L.SIG_COMPLEX_SUM).cpu().numpy()[r]
        got = cs[:, 0] + 1j * cs[:, 1]
        want = np.array([np.sum(oracle_choice(S[r, f].reshape(-1), ref, f)) for f in range(n_f)])
        rms = np.sqrt(np.mean(np.abs(want) ** 2))
        ratio = np.abs(got - want) / (TOL_RAY * (np.abs(want) + 1e-2 * rms))
        print("CSI element %d, %d subcarriers: worst error %.3g of the bar, relative L2 %.3g"
              % (r, n_f, ratio.max(), np.linalg.norm(got - want) / np.linalg.norm(want)))
        assert ratio.max() <= 1.0, ratio


def test_csi_100k_full_size_and_phase_step():
    """The CSI workload in the benchmark's configuration: 100,000 Gaussians, 8 arrays of
    4 elements, 64 subcarriers at 312.5 kHz around 5.2 GHz, 180 x 45 grid.  Sampled rays
    of two elements against the oracle at every subcarrier, and the stored FP64-reduced
    path phase of every (element, Gaussian) of two elements within 1e-6 rad."""
    cfg = synthetic.config_csi()
    out, R = render_mf(cfg["scene"], cfg["rx"], cfg["tx"], cfg["f0"], cfg["df"], cfg["n_f"], cfg["grid"])
    assert R.status().code == 0
    S = out.cpu().numpy()
    S = S[..., 0] + 1j * S[..., 1]
    g = oracle.make_grid(**cfg["grid"])
    rng = np.random.default_rng(9)
    n_rays = g.n_az * g.n_el
    for r in (0, 29):
        rays = np.sort(rng.choice(n_rays, 300, replace=False)).astype(np.int32)
        ref = oracle_pair(cfg["scene"], cfg["rx"][r], cfg["tx"], cfg["f0"], g, rays=rays, df=cfg["df"],
                          n_f=cfg["n_f"])
        for f in (0, 17, 32, 63):
            compare(S[r, f].reshape(-1)[rays], ref, f=f)
    # distance-to-phase step: recompute the projection with the records kept
    p = to_device(cfg["scene"])
    R.project(p, torch.tensor(cfg["rx"], device="cuda"), torch.tensor(cfg["tx"], device="cuda"))
    views = R.view_records().cpu().numpy()
    worst = 0.0
    for r in (0, 29):
        ph_ref = oracle.path_phase(cfg["scene"], cfg["rx"][r], cfg["tx"], cfg["f0"])
        vis = np.isfinite(views[r, :, 3])  # the records of Gaussians in some tile's list
        assert vis.sum() > 0.2 * vis.size
        ph_gpu = np.arctan2(-views[r, vis, 8], views[r, vis, 7])
        err = np.abs(np.angle(np.exp(1j * (ph_gpu - ph_ref[vis]))))
        worst = max(worst, float(err.max()))
    print("max |phase error| of the FP64 distance-to-phase step: %.3g rad" % worst)
    assert worst <= 1e-6
