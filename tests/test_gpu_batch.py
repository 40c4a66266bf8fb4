"""The batched persistent render (gsrf_render_batch) against the plain launch: every
job of a batch -- different scenes, receiver counts, grids, transmitters and carriers --
must come out bit-identical to its own gsrf_render_fwd, since both run the same per-ray
arithmetic in the same order; the composited-pair statistics must agree too."""
import math

import numpy as np
import pytest
import torch

from paper_2502_01826_gb300 import synthetic
from paper_2502_01826_gb300.render import BatchRender, Renderer, make_grid, to_device

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _job(K, seed, n_rx, spec, f0):
    scene = synthetic.tiny_scene(K, seed, box=(8.0, 6.0, 3.0), log_scale_mu=math.log(0.2))
    rng = np.random.default_rng(seed)
    rx = (rng.uniform(0, 1, (n_rx, 3)) * [8.0, 6.0, 3.0]).astype(np.float32)
    tx = (rng.uniform(0, 1, 3) * [8.0, 6.0, 3.0]).astype(np.float32)
    R = Renderer(K, n_rx, make_grid(**spec), f0)
    p = to_device(scene)
    rxd, txd = torch.tensor(rx, device="cuda"), torch.tensor(tx, device="cuda")
    R.ensure_capacity(p, rxd, txd)
    return R, p, rxd, txd


def test_batch_render_equals_plain_launches():
    jobs = [_job(3000, 301, 3, dict(n_az=360, n_el=90), 2.4e9),
            _job(800, 302, 1, dict(n_az=72, n_el=18), 5.2e9),
            _job(5000, 303, 5, dict(n_az=180, n_el=45), 915e6),
            _job(0, 304, 2, dict(n_az=36, n_el=9), 2.4e9),
            _job(2000, 305, 7, dict(n_az=100, n_el=37, az0_deg=-45.0, daz_deg=1.7, el0_deg=-30.0, del_deg=2.5),
                 2.4e9)]
    plain, plain_pairs = [], []
    for R, p, rx, tx in jobs:
        plain.append(R.forward(p, rx, tx).clone())
        plain_pairs.append(R.status().stats[1])
    B = BatchRender([R for R, _, _, _ in jobs])
    for rep in range(2):  # twice: the queue and the ordering are rebuilt every call
        outs = B.render()
        torch.cuda.synchronize()
        for (R, _, _, _), a, b, pp in zip(jobs, plain, outs, plain_pairs):
            assert torch.equal(a, b)
            assert R.status().stats[1] == pp


def test_batch_render_matches_oracle_on_mixed_scenes():
    """One gsrf_render_batch launch over problems of different scenes, receiver counts,
    grids, transmitters and carriers, each held to the oracle's per-ray bars (sampled
    rays on the full-resolution grid)."""
    import oracle
    from gpu_util import compare, oracle_pair

    oracle.build()
    specs = [(3000, 311, 3, dict(n_az=360, n_el=90), 2.4e9), (800, 312, 1, dict(n_az=72, n_el=18), 5.2e9),
             (2000, 313, 2, dict(n_az=100, n_el=37, az0_deg=-45.0, daz_deg=1.7, el0_deg=-30.0, del_deg=2.5),
              915e6)]
    jobs = [_job(*s) for s in specs]
    B = BatchRender([R for R, _, _, _ in jobs])
    outs = B.render()
    torch.cuda.synchronize()
    rng = np.random.default_rng(31)
    for (K, seed, n_rx, spec, f0), (R, p, rx, tx), out in zip(specs, jobs, outs):
        scene = synthetic.tiny_scene(K, seed, box=(8.0, 6.0, 3.0), log_scale_mu=math.log(0.2))
        S = out.cpu().numpy()
        S = (S[..., 0] + 1j * S[..., 1]).reshape(n_rx, -1)
        g = oracle.make_grid(**spec)
        n_rays = g.n_az * g.n_el
        rays = np.sort(rng.choice(n_rays, min(n_rays, 600), replace=False)).astype(np.int32)
        for r in sorted({0, n_rx - 1}):
            ref = oracle_pair(scene, rx[r].cpu().numpy(), tx.cpu().numpy(), f0, g, rays=rays)
            compare(S[r][rays], ref)


def test_batch_completion_stamps_and_many_jobs():
    """More jobs than one chunk of the job table (48), with completion stamps: every job
    finishes after the launch's first warp started, within the launch's span, and each job
    equals its plain launch bit for bit."""
    jobs = [_job(300 + 37 * (i % 5), 400 + i, 1 + i % 3, dict(n_az=72, n_el=18), 2.4e9 if i % 2 else 5.2e9)
            for i in range(61)]
    plain = []
    for R, p, rx, tx in jobs:
        plain.append(R.forward(p, rx, tx).clone())
    B = BatchRender([R for R, _, _, _ in jobs], stamps=True)
    for _ in range(2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        outs = B.render()
        b.record()
        torch.cuda.synchronize()
        for x, y in zip(plain, outs):
            assert torch.equal(x, y)
        t = B.job_done_ns.cpu().numpy().view(np.uint64)
        start, done = int(t[-1]), t[:-1].astype(np.int64)
        assert start != np.iinfo(np.uint64).max
        span_ns = a.elapsed_time(b) * 1e6
        assert np.all(done >= start) and np.all(done - start <= span_ns + 1e5)
        c = B.completion_ms()
        assert c.shape == (len(jobs),) and np.all(c >= 0.0)
    # the same jobs taken in their given order (heaviest first inside each): same outputs,
    # and the first jobs finish before the last ones
    Bo = BatchRender([R for R, _, _, _ in jobs], stamps=True, job_order=True)
    outs = Bo.render()
    torch.cuda.synchronize()
    for x, y in zip(plain, outs):
        assert torch.equal(x, y)
    c = Bo.completion_ms()
    assert np.mean(c[:10]) < np.mean(c[-10:]), c


def test_uneven_serving_requests_in_one_launch_match_oracle():
    """Requests of the uneven serving workload (its scenes of 12k to 688k Gaussians, 1-32
    receivers, 2.4 and 5.2 GHz, 360 x 90) rendered by ONE gsrf_render_batch launch in job
    order with completion stamps; sampled rays of the first and last receiver of four
    requests -- a 688k-Gaussian one at 5.2 GHz, a 287k one, a 101k one and a 12k one --
    against the oracle's per-ray bars."""
    import oracle
    from gpu_util import compare, oracle_pair

    oracle.build()
    cfg = synthetic.config_uneven()
    scenes = [to_device(sc) for sc in cfg["scenes"]]
    reqs = cfg["requests"][:24]
    jobs = []
    for q in reqs:
        R = Renderer(scenes[q["scene"]]["means"].shape[0], q["rx"].shape[0], make_grid(**cfg["grid"]), q["f0"],
                     pair_capacity=1024)
        rx, tx = torch.tensor(q["rx"], device="cuda"), torch.tensor(q["tx"], device="cuda")
        R.ensure_capacity(scenes[q["scene"]], rx, tx)
        jobs.append(R)
    B = BatchRender(jobs, stamps=True, job_order=True)
    outs = B.render()
    torch.cuda.synchronize()
    for R in jobs:
        assert R.status().code == 0
    assert np.all(B.completion_ms() > 0.0)
    g = oracle.make_grid(**cfg["grid"])
    rng = np.random.default_rng(41)
    for i in (23, 12, 0, 3):  # 688k at 5.2 GHz, 287k, 101k, 12k Gaussians
        q = reqs[i]
        S = outs[i].cpu().numpy()
        S = (S[..., 0] + 1j * S[..., 1]).reshape(q["rx"].shape[0], -1)
        rays = np.sort(rng.choice(S.shape[1], 200, replace=False)).astype(np.int32)
        for r in sorted({0, q["rx"].shape[0] - 1}):
            ref = oracle_pair(cfg["scenes"][q["scene"]], q["rx"][r], q["tx"], q["f0"], g, rays=rays)
            compare(S[r][rays], ref)
