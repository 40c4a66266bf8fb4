"""GPU parity of the hand-written backward (App. D) against the FP64 oracle gradient
and against central finite differences of the GPU forward, through the C ABI and the
torch.autograd.Function.

Bar: <= 1e-3 relative, norm-wise per parameter group, and per element against
|g_ref| + 10% of the group's rms.  Rays that pass within 0.05 of a 3-sigma boundary
(in m2), within 1 cm of the emitting sphere, or near the termination threshold get no
weight in the loss: the chord length 2 sqrt((9 - m2)/A) has an unbounded derivative at
grazing, so there FP32 and FP64 gradients (and finite differences) legitimately part.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2502_01826_gb300 import synthetic
from paper_2502_01826_gb300.render import Renderer, make_grid, render, to_device

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

NAMES = ("means", "log_scales", "quats", "opacity_logit", "coeffs", "phase_b")
MASK_BANDS = (0.0, 0.05, 1.0, 1e-2, 0.0, 0.05)  # m2 within 0.05, exit within 1 cm, ln Ta within 0.05


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    oracle.build()


def masked_upstream(scene, rx, tx, f0, spec, rng, eps_T=1e-4, n_f=1, fle_degree=0):
    """Random upstream dL/dS per ray (and subcarrier), zero on rays near a discrete
    decision.  Returns [n_rx, rays] for one frequency, else [n_rx, n_f, rays]."""
    g = oracle.make_grid(**spec, eps_T=eps_T, fle_degree=fle_degree)
    G = []
    for r in range(rx.shape[0]):
        out = oracle.render(scene, rx[r], tx, f0, g, bands=MASK_BANDS)
        shape = (n_f, out["S"].shape[1])
        Gr = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        Gr[:, out["flags"] != 0] = 0
        G.append(Gr[0] if n_f == 1 else Gr)
    return np.array(G), g


def gpu_grads(scene, rx, tx, f0, spec, G, eps_T=1e-4, df=0.0, n_f=1, **plan_kw):
    """Gradients of sum Re(conj(G) S) through the autograd Function."""
    K = scene["means"].shape[0]
    grid = make_grid(**spec, eps_T=eps_T)
    R = Renderer(K, rx.shape[0], grid, f0, df_hz=df, n_f=n_f, **plan_kw)
    p = {k: v.clone().requires_grad_(True) for k, v in to_device(scene).items()}
    rxd = torch.tensor(rx, device="cuda")
    txd = torch.tensor(tx, device="cuda")
    R.ensure_capacity({k: v.detach() for k, v in p.items()}, rxd, txd)
    S = render(R, p, rxd, txd)  # [n_rx, 1, n_el, n_az, 2]
    Gt = torch.tensor(np.stack([G.real, G.imag], -1), dtype=torch.float32, device="cuda")
    Gt = Gt.reshape(S.shape)
    loss = (S * Gt).sum()
    loss.backward()
    torch.cuda.synchronize()
    return {k: p[k].grad.cpu().numpy().astype(np.float64) for k in NAMES}


def oracle_grads(scene, rx, tx, f0, g, G, df=0.0, n_f=1):
    tot = None
    for r in range(rx.shape[0]):
        gr = oracle.render_grad(scene, rx[r], tx, f0, g, G[r].reshape(n_f, -1), df=df, n_f=n_f)
        tot = gr if tot is None else {k: tot[k] + gr[k] for k in tot}
    return tot


def compare_grads(gg, go, tol=1e-3):
    report = {}
    for k in NAMES:
        a, b = gg[k].ravel(), go[k].ravel()
        nb = np.linalg.norm(b)
        rel = np.linalg.norm(a - b) / max(nb, 1e-30)
        rms = np.sqrt(np.mean(b ** 2))
        worst = np.max(np.abs(a - b) / (np.abs(b) + 0.1 * rms + 1e-30))
        report[k] = (rel, worst)
        assert rel <= tol, "%s: relative error %.3g" % (k, rel)
        assert worst <= 10 * tol, "%s: worst element %.3g" % (k, worst)
    return report


def test_backward_matches_oracle_gradient_small():
    scene = synthetic.tiny_scene(300, 201, box=(6.0, 5.0, 3.0), log_scale_mu=math.log(0.25))
    rng = np.random.default_rng(1)
    rx = (rng.uniform(0, 1, (2, 3)) * [6.0, 5.0, 3.0]).astype(np.float32)
    tx = np.array([0.5, 4.0, 2.0], np.float32)
    spec = dict(n_az=72, n_el=18)
    G, g = masked_upstream(scene, rx, tx, 2.4e9, spec, rng)
    assert np.count_nonzero(G) > 0.5 * G.size
    compare_grads(gpu_grads(scene, rx, tx, 2.4e9, spec, G), oracle_grads(scene, rx, tx, 2.4e9, g, G))


@pytest.mark.parametrize("n_f,df", [(3, 2.0e7), (12, 2.0e6), (64, 312.5e3)])
def test_backward_multifrequency_matches_oracle(n_f, df):
    """Subcarriers f0 + s df, all in one reverse walk (3: an odd count, whose last pair is
    zero-padded; 64 at 312.5 kHz: the CSI workload's band): every subcarrier's upstream
    enters with its own suffix sum and its own 2 pi f_s / c."""
    scene = synthetic.tiny_scene(300, 203, box=(6.0, 5.0, 3.0), log_scale_mu=math.log(0.25))
    rng = np.random.default_rng(4)
    rx = (rng.uniform(0, 1, (2, 3)) * [6.0, 5.0, 3.0]).astype(np.float32)
    tx = np.array([5.5, 0.5, 2.5], np.float32)
    spec = dict(n_az=72, n_el=18)
    f0 = 5.2e9
    G, g = masked_upstream(scene, rx, tx, f0, spec, rng, n_f=n_f)
    assert np.count_nonzero(G) > 0.5 * G.size
    compare_grads(gpu_grads(scene, rx, tx, f0, spec, G, df=df, n_f=n_f),
                  oracle_grads(scene, rx, tx, f0, g, G, df=df, n_f=n_f))


def test_backward_matches_oracle_on_512_gaussian_training_subscene():
    """A 512-Gaussian sub-scene of the training workload (same box and distributions),
    16 receivers on the 360 x 90 grid, loss = complex MSE against targets the oracle
    renders from a separately seeded ground-truth set."""
    cfg = synthetic.config_train(K=512, n_rx=16)
    scene, gt = cfg["scene"], cfg["gt_scene"]
    rx, tx, f0 = cfg["rx"], cfg["tx"], cfg["f0"]
    spec = cfg["grid"]
    g = oracle.make_grid(**spec)
    rng = np.random.default_rng(2)
    # dL/dS for L = mean |S - S_gt|^2 is 2 (S - S_gt) / N, evaluated with the oracle
    G = []
    for r in range(rx.shape[0]):
        S = oracle.render(scene, rx[r], tx, f0, g, bands=MASK_BANDS)
        S_gt = oracle.render(gt, rx[r], tx, f0, g)["S"][0]
        Gr = 2.0 * (S["S"][0] - S_gt) / S_gt.size
        Gr[S["flags"] != 0] = 0
        G.append(Gr)
    G = np.array(G)
    assert np.count_nonzero(G) > 0.5 * G.size
    compare_grads(gpu_grads(scene, rx, tx, f0, spec, G), oracle_grads(scene, rx, tx, f0, g, G))


def central_difference_check(f0, seed, trunc):
    """Central differences (eps = 1e-3 relative, the training workload's setting) of the
    GPU forward on 32 random parameters against the hand-written backward.  Each quotient
    is held to 2e-2 (FP32 forward noise) plus `trunc`(h) of |g| + 10% of the rms of the
    checked gradients, where trunc(h) is the step's truncation error relative to the
    derivative.  A perturbation that changes the composited pairs or the candidate tests
    (a hit set, the discrete steps of the method) is not a derivative and is skipped."""
    scene = synthetic.tiny_scene(200, 202, box=(5.0, 5.0, 3.0), log_scale_mu=math.log(0.3))
    rng = np.random.default_rng(seed)
    rx = (rng.uniform(0, 1, (1, 3)) * [5.0, 5.0, 3.0]).astype(np.float32)
    tx = np.array([4.0, 0.5, 1.0], np.float32)
    spec = dict(n_az=72, n_el=18)
    G, g = masked_upstream(scene, rx, tx, f0, spec, rng, eps_T=0.0)
    grads = gpu_grads(scene, rx, tx, f0, spec, G, eps_T=0.0)
    K = scene["means"].shape[0]
    grid = make_grid(**spec, eps_T=0.0)
    R = Renderer(K, 1, grid, f0)
    rxd = torch.tensor(rx, device="cuda")
    txd = torch.tensor(tx, device="cuda")
    Gt = torch.tensor(np.stack([G.real, G.imag], -1), dtype=torch.float64, device="cuda")

    def loss_of(sc):
        p = to_device(sc)
        R.ensure_capacity(p, rxd, txd)
        S = R.forward(p, rxd, txd).double().reshape(Gt.shape)
        st = R.status()
        return float((S * Gt).sum().item()), (st.stats[0], st.stats[1])

    _, base = loss_of(scene)
    errs, checked, skipped = [], 0, 0
    for _ in range(300):
        name = NAMES[rng.integers(len(NAMES))]
        arr = scene[name]
        idx = tuple(rng.integers(n) for n in arr.shape)
        x0 = float(arr[idx])
        h = 1e-3 * max(1.0, abs(x0))
        sp = {k: v.copy() for k, v in scene.items()}
        sm = {k: v.copy() for k, v in scene.items()}
        sp[name][idx] = np.float32(x0 + h)
        sm[name][idx] = np.float32(x0 - h)
        (lp, cp), (lm, cm) = loss_of(sp), loss_of(sm)
        if cp != base or cm != base:
            skipped += 1
            continue
        hh = 0.5 * (float(sp[name][idx]) - float(sm[name][idx]))
        fd = (lp - lm) / (2.0 * hh)
        an = grads[name][idx]
        if abs(an) < 1e-12 and abs(fd) < 1e-9:
            continue
        errs.append((abs(fd - an), abs(an), trunc(name, hh)))
        checked += 1
        if checked >= 32:
            break
    errs = np.array(errs)
    rms = np.sqrt(np.mean(errs[:, 1] ** 2))
    bad = errs[:, 0] > (2e-2 + errs[:, 2]) * (errs[:, 1] + 0.1 * rms)
    print("central differences at %.3g GHz: %d checked, %d skipped (hit set changed), %d outside"
          % (f0 / 1e9, checked, skipped, int(bad.sum())))
    assert checked >= 24 and bad.sum() <= 2, errs[bad]


def test_backward_against_central_differences_of_the_gpu_forward():
    """At a 300 MHz carrier the path-phase curvature is well inside the step."""
    central_difference_check(3.0e8, 3, lambda name, h: 0.0)


def test_backward_against_central_differences_at_the_operating_carrier():
    """At the training workload's 2.4 GHz carrier.  A mean moved by h turns the path phase
    by up to 2 (2 pi f / c) h, whose third derivative makes the central quotient of
    e^{-j k x} err by (k h)^2 / 6 relative, k = 2 (2 pi f / c) (both legs of the path);
    the other parameters move the phase only through the transmittance's b dt, far less."""
    k = 2.0 * 2.0 * math.pi * 2.4e9 / 3.0e8
    central_difference_check(2.4e9, 5, lambda name, h: (k * h) ** 2 / 6.0 if name == "means" else 0.0)


def deep_scene():
    """Dense, large Gaussians around the receivers and no early termination: rays
    composite hundreds of pairs, so the recomputed transmittance runs over long walks."""
    scene = synthetic.tiny_scene(1500, 204, box=(3.0, 3.0, 2.0), log_scale_mu=math.log(0.3))
    scene["opacity_logit"] = (scene["opacity_logit"] - 3.0).astype(np.float32)  # thin: deep walks
    rng = np.random.default_rng(8)
    rx = (0.25 + rng.uniform(0, 1, (2, 3)) * [2.5, 2.5, 1.5]).astype(np.float32)
    tx = np.array([2.9, 0.1, 1.9], np.float32)
    return scene, rx, tx


def test_checkpoints_leave_the_forward_unchanged():
    scene, rx, tx = deep_scene()
    K = scene["means"].shape[0]
    outs = []
    for kw in (dict(), dict(ckpt_every=64, ckpt_slots=8)):
        R = Renderer(K, rx.shape[0], make_grid(72, 18, eps_T=0.0), 2.4e9, **kw)
        p = to_device(scene)
        rxd, txd = torch.tensor(rx, device="cuda"), torch.tensor(tx, device="cuda")
        R.ensure_capacity(p, rxd, txd)
        state = R.ray_state()
        outs.append(R.forward(p, rxd, txd, ray_state=state).cpu().numpy())
        rays = rx.shape[0] * 72 * 18
        assert state.numel() == rays * 32 + (rays * 8 * 16 if kw else 0)  # slots follow the ray states
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("every,slots", [(32, 64), (64, 4)])
def test_checkpointed_backward_on_deep_walks(every, slots):
    """Checkpoints every 32 positions (all of the walk covered) and every 64 with only 4
    slots (beyond them the division takes over): both gradients within the bar of the
    FP64 oracle's, and at least as close to it as the division-only backward."""
    scene, rx, tx = deep_scene()
    spec = dict(n_az=72, n_el=18)
    rng = np.random.default_rng(9)
    G, g = masked_upstream(scene, rx, tx, 2.4e9, spec, rng, eps_T=0.0)
    ref = oracle_grads(scene, rx, tx, 2.4e9, g, G)
    div = gpu_grads(scene, rx, tx, 2.4e9, spec, G, eps_T=0.0)
    ck = gpu_grads(scene, rx, tx, 2.4e9, spec, G, eps_T=0.0, ckpt_every=every, ckpt_slots=slots)
    compare_grads(ck, ref)
    e_div = sum(np.linalg.norm(div[k] - ref[k]) ** 2 for k in NAMES)
    e_ck = sum(np.linalg.norm(ck[k] - ref[k]) ** 2 for k in NAMES)
    print("squared gradient error vs oracle: division only %.3g, checkpoints %.3g" % (e_div, e_ck))
    assert e_ck <= 1.5 * e_div + 1e-30


@pytest.mark.parametrize("deg", [1, 2, 4, 5])
def test_backward_at_other_degrees_matches_oracle(deg):
    """The adjoint at Fourier-Legendre degree L = 1, 2, 4, 5 (Sec. 4.2's degree study):
    (L + 1)^2 coefficient gradients per Gaussian from the basis chunks of the reduction,
    and every other parameter group, against the FP64 oracle gradient at the same degree."""
    scene = synthetic.tiny_scene(300, 210 + deg, box=(6.0, 5.0, 3.0), log_scale_mu=math.log(0.25))
    scene["coeffs"] = np.random.default_rng(deg).normal(0.0, 0.1, (300, (deg + 1) ** 2, 2)).astype(np.float32)
    rng = np.random.default_rng(20 + deg)
    rx = (rng.uniform(0, 1, (2, 3)) * [6.0, 5.0, 3.0]).astype(np.float32)
    tx = np.array([0.5, 4.0, 2.0], np.float32)
    spec = dict(n_az=72, n_el=18)
    G, g = masked_upstream(scene, rx, tx, 2.4e9, spec, rng, fle_degree=deg)
    assert np.count_nonzero(G) > 0.5 * G.size
    ref = oracle_grads(scene, rx, tx, 2.4e9, g, G)
    got = gpu_grads(scene, rx, tx, 2.4e9, spec, G, fle_degree=deg)
    assert got["coeffs"].shape == ((300, (deg + 1) ** 2, 2))
    compare_grads(got, ref)


@pytest.mark.parametrize("variant", [2, 4, 6])
def test_backward_of_variant_readings_matches_oracle(variant):
    """The adjoint of the normalised-weight reading (2: o N with N = 1 / ((2 pi)^1.5 s0 s1
    s2), so the log-scales get an extra term) and of the paper's splatting-circle culling
    (4: the hit set only), against the FP64 oracle's gradient under the same reading."""
    scene = synthetic.tiny_scene(300, 230 + variant, box=(6.0, 5.0, 3.0), log_scale_mu=math.log(0.25))
    rng = np.random.default_rng(50 + variant)
    rx = (rng.uniform(0, 1, (2, 3)) * [6.0, 5.0, 3.0]).astype(np.float32)
    tx = np.array([0.5, 4.0, 2.0], np.float32)
    spec = dict(n_az=72, n_el=18)
    G, _ = masked_upstream(scene, rx, tx, 2.4e9, spec, rng)
    assert np.count_nonzero(G) > 0.5 * G.size
    g = oracle.make_grid(**spec, eps_T=1e-4, variant=variant)
    ref = oracle_grads(scene, rx, tx, 2.4e9, g, G)
    got = gpu_grads(scene, rx, tx, 2.4e9, spec, G, variant=variant)
    compare_grads(got, ref)
