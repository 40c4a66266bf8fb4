"""Host logic of the training loop (Sec. 4.4 losses, App. B updates) on CPU tensors:
each loss against what fixes it independently, the learning-rate schedule, the SGD
step per attribute, and the clone / split / prune rules."""
import math

import numpy as np
import pytest
import torch

from paper_2502_01826_gb300 import train


def test_fourier_loss_is_parseval():
    """(1/N) sum_f |F(a - b)|^2 = (1/N) sum |a - b|^2 (Parseval, unitary DFT), per map."""
    g = torch.Generator().manual_seed(0)
    a = torch.rand(3, 18, 72, generator=g, dtype=torch.float64)
    b = torch.rand(3, 18, 72, generator=g, dtype=torch.float64)
    ref = ((a - b) ** 2).mean()
    assert abs(float(train.fourier_loss(a, b) - ref)) <= 1e-12 * float(ref)


def test_ssim_matches_scipy_definition():
    """The Gaussian-window index recomputed with scipy's correlate (zero padding)."""
    from scipy.ndimage import correlate1d
    rng = np.random.default_rng(1)
    x = rng.random((18, 72))
    y = 0.7 * x + 0.3 * rng.random((18, 72))
    w = np.exp(-0.5 * ((np.arange(11) - 5) / 1.5) ** 2)
    w /= w.sum()

    def blur(t):
        return correlate1d(correlate1d(t, w, axis=1, mode="constant"), w, axis=0, mode="constant")

    L = y.max()
    c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    mx, my = blur(x), blur(y)
    sxx, syy, sxy = blur(x * x) - mx * mx, blur(y * y) - my * my, blur(x * y) - mx * my
    ref = (((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))).mean()
    got = float(train.ssim(torch.tensor(x), torch.tensor(y)))
    assert abs(got - ref) <= 1e-10
    assert abs(float(train.ssim(torch.tensor(x), torch.tensor(x))) - 1.0) <= 1e-12


def test_spectrum_loss_weights_and_zero():
    g = torch.Generator().manual_seed(2)
    a = torch.rand(2, 9, 36, generator=g, dtype=torch.float64)
    b = torch.rand(2, 9, 36, generator=g, dtype=torch.float64)
    assert float(train.spectrum_loss(a, a)) == 0.0
    l = train.spectrum_loss(a, b, 0.2, 0.1)
    ref = 0.7 * (a - b).abs().mean() + 0.2 * (1 - train.ssim(a, b)) + 0.1 * ((a - b) ** 2).mean()
    assert abs(float(l - ref)) <= 1e-12


def test_signal_loss_real_and_complex():
    p = torch.tensor([1.0, -2.0, 3.0], dtype=torch.float64)
    t = torch.tensor([0.5, -1.0, 5.0], dtype=torch.float64)
    assert float(train.signal_loss(p, t)) == 0.5 + 1.0 + 2.0
    pc = torch.tensor([1 + 1j, 2 - 1j])
    tc = torch.tensor([0 + 1j, 2 + 1j])
    assert abs(float(train.signal_loss(pc, tc)) - (1.0 + 4.0)) < 1e-6


def test_mean_lr_schedule():
    assert train.mean_lr(0) == pytest.approx(1.6e-4, rel=1e-12)
    assert train.mean_lr(30_000) == pytest.approx(1.6e-6, rel=1e-12)
    assert train.mean_lr(15_000) == pytest.approx(math.sqrt(1.6e-4 * 1.6e-6), rel=1e-12)
    assert train.mean_lr(60_000) == pytest.approx(1.6e-6, rel=1e-12)


def _model(n=6, seed=3):
    rng = np.random.default_rng(seed)
    p = dict(means=rng.uniform(0, 5, (n, 3)), log_scales=np.full((n, 3), math.log(0.2)),
             quats=rng.normal(0, 1, (n, 4)), opacity_logit=rng.normal(0, 1, n),
             coeffs=rng.normal(0, 0.1, (n, 16, 2)), phase_b=rng.normal(0, 0.1, n))
    return train.GaussianModel({k: torch.tensor(v, dtype=torch.float32) for k, v in p.items()}, device="cpu")


def test_sgd_step_uses_each_attributes_rate():
    m = _model()
    before = {k: v.detach().clone() for k, v in m.params.items()}
    for k, v in m.params.items():
        v.grad = torch.ones_like(v)
    m.step()
    assert torch.allclose(m.params["means"], before["means"] - train.mean_lr(0))
    for k, lr in train.LR.items():
        assert torch.allclose(m.params[k], before[k] - lr), k
    assert m.it == 1 and m.grad_cnt == 1
    assert torch.allclose(m.grad_sum, torch.full((6,), math.sqrt(3.0)))


def test_densify_clones_small_and_splits_large():
    m = _model(n=5)
    with torch.no_grad():
        m.params["log_scales"][3] = math.log(4.0)  # radius trace/3 = 16 > 10: large
    g = torch.zeros(5, 3)
    g[1] = torch.tensor([1e-3, 0.0, 0.0])  # selected, small: cloned
    g[3] = torch.tensor([0.0, 2e-3, 0.0])  # selected, large: split
    g[4] = torch.tensor([1e-5, 0.0, 0.0])  # below eps_mu: untouched
    m.params["means"].grad = g
    m.grad_sum += g.norm(dim=1)
    m.grad_cnt = 1
    old = {k: v.detach().clone() for k, v in m.params.items()}
    out = m.densify(generator=torch.Generator().manual_seed(0))
    assert out == {"cloned": 1, "split": 1}
    p = m.params
    assert p["means"].shape[0] == 5 + 1 + 2 - 1
    keep = [0, 1, 2, 4]
    assert torch.equal(p["means"][:4], old["means"][keep])
    # the clone: a copy of Gaussian 1 moved by one SGD step of the mean
    assert torch.allclose(p["means"][4], old["means"][1] - train.mean_lr(0) * g[1])
    assert torch.equal(p["coeffs"][4], old["coeffs"][1])
    # the split: two Gaussians with scales / 1.6, near the original
    assert torch.allclose(p["log_scales"][5:], old["log_scales"][3] - math.log(1.6))
    assert torch.all((p["means"][5:] - old["means"][3]).norm(dim=1) < 5 * 4.0 * math.sqrt(3))
    assert m.grad_cnt == 0 and m.grad_sum.shape[0] == 7


def test_prune_by_attenuation():
    m = _model(n=4)
    with torch.no_grad():
        m.params["opacity_logit"][:] = torch.tensor([0.0, -6.0, 2.0, -5.0])  # sigmoid: .5, .0025, .88, .0067
    assert m.prune() == 1
    assert m.n == 3
    assert torch.allclose(m.params["opacity_logit"], torch.tensor([0.0, 2.0, -5.0]))
