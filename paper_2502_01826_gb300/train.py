"""The training loop around the differentiable render: the loss functions of Sec. 4.4,
per-attribute SGD with the mean's exponential learning-rate decay, and the Gaussian
count updates of App. B (gradient-threshold clone / split, pruning by attenuation).

Only PyTorch tensor operations run here; the forward and backward of the render are the
library's kernels (``render.render``).  Readings where the paper leaves a value open:
  * lambda_1 = 0.2, lambda_2 = 0.1 for the spectrum loss (no values are given);
  * F in the Fourier term is the unitary DFT, so that with the paper's 1 / (N_az N_el)
    the term is a mean over frequency bins like the L1 term (with the unnormalised DFT
    it would be, by Parseval, the sum of squared differences over all rays);
  * SSIM with an 11 x 11 Gaussian window (sigma 1.5), zero padding, constants
    (0.01 L)^2 and (0.03 L)^2 with L the target's peak value;
  * the excess-phase coefficient b (part of the complex transmittance) takes the
    attenuation's learning rate, 0.01;
  * a cloned copy moves by one SGD step of the mean along the descent direction;
  * the "radius" of a Gaussian is the mean of its covariance diagonal, trace(Sigma) / 3;
  * attenuation below eps_rho means opacity sigmoid(logit) below it;
  * spatial spectra and complex signals enter the loss divided by the target's peak
    magnitude (spectra as images in [0, 1]), so the paper's learning rates apply
    whatever the scene's absolute signal level; RSSI in dB enters as it is.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F

from . import _lib as L
from .render import Renderer, make_grid, render

# App. B learning rates: attenuation 0.01, emission (FLE coefficients) 0.0025, scaling
# 0.01, rotation 0.005; the mean from 1.6e-4 down to 1.6e-6 over 30,000 iterations
LR = {"opacity_logit": 0.01, "coeffs": 0.0025, "log_scales": 0.01, "quats": 0.005, "phase_b": 0.01}
MEAN_LR0, MEAN_LR1, MEAN_LR_STEPS = 1.6e-4, 1.6e-6, 30_000

# App. B table of hyperparameters
EPS_MU, EPS_R, EPS_RHO, N_MU, N_RHO, PHI = 2e-4, 10.0, 0.004, 100, 100, 1.6


def mean_lr(it: int, lr0: float = MEAN_LR0, lr1: float = MEAN_LR1, steps: int = MEAN_LR_STEPS) -> float:
    """Exponential decay from lr0 at iteration 0 to lr1 at ``steps`` (held after)."""
    t = min(max(it, 0) / steps, 1.0)
    return math.exp((1.0 - t) * math.log(lr0) + t * math.log(lr1))


# ----------------------------------------------------------------------------- losses

def l1_loss(pred: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """Mean absolute difference over all entries (the L1 term of Sec. 4.4)."""
    return (pred - target).abs().mean()


def _gauss_window(size: int, sigma: float, device, dtype) -> torch.Tensor:
    x = torch.arange(size, device=device, dtype=dtype) - (size - 1) / 2.0
    g = torch.exp(-0.5 * (x / sigma) ** 2)
    g = g / g.sum()
    return g


def ssim(pred: torch.Tensor, target: torch.Tensor, window: int = 11, sigma: float = 1.5,
         data_range: float | None = None) -> torch.Tensor:
    """Mean structural similarity of two stacks of 2-D maps [..., H, W] (Wang et al.'s
    index with a Gaussian window and zero padding)."""
    if data_range is None:
        data_range = float(target.detach().abs().max().clamp_min(1e-12))
    c1, c2 = (0.01 * data_range) ** 2, (0.03 * data_range) ** 2
    shape = pred.shape
    x = pred.reshape(-1, 1, shape[-2], shape[-1])
    y = target.reshape(-1, 1, shape[-2], shape[-1])
    g = _gauss_window(window, sigma, x.device, x.dtype)
    kx, ky = g.view(1, 1, 1, -1), g.view(1, 1, -1, 1)

    def blur(t):
        return F.conv2d(F.conv2d(t, kx, padding=(0, window // 2)), ky, padding=(window // 2, 0))

    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return s.mean()


def fourier_loss(pred: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """(1 / (N_az N_el)) sum over the 2-D frequency grid of |F(pred) - F(target)|^2 with F
    the unitary 2-D DFT, per map, averaged over the stack [..., N_el, N_az] (the Fourier
    term of Sec. 4.4): a mean over frequency bins, on the scale of the L1 term."""
    d = torch.fft.fft2(pred - target, norm="ortho")
    n = pred.shape[-1] * pred.shape[-2]
    return (d.real ** 2 + d.imag ** 2).sum(dim=(-2, -1)).mean() / n


def spectrum_loss(pred: torch.Tensor, target: torch.Tensor, lam1: float = 0.2, lam2: float = 0.1) -> torch.Tensor:
    """Antenna-array loss of Sec. 4.4 on spatial spectra [..., N_el, N_az]:
    (1 - lam1 - lam2) L1 + lam1 (1 - SSIM) + lam2 L_Fourier."""
    return ((1.0 - lam1 - lam2) * l1_loss(pred, target) + lam1 * (1.0 - ssim(pred, target))
            + lam2 * fourier_loss(pred, target))


def signal_loss(pred: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """Single-antenna loss of Sec. 4.4: |pred - target| summed for real power, |pred -
    target|^2 summed for a complex signal (a complex tensor, or real pairs [..., 2])."""
    if torch.is_complex(pred):
        return ((pred - target).abs() ** 2).sum()
    return (pred - target).abs().sum()


def spectrum_of(rays: torch.Tensor) -> torch.Tensor:
    """|S| per ray from the render's interleaved output [..., n_el, n_az, 2]."""
    return torch.sqrt(rays[..., 0] ** 2 + rays[..., 1] ** 2 + 1e-30)


# ----------------------------------------------------------------------------- Gaussian model

class GaussianModel:
    """The Gaussian parameters as leaf tensors, their SGD optimiser and the mean-gradient
    statistics that drive the count updates of App. B."""

    def __init__(self, params: dict, device="cuda", lr_scale: float = 1.0):
        self.params = {k: (v.detach().clone() if torch.is_tensor(v) else torch.as_tensor(v)).to(device).float()
                       .requires_grad_(True) for k, v in params.items() if v is not None}
        self.it = 0
        self.lr_scale = lr_scale
        self._reset_stats()
        self._make_optimizer()

    @property
    def n(self) -> int:
        return int(self.params["means"].shape[0])

    def _make_optimizer(self):
        groups = [{"params": [self.params["means"]], "lr": self.lr_scale * mean_lr(self.it), "name": "means"}]
        for k, lr in LR.items():
            if k in self.params:
                groups.append({"params": [self.params[k]], "lr": self.lr_scale * lr, "name": k})
        self.opt = torch.optim.SGD(groups, lr=0.0)

    def _reset_stats(self):
        dev = self.params["means"].device
        self.grad_sum = torch.zeros(self.n, device=dev)
        self.grad_cnt = 0

    def zero_grad(self):
        for v in self.params.values():
            v.grad = None

    def step(self):
        """One SGD update (App. B), the mean's learning rate taken at this iteration; adds
        |dL/dmu| per Gaussian to the statistics."""
        g = self.params["means"].grad
        if g is not None:
            self.grad_sum += g.detach().norm(dim=1)
            self.grad_cnt += 1
        for grp in self.opt.param_groups:
            if grp["name"] == "means":
                grp["lr"] = self.lr_scale * mean_lr(self.it)
        self.opt.step()
        self.it += 1

    def _replace(self, new: dict):
        self.params = {k: v.detach().contiguous().requires_grad_(True) for k, v in new.items()}
        self._reset_stats()
        self._make_optimizer()

    @torch.no_grad()
    def densify(self, eps_mu: float = EPS_MU, eps_r: float = EPS_R, phi: float = PHI, generator=None) -> dict:
        """Clone or split the Gaussians whose average mean gradient since the last update
        exceeds eps_mu (App. B): radius trace(Sigma)/3 <= eps_r clones, with the copy moved
        by one SGD step of the mean; larger ones split into two, scales / phi, positions
        drawn from the original's density.  Returns the counts."""
        p = {k: v.detach() for k, v in self.params.items()}
        if self.grad_cnt == 0:
            return {"cloned": 0, "split": 0}
        avg = self.grad_sum / self.grad_cnt
        sel = avg > eps_mu
        radius = torch.exp(2.0 * p["log_scales"]).mean(dim=1)  # trace(R S S^T R^T) / 3
        small = sel & (radius <= eps_r)
        large = sel & (radius > eps_r)
        parts = [p]
        if small.any():
            g = self.params["means"].grad
            step = self.lr_scale * mean_lr(self.it) * (g.detach()[small] if g is not None
                                                       else torch.zeros_like(p["means"][small]))
            c = {k: v[small].clone() for k, v in p.items()}
            c["means"] = c["means"] - step
            parts.append(c)
        n_large = int(large.sum())
        if n_large:
            q = p["quats"][large]
            q = q / q.norm(dim=1, keepdim=True).clamp_min(1e-12)
            R = _quat_to_rot(q)
            s = torch.exp(p["log_scales"][large])
            for _ in range(2):
                z = torch.randn(n_large, 3, device=q.device, generator=generator)
                c = {k: v[large].clone() for k, v in p.items()}
                c["means"] = c["means"] + torch.einsum("nij,nj->ni", R, s * z)
                c["log_scales"] = c["log_scales"] - math.log(phi)
                parts.append(c)
            keep = ~large
            parts[0] = {k: v[keep] for k, v in p.items()}
        new = {k: torch.cat([part[k] for part in parts]) for k in p}
        self._replace(new)
        return {"cloned": int(small.sum()), "split": n_large}

    @torch.no_grad()
    def prune(self, eps_rho: float = EPS_RHO) -> int:
        """Remove Gaussians whose attenuation (opacity) is below eps_rho (App. B)."""
        keep = torch.sigmoid(self.params["opacity_logit"].detach()) >= eps_rho
        removed = int((~keep).sum())
        if removed:
            self._replace({k: v.detach()[keep] for k, v in self.params.items()})
        return removed


def _quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1).reshape(q.shape[:-1] + (3, 3))


# ----------------------------------------------------------------------------- trainer

class Trainer:
    """One scene, fixed receivers and transmitter, a target per receiver; ``step`` runs
    forward + loss + backward + SGD and, in the first half of ``total_iters``, the count
    updates every N_mu / N_rho iterations.

    mode: "spectrum" (antenna arrays: target = |S| per ray, [n_rx, n_el, n_az]),
          "complex" (single antenna: target = the complex received signal per receiver and
          subcarrier, [n_rx, n_f]), or "power" (single antenna: target = RSSI in dB, [n_rx])."""

    def __init__(self, params: dict, rx, tx, grid_spec: dict, f0: float, df: float = 0.0, n_f: int = 1,
                 mode: str = "spectrum", lam1: float = 0.2, lam2: float = 0.1, total_iters: int = 30_000,
                 densify: bool = True, seed: int = 0, device="cuda", lr_scale: float = 1.0, n_mu: int = N_MU,
                 n_rho: int = N_RHO, eps_mu: float = EPS_MU, eps_r: float = EPS_R, eps_rho: float = EPS_RHO,
                 phi: float = PHI):
        if mode not in ("spectrum", "complex", "power"):
            raise ValueError("mode must be spectrum, complex or power")
        self.model = GaussianModel(params, device=device, lr_scale=lr_scale)
        self.n_mu, self.n_rho, self.eps_mu, self.eps_r, self.eps_rho, self.phi = n_mu, n_rho, eps_mu, eps_r, eps_rho, phi
        self.counts = {"cloned": 0, "split": 0, "pruned": 0}
        self.rx = torch.as_tensor(rx, dtype=torch.float32, device=device).reshape(-1, 3).contiguous()
        self.tx = torch.as_tensor(tx, dtype=torch.float32, device=device).reshape(3).contiguous()
        self.grid = make_grid(**grid_spec)
        self.f0, self.df, self.n_f = f0, df, n_f
        self.mode, self.lam1, self.lam2 = mode, lam1, lam2
        self.scale = None  # the target's peak magnitude, fixed at the first step
        self.total_iters = total_iters
        self.densify_on = densify
        self.gen = torch.Generator(device=device).manual_seed(seed)
        self.renderer = None
        self._renderer_for_model()

    def _renderer_for_model(self):
        p = {k: v.detach() for k, v in self.model.params.items()}
        self.renderer = Renderer(self.model.n, self.rx.shape[0], self.grid, self.f0, df_hz=self.df, n_f=self.n_f)
        self.renderer.ensure_capacity(p, self.rx, self.tx)

    def predict(self):
        """The differentiable prediction for the current mode."""
        S = render(self.renderer, self.model.params, self.rx, self.tx)  # [n_rx, n_f, n_el, n_az, 2]
        if self.mode == "spectrum":
            return spectrum_of(S[:, 0])
        tot = S.sum(dim=(2, 3))  # [n_rx, n_f, 2]
        if self.mode == "complex":
            return torch.view_as_complex(tot.contiguous())
        return 10.0 * torch.log10(tot[:, 0, 0] ** 2 + tot[:, 0, 1] ** 2 + 1e-30)  # RSSI dB

    def loss(self, pred, target):
        if self.mode == "power":
            return signal_loss(pred, target)
        if self.scale is None:
            self.scale = float(target.detach().abs().max().clamp_min(1e-30))
        if self.mode == "spectrum":
            return spectrum_loss(pred / self.scale, target / self.scale, self.lam1, self.lam2)
        return signal_loss(pred / self.scale, target / self.scale)

    def step(self, target) -> float:
        """One iteration; returns the loss (a host float: one device-to-host read).  When
        the moved Gaussians no longer fit the pair capacity, the workspace grows and the
        iteration runs again."""
        for _ in range(2):
            self.model.zero_grad()
            pred = self.predict()
            loss = self.loss(pred, target)
            loss.backward()
            st = self.renderer.status()
            if st.code != L.GSRF_ERR_CAPACITY:
                break
            self.renderer.ensure_capacity({k: v.detach() for k, v in self.model.params.items()}, self.rx, self.tx)
        L.check("render (device status)", st.code)
        self.model.step()
        it = self.model.it
        if self.densify_on and it < self.total_iters // 2:
            changed = False
            if it % self.n_mu == 0:
                c = self.model.densify(self.eps_mu, self.eps_r, self.phi, generator=self.gen)
                self.counts["cloned"] += c["cloned"]
                self.counts["split"] += c["split"]
                changed = c["cloned"] + c["split"] > 0
            if it % self.n_rho == 0:
                pr = self.model.prune(self.eps_rho)
                self.counts["pruned"] += pr
                changed = changed or pr > 0
            if changed:
                self._renderer_for_model()
        return float(loss.detach())
