"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI, run
the oracle on the same seeded inputs, compare with the stated tolerances.  Every
comparison is recorded in PARITY (test, rays compared and excluded, L2, worst per-ray
ratio, rays outside the plain relative bar); conftest prints the summary at the end of
the run."""
from __future__ import annotations

import os

import numpy as np
import torch

import oracle
from paper_2502_01826_gb300 import _lib as L
from paper_2502_01826_gb300.render import Renderer, make_grid, received_signal, to_device

# FP32 forward vs FP64 oracle.  The bar (the benchmark spec): relative L2 error of the per-ray
# complex signal over the compared rays <= 1e-4.  Per ray, the error of a sum scales
# with the sum of its terms' magnitudes, sum_k |z_k| (the oracle's Sabs), and with the
# conditioning of the ray: an FP32 error delta_k in a pair's closest approach m2 moves
# its weight, the 1 - alpha of every pair behind it and, through the chord
# dt = 2 sqrt((9 - m2)/A), the transmittance phase 2 pi f b dt / c of everything behind
# it -- steeply for a grazing pair.  The oracle propagates delta_k = 1e-6 sqrt(C_k)
# (~ FP32 rounding of a whitened offset sqrt(C_k) long) to first order (Scond); each
# ray is held to |S_gpu - S_ref| <= 1e-4 Sabs + 4 Scond.
TOL_L2 = 1e-4
TOL_RAY = 1e-4
COND_MULT = 4.0
TOL_DB = 0.01
# Discrete decisions FP32 may take differently: the closest approach within 4 delta_k
# of the 3-sigma boundary, the exit point within 1e-5 m of the emitting sphere,
# ln prod(1 - alpha) within 4 times its propagated error (+1e-5) of ln eps_T.  A ray
# with one such decision must match the oracle with that decision taken either way;
# a ray with two or more is not compared (and counted): at most 0.1% of the rays, plus two.
BANDS = (1e-6, 1e-7, 4.0, 1e-5, 4.0, 1e-5)
MAX_EXCLUDED = 1e-3
# The plain per-ray bar |dS| <= 1e-4 (|S_ref| + 1e-2 rms(S_ref)) is reported beside the
# conditioning-aware one for every comparison (rays outside it: "plain_bar_misses").
PARITY: list = []


def oracle_pair(scene, rx, tx, f0, grid, rays=None, **kw):
    """The oracle's render and its render with every in-band decision flipped."""
    ref = oracle.render(scene, rx, tx, f0, grid, rays=rays, bands=BANDS, **kw)
    alt = oracle.render(scene, rx, tx, f0, grid, rays=rays, bands=BANDS, flip=True, **kw)
    ref["S_alt"] = alt["S"]
    ref["Sabs_alt"] = alt["Sabs"]
    ref["Scond_alt"] = alt["Scond"]
    return ref


def require_gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    L.load(build_if_missing=True)


def oracle_grid(spec: dict, **kw):
    args = dict(spec)
    args.update(kw)
    return oracle.make_grid(**args)


def gpu_render(scene: dict, rx, tx, f0, grid_spec: dict, cap=None, variant=0, fle_degree=0, **grid_kw):
    """Render all receivers on the GPU.  Returns (rays complex [n_rx, n_el*n_az], renderer,
    params on device)."""
    rx = np.asarray(rx, np.float32).reshape(-1, 3)
    grid = make_grid(**{**grid_spec, **grid_kw})
    K = scene["means"].shape[0]
    R = Renderer(K, rx.shape[0], grid, f0, pair_capacity=cap, variant=variant, fle_degree=fle_degree)
    p = to_device(scene)
    rxd = torch.tensor(rx, device="cuda")
    txd = torch.tensor(np.asarray(tx, np.float32), device="cuda")
    if cap is None:
        R.ensure_capacity(p, rxd, txd)
    out = R.forward(p, rxd, txd)
    torch.cuda.synchronize()
    S = out.cpu().numpy()
    with np.errstate(invalid="ignore"):  # outputs of a refused (non-finite) input are undefined
        S = S[..., 0] + 1j * S[..., 1]
    return S.reshape(rx.shape[0], -1), R, p, out


def compare(S_gpu: np.ndarray, ref: dict, f: int = 0, tol_l2=TOL_L2, tol_ray=TOL_RAY,
            max_excluded=MAX_EXCLUDED):
    """Compare one receiver's rays at frequency index f against ``oracle_pair``."""
    namb = ref["flags"] >> 8
    keep = namb <= 1
    S_ref = ref["S"][f].copy()
    bound = tol_ray * ref["Sabs"] + COND_MULT * ref["Scond"]
    if "S_alt" in ref:
        alt = ref["S_alt"][f]
        use_alt = (namb == 1) & (np.abs(S_gpu - alt) < np.abs(S_gpu - S_ref))
        S_ref[use_alt] = alt[use_alt]
        bound = np.maximum(bound, tol_ray * ref["Sabs_alt"] + COND_MULT * ref["Scond_alt"])
    else:
        keep = namb == 0
    a, b = S_gpu[keep], S_ref[keep]
    err = np.abs(a - b)
    nb = np.linalg.norm(b)
    l2 = np.linalg.norm(a - b) / nb if nb > 0 else (np.max(err) if err.size else 0.0)
    worst = np.max(err / (bound[keep] + 1e-30)) * tol_ray if a.size else 0.0
    excluded = int((~keep).sum())
    rms = np.sqrt(np.mean(np.abs(b) ** 2)) if b.size else 0.0
    plain_miss = int(np.sum(err > tol_ray * (np.abs(b) + 1e-2 * rms))) if a.size else 0
    rec = dict(test=os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0], l2=float(l2),
               worst=float(worst), compared=int(keep.sum()), excluded=excluded,
               ambiguous=int((namb == 1).sum()), plain_bar_misses=plain_miss)
    PARITY.append(rec)
    assert l2 <= tol_l2, "relative L2 error %.3g > %.3g" % (l2, tol_l2)
    assert worst <= tol_ray, "worst per-ray error %.3g > %.3g" % (worst, tol_ray)
    assert excluded <= max_excluded * len(keep) + 2, "%d of %d rays excluded" % (excluded, len(keep))
    return rec


def oracle_choice(S_gpu: np.ndarray, ref: dict, f: int = 0) -> np.ndarray:
    """The oracle's rays at frequency index f with, on every ray holding an in-band
    discrete decision, whichever of the two readings of it (``oracle_pair``) lies closer
    to the GPU's ray: the reference for sums over rays (CSI, RSSI)."""
    S_ref = ref["S"][f].copy()
    if "S_alt" in ref:
        alt = ref["S_alt"][f]
        use_alt = ((ref["flags"] >> 8) >= 1) & (np.abs(S_gpu - alt) < np.abs(S_gpu - S_ref))
        S_ref[use_alt] = alt[use_alt]
    return S_ref


def parity_summary() -> list[str]:
    """Lines summarising every comparison of the run (printed by conftest)."""
    if not PARITY:
        return []
    comp = sum(r["compared"] for r in PARITY)
    excl = sum(r["excluded"] for r in PARITY)
    amb = sum(r["ambiguous"] for r in PARITY)
    miss = sum(r["plain_bar_misses"] for r in PARITY)
    w = max(PARITY, key=lambda r: r["worst"])
    l2 = max(PARITY, key=lambda r: r["l2"])
    fr = max(PARITY, key=lambda r: r["excluded"] / max(1, r["compared"] + r["excluded"]))
    return ["parity vs the FP64 oracle: %d comparisons, %d rays compared, %d excluded (%.2g%%; largest share "
            "%.2g%% in %s), %d compared with one decision taken either way"
            % (len(PARITY), comp, excl, 100.0 * excl / max(1, comp + excl),
               100.0 * fr["excluded"] / max(1, fr["compared"] + fr["excluded"]), fr["test"], amb),
            "  largest relative L2 %.3g (%s); worst per-ray error %.3g of the 1e-4 bar (%s)"
            % (l2["l2"], l2["test"], w["worst"] / TOL_RAY, w["test"]),
            "  rays outside the plain bar 1e-4 (|S| + 1e-2 rms): %d of %d (%.3g%%)"
            % (miss, comp, 100.0 * miss / max(1, comp))]


def rssi_db(S) -> float:
    return float(20 * np.log10(np.abs(np.sum(np.asarray(S, np.complex128)))))
