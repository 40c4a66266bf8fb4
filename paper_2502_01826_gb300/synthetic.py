"""Seeded synthetic inputs shaped like the paper's RFID / BLE / CSI workloads.

This module only draws random numbers and lays out positions; it holds none of the
render's arithmetic.  Both the CUDA path (tests, benchmark) and the oracle consume
what it returns, which is why it lives on its own.

The paper's datasets (RFID and BLE from NeRF^2, Argos CSI) are not available here;
these scenes stand in for them with the paper's shapes: a 360x90 one-degree receiving
grid over the front hemisphere, 915 MHz / 2.4 GHz / 5.2 GHz carriers, single
antennas and four-element arrays, many receivers against one transmitter.

Draw order for a scene of K Gaussians, numpy PCG64(seed):
    means        U([0,10] x [0,8] x [0,3]) m          [K,3]
    log_scales   N(ln 0.15, 0.5)  (standard deviation) [K,3]
    quats        N(0,1)^4, normalised to unit length    [K,4]  (w, x, y, z)
    opacity      logit ~ N(0,1)                         [K]
    coeffs       N(0, 0.1) real and imaginary parts     [K,16,2]
    phase_b      N(0, 0.1)                              [K]
then receiver positions U(box) [n_rx,3], then the transmitter U(box) [3].
"""
from __future__ import annotations

import math

import numpy as np

BOX = (10.0, 8.0, 3.0)
BASE_SEED = 2502_01826
C_LIGHT = 3.0e8


def scene(K: int, seed: int, fle_degree: int = 3) -> dict:
    """K Gaussians in the box; (L + 1)^2 complex Fourier-Legendre coefficients each for
    degree L = fle_degree (16 for the paper's L = 3)."""
    g = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(BOX, np.float64)
    means = g.uniform(0.0, 1.0, size=(K, 3)) * box
    log_scales = g.normal(math.log(0.15), 0.5, size=(K, 3))
    q = g.normal(0.0, 1.0, size=(K, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity_logit = g.normal(0.0, 1.0, size=K)
    coeffs = g.normal(0.0, 0.1, size=(K, (fle_degree + 1) ** 2, 2))
    phase_b = g.normal(0.0, 0.1, size=K)
    return dict(means=means.astype(np.float32), log_scales=log_scales.astype(np.float32),
                quats=q.astype(np.float32), opacity_logit=opacity_logit.astype(np.float32),
                coeffs=coeffs.astype(np.float32), phase_b=phase_b.astype(np.float32),
                _rng=g)


def positions(g: np.random.Generator, n: int) -> np.ndarray:
    return (g.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(BOX)).astype(np.float32)


def grid_spec(n_az: int, n_el: int) -> dict:
    """Receiving-plane grid over azimuth [0, 360) and elevation [0, 90)."""
    return dict(n_az=n_az, n_el=n_el, az0_deg=0.0, daz_deg=360.0 / n_az, el0_deg=0.0,
                del_deg=90.0 / n_el)


def strip(s: dict) -> dict:
    return {k: v for k, v in s.items() if not k.startswith("_")}


def config_plain(seed_offset: int = 0) -> dict:
    """Plain forward, one receiver: 2,048 Gaussians, 36x9 (10 degree) grid, 2.4 GHz."""
    s = scene(2048, BASE_SEED + 0 + seed_offset)
    rx = positions(s["_rng"], 1)
    tx = positions(s["_rng"], 1)[0]
    return dict(name="plain_fwd_2k_36x9", scene=strip(s), rx=rx, tx=tx, f0=2.4e9, df=0.0,
                n_f=1, grid=grid_spec(36, 9))


def config_ble(K: int = 50_000, n_rx: int = 64, seed_offset: int = 0) -> dict:
    """BLE-RSSI shaped: 50,000 Gaussians, 64 receivers, 360x90 grid, 2.4 GHz."""
    s = scene(K, BASE_SEED + 1 + seed_offset)
    rx = positions(s["_rng"], n_rx)
    tx = positions(s["_rng"], 1)[0]
    return dict(name="ble_50k_64rx_360x90", scene=strip(s), rx=rx, tx=tx, f0=2.4e9, df=0.0,
                n_f=1, grid=grid_spec(360, 90))


def config_train(K: int = 200_000, n_rx: int = 16) -> dict:
    """Training step: 200,000 Gaussians, 16 receivers, 360x90, 2.4 GHz, plus a
    separately seeded ground-truth set of the same size."""
    s = scene(K, BASE_SEED + 2)
    rx = positions(s["_rng"], n_rx)
    tx = positions(s["_rng"], 1)[0]
    gt = scene(K, BASE_SEED + 2 + 1000)
    return dict(name="train_%dk_%drx_360x90" % (K // 1000, n_rx), scene=strip(s), gt_scene=strip(gt), rx=rx, tx=tx,
                f0=2.4e9, df=0.0, n_f=1, grid=grid_spec(360, 90))


def config_csi(K: int = 100_000, gt: bool = False) -> dict:
    """CSI shaped: 100,000 Gaussians, 8 receivers x 4 elements spaced half a carrier
    wavelength along x, 64 subcarriers at 312.5 kHz around 5.2 GHz, 180x45 grid.  With
    gt=True also a separately seeded ground-truth set of the same size."""
    s = scene(K, BASE_SEED + 3)
    centres = positions(s["_rng"], 8)
    tx = positions(s["_rng"], 1)[0]
    lam = C_LIGHT / 5.2e9
    off = (np.arange(4) - 1.5) * lam / 2.0
    rx = np.repeat(centres.astype(np.float64), 4, axis=0)
    rx[:, 0] += np.tile(off, 8)
    out = dict(name="csi_100k_8x4rx_64sc_180x45", scene=strip(s), rx=rx.astype(np.float32),
               tx=tx, f0=5.2e9 - 32 * 312.5e3, df=312.5e3, n_f=64, grid=grid_spec(180, 45))
    if gt:
        out["gt_scene"] = strip(scene(K, BASE_SEED + 3 + 1000))
    return out


def config_million(n_rx: int = 8) -> dict:
    """Training at the top of the uneven workload's range: 1,000,000 Gaussians from the
    same distributions, n_rx receivers, 360x90, 2.4 GHz, and a separately seeded
    ground-truth set of the same size."""
    K = 1_000_000
    s = scene(K, BASE_SEED + 5)
    rx = positions(s["_rng"], n_rx)
    tx = positions(s["_rng"], 1)[0]
    gt = scene(K, BASE_SEED + 5 + 1000)
    return dict(name="train_1m_%drx_360x90" % n_rx, scene=strip(s), gt_scene=strip(gt), rx=rx, tx=tx, f0=2.4e9,
                df=0.0, n_f=1, grid=grid_spec(360, 90))


def config_uneven(n_scenes: int = 8, n_req: int = 256, k_lo: float = 1e4, k_hi: float = 1e6):
    """Uneven serving stress: scenes with log-uniform Gaussian counts, requests with
    1-32 receivers and a 2.4 or 5.2 GHz carrier, 360x90 grids."""
    g = np.random.Generator(np.random.PCG64(BASE_SEED + 4))
    Ks = np.exp(g.uniform(math.log(k_lo), math.log(k_hi), size=n_scenes)).astype(np.int64)
    scenes = [strip(scene(int(K), BASE_SEED + 4 + 100 + i)) for i, K in enumerate(Ks)]
    reqs = []
    for _ in range(n_req):
        si = int(g.integers(0, n_scenes))
        nrx = int(g.integers(1, 33))
        f = float(g.choice([2.4e9, 5.2e9]))
        rx = positions(g, nrx)
        tx = positions(g, 1)[0]
        reqs.append(dict(scene=si, rx=rx, tx=tx, f0=f))
    return dict(name="uneven_8scenes_256req", scenes=scenes, requests=reqs,
                grid=grid_spec(360, 90))


def tiny_scene(K: int, seed: int, box=(4.0, 4.0, 2.0), log_scale_mu=math.log(0.3)) -> dict:
    """Small scenes for brute-force pins and edge cases."""
    g = np.random.Generator(np.random.PCG64(seed))
    means = g.uniform(0.0, 1.0, size=(K, 3)) * np.asarray(box)
    log_scales = g.normal(log_scale_mu, 0.4, size=(K, 3))
    q = g.normal(0.0, 1.0, size=(K, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return dict(means=means.astype(np.float32), log_scales=log_scales.astype(np.float32),
                quats=q.astype(np.float32),
                opacity_logit=g.normal(0.0, 1.0, size=K).astype(np.float32),
                coeffs=g.normal(0.0, 0.1, size=(K, 16, 2)).astype(np.float32),
                phase_b=g.normal(0.0, 0.1, size=K).astype(np.float32))
