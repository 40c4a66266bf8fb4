"""FP64 CPU oracle for the GSRF per-receiver render (arXiv 2502.01826).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg of
``bench.py`` load this module; the library under ``paper_2502_01826_gb300`` never
does.  It shares no code with the CUDA path: the C sources here are the whole
oracle, this file only marshals numpy arrays into them.

Parity status of each function (what pins it) is listed in ``tests/test_oracle_pins.py``;
every entry point here is pinned by at least one closed form, library routine or
brute-force check there.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = ["oracle.c", "oracle_f32.c"]
_DEPS = _SRC + ["oracle_grad.inc", "gsrf_oracle.h"]

C_LIGHT = 3.0e8


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no contraction into FMA anywhere)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    deps = [os.path.join(_HERE, s) for s in _DEPS]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(d) <= so_t for d in deps):
            return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-pthread", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Grid(C.Structure):
    _fields_ = [("n_az", C.c_int32), ("n_el", C.c_int32),
                ("az0_deg", C.c_float), ("daz_deg", C.c_float),
                ("el0_deg", C.c_float), ("del_deg", C.c_float),
                ("r_rx", C.c_float), ("eps_T", C.c_float), ("alpha_max", C.c_float),
                ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("variant", C.c_int32),
                ("fle_degree", C.c_int32)]


class Scene(C.Structure):
    _fields_ = [("n", C.c_int64),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("coeffs", C.c_void_p), ("phase_b", C.c_void_p)]


class Bands(C.Structure):
    _fields_ = [("m2_err", C.c_double), ("m2_abs", C.c_double), ("m2_mult", C.c_double),
                ("t_band", C.c_double),
                ("term_mult", C.c_double), ("term_abs", C.c_double), ("flip", C.c_int32),
                ("m2_shift", C.c_void_p), ("shift_stride", C.c_int32)]


FLAG_M2, FLAG_TOUT, FLAG_TERM = 1, 2, 4

_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.or_legendre.restype = dbl
        L.or_legendre.argtypes = [C.c_int, C.c_int, dbl]
        L.or_basis.restype = None
        L.or_basis.argtypes = [dbl, dbl, vp]
        L.or_basis_l.restype = None
        L.or_basis_l.argtypes = [dbl, dbl, i32, vp]
        L.or_gaussian.restype = None
        L.or_gaussian.argtypes = [vp, i64, vp, vp, vp]
        L.or_intersect.restype = C.c_int
        L.or_intersect.argtypes = [vp, vp, vp, vp, dbl, vp]
        for nm, na in (("or_det_exp", 1), ("or_det_atan2", 2), ("or_det_asin", 1)):
            fn = getattr(L, nm)
            fn.restype = C.c_float
            fn.argtypes = [C.c_float] * na
        L.or_depth_key_f32.restype = C.c_uint32
        L.or_depth_key_f32.argtypes = [vp, vp]
        L.or_cover_f32.restype = i32
        L.or_cover_f32.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.or_circle_f32.restype = None
        L.or_circle_f32.argtypes = [vp, vp, vp, vp, vp, vp]
        L.or_bin.restype = i64
        L.or_bin.argtypes = [vp, vp, vp, vp, vp, i64, vp]
        L.or_path_phase.restype = None
        L.or_path_phase.argtypes = [vp, vp, vp, dbl, vp]
        L.or_render.restype = C.c_int
        L.or_render.argtypes = [vp, vp, vp, dbl, dbl, i32, vp, i32, vp, i64, i32, vp,
                                vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_render_grad.restype = C.c_int
        L.or_render_grad.argtypes = [vp, vp, vp, dbl, dbl, i32, vp, i32, vp, i64, i32, vp,
                                     vp, vp, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def make_grid(n_az, n_el, az0_deg=0.0, daz_deg=None, el0_deg=0.0, del_deg=None, r_rx=1.0,
              eps_T=1e-4, alpha_max=0.99, tile_w=16, tile_h=16, variant=0, fle_degree=0) -> Grid:
    """variant: bit 1 = radiance at the Gaussian's direction, bit 2 = normalised weight,
    bit 4 = the paper's splatting-circle culling; fle_degree: L of the radiance, 0 = 3
    (see or_grid in gsrf_oracle.h)."""
    if daz_deg is None:
        daz_deg = 360.0 / n_az
    if del_deg is None:
        del_deg = 90.0 / n_el
    return Grid(n_az, n_el, az0_deg, daz_deg, el0_deg, del_deg, r_rx, eps_T, alpha_max,
                tile_w, tile_h, variant, fle_degree)


def _check_coeffs(scene: dict, grid: Grid):
    """The scene's coefficients must match the grid's degree (the C code reads
    (L + 1)^2 complex values per Gaussian)."""
    deg = grid.fle_degree if grid.fle_degree > 0 else 3
    c = np.asarray(scene["coeffs"])
    if c.ndim != 3 or c.shape[1:] != ((deg + 1) ** 2, 2):
        raise ValueError("coefficients %s do not match degree %d" % (c.shape, deg))


class _SceneRef:
    """Keeps float32 copies alive for the duration of a call."""

    def __init__(self, scene: dict):
        self.arrs = {k: _f32(scene[k]) for k in ("means", "log_scales", "quats",
                                                  "opacity_logit", "coeffs")}
        pb = scene.get("phase_b")
        self.arrs["phase_b"] = None if pb is None else _f32(pb)
        n = self.arrs["means"].shape[0]
        self.n = n
        self.c = Scene(n, _p(self.arrs["means"]), _p(self.arrs["log_scales"]),
                       _p(self.arrs["quats"]), _p(self.arrs["opacity_logit"]),
                       _p(self.arrs["coeffs"]), _p(self.arrs["phase_b"]))


def legendre(l: int, m: int, x: float) -> float:
    return lib().or_legendre(l, m, x)


def basis(alpha: float, x: float, L: int = 3) -> np.ndarray:
    Y = np.zeros(((L + 1) ** 2, 2))
    lib().or_basis_l(alpha, x, L, _p(Y))
    return Y[:, 0] + 1j * Y[:, 1]


def gaussian(scene: dict, k: int):
    s = _SceneRef(scene)
    Sg = np.zeros(9)
    Si = np.zeros(9)
    o = np.zeros(1)
    lib().or_gaussian(C.byref(s.c), k, _p(Sg), _p(Si), _p(o))
    return Sg.reshape(3, 3), Si.reshape(3, 3), float(o[0])


def intersect(Sinv, mu, r, v, r_rx):
    out = np.zeros(10)
    Si = np.ascontiguousarray(Sinv, dtype=np.float64).reshape(9)
    hit = lib().or_intersect(_p(Si), _p(np.ascontiguousarray(mu, np.float64)),
                             _p(np.ascontiguousarray(r, np.float64)),
                             _p(np.ascontiguousarray(v, np.float64)), r_rx, _p(out))
    names = ("t_in", "t_out", "t_a", "dt", "t_rep", "m2", "m2_rep", "g", "A", "C")
    return bool(hit), dict(zip(names, out))


def det_exp(x: float) -> float:
    return lib().or_det_exp(x)


def det_atan2(y: float, x: float) -> float:
    return lib().or_det_atan2(y, x)


def det_asin(s: float) -> float:
    return lib().or_det_asin(s)


def depth_key_f32(mu, r) -> int:
    return int(lib().or_depth_key_f32(_p(_f32(mu)), _p(_f32(r))))


def cover_f32(mu, log_scale, r, grid: Grid):
    mask = np.zeros(1, np.uint64)
    lo = np.zeros(1, np.int32)
    hi = np.zeros(1, np.int32)
    n = lib().or_cover_f32(_p(_f32(mu)), _p(_f32(log_scale)), _p(_f32(r)), C.byref(grid),
                           _p(mask), _p(lo), _p(hi))
    return int(n), int(mask[0]), int(lo[0]), int(hi[0])


def circle_f32(mu, log_scale, quat, r, grid: Grid):
    """The paper's splatting circle (u_k, v_k, r_k^2) in bins, decided in FP32."""
    out = np.zeros(3, np.float32)
    lib().or_circle_f32(_p(_f32(mu)), _p(_f32(log_scale)), _p(_f32(quat)), _p(_f32(r)), C.byref(grid), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def n_tiles(grid: Grid):
    ntu = (grid.n_az + grid.tile_w - 1) // grid.tile_w
    ntv = (grid.n_el + grid.tile_h - 1) // grid.tile_h
    return ntu, ntv


def bin_pairs(scene: dict, rx, grid: Grid):
    """Sorted (keys uint64, ids uint32, tile_start int64[n_tiles+1]) for one receiver."""
    s = _SceneRef(scene)
    ntu, ntv = n_tiles(grid)
    ts = np.zeros(ntu * ntv + 1, np.int64)
    rxa = _f32(rx)
    tot = -lib().or_bin(C.byref(s.c), _p(rxa), C.byref(grid), None, None, -1, _p(ts))
    keys = np.zeros(max(tot, 1), np.uint64)
    ids = np.zeros(max(tot, 1), np.uint32)
    got = lib().or_bin(C.byref(s.c), _p(rxa), C.byref(grid), _p(keys), _p(ids), tot, _p(ts))
    assert got == tot
    return keys[:tot], ids[:tot], ts


def path_phase(scene: dict, rx, tx, f: float) -> np.ndarray:
    """phi_k = 2 pi f (|t - mu_k| + |mu_k - r|) / c in [0, 2 pi), FP64."""
    s = _SceneRef(scene)
    out = np.zeros(s.n)
    lib().or_path_phase(C.byref(s.c), _p(_f32(rx)), _p(_f32(tx)), float(f), _p(out))
    return out


def render(scene: dict, rx, tx, f0: float, grid: Grid, df: float = 0.0, n_f: int = 1,
           mode: int = 0, rays=None, threads: int | None = None, bands=None, flip: bool = False,
           m2_shift=None):
    """Render one receiver.  Returns dict with S [n_f, n_rays] complex, T, Ta, Sabs, Scond,
    nhit, ntest, flags.  ``bands``: (m2_err, m2_abs, m2_mult, t_band, term_mult, term_abs).
    ``rays``: optional int array of ray indices (v * n_az + u).  ``m2_shift`` (needs
    ``bands``): [n_rays, J] array; the m2 of the j-th composited pair of each ray is moved
    by m2_shift[i, j] times its delta_k (the perturbation study of the rounding model)."""
    _check_coeffs(scene, grid)
    s = _SceneRef(scene)
    n_rays = grid.n_az * grid.n_el if rays is None else len(rays)
    ridx = None if rays is None else np.ascontiguousarray(rays, np.int32)
    S = np.zeros((n_f, n_rays, 2))
    T = np.zeros((n_f, n_rays, 2))
    Ta = np.zeros(n_rays)
    Sabs = np.zeros(n_rays)
    Scond = np.zeros(n_rays)
    nhit = np.zeros(n_rays, np.int32)
    ntest = np.zeros(n_rays, np.int32)
    flags = np.zeros(n_rays, np.uint32)
    b = None
    if bands is not None:
        b = Bands(*bands, 1 if flip else 0)
        if m2_shift is not None:
            shift = np.ascontiguousarray(m2_shift, np.float64)
            assert shift.ndim == 2 and shift.shape[0] == n_rays
            b.m2_shift = shift.ctypes.data
            b.shift_stride = shift.shape[1]
    th = threads if threads else (os.cpu_count() or 1)
    rc = lib().or_render(C.byref(s.c), _p(_f32(rx)), _p(_f32(tx)), float(f0), float(df), n_f,
                         C.byref(grid), mode, _p(ridx), n_rays, th,
                         None if b is None else C.byref(b),
                         _p(S), _p(T), _p(Ta), _p(Sabs), _p(Scond), _p(nhit), _p(ntest), _p(flags))
    if rc != 0:
        raise ValueError("or_render rejected its arguments")
    return dict(S=S[..., 0] + 1j * S[..., 1], T=T[..., 0] + 1j * T[..., 1], Ta=Ta, Sabs=Sabs,
                Scond=Scond, nhit=nhit, ntest=ntest, flags=flags)


def render_grad(scene: dict, rx, tx, f0: float, grid: Grid, G, df: float = 0.0, n_f: int = 1,
                mode: int = 0, rays=None, threads: int | None = None):
    """Gradient of sum Re(conj(G) S) with respect to the raw parameters (FP64)."""
    _check_coeffs(scene, grid)
    s = _SceneRef(scene)
    n = s.n
    n_rays = grid.n_az * grid.n_el if rays is None else len(rays)
    ridx = None if rays is None else np.ascontiguousarray(rays, np.int32)
    G = np.asarray(G).reshape(n_f, n_rays)
    Gr = np.ascontiguousarray(np.stack([G.real, G.imag], -1), np.float64)
    deg = grid.fle_degree if grid.fle_degree > 0 else 3
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logit=np.zeros(n), coeffs=np.zeros((n, (deg + 1) ** 2, 2)), phase_b=np.zeros(n))
    th = threads if threads else (os.cpu_count() or 1)
    rc = lib().or_render_grad(C.byref(s.c), _p(_f32(rx)), _p(_f32(tx)), float(f0), float(df),
                              n_f, C.byref(grid), mode, _p(ridx), n_rays, th, _p(Gr),
                              _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
                              _p(out["opacity_logit"]), _p(out["coeffs"]), _p(out["phase_b"]))
    if rc != 0:
        raise ValueError("or_render_grad rejected its arguments")
    return out


def received_signal(S: np.ndarray) -> np.ndarray:
    """Single-antenna received signal: the complex sum over rays (Sec. 4.4), FP64."""
    return np.sum(np.asarray(S, np.complex128), axis=-1)


def rssi_db(S_hat: np.ndarray) -> np.ndarray:
    """Coherent received power in dB re unit amplitude: 20 log10 |S_hat|."""
    return 20.0 * np.log10(np.abs(S_hat))
