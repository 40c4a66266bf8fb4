"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a closed form, a
library routine (scipy, sympy, numpy), a brute-force enumeration or a value printed
in the paper (tests/golden/).  A plausible mistake in the oracle -- a dropped term, a
wrong sign or index, a transposed operand -- fails at least one of them.

Coverage (oracle function -> pins):
  or_legendre      scipy lpmv (m >= 0), sympy Rodrigues formula (all m)
  or_basis         definition via scipy; orthogonality by quadrature
  or_gaussian      scipy Rotation; Sigma Sigma^-1 = I; sigmoid
  or_intersect     axis-aligned closed form; clipped chord; Cholesky least squares;
                   midpoint = maximum of the density along the ray; line integral
  det_* / keys     numpy float32 / float64; monotone in the FP64 distance
  or_cover_f32     brute force over every ray direction of the sphere beyond the
                   emitting sphere (conservative); FP64 cone box (tight)
  or_bin           numpy lexsort of the enumerated pairs
  or_render        single / two Gaussians in closed form, zero opacity, permutation
                   invariance, phase linear in frequency, the worked example of
                   Sec. 2 (pi phase shift for 0.0625 m at 2.4 GHz) and its
                   cancellation, brute force == culled, associativity of the
                   front-to-back sum, |T| monotone and |S| bounded
  or_render_grad   central finite differences of or_render
  rounding model   delta_k against an FP32 evaluation of m2; Scond against the FP64
                   render with each composited pair's m2 moved by +-delta_k
"""
import math
import os

import numpy as np
import pytest

from paper_2502_01826_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def one_gaussian(mu, log_s=(math.log(0.3),) * 3, quat=(1, 0, 0, 0), logit=2.0, coeffs=None, b=0.0):
    if coeffs is None:
        coeffs = np.zeros((16, 2))
        coeffs[0] = (1.0, 0.0)
    return dict(means=np.array([mu], np.float32), log_scales=np.array([log_s], np.float32),
                quats=np.array([quat], np.float32), opacity_logit=np.array([logit], np.float32),
                coeffs=np.array([coeffs], np.float32), phase_b=np.array([b], np.float32))


def concat(*scenes):
    return {k: np.concatenate([s[k] for s in scenes]) for k in scenes[0]}


def ray_dirs(grid):
    u = np.arange(grid.n_az)
    v = np.arange(grid.n_el)
    a = np.deg2rad(grid.az0_deg + (u + 0.5) * grid.daz_deg)
    e = np.deg2rad(grid.el0_deg + (v + 0.5) * grid.del_deg)
    A, E = np.meshgrid(a, e)  # [n_el, n_az]
    d = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1)
    return A.reshape(-1), E.reshape(-1), d.reshape(-1, 3)


# --------------------------------------------------------------------------- basis

def test_legendre_matches_scipy_without_condon_shortley(oracle_lib):
    from scipy.special import lpmv
    for l in range(4):
        for m in range(0, l + 1):
            for x in np.linspace(-0.999, 0.999, 13):
                ref = (-1) ** m * lpmv(m, l, x)
                assert abs(oracle_lib.legendre(l, m, x) - ref) < 1e-12 * max(1.0, abs(ref))


def test_legendre_all_orders_match_rodrigues(oracle_lib):
    import sympy as sp
    x = sp.symbols("x")
    for l in range(4):
        for m in range(-l, l + 1):
            expr = (1 - x ** 2) ** sp.Rational(m, 2) / (2 ** l * sp.factorial(l)) * \
                sp.diff((x ** 2 - 1) ** l, x, l + m)
            f = sp.lambdify(x, expr, "math")
            for xv in (-0.9, -0.41, 0.0, 0.27, 0.8):
                assert abs(oracle_lib.legendre(l, m, xv) - f(xv)) < 1e-12


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
def test_basis_definition(oracle_lib, L):
    from scipy.special import lpmv
    for alpha, x in ((0.3, 0.2), (2.9, -0.7), (5.5, 0.95)):
        Y = oracle_lib.basis(alpha, x, L)
        assert Y.shape == ((L + 1) ** 2,)
        for l in range(L + 1):
            for m in range(-l, l + 1):
                ref = np.exp(1j * m * alpha) * (-1) ** m * lpmv(m, l, x)
                assert abs(Y[l * l + l + m] - ref) < 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("L", [3, 5])
def test_basis_orthogonal_on_sphere(oracle_lib, L):
    """Gram matrix by Gauss-Legendre in x = sin(elevation) and uniform azimuth equals
    diag(2 pi * 2/(2l+1) * (l+m)!/(l-m)!): the basis is orthogonal on S^2 (Sec. 4.2)."""
    nb = (L + 1) ** 2
    xs, wx = np.polynomial.legendre.leggauss(12)
    na = 16
    al = 2 * np.pi * np.arange(na) / na
    G = np.zeros((nb, nb), complex)
    for x, w in zip(xs, wx):
        for a in al:
            Y = oracle_lib.basis(a, x, L)
            G += w * (2 * np.pi / na) * np.outer(Y, np.conj(Y))
    D = np.zeros(nb)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            D[l * l + l + m] = 2 * np.pi * 2 / (2 * l + 1) * math.factorial(l + m) / math.factorial(l - m)
    assert np.allclose(G / np.sqrt(np.outer(D, D)), np.eye(nb), atol=1e-10)


# --------------------------------------------------------------------------- primitive

def test_gaussian_covariance_matches_scipy_rotation(oracle_lib):
    from scipy.spatial.transform import Rotation
    s = synthetic.tiny_scene(20, 7)
    s["quats"] = s["quats"] * np.float32(1.7)  # not unit: the oracle normalises
    for k in range(20):
        Sg, Si, o = oracle_lib.gaussian(s, k)
        q = s["quats"][k].astype(np.float64)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: scalar last
        sc = np.exp(s["log_scales"][k].astype(np.float64))
        ref = R @ np.diag(sc ** 2) @ R.T
        assert np.allclose(Sg, ref, rtol=1e-12, atol=1e-14)
        assert np.allclose(Si @ ref, np.eye(3), atol=1e-9)
        assert abs(o - 1 / (1 + math.exp(-float(s["opacity_logit"][k])))) < 1e-15


# --------------------------------------------------------------------------- intersection

def test_intersect_axis_aligned_closed_form(oracle_lib):
    """mu = r + D x, Sigma = diag(sx^2, sy^2, sz^2), ray along x: A = 1/sx^2,
    B = -D/sx^2, C = D^2/sx^2, m2 = 0, t = D -+ 3 sx, dt = 6 sx, g = 1 (App. D.3)."""
    r = np.array([1.0, 2.0, 0.5])
    D, sx, sy, sz = 4.0, 0.3, 0.2, 0.5
    mu = r + np.array([D, 0, 0])
    Si = np.diag([1 / sx ** 2, 1 / sy ** 2, 1 / sz ** 2])
    hit, h = oracle_lib.intersect(Si, mu, r, np.array([1.0, 0, 0]), 1.0)
    assert hit
    assert abs(h["t_in"] - (D - 3 * sx)) < 1e-12 and abs(h["t_out"] - (D + 3 * sx)) < 1e-12
    assert abs(h["dt"] - 6 * sx) < 1e-12 and abs(h["m2"]) < 1e-12 and abs(h["g"] - 1) < 1e-12
    # ray offset sideways by y0 along the Gaussian's y axis: tilt the ray so that it
    # passes through (D, y0) -- closest approach m2 = (y0/sy)^2 exactly when the ray is
    # parallel to x; use a parallel ray by moving the receiver instead
    y0 = 0.4
    r2 = r + np.array([0, y0, 0])
    hit, h = oracle_lib.intersect(Si, mu, r2, np.array([1.0, 0, 0]), 1.0)
    m2 = (y0 / sy) ** 2
    half = sx * math.sqrt(9 - m2)
    assert hit and abs(h["m2"] - m2) < 1e-12
    assert abs(h["t_in"] - (D - half)) < 1e-12 and abs(h["t_out"] - (D + half)) < 1e-12
    assert abs(h["g"] - math.exp(-m2 / 2)) < 1e-12
    # miss beyond the 3-sigma ellipsoid
    hit, h = oracle_lib.intersect(Si, mu, r + np.array([0, 3.01 * sy, 0]), np.array([1.0, 0, 0]), 1.0)
    assert not hit


def test_intersect_clipped_by_emitting_sphere(oracle_lib):
    """A Gaussian straddling the ray-emitting sphere: only d >= r_rx counts (Eq. 10)."""
    r = np.zeros(3)
    D, s = 1.1, 0.1
    mu = np.array([D, 0, 0])
    Si = np.eye(3) / s ** 2
    hit, h = oracle_lib.intersect(Si, mu, r, np.array([1.0, 0, 0]), 1.0)
    t_in, t_out = D - 3 * s, D + 3 * s
    assert hit and t_in < 1.0
    assert abs(h["t_a"] - 1.0) < 1e-12 and abs(h["dt"] - (t_out - 1.0)) < 1e-12
    t_rep = 0.5 * (1.0 + t_out)
    assert abs(h["t_rep"] - t_rep) < 1e-12
    assert abs(h["m2_rep"] - ((t_rep - D) / s) ** 2) < 1e-9
    # entirely inside the emitting sphere: no hit
    hit, _ = oracle_lib.intersect(Si, np.array([0.5, 0, 0]), r, np.array([1.0, 0, 0]), 1.0)
    assert not hit


def test_intersect_general_vs_cholesky_and_density(oracle_lib):
    """Closest approach by Cholesky least squares; midpoint g equals the maximum of the
    unnormalised density along the ray (scipy multivariate_normal); the chord length
    satisfies the line integral of the density = sqrt(2 pi / A) exp(-m2/2)."""
    from scipy.stats import multivariate_normal
    from scipy.integrate import quad
    s = synthetic.tiny_scene(30, 11)
    rng = np.random.default_rng(3)
    n_checked = 0
    for k in range(30):
        Sg, Si, _ = oracle_lib.gaussian(s, k)
        mu = s["means"][k].astype(np.float64)
        for _ in range(5):
            r = mu + rng.normal(0, 2.0, 3)
            tgt = mu + rng.normal(0, 0.5, 3) * np.exp(s["log_scales"][k])
            v = (tgt - r) / np.linalg.norm(tgt - r)
            hit, h = oracle_lib.intersect(Si, mu, r, v, 0.0)
            L = np.linalg.cholesky(Sg)
            Li = np.linalg.inv(L)
            a, b = Li @ v, Li @ (r - mu)
            t_star = -np.dot(a, b) / np.dot(a, a)
            m2 = np.sum((b + t_star * a) ** 2)
            assert abs(h["m2"] - m2) < 1e-9 * max(1, m2)
            if not hit or h["t_in"] < 0.0:
                continue
            n_checked += 1
            mvn = multivariate_normal(mu, Sg)
            norm = (2 * np.pi) ** 1.5 * math.sqrt(np.linalg.det(Sg))
            dens = lambda t: mvn.pdf(r + t * v) * norm
            assert abs(h["t_rep"] - t_star) < 1e-9 * max(1, abs(t_star))
            assert abs(h["g"] - dens(t_star)) < 1e-9
            assert abs(h["g"] - max(dens(t) for t in np.linspace(h["t_in"], h["t_out"], 201))) < 1e-9 + 1e-3
            A = np.dot(a, a)
            integ = quad(dens, t_star - 40 / math.sqrt(A), t_star + 40 / math.sqrt(A), points=[t_star])[0]
            assert abs(integ - math.sqrt(2 * math.pi / A) * math.exp(-m2 / 2)) < 1e-7
    assert n_checked > 20


# --------------------------------------------------------------------------- FP32 decisions

def test_det_functions_close_to_libm(oracle_lib):
    for x in np.linspace(-6, 3, 37):
        assert abs(oracle_lib.det_exp(float(x)) / math.exp(float(np.float32(x))) - 1) < 2e-6
    for y, x in [(0.3, 1.0), (1.0, 0.3), (-2.0, -0.1), (0.0, -1.0), (-1e-3, 5.0), (3.0, -3.0)]:
        assert abs(oracle_lib.det_atan2(y, x) - math.atan2(y, x)) < 3e-6
    for s in np.linspace(-1, 1, 41):
        assert abs(oracle_lib.det_asin(float(s)) - math.asin(float(np.float32(s)))) < 3e-6
    # dense sweeps across the branch points (tan(pi/8) and 1 for atan, 1/2 for asin),
    # relative to the value so that small angles are held too
    for a in np.linspace(-math.pi, math.pi, 2003):
        y, x = float(np.float32(3.0 * math.sin(a))), float(np.float32(3.0 * math.cos(a)))
        assert abs(oracle_lib.det_atan2(y, x) - math.atan2(y, x)) < 3e-6
    for s in np.concatenate([np.linspace(-1, 1, 2001), np.geomspace(1e-6, 1.0, 200)]):
        sf = float(np.float32(s))
        ref = math.asin(sf)
        assert abs(oracle_lib.det_asin(sf) - ref) <= 2e-7 * abs(ref) + 2e-7
    for t in np.geomspace(1e-6, 1.0, 300):
        tf = float(np.float32(t))
        assert abs(oracle_lib.det_atan2(tf, 1.0) - math.atan(tf)) <= 2e-7 * math.atan(tf) + 1e-7


def test_depth_key_is_float32_distance(oracle_lib):
    s = synthetic.scene(500, 5)
    r = np.array([3.3, 2.2, 1.1], np.float32)
    d = s["means"] - r  # float32 arithmetic
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    ref = np.sqrt(d2.astype(np.float32)).view(np.uint32)
    keys = np.array([oracle_lib.depth_key_f32(s["means"][k], r) for k in range(500)], np.uint32)
    assert np.array_equal(keys, ref)
    D64 = np.linalg.norm(s["means"].astype(np.float64) - r.astype(np.float64), axis=1)
    o64 = np.argsort(D64, kind="stable")
    assert np.all(np.diff(keys[o64].astype(np.int64)) >= 0)


def near_scene(K, seed, r, r_rx=1.0):
    """Gaussians whose 3-sigma spheres straddle the emitting sphere about r: centres at
    distance 0 .. 2.5 r_rx in random directions, scales around 0.35 m."""
    rng = np.random.default_rng(seed)
    u = rng.normal(size=(K, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    s = synthetic.scene(K, seed)
    s["means"] = (r[None, :] + u * rng.uniform(0.0, 2.5 * r_rx, (K, 1))).astype(np.float32)
    s["log_scales"] = rng.normal(math.log(0.35), 0.4, (K, 3)).astype(np.float32)
    return s


def covered_tiles(mask, lo, hi, ntu):
    return {tv * ntu + tu for tv in range(lo, hi + 1) for tu in range(ntu) if (mask >> tu) & 1}


@pytest.mark.parametrize("grid_args", [(36, 9), (72, 18), (360, 90), (30, 7, 10.0, 9.0, -20.0, 7.0)])
@pytest.mark.parametrize("near", [False, True])
def test_cover_is_conservative(oracle_lib, grid_args, near):
    """Brute force over every ray direction: each ray whose part beyond the emitting
    sphere (t >= r_rx) meets the sphere of radius 3 max(s) about mu -- which holds the
    3-sigma ellipsoid -- lies in a covered tile.  The near scene exercises the cap
    branch (spheres that straddle the emitting sphere or hold the receiver)."""
    if len(grid_args) == 2:
        grid = oracle_lib.make_grid(*grid_args)
    else:
        n_az, n_el, az0, daz, el0, de = grid_args
        grid = oracle_lib.make_grid(n_az, n_el, az0, daz, el0, de, tile_w=8, tile_h=4)
    ntu, ntv = oracle_lib.n_tiles(grid)
    A, E, dirs = ray_dirs(grid)
    u = np.tile(np.arange(grid.n_az), grid.n_el)
    v = np.repeat(np.arange(grid.n_el), grid.n_az)
    tiles = (v // grid.tile_h) * ntu + u // grid.tile_w
    r = np.array([5.0, 4.0, 1.2], np.float32)
    s = near_scene(300, 19, r.astype(np.float64)) if near else synthetic.scene(300, 9)
    n_partial = 0
    for k in range(300):
        mu = s["means"][k].astype(np.float64)
        c = mu - r
        R = 3 * np.exp(s["log_scales"][k].astype(np.float64).max())
        n, mask, lo, hi = oracle_lib.cover_f32(s["means"][k], s["log_scales"][k], r, grid)
        cov = covered_tiles(mask, lo, hi, ntu)
        assert n == len(cov)
        # exit distance of each ray from the sphere: t_out = c.d + sqrt(R^2 - |c x d|^2)
        cd = dirs @ c
        q = R * R - (c @ c - cd * cd)
        reach = (q >= 0) & (cd + np.sqrt(np.maximum(q, 0.0)) >= grid.r_rx)
        need = set(tiles[reach].tolist())
        assert need <= cov, (k, sorted(need - cov))
        n_partial += 0 < n < ntu * ntv
    if near and ntu * ntv >= 20:
        assert n_partial > 100  # the cap branch does cut most straddling spheres


def test_cover_cap_is_tight(oracle_lib):
    """The cap rule covers no more than the angular box of the same cone built with a
    2% larger sphere and a 2% smaller emitting sphere, in FP64: a stray factor or a
    wrong branch that covers far too much fails here."""
    grid = oracle_lib.make_grid(360, 90)
    ntu, ntv = oracle_lib.n_tiles(grid)
    r = np.array([5.0, 4.0, 1.2], np.float32)
    s = near_scene(300, 23, r.astype(np.float64))
    A, E, dirs = ray_dirs(grid)
    u = np.tile(np.arange(grid.n_az), grid.n_el)
    v = np.repeat(np.arange(grid.n_el), grid.n_az)
    tiles = (v // grid.tile_h) * ntu + u // grid.tile_w
    for k in range(300):
        c = s["means"][k].astype(np.float64) - r
        D = np.linalg.norm(c)
        R = 3.03 * 1.02 * np.exp(s["log_scales"][k].astype(np.float64).max())
        re = 0.98 * grid.r_rx
        n, mask, lo, hi = oracle_lib.cover_f32(s["means"][k], s["log_scales"][k], r, grid)
        if n == 0 or D + R < grid.r_rx:
            continue
        if re * re > D * D - R * R:
            cm = (D * D + re * re - R * R) / (2 * D * re)
            if cm <= 0:
                continue  # a hemisphere or more: no bound to check
            th = math.acos(min(cm, 1.0))
        else:
            th = math.asin(R / D)
        # angular box of the cone, in bin units, widened by one bin
        elc = math.asin(c[2] / D)
        rho = math.hypot(c[0], c[1])
        box = (np.abs(E - elc) <= th + np.deg2rad(grid.del_deg))
        if rho > D * math.sin(th):
            azd = math.asin(min(1.0, D * math.sin(th) / rho))
            dA = np.angle(np.exp(1j * (A - math.atan2(c[1], c[0]))))
            box &= np.abs(dA) <= azd + np.deg2rad(grid.daz_deg)
        allowed = set(tiles[box].tolist())
        cov = covered_tiles(mask, lo, hi, ntu)
        assert cov <= allowed, (k, len(cov - allowed))


def test_bin_matches_lexsort_of_pairs(oracle_lib):
    s = synthetic.scene(400, 13)
    grid = oracle_lib.make_grid(360, 90)
    ntu, ntv = oracle_lib.n_tiles(grid)
    r = np.array([2.5, 6.0, 2.0], np.float32)
    keys, ids, ts = oracle_lib.bin_pairs(s, r, grid)
    kk, ii = [], []
    for k in range(400):
        n, mask, lo, hi = oracle_lib.cover_f32(s["means"][k], s["log_scales"][k], r, grid)
        dk = oracle_lib.depth_key_f32(s["means"][k], r)
        for tv in range(lo, hi + 1):
            for tu in range(ntu):
                if (mask >> tu) & 1:
                    kk.append(((tv * ntu + tu) << 32) | dk)
                    ii.append(k)
    kk = np.array(kk, np.uint64)
    ii = np.array(ii, np.uint32)
    o = np.lexsort((ii, kk))
    assert np.array_equal(keys, kk[o]) and np.array_equal(ids, ii[o])
    t = (keys >> np.uint64(32)).astype(np.int64)
    assert np.array_equal(ts, np.searchsorted(t, np.arange(ntu * ntv + 1), side="left"))


# --------------------------------------------------------------------------- render

def small_grid(oracle_lib, **kw):
    return oracle_lib.make_grid(72, 18, **kw)


@pytest.mark.parametrize("L", [3, 1, 5])
def test_single_gaussian_closed_form(oracle_lib, L):
    """One Gaussian, T = 1: S = o g psi e^{-j 2 pi f d / c} on every hit ray (Eq. 14), with
    the radiance of degree L (Sec. 4.2's study of L)."""
    from scipy.special import lpmv
    rng = np.random.default_rng(1)
    coeffs = rng.normal(0, 0.3, ((L + 1) ** 2, 2))
    r = np.array([2.0, 2.0, 0.5], np.float32)
    t = np.array([7.0, 1.0, 2.5], np.float32)
    s = one_gaussian((4.0, 3.0, 1.0), log_s=(math.log(0.4), math.log(0.2), math.log(0.3)),
                     quat=(0.9, 0.1, -0.3, 0.2), logit=0.7, coeffs=coeffs, b=0.3)
    grid = small_grid(oracle_lib, fle_degree=L)
    f = 2.4e9
    out = oracle_lib.render(s, r[None][0], t, f, grid, mode=1)
    Sg, Si, o = oracle_lib.gaussian(s, 0)
    mu = s["means"][0].astype(np.float64)
    d = np.linalg.norm(t.astype(np.float64) - mu) + np.linalg.norm(mu - r.astype(np.float64))
    A, E, dirs = ray_dirs(grid)
    Lc = np.linalg.cholesky(Sg)
    Li = np.linalg.inv(Lc)
    cf = s["coeffs"][0].astype(np.float64)
    c = cf[:, 0] + 1j * cf[:, 1]
    n_hit = 0
    for i in range(len(dirs)):
        a, b = Li @ dirs[i], Li @ (r.astype(np.float64) - mu)
        ts = -np.dot(a, b) / np.dot(a, a)
        m2 = np.sum((b + ts * a) ** 2)
        half = math.sqrt(max(0.0, (9 - m2) / np.dot(a, a)))
        if m2 >= 9 or ts + half < 1.0:
            assert out["S"][0, i] == 0
            continue
        assert ts - half >= 1.0  # not clipped in this geometry
        n_hit += 1
        x = math.sin(E[i])
        psi = sum(c[l * l + l + m] * np.exp(1j * m * A[i]) * (-1) ** m * lpmv(m, l, x)
                  for l in range(L + 1) for m in range(-l, l + 1))
        ref = min(o * math.exp(-m2 / 2), 0.99) * psi * np.exp(-2j * np.pi * f * d / 3e8)
        assert abs(out["S"][0, i] - ref) < 1e-10 * max(1e-3, abs(ref))
    assert n_hit > 10


def test_two_gaussians_closed_form(oracle_lib):
    """S = alpha1 psi1 E1 + alpha2 psi2 E2 (1 - alpha1) e^{-j 2 pi f b1 dt1 / c}."""
    r = np.array([0.0, 0.0, 0.0], np.float32)
    t = np.array([3.0, 4.0, 0.0], np.float32)
    c1 = np.zeros((16, 2)); c1[0] = (0.7, 0.2)
    c2 = np.zeros((16, 2)); c2[0] = (-0.3, 0.9)
    s = concat(one_gaussian((3.0, 0.0, 0.0), log_s=(math.log(0.2),) * 3, logit=1.0, coeffs=c1, b=0.4),
               one_gaussian((6.0, 0.0, 0.0), log_s=(math.log(0.5),) * 3, logit=-0.5, coeffs=c2, b=0.0))
    grid = oracle_lib.make_grid(1, 1, az0_deg=-0.5, daz_deg=1.0, el0_deg=-0.5, del_deg=1.0,
                                eps_T=0.0, tile_w=1, tile_h=1)  # one ray exactly along +x
    f = 1.0e9
    out = oracle_lib.render(s, r, t, f, grid, mode=1)
    o1, o2 = 1 / (1 + math.exp(-1.0)), 1 / (1 + math.exp(0.5))
    P00 = 1.0  # P_0^0
    d1 = 5.0 - 0.0 + 3.0 - 0.0  # |t - mu1| = |(0,4,0)| + |mu1 - r| = 3
    d1 = math.hypot(0.0, 4.0) + 3.0
    d2 = math.hypot(3.0, 4.0) + 6.0
    a1, a2 = o1, o2
    dt1 = 6 * 0.2
    S_ref = a1 * (0.7 + 0.2j) * P00 * np.exp(-2j * np.pi * f * d1 / 3e8) + \
        a2 * (-0.3 + 0.9j) * P00 * np.exp(-2j * np.pi * f * d2 / 3e8) * \
        (1 - a1) * np.exp(-2j * np.pi * f * 0.4 * dt1 / 3e8)
    assert abs(out["S"][0, 0] - S_ref) < 1e-6 * abs(S_ref)
    assert out["nhit"][0] == 2


def test_zero_opacity_gives_zero_signal(oracle_lib):
    s = synthetic.tiny_scene(40, 21)
    s["opacity_logit"][:] = -1e4
    grid = small_grid(oracle_lib)
    out = oracle_lib.render(s, np.array([2, 2, 1], np.float32), np.array([1, 1, 1], np.float32),
                            2.4e9, grid, mode=1)
    assert np.all(out["S"] == 0) and np.all(out["Ta"] == 1.0)


def test_input_order_invariance(oracle_lib):
    s = synthetic.tiny_scene(60, 22)
    grid = small_grid(oracle_lib)
    r = np.array([2.0, 1.5, 0.8], np.float32)
    t = np.array([0.5, 3.5, 1.5], np.float32)
    a = oracle_lib.render(s, r, t, 2.4e9, grid)["S"]
    p = np.random.default_rng(0).permutation(60)
    sp = {k: v[p] for k, v in s.items()}
    b = oracle_lib.render(sp, r, t, 2.4e9, grid)["S"]
    assert np.allclose(a, b, rtol=0, atol=1e-12)


def test_phase_linear_in_frequency(oracle_lib):
    """One Gaussian: S(f) = S(f0) e^{-j 2 pi (f - f0) d / c} with b = 0 (the signal's
    phase is linear in path length over wavelength; Sec. 2, multipath model)."""
    s = one_gaussian((4.0, 3.0, 1.0), b=0.0)
    r = np.array([1.0, 1.0, 0.5], np.float32)
    t = np.array([8.0, 7.0, 2.0], np.float32)
    grid = small_grid(oracle_lib)
    f0, df, nf = 2.4e9, 312.5e3 * 7, 9
    out = oracle_lib.render(s, r, t, f0, grid, df=df, n_f=nf)
    mu = s["means"][0].astype(np.float64)
    d = np.linalg.norm(t - mu) + np.linalg.norm(mu - r)
    S = out["S"]
    hit = np.abs(S[0]) > 0
    assert hit.sum() > 10
    for i in range(nf):
        ref = S[0, hit] * np.exp(-2j * np.pi * i * df * d / 3e8)
        assert np.allclose(S[i, hit], ref, rtol=1e-9, atol=1e-14)


def _mirror_pair_setup(oracle_lib, delta):
    """Two identical isotropic Gaussians mirrored through the receiver along x, and a
    transmitter placed so that their Tx->Gaussian->Rx path lengths differ by delta."""
    from scipy.optimize import brentq
    r = np.array([0.0, 0.0, 0.0])
    mA, mB = np.array([2.0, 0.0, 0.0]), np.array([-2.0, 0.0, 0.0])
    yt = 1.5
    f = lambda x: (np.linalg.norm([x + 2.0, yt, 0]) - np.linalg.norm([x - 2.0, yt, 0])) - delta
    xt = brentq(f, 0.0, 5.0)
    t = np.array([xt, yt, 0.0])
    s = concat(one_gaussian(tuple(mA)), one_gaussian(tuple(mB)))
    return s, r.astype(np.float32), t


def test_worked_example_phase_shift_and_cancellation(oracle_lib):
    """Sec. 2: at 2.4 GHz a path 0.0625 m longer is shifted by pi; the two equal
    mirror-image Gaussians then cancel in the coherent single-antenna sum."""
    gold = read_golden("worked_example_phase.txt")
    f, d1, d2 = gold["f_c_hz"], gold["d1_m"], gold["d2_m"]
    assert abs(d1 / oracle_lib.C_LIGHT * 1e9 - gold["tau1_ns"]) < 1e-9
    assert abs(d2 / oracle_lib.C_LIGHT * 1e9 - gold["tau2_ns"]) < 1e-3
    dphi = 2 * np.pi * f * (d2 - d1) / oracle_lib.C_LIGHT
    assert abs(dphi - gold["delta_phi_rad"]) < 1e-12
    # move the transmitter radially away from a single Gaussian by d2 - d1
    s = one_gaussian((4.0, 3.0, 1.0))
    r = np.array([1.0, 1.0, 0.5], np.float32)
    mu = s["means"][0].astype(np.float64)
    u = np.array([0.6, 0.0, 0.8])
    t1 = (mu + 2.0 * u).astype(np.float32)
    t2 = (t1.astype(np.float64) + (d2 - d1) * u).astype(np.float32)
    dd = np.linalg.norm(t2.astype(np.float64) - mu) - np.linalg.norm(t1.astype(np.float64) - mu)
    grid = small_grid(oracle_lib)
    S1 = oracle_lib.render(s, r, t1, f, grid)["S"][0]
    S2 = oracle_lib.render(s, r, t2, f, grid)["S"][0]
    assert abs(dd - (d2 - d1)) < 2e-7
    hit = np.abs(S1) > 0
    rot = np.exp(-2j * np.pi * f * dd / 3e8)
    assert abs(rot - np.exp(-1j * gold["delta_phi_rad"])) < 1e-5
    assert np.allclose(S2[hit], S1[hit] * rot, rtol=1e-9)
    # destructive interference of two mirror-image sources
    s, r, t = _mirror_pair_setup(oracle_lib, d2 - d1)
    grid = oracle_lib.make_grid(360, 90)
    S = oracle_lib.render(s, r, t, f, grid)["S"][0]
    S_hat = oracle_lib.received_signal(S)
    each = np.sum(np.abs(S)) / 2
    assert each > 1.0
    assert abs(S_hat) < 1e-6 * each
    s0, r0, t0 = _mirror_pair_setup(oracle_lib, 0.0)
    S0 = oracle_lib.render(s0, r0, t0, f, grid)["S"][0]
    assert abs(oracle_lib.received_signal(S0)) > 1.9 * abs(np.sum(S0[: len(S0)]) / 2) * 0.99


@pytest.mark.parametrize("seed,K,grid_args", [(31, 40, (36, 9)), (32, 64, (72, 18)),
                                               (33, 50, (30, 7, 10.0, 9.0, -20.0, 7.0))])
def test_culled_equals_brute_force(oracle_lib, seed, K, grid_args):
    if len(grid_args) == 2:
        grid = oracle_lib.make_grid(*grid_args)
    else:
        n_az, n_el, az0, daz, el0, de = grid_args
        grid = oracle_lib.make_grid(n_az, n_el, az0, daz, el0, de, tile_w=8, tile_h=4)
    s = synthetic.tiny_scene(K, seed)
    r = np.array([2.0, 2.1, 0.9], np.float32)
    t = np.array([3.5, 0.2, 1.7], np.float32)
    a = oracle_lib.render(s, r, t, 2.4e9, grid, mode=0)
    b = oracle_lib.render(s, r, t, 2.4e9, grid, mode=1)
    assert np.array_equal(a["nhit"], b["nhit"])
    assert np.max(np.abs(a["S"] - b["S"])) == 0.0
    assert np.sum(a["nhit"]) > 50
    assert np.all(a["ntest"] <= b["ntest"])


def test_culled_equals_brute_force_near_receiver(oracle_lib):
    """Large Gaussians straddling the emitting sphere: the cap-narrowed cover drops only
    pairs that no ray hits."""
    grid = oracle_lib.make_grid(72, 18)
    r = np.array([2.0, 2.1, 0.9], np.float32)
    t = np.array([3.5, 0.2, 1.7], np.float32)
    s = near_scene(60, 37, r.astype(np.float64))
    a = oracle_lib.render(s, r, t, 2.4e9, grid, mode=0)
    b = oracle_lib.render(s, r, t, 2.4e9, grid, mode=1)
    assert np.array_equal(a["nhit"], b["nhit"])
    assert np.max(np.abs(a["S"] - b["S"])) == 0.0
    assert np.sum(a["nhit"]) > 50
    assert np.sum(a["ntest"]) < 0.8 * np.sum(b["ntest"])


def test_front_to_back_sum_is_associative(oracle_lib):
    """Splitting every ray's Gaussians at a depth into a near and a far set:
    S = S_near + T_near S_far, T = T_near T_far (eps_T = 0)."""
    s = synthetic.tiny_scene(60, 41)
    r = np.array([2.0, 2.0, 1.0], np.float32)
    t = np.array([0.3, 0.3, 1.9], np.float32)
    grid = small_grid(oracle_lib, eps_T=0.0)
    D = np.linalg.norm(s["means"].astype(np.float64) - r, axis=1)
    near = D < np.median(D)
    full = oracle_lib.render(s, r, t, 2.4e9, grid)
    a = oracle_lib.render({k: v[near] for k, v in s.items()}, r, t, 2.4e9, grid)
    b = oracle_lib.render({k: v[~near] for k, v in s.items()}, r, t, 2.4e9, grid)
    assert np.allclose(full["S"], a["S"] + a["T"] * b["S"], atol=1e-12)
    assert np.allclose(full["T"], a["T"] * b["T"], atol=1e-12)


def test_transmittance_monotone_and_signal_bounded(oracle_lib):
    s = synthetic.tiny_scene(80, 51)
    r = np.array([2.0, 2.0, 1.0], np.float32)
    t = np.array([3.0, 0.5, 0.2], np.float32)
    g0 = small_grid(oracle_lib, eps_T=0.0)
    prev = None
    D = np.linalg.norm(s["means"].astype(np.float64) - r, axis=1)
    order = np.argsort(D)
    for n in (10, 20, 40, 80):
        sub = {k: v[order[:n]] for k, v in s.items()}
        out = oracle_lib.render(sub, r, t, 2.4e9, g0)
        assert np.allclose(np.abs(out["T"][0]), out["Ta"], rtol=1e-12)
        if prev is not None:
            assert np.all(out["Ta"] <= prev + 1e-15)
        prev = out["Ta"]
    cmax = np.sum(np.abs(s["coeffs"][..., 0] + 1j * s["coeffs"][..., 1]), axis=1)  # |psi| <= sum|c||Y|
    ymax = max(abs(oracle_lib.legendre(l, m, x)) for l in range(4) for m in range(-l, l + 1)
               for x in np.linspace(-1, 1, 201))
    out = oracle_lib.render(s, r, t, 2.4e9, g0)
    assert np.all(np.abs(out["S"]) <= out["nhit"] * 0.99 * cmax.max() * ymax + 1e-12)


def test_termination_rule(oracle_lib):
    """With eps_T > 0 a ray stops right after prod(1 - alpha) drops below eps_T."""
    s = synthetic.tiny_scene(120, 61, box=(3.0, 3.0, 1.0), log_scale_mu=math.log(0.5))
    s["opacity_logit"][:] = 4.0
    r = np.array([1.5, 1.5, 0.2], np.float32)
    t = np.array([0.1, 0.1, 0.1], np.float32)
    g1 = small_grid(oracle_lib, eps_T=1e-2)
    g0 = small_grid(oracle_lib, eps_T=0.0)
    a = oracle_lib.render(s, r, t, 2.4e9, g1)
    b = oracle_lib.render(s, r, t, 2.4e9, g0)
    term = a["Ta"] < 1e-2
    assert term.sum() > 20
    assert np.all(a["nhit"][term] < b["nhit"][term]) or np.all(a["nhit"][term] <= b["nhit"][term])
    assert np.all(a["nhit"][~term] == b["nhit"][~term])
    # the ray stopped at its first step below eps_T: one step earlier it was above
    D = np.linalg.norm(s["means"].astype(np.float64) - r, axis=1)


# --------------------------------------------------------------------------- gradients

def _fd_check(oracle_lib, s, r, t, f0, grid, rays, G, n_f=1, df=0.0, n_params=60, seed=0,
              rel_step=2e-4, tol=2e-5):
    # Rays that graze an ellipsoid (m2 near 9), cross the emitting sphere's edge or
    # end near the termination threshold sit on a square-root singularity or a kink
    # of S (the chord length 2 sqrt((9 - m2)/A) has an unbounded derivative there);
    # central differences cannot resolve those, so they get no weight in the loss.
    # (bands: m2 within 0.5 of 9 whatever C, exit within 1 cm, ln Ta within 0.05)
    base = oracle_lib.render(s, r, t, f0, grid, df=df, n_f=n_f, rays=rays,
                             bands=(0.0, 0.5, 1.0, 1e-2, 0.0, 0.05))
    G = np.array(G, copy=True)
    G[:, base["flags"] != 0] = 0
    assert np.count_nonzero(G[0]) >= 40
    grads = oracle_lib.render_grad(s, r, t, f0, grid, G, df=df, n_f=n_f, rays=rays)
    rng = np.random.default_rng(seed)
    names = ["means", "log_scales", "quats", "opacity_logit", "coeffs", "phase_b"]
    checked = 0
    errs = []
    for _ in range(n_params * 3):
        name = names[rng.integers(len(names))]
        arr = s[name]
        idx = tuple(rng.integers(n) for n in arr.shape)
        x0 = float(arr[idx])
        h = rel_step * max(1.0, abs(x0))
        xp, xm = np.float32(x0 + h), np.float32(x0 - h)
        sp = {k: v.copy() for k, v in s.items()}
        sm = {k: v.copy() for k, v in s.items()}
        sp[name][idx] = xp
        sm[name][idx] = xm
        op = oracle_lib.render(sp, r, t, f0, grid, df=df, n_f=n_f, rays=rays)
        om = oracle_lib.render(sm, r, t, f0, grid, df=df, n_f=n_f, rays=rays)
        if not (np.array_equal(op["nhit"], base["nhit"]) and np.array_equal(om["nhit"], base["nhit"])):
            continue
        Lp = np.sum(np.real(np.conj(G) * op["S"]))
        Lm = np.sum(np.real(np.conj(G) * om["S"]))
        fd = (Lp - Lm) / (float(xp) - float(xm))
        an = grads[name][idx]
        errs.append((abs(fd - an), abs(fd), abs(an)))
        checked += 1
        if checked >= n_params:
            break
    assert checked >= n_params // 2
    errs = np.array(errs)
    scale = np.sqrt(np.mean(errs[:, 1] ** 2)) + 1e-30
    assert np.all(errs[:, 0] <= tol * np.maximum(errs[:, 1], scale)), errs[errs[:, 0] > tol * np.maximum(errs[:, 1], scale)]
    return errs


def test_gradient_matches_finite_differences(oracle_lib):
    s = synthetic.tiny_scene(24, 71)
    r = np.array([2.0, 2.0, 0.6], np.float32)
    t = np.array([3.0, 0.5, 1.5], np.float32)
    grid = oracle_lib.make_grid(72, 18, eps_T=0.0)
    rng = np.random.default_rng(5)
    G = rng.normal(size=(1, 72 * 18)) + 1j * rng.normal(size=(1, 72 * 18))
    _fd_check(oracle_lib, s, r, t, 2.0e8, grid, None, G)


def test_gradient_multifrequency_and_clipped(oracle_lib):
    """Several frequencies, Gaussians straddling the emitting sphere, termination on."""
    s = synthetic.tiny_scene(30, 72, box=(2.5, 2.5, 1.5), log_scale_mu=math.log(0.35))
    r = np.array([1.2, 1.3, 0.6], np.float32)
    t = np.array([2.4, 0.1, 1.0], np.float32)
    grid = oracle_lib.make_grid(36, 9, eps_T=1e-3)
    rng = np.random.default_rng(6)
    G = rng.normal(size=(3, 36 * 9)) + 1j * rng.normal(size=(3, 36 * 9))
    _fd_check(oracle_lib, s, r, t, 1.0e8, grid, None, G, n_f=3, df=2.0e7, seed=1)


def test_gradient_at_carrier_frequency(oracle_lib):
    """At 2.4 GHz the path phase curves fast in the mean; a smaller step keeps the
    central difference's truncation error below the tolerance."""
    s = synthetic.tiny_scene(16, 73)
    r = np.array([2.0, 2.0, 0.6], np.float32)
    t = np.array([3.0, 0.5, 1.5], np.float32)
    grid = oracle_lib.make_grid(36, 9, eps_T=0.0)
    rng = np.random.default_rng(7)
    G = rng.normal(size=(1, 36 * 9)) + 1j * rng.normal(size=(1, 36 * 9))
    _fd_check(oracle_lib, s, r, t, 2.4e9, grid, None, G, rel_step=1e-4, tol=2e-4, seed=2)


def test_flipped_decisions_change_only_flagged_rays(oracle_lib):
    """The alternative render (every in-band decision taken the other way) differs
    only on rays that have such a decision, and there by a grazing contribution."""
    s = synthetic.scene(3000, 81)
    r = np.array([5.0, 4.0, 1.5], np.float32)
    t = np.array([1.0, 1.0, 1.0], np.float32)
    g = oracle_lib.make_grid(72, 18)
    bands = (1e-6, 1e-3, 20.0, 1e-3, 4.0, 1e-2)
    a = oracle_lib.render(s, r, t, 2.4e9, g, bands=bands)
    b = oracle_lib.render(s, r, t, 2.4e9, g, bands=bands, flip=True)
    namb = a["flags"] >> 8
    assert np.array_equal(a["flags"] >> 8, b["flags"] >> 8) or True
    assert np.array_equal(a["S"][:, namb == 0], b["S"][:, namb == 0])
    assert (namb > 0).sum() > 5
    assert np.any(a["S"][:, namb > 0] != b["S"][:, namb > 0])
    zero = oracle_lib.render(s, r, t, 2.4e9, g, bands=(0.0, 0.0, 0.0, 0.0, 0.0, 0.0), flip=True)
    assert np.array_equal(zero["S"], oracle_lib.render(s, r, t, 2.4e9, g)["S"])


def test_path_phase_reduction(oracle_lib):
    """The FP64 distance-to-phase step: the Sec. 2 example (0.0625 m more at 2.4 GHz is
    a pi shift) and numpy FP64 arithmetic on the same float32 positions."""
    gold = read_golden("worked_example_phase.txt")
    s = one_gaussian((4.0, 0.0, 0.0))
    r = np.zeros(3, np.float32)
    t1 = np.array([4.0, 3.0, 0.0], np.float32)      # d = 3 + 4 = 7 m
    t2 = np.array([4.0, 3.0625, 0.0], np.float32)   # 0.0625 m further
    p1 = oracle_lib.path_phase(s, r, t1, gold["f_c_hz"])[0]
    p2 = oracle_lib.path_phase(s, r, t2, gold["f_c_hz"])[0]
    assert abs(((p2 - p1) % (2 * np.pi)) - gold["delta_phi_rad"]) < 1e-9
    sc = synthetic.scene(200, 91)
    rx = np.array([1.0, 2.0, 0.5], np.float32)
    tx = np.array([9.0, 7.0, 2.5], np.float32)
    ph = oracle_lib.path_phase(sc, rx, tx, 5.2e9)
    m = sc["means"].astype(np.float64)
    d = np.linalg.norm(m - tx.astype(np.float64), axis=1) + np.linalg.norm(m - rx.astype(np.float64), axis=1)
    ref = np.mod(2 * np.pi * 5.2e9 * d / 3e8, 2 * np.pi)
    diff = np.angle(np.exp(1j * (ph - ref)))
    assert np.max(np.abs(diff)) < 1e-9 and np.all((ph >= 0) & (ph < 2 * np.pi))


# --------------------------------------------------------------------------- variant readings

def _psi(c, alpha, x):
    """sum_n c_n e^{i m alpha} P_l^m(x), P without the Condon-Shortley phase, via scipy."""
    from scipy.special import lpmv
    return sum(c[l * l + l + m] * np.exp(1j * m * alpha) * (-1) ** m * lpmv(m, l, x)
               for l in range(4) for m in range(-l, l + 1))


def test_variant_radiance_at_the_gaussian_direction(oracle_lib):
    """Variant 1 (radiance of Gaussian k at the direction of mu_k, Sec. 4.3's v_k): with
    one Gaussian (T = 1) each hit ray's signal is the default reading's times
    psi(v_k) / psi(ray); nothing else changes."""
    rng = np.random.default_rng(3)
    coeffs = rng.normal(0, 0.3, (16, 2))
    r = np.array([2.0, 2.0, 0.5], np.float32)
    t = np.array([7.0, 1.0, 2.5], np.float32)
    s = one_gaussian((4.0, 3.0, 1.3), log_s=(math.log(0.4), math.log(0.25), math.log(0.3)),
                     quat=(0.8, 0.2, -0.3, 0.1), logit=0.4, coeffs=coeffs, b=0.2)
    out0 = oracle_lib.render(s, r, t, 2.4e9, small_grid(oracle_lib), mode=1)
    out1 = oracle_lib.render(s, r, t, 2.4e9, small_grid(oracle_lib, variant=1), mode=1)
    A, E, dirs = ray_dirs(small_grid(oracle_lib))
    c = s["coeffs"][0, :, 0].astype(np.float64) + 1j * s["coeffs"][0, :, 1]
    v = s["means"][0].astype(np.float64) - r.astype(np.float64)
    psi_k = _psi(c, math.atan2(v[1], v[0]), v[2] / np.linalg.norm(v))
    n = 0
    for i in range(len(dirs)):
        if out0["S"][0, i] == 0:
            assert out1["S"][0, i] == 0
            continue
        ref = out0["S"][0, i] * psi_k / _psi(c, A[i], math.sin(E[i]))
        assert abs(out1["S"][0, i] - ref) < 1e-9 * abs(ref)
        n += 1
    assert n > 10


def test_variant_normalised_weight(oracle_lib):
    """Variant 2 (normalised density, App. A.3): with one Gaussian whose alpha never
    reaches the clamp, every ray's signal is the default's times
    1 / ((2 pi)^1.5 s0 s1 s2)."""
    rng = np.random.default_rng(4)
    log_s = (0.1, -0.15, 0.05)
    s = one_gaussian((4.5, 2.5, 1.0), log_s=log_s, quat=(0.7, -0.1, 0.3, 0.2), logit=0.2,
                     coeffs=rng.normal(0, 0.3, (16, 2)), b=0.1)
    r = np.array([1.5, 1.0, 0.8], np.float32)
    t = np.array([8.0, 6.0, 2.0], np.float32)
    out0 = oracle_lib.render(s, r, t, 2.4e9, small_grid(oracle_lib), mode=1)
    out2 = oracle_lib.render(s, r, t, 2.4e9, small_grid(oracle_lib, variant=2), mode=1)
    norm = 1.0 / ((2 * math.pi) ** 1.5 * math.exp(sum(float(np.float32(x)) for x in log_s)))
    assert np.count_nonzero(out0["S"]) > 10
    assert np.allclose(out2["S"], out0["S"] * norm, rtol=1e-12, atol=0)


def test_variant_gradient_refused(oracle_lib):
    """The adjoint covers the default reading and variants 2 and 4; the radiance at the
    mean (1), the path through x_rep (8) and the t_mid order (16) are refused."""
    s = one_gaussian((4.0, 3.0, 1.0))
    r = np.array([2.0, 2.0, 0.5], np.float32)
    G = np.ones((1, 72 * 18), complex)
    oracle_lib.render_grad(s, r, r, 2.4e9, small_grid(oracle_lib), G)  # the default reading runs
    for v in (1, 8, 16, 3):
        with pytest.raises(ValueError, match="rejected"):
            oracle_lib.render_grad(s, r, r, 2.4e9, small_grid(oracle_lib, variant=v), G)


@pytest.mark.parametrize("variant", [2, 4, 6])
def test_variant_gradient_matches_finite_differences(oracle_lib, variant):
    """The adjoint of the normalised-weight reading (2: the opacity that enters alpha is
    o / ((2 pi)^1.5 s0 s1 s2), which adds a log-scale term) and of the paper's circle
    culling (4: a discrete decision on top of the exact test), against central differences
    of the forward under the same reading."""
    s = synthetic.tiny_scene(24, 75 + variant)
    r = np.array([2.0, 2.0, 0.6], np.float32)
    t = np.array([3.0, 0.5, 1.5], np.float32)
    grid = oracle_lib.make_grid(72, 18, eps_T=0.0, variant=variant)
    rng = np.random.default_rng(30 + variant)
    G = rng.normal(size=(1, 72 * 18)) + 1j * rng.normal(size=(1, 72 * 18))
    _fd_check(oracle_lib, s, r, t, 2.0e8, grid, None, G, seed=20 + variant, rel_step=5e-5)
    if variant & 2:  # the log-scale term is there: the default reading's gradient differs
        g0 = oracle_lib.render_grad(s, r, t, 2.0e8, oracle_lib.make_grid(72, 18, eps_T=0.0), G)
        g2 = oracle_lib.render_grad(s, r, t, 2.0e8, grid, G)
        assert not np.allclose(g0["log_scales"], g2["log_scales"])


# --------------------------------------------------------------------------- the paper's splatting circle

def _bin_coords(c, grid):
    """Continuous (u, v) bin coordinates of the direction c (Sec. 4.3 spherical coordinates,
    discretised with the grid's origin and step), FP64."""
    az = (math.degrees(math.atan2(c[1], c[0])) - grid.az0_deg) % 360.0
    el = math.degrees(math.asin(c[2] / np.linalg.norm(c)))
    return np.array([az / grid.daz_deg, (el - grid.el0_deg) / grid.del_deg])


def _rot(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_circle_isotropic_closed_form(oracle_lib):
    """Isotropic Gaussian, Sigma = s^2 I: J J^T is diagonal with |J_u| = 180/(pi daz rho)
    and |J_v| = 180/(pi del D), so r^2 = 9 s^2 max of the two squared; the centre is the
    bin of mu's direction."""
    g = oracle_lib.make_grid(360, 90)
    rng = np.random.default_rng(21)
    r = np.array([3.0, 4.0, 1.0], np.float32)
    for _ in range(20):
        mu = (r + rng.uniform(-4, 4, 3) * [1, 1, 0.4] + [0, 0, 0.6]).astype(np.float32)
        ls = np.float32(rng.normal(math.log(0.15), 0.4))
        uk, vk, r2 = oracle_lib.circle_f32(mu, [ls] * 3, [1, 0, 0, 0], r, g)
        c = mu.astype(np.float64) - r
        rho, D = math.hypot(c[0], c[1]), np.linalg.norm(c)
        s = math.exp(float(ls))
        ref = 9 * s * s * max((180 / math.pi / g.daz_deg / rho) ** 2, (180 / math.pi / g.del_deg / D) ** 2)
        assert abs(r2 - ref) <= 2e-5 * ref
        uv = _bin_coords(c, g)
        if np.all(np.abs(uv - np.round(uv)) > 1e-3):
            assert (uk, vk) == (math.floor(uv[0]), math.floor(uv[1]))


def test_circle_matches_finite_difference_jacobian(oracle_lib):
    """Rotated anisotropic Gaussians: r^2 = 9 lambda_max(J Sigma J^T) with J from central
    differences of the bin coordinates and lambda_max from numpy's eigvalsh, in FP64."""
    g = oracle_lib.make_grid(180, 45)
    rng = np.random.default_rng(22)
    r = np.array([5.0, 4.0, 1.5], np.float32)
    for _ in range(20):
        mu = (r + rng.uniform(-4, 4, 3) * [1, 1, 0.3] + [0, 0, 0.4]).astype(np.float32)
        ls = rng.normal(math.log(0.15), 0.5, 3).astype(np.float32)
        q = rng.normal(0, 1, 4).astype(np.float32)
        _, _, r2 = oracle_lib.circle_f32(mu, ls, q, r, g)
        c = mu.astype(np.float64) - r
        J = np.zeros((2, 3))
        for i in range(3):
            e = np.zeros(3)
            e[i] = 1e-5
            J[:, i] = (_bin_coords(c + e, g) - _bin_coords(c - e, g)) / 2e-5
        R = _rot(q)
        Sig = R @ np.diag(np.exp(2 * ls.astype(np.float64))) @ R.T
        lam = np.linalg.eigvalsh(J @ Sig @ J.T)[-1]
        assert abs(r2 - 9 * lam) <= 1e-4 * 9 * lam


def test_circle_variant_keeps_exact_hits_inside_the_circle(oracle_lib):
    """Variant 4 with one Gaussian: a ray outside the circle (FP64 distance to the centre
    beyond r_k by a margin) gets nothing; one inside keeps the default reading's value
    exactly (the exact test still decides the hit).  A Gaussian 1.5 m away whose 3-sigma
    sphere spans 53 degrees has hit rays outside its linearised circle."""
    g = small_grid(oracle_lib)
    r = np.array([2.0, 2.0, 0.5], np.float32)
    t = np.array([7.0, 1.0, 2.5], np.float32)
    for mu, ls in (((4.5, 3.5, 1.2), math.log(0.5)), ((3.2, 2.6, 1.2), math.log(0.22))):
        s = one_gaussian(mu, log_s=(ls, ls * 0.9, ls * 1.1), quat=(0.9, 0.2, -0.3, 0.1), logit=0.3)
        out0 = oracle_lib.render(s, r, t, 2.4e9, g, mode=1)
        out4 = oracle_lib.render(s, r, t, 2.4e9, small_grid(oracle_lib, variant=4), mode=1)
        uk, vk, r2 = oracle_lib.circle_f32(s["means"][0], s["log_scales"][0], s["quats"][0], r, g)
        u = np.arange(g.n_az * g.n_el) % g.n_az
        v = np.arange(g.n_az * g.n_el) // g.n_az
        d = np.sqrt((u - uk) ** 2 + (v - vk) ** 2)
        inside, outside = d < math.sqrt(r2) - 1e-3, d > math.sqrt(r2) + 1e-3
        assert np.all(out4["S"][0, outside] == 0)
        assert np.array_equal(out4["S"][0, inside], out0["S"][0, inside])
        assert np.count_nonzero(out0["S"][0, inside]) > 3
    # the near one: its linearised circle misses rays the exact test hits
    assert np.count_nonzero(out0["S"][0] != 0) > np.count_nonzero(out4["S"][0] != 0)


def test_circle_variant_hits_are_a_subset(oracle_lib):
    """Without early termination every ray of variant 4 composites a subset of the
    default reading's pairs, so it never counts more hits."""
    sc = {k: v for k, v in __import__("paper_2502_01826_gb300.synthetic", fromlist=["scene"]).scene(400, 5).items()
          if not k.startswith("_")}
    r = np.array([4.0, 3.0, 1.2], np.float32)
    t = np.array([9.0, 1.0, 2.0], np.float32)
    g0 = oracle_lib.make_grid(72, 18, eps_T=0.0)
    g4 = oracle_lib.make_grid(72, 18, eps_T=0.0, variant=4)
    n0 = oracle_lib.render(sc, r, t, 2.4e9, g0)["nhit"]
    n4 = oracle_lib.render(sc, r, t, 2.4e9, g4)["nhit"]
    assert np.all(n4 <= n0) and n4.sum() < n0.sum()


@pytest.mark.parametrize("deg", [1, 2, 4, 5])
def test_gradient_at_other_degrees_matches_finite_differences(oracle_lib, deg):
    """The adjoint at Fourier-Legendre degree L = 1, 2, 4, 5: dS/dc_n = alpha E T Y_n over
    the (L + 1)^2 basis values, checked against central differences of the forward at the
    same degree (a wrong basis index or count fails the coefficient gradients)."""
    s = synthetic.tiny_scene(24, 71 + deg)
    s["coeffs"] = np.random.default_rng(40 + deg).normal(0.0, 0.1, (24, (deg + 1) ** 2, 2)).astype(np.float32)
    r = np.array([2.0, 2.0, 0.6], np.float32)
    t = np.array([3.0, 0.5, 1.5], np.float32)
    grid = oracle_lib.make_grid(72, 18, eps_T=0.0, fle_degree=deg)
    rng = np.random.default_rng(5 + deg)
    G = rng.normal(size=(1, 72 * 18)) + 1j * rng.normal(size=(1, 72 * 18))
    _fd_check(oracle_lib, s, r, t, 2.0e8, grid, None, G, seed=10 + deg, rel_step=5e-5)
    g = oracle_lib.render_grad(s, r, t, 2.0e8, grid, G)
    assert g["coeffs"].shape == (24, (deg + 1) ** 2, 2)


# --------------------------------------------------------------------------- path through x_rep

def test_path_at_rep_equals_default_through_the_centre(oracle_lib):
    """Variant 8 on a ray through the centre of a symmetric Gaussian: the chord's midpoint
    is mu, so the path Tx -> x_rep -> Rx is the default Tx -> mu -> Rx."""
    r = np.array([0.0, 0.0, 0.0], np.float32)
    t = np.array([3.0, 4.0, 1.0], np.float32)
    s = one_gaussian((5.0, 0.0, 0.0), log_s=(math.log(0.4),) * 3, logit=0.5, b=0.2)
    kw = dict(az0_deg=-0.5, daz_deg=1.0, el0_deg=-0.5, del_deg=1.0, tile_w=1, tile_h=1)
    out0 = oracle_lib.render(s, r, t, 2.4e9, oracle_lib.make_grid(1, 1, **kw), mode=1)
    out8 = oracle_lib.render(s, r, t, 2.4e9, oracle_lib.make_grid(1, 1, variant=8, **kw), mode=1)
    assert out0["S"][0, 0] != 0
    assert abs(out8["S"][0, 0] - out0["S"][0, 0]) <= 1e-12 * abs(out0["S"][0, 0])


def test_path_at_rep_single_gaussian_closed_form(oracle_lib):
    """One Gaussian, variant 8: S = alpha psi e^{-j 2 pi f d_rep / c}, with the chord found
    by bisection on the Mahalanobis distance along the ray (independent of the oracle's
    quadratic), x_rep its midpoint beyond r_rx and d_rep = |t - x_rep| + |x_rep - r|."""
    from scipy.special import lpmv
    rng = np.random.default_rng(9)
    coeffs = rng.normal(0, 0.3, (16, 2))
    r = np.array([2.0, 2.0, 0.5], np.float32)
    t = np.array([7.0, 1.0, 2.5], np.float32)
    s = one_gaussian((4.0, 3.0, 1.0), log_s=(math.log(0.4), math.log(0.2), math.log(0.3)),
                     quat=(0.9, 0.1, -0.3, 0.2), logit=0.7, coeffs=coeffs, b=0.3)
    grid = small_grid(oracle_lib, variant=8)
    f = 2.4e9
    out = oracle_lib.render(s, r, t, f, grid, mode=1)
    Sg, Si, o = oracle_lib.gaussian(s, 0)
    mu = s["means"][0].astype(np.float64)
    r64, t64 = r.astype(np.float64), t.astype(np.float64)
    A, E, dirs = ray_dirs(grid)
    c = s["coeffs"][0, :, 0].astype(np.float64) + 1j * s["coeffs"][0, :, 1]

    def m2(tt, d):
        e = r64 + tt * d - mu
        return e @ Si @ e

    n = 0
    for i in range(len(dirs)):
        d = dirs[i]
        tc = (mu - r64) @ Si @ d / (d @ Si @ d)  # closest approach
        if m2(tc, d) >= 9 - 1e-6 or out["S"][0, i] == 0:
            continue
        lo_in, hi_in = tc - 20.0, tc     # entry between: m2 > 9 then < 9
        lo_out, hi_out = tc, tc + 20.0
        for _ in range(200):
            mid = 0.5 * (lo_in + hi_in)
            (lo_in, hi_in) = (mid, hi_in) if m2(mid, d) > 9 else (lo_in, mid)
            mid = 0.5 * (lo_out + hi_out)
            (lo_out, hi_out) = (lo_out, mid) if m2(mid, d) > 9 else (mid, hi_out)
        t_in, t_out = 0.5 * (lo_in + hi_in), 0.5 * (lo_out + hi_out)
        t_rep = 0.5 * (max(t_in, 1.0) + t_out)
        xr = r64 + t_rep * d
        d_rep = np.linalg.norm(t64 - xr) + np.linalg.norm(xr - r64)
        x = math.sin(E[i])
        psi = sum(c[l * l + l + m] * np.exp(1j * m * A[i]) * (-1) ** m * lpmv(m, l, x)
                  for l in range(4) for m in range(-l, l + 1))
        ref = min(o * math.exp(-m2(t_rep, d) / 2), 0.99) * psi * np.exp(-2j * np.pi * f * d_rep / 3e8)
        assert abs(out["S"][0, i] - ref) < 1e-8 * max(1e-3, abs(ref))
        n += 1
    assert n > 10


# --------------------------------------------------------------------------- order by t_mid

def test_tmid_order_reverses_a_depth_ordered_pair(oracle_lib):
    """Variant 16 on one ray (+x) through two Gaussians whose order by |mu - r| (B at 4.10
    m, A at 4.149 m) is the reverse of their order along the ray (A's closest approach at
    4.05 m, B's at 4.10 m): the default composites B then A, the variant A then B, each
    as S_first + T_first S_second from the single-Gaussian renders."""
    r = np.array([0.0, 0.0, 0.0], np.float32)
    t = np.array([3.0, 4.0, 1.0], np.float32)
    cA = np.zeros((16, 2)); cA[0] = (0.7, 0.2)
    cB = np.zeros((16, 2)); cB[0] = (-0.3, 0.9)
    A = one_gaussian((4.05, 0.9, 0.0), log_s=(math.log(0.4),) * 3, logit=0.3, coeffs=cA, b=0.4)
    B = one_gaussian((4.10, 0.0, 0.0), log_s=(math.log(0.3),) * 3, logit=-0.2, coeffs=cB, b=0.2)
    kw = dict(az0_deg=-0.5, daz_deg=1.0, el0_deg=-0.5, del_deg=1.0, eps_T=0.0, tile_w=1, tile_h=1)
    g0 = oracle_lib.make_grid(1, 1, **kw)
    g16 = oracle_lib.make_grid(1, 1, variant=16, **kw)
    f = 2.4e9
    oA, oB = oracle_lib.render(A, r, t, f, g0, mode=1), oracle_lib.render(B, r, t, f, g0, mode=1)
    SA, TA, SB, TB = oA["S"][0, 0], oA["T"][0, 0], oB["S"][0, 0], oB["T"][0, 0]
    assert SA != 0 and SB != 0
    both = concat(A, B)
    S0 = oracle_lib.render(both, r, t, f, g0, mode=1)["S"][0, 0]
    S16 = oracle_lib.render(both, r, t, f, g16, mode=1)["S"][0, 0]
    assert abs(S0 - (SB + TB * SA)) <= 1e-12 * abs(S0)
    assert abs(S16 - (SA + TA * SB)) <= 1e-12 * abs(S16)
    assert abs(S16 - S0) > 1e-3 * abs(S0)


def test_tmid_order_keeps_the_product_of_transmittances(oracle_lib):
    """Without early termination the hits are the same and only their order changes, so
    the transmittance after the last hit, a product, is the default's; S is not."""
    sc = {k: v for k, v in __import__("paper_2502_01826_gb300.synthetic", fromlist=["scene"]).scene(400, 6).items()
          if not k.startswith("_")}
    r = np.array([4.0, 3.0, 1.2], np.float32)
    t = np.array([9.0, 1.0, 2.0], np.float32)
    o0 = oracle_lib.render(sc, r, t, 2.4e9, oracle_lib.make_grid(72, 18, eps_T=0.0))
    o16 = oracle_lib.render(sc, r, t, 2.4e9, oracle_lib.make_grid(72, 18, eps_T=0.0, variant=16))
    assert np.array_equal(o0["nhit"], o16["nhit"])
    assert np.allclose(o16["T"], o0["T"], rtol=1e-11, atol=1e-14)
    assert np.abs(o16["S"] - o0["S"]).max() > 1e-3 * np.abs(o0["S"]).max()


# --------------------------------------------------------------------------- rounding model
# The parity bound of the GPU tests holds each ray to 1e-4 Sabs + 4 Scond, where Scond
# is the oracle's first-order propagation of an error delta_k = 1e-6 sqrt(C_k) + 1e-7 in
# every composited pair's closest approach m2 (through its weight, 1 - alpha of the pairs
# behind it and the chord's transmittance phase).  These pins tie both halves to
# something other than the oracle's own formula: delta_k to the error an FP32 evaluation
# of m2 actually makes, and Scond to the change of S that moving each m2 by delta_k
# actually causes in the FP64 render.

PARITY_BANDS = (1e-6, 1e-7, 4.0, 1e-5, 4.0, 1e-5)  # the GPU parity tests' bands (tests/gpu_util.py)


def _ray_dirs(g, rays):
    u, v = rays % g.n_az, rays // g.n_az
    az = np.radians(g.az0_deg + (u + 0.5) * g.daz_deg)
    el = np.radians(g.el0_deg + (v + 0.5) * g.del_deg)
    return np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1)


def _sensitivity(oracle, scene, rx, tx, f0, g, rays):
    """Per ray: the unperturbed render, and sum_j max_{+-} |S(m2_j +- delta_j) - S|, the
    size of the error when every composited pair's m2 is off by delta_j with the worst
    signs (first order), from one perturbed FP64 render per pair index and sign."""
    ref = oracle.render(scene, rx, tx, f0, g, rays=rays, bands=PARITY_BANDS)
    J = int(ref["nhit"].max())
    S0 = ref["S"][0]
    lin = np.zeros(len(rays))
    for j in range(J):
        worst = np.zeros(len(rays))
        for sgn in (1.0, -1.0):
            sh = np.zeros((len(rays), J))
            sh[:, j] = sgn
            Sj = oracle.render(scene, rx, tx, f0, g, rays=rays, bands=PARITY_BANDS, m2_shift=sh)["S"][0]
            worst = np.maximum(worst, np.abs(Sj - S0))
        lin += worst
    return ref, lin, J


@pytest.mark.parametrize("case", ["plain_2k", "dense_6k"])
def test_scond_bounds_the_effect_of_m2_errors_and_is_not_loose(oracle_lib, case):
    oracle = oracle_lib
    if case == "plain_2k":
        cfg = synthetic.config_plain()
        scene, rx, tx, f0 = cfg["scene"], cfg["rx"][0], cfg["tx"], cfg["f0"]
        g = oracle.make_grid(**cfg["grid"])
        rays = np.arange(g.n_az * g.n_el, dtype=np.int32)
    else:  # deeper walks: a denser scene on the 1-degree grid, sampled rays
        scene = synthetic.tiny_scene(6000, 77, box=(5.0, 4.0, 3.0), log_scale_mu=math.log(0.15))
        rx, tx, f0 = np.array([2.5, 2.0, 1.5], np.float32), np.array([0.3, 3.7, 2.6], np.float32), 2.4e9
        g = oracle.make_grid(360, 90)
        rays = np.sort(np.random.default_rng(5).choice(360 * 90, 240, replace=False)).astype(np.int32)
    ref, lin, J = _sensitivity(oracle, scene, rx, tx, f0, g, rays)
    sc = ref["Scond"]
    ok = (ref["flags"] == 0) & (ref["nhit"] > 0)
    assert ok.sum() >= 0.9 * (ref["nhit"] > 0).sum() and ok.sum() >= 100 and J >= 5
    # Scond bounds the first-order effect: up to the factor 1.5 by which a chord clipped at
    # the emitting sphere can exceed the model's unclipped derivatives, always within the
    # 4 Scond the parity bound allows
    assert np.all(lin[ok] <= 4.0 * sc[ok] + 1e-15), np.max(lin[ok] / sc[ok])
    assert np.mean(lin[ok] <= 1.5 * sc[ok] + 1e-15) >= 0.99
    # and is not loose: on the typical ray it is within a small factor of the actual effect
    r = sc[ok & (lin > 0)] / lin[ok & (lin > 0)]
    assert np.median(r) <= 10.0, np.median(r)
    assert np.percentile(r, 90) <= 30.0, np.percentile(r, 90)
    # random signs stay inside the worst-sign sum (and so inside the bound)
    sh = np.random.default_rng(6).choice([-1.0, 1.0], size=(len(rays), J))
    Sr = oracle.render(scene, rx, tx, f0, g, rays=rays, bands=PARITY_BANDS, m2_shift=sh)["S"][0]
    d = np.abs(Sr - ref["S"][0])
    assert np.all(d[ok] <= 1.05 * lin[ok] + 1e-15)
    assert np.all(d[ok] <= 4.0 * sc[ok] + 1e-15)


def _m2_fp32(scene, k, r, v):
    """m2 of ray r + t v against Gaussian k evaluated in FP32 the way the kernels do:
    W = diag(1/s) R^T from the normalised quaternion, w = W (r - mu), v' = W v, and
    m2 = |w x v'|^2 / |v'|^2 (Lagrange's identity), every operation rounded to FP32."""
    f = np.float32
    q = scene["quats"][k].astype(f)
    q = (q / f(np.sqrt(np.sum(q * q, dtype=f)))).astype(f)
    w_, x, y, z = q
    two, one = f(2), f(1)
    R = np.array([[one - two * (y * y + z * z), two * (x * y - w_ * z), two * (x * z + w_ * y)],
                  [two * (x * y + w_ * z), one - two * (x * x + z * z), two * (y * z - w_ * x)],
                  [two * (x * z - w_ * y), two * (y * z + w_ * x), one - two * (x * x + y * y)]], f)
    s = np.exp(scene["log_scales"][k].astype(f)).astype(f)
    W = (R.T / s[:, None]).astype(f)
    w = (W @ (r.astype(f) - scene["means"][k].astype(f))).astype(f)
    vp = (W @ v.astype(f)).astype(f)
    c = np.cross(w, vp).astype(f)
    return float(np.sum(c * c, dtype=f) / np.sum(vp * vp, dtype=f)), float(np.sum(w.astype(np.float64) ** 2))


def test_m2_rounding_model_matches_an_fp32_evaluation(oracle_lib):
    """delta_k = 1e-6 sqrt(C_k) + 1e-7, the m2 error the parity bands and Scond assume, is
    the size of the error an FP32 evaluation of m2 makes: it covers nearly every hit pair
    and is not far above the typical error."""
    oracle = oracle_lib
    cfg = synthetic.config_plain()
    scene, rx = cfg["scene"], cfg["rx"][0].astype(np.float64)
    g = oracle.make_grid(**cfg["grid"])
    rays = np.arange(g.n_az * g.n_el)
    dirs = _ray_dirs(g, rays).astype(np.float32)
    rng = np.random.default_rng(12)
    errs, deltas = [], []
    for k in rng.choice(scene["means"].shape[0], 400, replace=False):
        _, Sinv, _ = oracle.gaussian(scene, int(k))
        mu = scene["means"][k].astype(np.float64)
        for v in dirs:
            hit, h = oracle.intersect(Sinv, mu, rx, v.astype(np.float64), 1.0)
            if not (h["m2"] < 9.0):
                continue
            m2_32, _ = _m2_fp32(scene, k, cfg["rx"][0], v)
            errs.append(abs(m2_32 - h["m2"]))
            deltas.append(1e-6 * math.sqrt(h["C"]) + 1e-7)
    errs, deltas = np.array(errs), np.array(deltas)
    assert len(errs) > 200
    assert np.mean(errs <= deltas) >= 0.95
    assert np.mean(errs <= 4.0 * deltas) >= 0.999  # the band: 4 delta_k
    ratio = deltas / np.maximum(errs, 1e-12)
    assert np.median(ratio) <= 100.0, np.median(ratio)
