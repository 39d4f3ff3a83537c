"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` instance and raises
AssertionError when the oracle disagrees with:
  * closed forms of a single Gaussian (projection, EWA Jacobian, rotation
    conventions, blended value, Eq. 10 threshold and the adjusted radius),
  * adaptive quadrature of the annulus integral behind Eq. 8-9 and the pixel
    (Riemann) sum it replaces,
  * the textbook table of real spherical harmonics (Condon-Shortley phase) and
    their orthonormality on the sphere,
  * brute-force enumeration (pixel coverage of the tile rectangle, untiled
    rendering, and an ideal render with no footprint at all),
  * the ellipse tile test against the closed form of an axis-aligned conic and
    a dense sampling of every tile (and plain mode with it rendering exactly
    the square-footprint image),
  * invariants stated by the paper (Th >= tau, Th > sigma culls, larger K drops
    pairs, the blend always uses the unscaled covariance),
  * FP64 central finite differences of the forward (backward pin).

The same functions run against deliberately broken oracle builds in
``test_oracle_mutants.py`` to show that plausible mistakes are caught.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from paper_2604_18980_gb300 import synth

TAU = oracle.TAU
C0 = 0.5 / math.sqrt(math.pi)     # Y_0^0


def axis_camera(W, H, f, R=None, campos=(0.0, 0.0, 0.0)):
    R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
    c = np.asarray(campos, dtype=np.float64)
    vm = np.concatenate([R, (-R @ c)[:, None]], 1)
    return dict(width=W, height=H, fx=f, fy=f, cx=(W - 1) / 2.0, cy=(H - 1) / 2.0, viewmat=vm,
                campos=c, near=0.2)


def one_gaussian(pos, scales, quat=(1.0, 0.0, 0.0, 0.0), opacity=0.7, dc=(0.2, -0.3, 0.4), extra_sh=None):
    sh = np.zeros((16, 3, 1))
    sh[0, :, 0] = dc
    if extra_sh is not None:
        sh[:, :, 0] += extra_sh
    return dict(mean=np.asarray(pos, dtype=np.float64).reshape(3, 1),
                log_scale=np.log(np.asarray(scales, dtype=np.float64)).reshape(3, 1),
                quat=np.asarray(quat, dtype=np.float64).reshape(4, 1),
                opacity_logit=np.array([math.log(opacity / (1.0 - opacity))]), sh=sh)


def concat(*scenes):
    out = {}
    for k in scenes[0]:
        out[k] = np.concatenate([s[k] for s in scenes], axis=-1)
    return out


# --------------------------------------------------------------------------
# Closed form 1: isotropic Gaussian on the optical axis, mean at a pixel centre
# --------------------------------------------------------------------------
def pin_isotropic_on_axis(orc):
    W = H = 65
    f, d, s, sig = 80.0, 2.0, 0.05, 0.7
    cam = axis_camera(W, H, f)
    sc = one_gaussian((0.0, 0.0, d), (s, s, s), quat=(0.3, -0.5, 0.2, 0.7), opacity=sig)
    lam = (f * s / d) ** 2 + 0.3
    rgb = np.array([0.2, -0.3, 0.4]) * C0 + 0.5
    par = oracle.params(cam, scale_mode=0)
    out = orc.render(sc, cam, par)
    g = out["dbl"][0]
    np.testing.assert_allclose([g[oracle.F_U], g[oracle.F_V]], [32.0, 32.0], atol=1e-12)
    np.testing.assert_allclose(g[oracle.F_DEPTH], d, rtol=1e-14)
    np.testing.assert_allclose([g[oracle.F_COVA], g[oracle.F_COVB], g[oracle.F_COVC]], [lam, 0.0, lam],
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose([g[oracle.F_A], g[oracle.F_B], g[oracle.F_C]], [1 / lam, 0.0, 1 / lam],
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g[oracle.F_DET], lam * lam, rtol=1e-12)
    np.testing.assert_allclose(g[oracle.F_OPAC], sig, rtol=1e-12)
    np.testing.assert_allclose(g[oracle.F_R:oracle.F_BL + 1], rgb, rtol=1e-12)
    r = math.ceil(3 * math.sqrt(lam))
    ir = out["irec"][0]
    assert ir[oracle.I_RADIUS] == r
    # pixel centres 32-r .. 32+r -> tiles
    assert (ir[oracle.I_X0], ir[oracle.I_X1]) == ((32 - r) // 16, (32 + r) // 16 + 1)
    img = out["image"]
    np.testing.assert_allclose(img[:, 32, 32], min(0.99, sig) * rgb, rtol=1e-12)
    for k in range(1, 9):
        a = sig * math.exp(-k * k / (2 * lam))
        exp = a * rgb if a >= TAU else np.zeros(3)
        np.testing.assert_allclose(img[:, 32, 32 + k], exp, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(img[:, 32 - k, 32], exp, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["final_T"][32, 32], 1 - sig, rtol=1e-12)

    # AdaGScale with T_up = 1: Th = K / (2 pi lambda) + tau (sqrt(det) = lambda)
    for K in (0.05, 0.5, 2.0):
        par = oracle.params(cam, scale_mode=1, K=K)
        o2 = orc.render(sc, cam, par)
        th = K / (2 * math.pi * lam) + TAU
        np.testing.assert_allclose(o2["dbl"][0][oracle.F_TH], th, rtol=1e-12)
        ra = math.ceil(math.sqrt(lam) * min(3.0, math.sqrt(2 * math.log(sig / th))))
        assert o2["irec"][0][oracle.I_RADIUS] == ra
        assert (o2["irec"][0][oracle.I_X0], o2["irec"][0][oracle.I_X1]) == ((32 - ra) // 16, (32 + ra) // 16 + 1)
        assert len(o2["ids"]) == ((32 + ra) // 16 + 1 - (32 - ra) // 16) ** 2
        # dual size: the blend is unchanged where the pair survives
        np.testing.assert_array_equal(o2["image"][:, 32, 32], img[:, 32, 32])
    # K large enough that Th > sigma: culled
    Kc = (sig - TAU) * 2 * math.pi * lam * 1.001
    o3 = orc.render(sc, cam, oracle.params(cam, scale_mode=1, K=Kc))
    assert o3["irec"][0][oracle.I_CULL] == oracle.CULL_TH and len(o3["ids"]) == 0
    # LUT: depth 2 falls in bin floor(2 / 5) = 0 of 20 bins over [0, 100]
    lut = np.ones(20)
    lut[0] = 0.25
    o4 = orc.render(sc, cam, oracle.params(cam, scale_mode=1, K=0.5, lut=lut))
    np.testing.assert_allclose(o4["dbl"][0][oracle.F_TH], 0.5 / (0.25 * 2 * math.pi * lam) + TAU, rtol=1e-12)
    lut = np.ones(20)
    lut[1] = 0.25   # bin 1 must not be used at depth 2
    o5 = orc.render(sc, cam, oracle.params(cam, scale_mode=1, K=0.5, lut=lut))
    np.testing.assert_allclose(o5["dbl"][0][oracle.F_TH], 0.5 / (2 * math.pi * lam) + TAU, rtol=1e-12)
    # T_up = 0 for the bin: Th infinite -> culled
    lut[0] = 0.0
    o6 = orc.render(sc, cam, oracle.params(cam, scale_mode=1, K=0.5, lut=lut))
    assert o6["irec"][0][oracle.I_CULL] == oracle.CULL_TUP


# --------------------------------------------------------------------------
# Closed form 2: off-axis isotropic Gaussian (the off-diagonal Jacobian terms)
# and the 1.3 tan(fov/2) frustum clamp
# --------------------------------------------------------------------------
def pin_off_axis_jacobian(orc):
    W, H, f = 200, 120, 150.0
    cam = axis_camera(W, H, f)
    for (x, y, d, s) in ((0.3, -0.2, 2.0, 0.02), (-0.5, 0.25, 3.0, 0.04)):
        sc = one_gaussian((x, y, d), (s, s, s), quat=(0.1, 0.9, -0.3, 0.2))
        g = orc.preprocess(sc, cam, oracle.params(cam))[0][0]
        JJ = np.array([[f * f / d ** 2 * (1 + x * x / d ** 2), f * f * x * y / d ** 4],
                       [f * f * x * y / d ** 4, f * f / d ** 2 * (1 + y * y / d ** 2)]])
        S = s * s * JJ + 0.3 * np.eye(2)
        np.testing.assert_allclose([g[oracle.F_COVA], g[oracle.F_COVB], g[oracle.F_COVC]],
                                   [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-12)
        np.testing.assert_allclose([g[oracle.F_U], g[oracle.F_V]], [f * x / d + (W - 1) / 2, f * y / d + (H - 1) / 2],
                                   rtol=1e-13)
        Si = np.linalg.inv(S)
        np.testing.assert_allclose([g[oracle.F_A], g[oracle.F_B], g[oracle.F_C]], [Si[0, 0], Si[0, 1], Si[1, 1]],
                                   rtol=1e-11)
        lam = 0.5 * (S[0, 0] + S[1, 1]) + math.sqrt(max(0.1, (0.5 * (S[0, 0] + S[1, 1])) ** 2 - np.linalg.det(S)))
        np.testing.assert_allclose(g[oracle.F_LAMBDA], lam, rtol=1e-12)
    # clamp: x/z beyond 1.3 * (W/2)/f -> the Jacobian uses the clamped x, the mean does not
    d, s = 2.0, 0.05
    lim = 1.3 * (0.5 * W / f)
    x = 1.6 * lim * d
    sc = one_gaussian((x, 0.0, d), (s, s, s))
    g = orc.preprocess(sc, cam, oracle.params(cam))[0][0]
    xc = lim * d
    np.testing.assert_allclose(g[oracle.F_COVA], s * s * f * f / d ** 2 * (1 + xc * xc / d ** 2) + 0.3, rtol=1e-12)
    np.testing.assert_allclose(g[oracle.F_U], f * x / d + (W - 1) / 2, rtol=1e-13)


# --------------------------------------------------------------------------
# Closed form 3: quaternion convention (w, x, y, z) and the camera rotation W
# --------------------------------------------------------------------------
def pin_rotation_conventions(orc):
    W = H = 101
    f, d = 120.0, 2.5
    cam = axis_camera(W, H, f)
    th = math.radians(30.0)
    s1, s2, s3 = 0.06, 0.02, 0.01
    sc = one_gaussian((0.0, 0.0, d), (s1, s2, s3), quat=(math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)))
    g = orc.preprocess(sc, cam, oracle.params(cam))[0][0]
    c, s = math.cos(th), math.sin(th)
    Sxy = np.array([[c * c * s1 ** 2 + s * s * s2 ** 2, c * s * (s1 ** 2 - s2 ** 2)],
                    [c * s * (s1 ** 2 - s2 ** 2), s * s * s1 ** 2 + c * c * s2 ** 2]])
    S = (f / d) ** 2 * Sxy + 0.3 * np.eye(2)
    np.testing.assert_allclose([g[oracle.F_COVA], g[oracle.F_COVB], g[oracle.F_COVC]],
                               [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-12)
    # an un-normalised quaternion describes the same rotation
    sc2 = one_gaussian((0.0, 0.0, d), (s1, s2, s3), quat=(3 * math.cos(th / 2), 0.0, 0.0, 3 * math.sin(th / 2)))
    g2 = orc.preprocess(sc2, cam, oracle.params(cam))[0][0]
    np.testing.assert_allclose(g2[oracle.F_COVA:oracle.F_COVC + 1], g[oracle.F_COVA:oracle.F_COVC + 1], rtol=1e-12)
    # camera looking along world +x with z up: camera x = -world y, camera y = -world z
    Rc = np.array([[0.0, -1.0, 0.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0]])
    cam2 = axis_camera(W, H, f, R=Rc)
    sx, sy, sz = 0.03, 0.05, 0.02
    sc3 = one_gaussian((d, 0.0, 0.0), (sx, sy, sz))
    g3 = orc.preprocess(sc3, cam2, oracle.params(cam2))[0][0]
    np.testing.assert_allclose([g3[oracle.F_COVA], g3[oracle.F_COVB], g3[oracle.F_COVC]],
                               [(f / d) ** 2 * sy ** 2 + 0.3, 0.0, (f / d) ** 2 * sz ** 2 + 0.3], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g3[oracle.F_DEPTH], d, rtol=1e-14)
    # a point at world (d, 0.1, 0.05) lands left of and above the centre
    sc4 = one_gaussian((d, 0.1, 0.05), (sx, sy, sz))
    g4 = orc.preprocess(sc4, cam2, oracle.params(cam2))[0][0]
    np.testing.assert_allclose([g4[oracle.F_U], g4[oracle.F_V]], [50.0 - f * 0.1 / d, 50.0 - f * 0.05 / d], rtol=1e-13)


# --------------------------------------------------------------------------
# Eq. 8-10: the annulus integral, by adaptive quadrature and by pixel sums
# --------------------------------------------------------------------------
def _annulus_integral(A, B, C, sig, lo, hi):
    """Integral of sig*exp(-Q/2) over tau_lo <= alpha < hi, Q = A dx^2 + 2B dx dy + C dy^2."""
    from scipy import integrate

    def radial(phi):
        rho = A * math.cos(phi) ** 2 + 2 * B * math.cos(phi) * math.sin(phi) + C * math.sin(phi) ** 2
        r_out = math.sqrt(2 * math.log(sig / lo) / rho)
        r_in = math.sqrt(2 * math.log(sig / hi) / rho) if hi < sig else 0.0
        val, _ = integrate.quad(lambda r: sig * math.exp(-0.5 * r * r * rho) * r, r_in, r_out,
                                epsabs=1e-13, epsrel=1e-11)
        return val

    val, _ = integrate.quad(radial, 0.0, 2 * math.pi, epsabs=1e-12, epsrel=1e-10, limit=200)
    return val


def pin_eq9_quadrature(orc):
    W = H = 257
    f, d = 300.0, 2.0
    cam = axis_camera(W, H, f)
    sig = 0.8
    sc = one_gaussian((0.0, 0.0, d), (0.07, 0.03, 0.02), quat=(0.9, 0.1, 0.2, 0.35), opacity=sig)
    for K in (0.5, 5.0):
        lut = np.full(20, 0.6)
        g = orc.preprocess(sc, cam, oracle.params(cam, scale_mode=1, K=K, lut=lut))[0][0]
        A, B, C = g[oracle.F_A], g[oracle.F_B], g[oracle.F_C]
        th = g[oracle.F_TH]
        assert TAU <= th < sig
        # Eq. 5 with the integral form (Eq. 8): T_up * integral_{tau <= alpha < Th} alpha = K
        ps = 0.6 * _annulus_integral(A, B, C, sig, TAU, th)
        np.testing.assert_allclose(ps, K, rtol=1e-7)
        # Eq. 9 at other levels x
        for x in (0.01, 0.1, 0.5, sig):
            np.testing.assert_allclose(_annulus_integral(A, B, C, sig, TAU, x),
                                       2 * math.pi * math.sqrt(g[oracle.F_DET]) * (x - TAU), rtol=1e-7)


def pin_eq8_riemann_pixels(orc):
    """Pixel sum of alpha over tau <= alpha < x is within 1% of Eq. 9 for a large Gaussian."""
    W = H = 161
    f, d, sig = 200.0, 2.0, 0.3          # sigma <= 0.35: the 3-sigma square covers alpha >= tau
    cam = axis_camera(W, H, f)
    dc = (0.5 / C0,) * 3                 # colour 1 in every channel: image = alpha
    sc = one_gaussian((0.013, -0.007, d), (0.2, 0.11, 0.05), quat=(0.8, 0.0, 0.0, 0.6), opacity=sig, dc=dc)
    out = orc.render(sc, cam, oracle.params(cam))
    g = out["dbl"][0]
    lam = g[oracle.F_LAMBDA]
    assert 300 < lam < 500
    a = out["image"][0]
    np.testing.assert_allclose(out["image"][1], a, rtol=1e-13)
    for x in (0.02, 0.1, 0.2, sig + 1e-9):
        sel = (a >= TAU) & (a < x)
        approx = 2 * math.pi * math.sqrt(g[oracle.F_DET]) * (min(x, sig) - TAU)
        np.testing.assert_allclose(a[sel].sum(), approx, rtol=1e-2)


# --------------------------------------------------------------------------
# Spherical harmonics: textbook table (Condon-Shortley phase) + orthonormality
# --------------------------------------------------------------------------
def sh_table(x, y, z):
    p = math.pi
    return np.array([
        0.5 / math.sqrt(p),
        -math.sqrt(3 / (4 * p)) * y, math.sqrt(3 / (4 * p)) * z, -math.sqrt(3 / (4 * p)) * x,
        0.5 * math.sqrt(15 / p) * x * y, -0.5 * math.sqrt(15 / p) * y * z,
        0.25 * math.sqrt(5 / p) * (3 * z * z - 1), -0.5 * math.sqrt(15 / p) * x * z,
        0.25 * math.sqrt(15 / p) * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * p)) * y * (3 * x * x - y * y), 0.5 * math.sqrt(105 / p) * x * y * z,
        -0.25 * math.sqrt(21 / (2 * p)) * y * (5 * z * z - 1), 0.25 * math.sqrt(7 / p) * (5 * z ** 3 - 3 * z),
        -0.25 * math.sqrt(21 / (2 * p)) * x * (5 * z * z - 1), 0.25 * math.sqrt(105 / p) * z * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * p)) * x * (x * x - 3 * y * y),
    ])


def pin_sh_basis(orc):
    rng = np.random.default_rng(7)
    dirs = rng.standard_normal((40, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    dirs = np.concatenate([dirs, np.eye(3), -np.eye(3)])
    Y = orc.sh_basis(3, dirs)
    for i, d in enumerate(dirs):
        np.testing.assert_allclose(Y[i], sh_table(*d), rtol=1e-12, atol=1e-14)
    # orthonormality: Gauss-Legendre in z times uniform phi (exact for these degrees)
    zs, wz = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * (2 * math.pi / 32)
    pts, wts = [], []
    for z, w in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            pts.append((r * math.cos(ph), r * math.sin(ph), z))
            wts.append(w * 2 * math.pi / 32)
    Yq = orc.sh_basis(3, np.array(pts))
    G = (Yq * np.array(wts)[:, None]).T @ Yq
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def pin_sh_colour(orc):
    """Colour = sum_k sh_k Y_k(dir) + 0.5, clamped at zero, with dir from the camera centre."""
    W = H = 33
    cam = axis_camera(W, H, 40.0, campos=(0.1, -0.2, -1.0))
    rng = np.random.default_rng(3)
    extra = rng.normal(0, 0.3, size=(16, 3))
    extra[0] = 0.0
    pos = np.array([0.2, 0.1, 1.5])
    sc = one_gaussian(pos, (0.01, 0.01, 0.01), dc=(0.1, -2.5, 0.3), extra_sh=extra)
    dbl, irec = orc.preprocess(sc, cam, oracle.params(cam))
    d = pos - np.array([0.1, -0.2, -1.0])
    d /= np.linalg.norm(d)
    sh = sc["sh"][:, :, 0]
    rgb = sh_table(*d) @ sh + 0.5
    clamped = rgb < 0
    rgb = np.maximum(rgb, 0.0)
    np.testing.assert_allclose(dbl[0, oracle.F_R:oracle.F_BL + 1], rgb, rtol=1e-12, atol=1e-14)
    assert (irec[0, oracle.I_CLAMP] & 7) == sum(1 << c for c in range(3) if clamped[c])
    assert clamped[1]


# --------------------------------------------------------------------------
# Brute force: tile rectangles by pixel enumeration; untiled and ideal renders
# --------------------------------------------------------------------------
def tiny_scene(n, seed, opacity_max=None, W=64, H=48):
    scene = synth.scene_uniform_cube(n, seed)
    scene["mean"] *= 0.6
    scene["log_scale"] += 1.0
    if opacity_max is not None:
        sig = 1.0 / (1.0 + np.exp(-scene["opacity_logit"].astype(np.float64)))
        sig = np.minimum(sig, opacity_max)
        scene["opacity_logit"] = np.log(sig / (1 - sig)).astype(np.float32)
    cam = synth.cams_sphere(1, seed + 1, 3.0, W, H)[0]
    return scene, cam


def pin_rect_enumeration(orc):
    for mode, K in ((0, 0.0), (1, 0.2)):
        scene, cam = tiny_scene(300, 11)
        W, H = cam["width"], cam["height"]
        dbl, irec = orc.preprocess(scene, cam, oracle.params(cam, scale_mode=mode, K=K))
        px, py = np.meshgrid(np.arange(W), np.arange(H))
        for i in range(len(irec)):
            r = irec[i, oracle.I_RADIUS]
            if irec[i, oracle.I_CULL] not in (oracle.CULL_NONE, oracle.CULL_EMPTY):
                continue
            u, v = dbl[i, oracle.F_U], dbl[i, oracle.F_V]
            inside = (np.abs(px - u) <= r) & (np.abs(py - v) <= r) if r > 0 else np.zeros_like(px, bool)
            tiles = set(zip((px[inside] // 16).tolist(), (py[inside] // 16).tolist()))
            x0, y0, x1, y1 = (irec[i, k] for k in (oracle.I_X0, oracle.I_Y0, oracle.I_X1, oracle.I_Y1))
            got = {(tx, ty) for tx in range(x0, x1) for ty in range(y0, y1)} if irec[i, oracle.I_TOUCHED] else set()
            assert got == tiles, (i, got, tiles)


def _ideal_render(dbl, irec, W, H, cull_ok):
    """Blend every Gaussian at every pixel in (fp32 depth, id) order; no footprint test."""
    order = sorted([i for i in range(len(dbl)) if cull_ok(irec[i])],
                   key=lambda i: (np.float32(dbl[i, oracle.F_DEPTH]), i))
    img = np.zeros((3, H, W))
    for y in range(H):
        for x in range(W):
            T, col = 1.0, np.zeros(3)
            for i in order:
                g = dbl[i]
                dx, dy = g[oracle.F_U] - x, g[oracle.F_V] - y
                p = -0.5 * (g[oracle.F_A] * dx * dx + g[oracle.F_C] * dy * dy) - g[oracle.F_B] * dx * dy
                if p > 0:
                    continue
                a = min(0.99, g[oracle.F_OPAC] * math.exp(p))
                if a < TAU:
                    continue
                tT = T * (1 - a)
                if tT < 1e-4:
                    break
                col += g[oracle.F_R:oracle.F_BL + 1] * a * T
                T = tT
            img[:, y, x] = col
    return img


def pin_bruteforce(orc):
    scene, cam = tiny_scene(160, 21)
    par = oracle.params(cam, bg=(0.1, 0.2, 0.3))
    tiled = orc.render(scene, cam, par)["image"]
    brute = orc.render_bruteforce(scene, cam, par)
    np.testing.assert_array_equal(tiled, brute)
    par = oracle.params(cam, scale_mode=1, K=0.05)
    np.testing.assert_array_equal(orc.render(scene, cam, par)["image"], orc.render_bruteforce(scene, cam, par))


def pin_ideal_render(orc):
    """With opacities <= 0.35 the 3-sigma square covers all alpha >= tau: tiling loses nothing."""
    scene, cam = tiny_scene(120, 31, opacity_max=0.35, W=48, H=40)
    par = oracle.params(cam)
    out = orc.render(scene, cam, par)
    ideal = _ideal_render(out["dbl"], out["irec"], cam["width"], cam["height"],
                          lambda r: r[oracle.I_CULL] in (oracle.CULL_NONE, oracle.CULL_EMPTY))
    np.testing.assert_allclose(out["image"], ideal, rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------
def _pairs(out, W):
    ts, ids = out["tile_start"], out["ids"]
    tile = np.repeat(np.arange(len(ts) - 1), np.diff(ts))
    return set(zip(tile.tolist(), ids.tolist()))


def pin_invariants(orc):
    scene, cams, _ = synth.workload("c1_cube16k_256", n=3000, width=96, height=80)
    cam = cams[0]
    plain = orc.render(scene, cam, oracle.params(cam))
    P = _pairs(plain, cam["width"])
    prev = None
    for K in (0.0, 0.1, 0.3, 1.0, 3.0, 10.0):
        par = oracle.params(cam, scale_mode=1, K=K)
        ada = orc.render(scene, cam, par)
        A = _pairs(ada, cam["width"])
        assert A <= P, "AdaGScale added a pair"
        if prev is not None:
            assert A <= prev, "pair set not monotone in K"
        prev = A
        live = ada["irec"][:, oracle.I_CULL] != oracle.CULL_NONFINITE
        th = ada["dbl"][live, oracle.F_TH]
        assert np.all(th[np.isfinite(th)] >= TAU)                       # Th >= tau (Sec. 3.3)
        culled = ada["irec"][:, oracle.I_CULL] == oracle.CULL_TH
        np.testing.assert_array_equal(culled, ada["dbl"][:, oracle.F_TH] > ada["dbl"][:, oracle.F_OPAC])
        # dual size: features of surviving Gaussians identical to plain mode
        surv = ada["irec"][:, oracle.I_CULL] == oracle.CULL_NONE
        np.testing.assert_array_equal(ada["dbl"][surv, :oracle.F_DEPTH + 1], plain["dbl"][surv, :oracle.F_DEPTH + 1])
        # the blend of a given list does not depend on K or the mode
        r1 = orc.rasterize(plain["dbl"], ada["tile_start"], ada["ids"], cam["width"], cam["height"],
                           oracle.params(cam))
        np.testing.assert_array_equal(r1["image"], ada["image"])
        if K == 0.0:
            # K = 0: Th = tau, dropped tiles held only alpha < tau pixels
            np.testing.assert_array_equal(ada["image"], plain["image"])
            sig = plain["dbl"][:, oracle.F_OPAC]
            assert np.all(ada["irec"][sig < TAU, oracle.I_CULL] == oracle.CULL_TH)
    assert len(prev) < len(P)


def pin_low_opacity_invisible(orc):
    """Gaussians with opacity < tau never change the image (and AdaGScale culls them)."""
    scene, cam = tiny_scene(150, 41)
    faint, _ = tiny_scene(60, 42)
    faint["opacity_logit"][:] = math.log((TAU * 0.9) / (1 - TAU * 0.9))
    both = concat(scene, faint)
    par = oracle.params(cam)
    np.testing.assert_array_equal(orc.render(both, cam, par)["image"], orc.render(scene, cam, par)["image"])
    ada = orc.render(both, cam, oracle.params(cam, scale_mode=1, K=0.0))
    assert np.all(ada["irec"][150:, oracle.I_CULL] == oracle.CULL_TH)


def pin_max_T(orc):
    """Calibration statistic: max T before blending over the pixels where a Gaussian blends."""
    W = H = 65
    f = 80.0
    cam = axis_camera(W, H, f)
    lam_f = (f * 0.3 / 2.0) ** 2 + 0.3       # front: wide, depth 2
    s_b = 0.02                                # back: small, depth 3
    lam_b = (f * s_b / 3.0) ** 2 + 0.3
    sc = concat(one_gaussian((0, 0, 2.0), (0.3, 0.3, 0.3), opacity=0.5),
                one_gaussian((0, 0, 3.0), (s_b, s_b, s_b), opacity=0.9))
    out = orc.render(sc, cam, oracle.params(cam), want_max_T=True)
    k = np.arange(-32, 33)
    dx, dy = np.meshgrid(k, k)
    r2 = dx * dx + dy * dy
    blended = 0.9 * np.exp(-r2 / (2 * lam_b)) >= TAU
    exp_back = (1 - 0.5 * np.exp(-r2[blended] / (2 * lam_f))).max()
    np.testing.assert_allclose(out["max_T"], [1.0, exp_back], rtol=1e-12)


# --------------------------------------------------------------------------
# Backward: FP64 central differences of the forward with frozen lists
# --------------------------------------------------------------------------
def pin_backward_fd(orc, n_check=None, seed=5):
    scene, cam = synth.fd_subscene()
    scene = {k: v.astype(np.float64) for k, v in scene.items()}
    scene["opacity_logit"][:4] = 5.5        # opacity 0.996: alpha hits the 0.99 clamp near the centre
    W, H = cam["width"], cam["height"]
    par = oracle.params(cam, bg=(0.05, 0.1, 0.15))
    base = orc.render(scene, cam, par, want_state=True)
    ts, ids = base["tile_start"], base["ids"]
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(3, H, W))
    grads = orc.backward(scene, cam, par, ts, ids, w)

    def loss_and_state(sc):
        dbl, irec = orc.preprocess(sc, cam, par)
        r = orc.rasterize(dbl, ts, ids, W, H, par, want_state=True)
        return float((w * r["image"]).sum()), (r["state"].tobytes(), irec[:, oracle.I_CLAMP].tobytes(),
                                               irec[:, oracle.I_CULL].tobytes())

    n = scene["opacity_logit"].shape[0]
    coords = []
    for key, rows in (("mean", 3), ("log_scale", 3), ("quat", 4), ("opacity_logit", 1)):
        for r in range(rows):
            for i in range(n):
                coords.append((key, r, i))
    for _ in range(96):
        coords.append(("sh", (int(rng.integers(0, 16)), int(rng.integers(0, 3))), int(rng.integers(0, n))))
    if n_check is not None:
        keep = [c for c in coords if c[2] < 4 and c[0] != "sh"]
        coords = keep + [coords[j] for j in rng.choice(len(coords), n_check, replace=False)]
    gmax = max(np.abs(grads[k]).max() for k in ("mean", "log_scale", "quat", "opacity_logit", "sh"))
    checked = skipped = 0
    for key, r, i in coords:
        arr = scene[key]
        idx = (i,) if arr.ndim == 1 else ((r, i) if arr.ndim == 2 else (r[0], r[1], i))
        th = arr[idx]
        h = 1e-6 * max(1.0, abs(th))
        arr[idx] = th + h
        lp, sp = loss_and_state(scene)
        arr[idx] = th - h
        lm, sm = loss_and_state(scene)
        arr[idx] = th
        if sp != sm:
            skipped += 1
            continue
        fd = (lp - lm) / (2 * h)
        g = grads[key][idx]
        assert abs(fd - g) <= 1e-5 * abs(g) + 1e-7 * gmax, (key, r, i, fd, g)
        checked += 1
    assert checked > 0.9 * len(coords), (checked, skipped)
    return checked, skipped


# --------------------------------------------------------------------------
# Ellipse tile test (tile_test 1)
# --------------------------------------------------------------------------
def _interval_dist(lo, hi):
    """Distance from 0 to the interval [lo, hi]."""
    return 0.0 if lo <= 0.0 <= hi else min(abs(lo), abs(hi))


def pin_ellipse_tiles(orc):
    """The kept tiles against (a) the closed form of an axis-aligned conic, whose
    minimum over a rectangle is A dx^2 + C dy^2 with dx, dy the distances from
    the centre to the rectangle's x and y ranges, and (b) a dense sampling of
    each tile's pixel-centre rectangle for rotated conics: a tile is kept iff the
    sampled minimum reaches Q, up to the sampling error."""
    # (a) axis-aligned Gaussians (on the y = 0 plane, so B = 0): one stretched
    # along x, one thin in x just beyond the last pixel column of a ragged
    # image, whose square reaches the clipped last tile column but whose
    # ellipse misses its pixel centres
    W, H = 100, 64
    cam = axis_camera(W, H, 80.0)
    scene = concat(one_gaussian((0.31, 0.0, 2.0), (0.35, 0.1, 0.1), opacity=0.9),
                   one_gaussian((1.3375, 0.0, 2.0), (0.01, 0.2, 0.01), opacity=0.9))
    par = oracle.params(cam, tile_test=oracle.TILE_ELLIPSE)
    dbl, irec = orc.preprocess(scene, cam, par)
    total = 0
    for i in range(2):
        g = dbl[i]
        assert g[oracle.F_B] == 0.0
        Q = 2 * math.log(g[oracle.F_OPAC] / TAU)
        assert abs(g[oracle.F_QELL] - Q) < 1e-12
        x0, y0, x1, y1 = (irec[i, k] for k in (oracle.I_X0, oracle.I_Y0, oracle.I_X1, oracle.I_Y1))
        kept_cf = 0
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                dx = _interval_dist(16 * tx - g[oracle.F_U], min(16 * tx + 15, W - 1) - g[oracle.F_U])
                dy = _interval_dist(16 * ty - g[oracle.F_V], min(16 * ty + 15, H - 1) - g[oracle.F_V])
                kept_cf += g[oracle.F_A] * dx * dx + g[oracle.F_C] * dy * dy <= Q
        assert irec[i, oracle.I_TOUCHED] == kept_cf and 0 <= kept_cf < (x1 - x0) * (y1 - y0)
        total += kept_cf
    assert irec[0, oracle.I_TOUCHED] > 0 and dbl[1, oracle.F_U] - W + 1 > 1.0 and irec[1, oracle.I_X1] == 7
    out = orc.render(scene, cam, par)
    assert len(out["ids"]) == total
    # (b) rotated conics, both modes: dense sampling of every tile of the square
    for mode, K in ((0, 0.0), (1, 0.1)):
        scene, cam = tiny_scene(60, 71, W=70, H=52)
        W, H = cam["width"], cam["height"]
        par = oracle.params(cam, scale_mode=mode, K=K, tile_test=oracle.TILE_ELLIPSE)
        dbl, irec = orc.preprocess(scene, cam, par)
        _, irq = orc.preprocess(scene, cam, oracle.params(cam, scale_mode=mode, K=K))
        ts, ids = orc.tile_lists(dbl, irec, W, H)
        gx = (W + 15) // 16
        kept_tiles = {(int(t), int(i)) for t, i in zip(np.repeat(np.arange(len(ts) - 1), np.diff(ts)), ids)}
        s = np.linspace(0.0, 1.0, 121)
        checked = 0
        for i in range(len(dbl)):
            if irq[i, oracle.I_TOUCHED] <= 0:
                continue
            g = dbl[i]
            Q = g[oracle.F_QELL]
            x0, y0, x1, y1 = (irq[i, k] for k in (oracle.I_X0, oracle.I_Y0, oracle.I_X1, oracle.I_Y1))
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    xs = 16 * tx + s * (min(16 * tx + 15, W - 1) - 16 * tx) - g[oracle.F_U]
                    ys = 16 * ty + s * (min(16 * ty + 15, H - 1) - 16 * ty) - g[oracle.F_V]
                    X, Y = np.meshgrid(xs, ys)
                    q = g[oracle.F_A] * X * X + 2 * g[oracle.F_B] * X * Y + g[oracle.F_C] * Y * Y
                    qmin = q.min()
                    # sampling error bound: |grad q| * half the sample spacing (diagonal)
                    step = 15.0 / 120.0
                    grad = 2.0 * math.sqrt((g[oracle.F_A] + g[oracle.F_C]) * max(qmin, 0.0) + 1e-300)
                    slack = grad * step + (g[oracle.F_A] + g[oracle.F_C]) * step * step
                    kept = ((ty * gx + tx), i) in kept_tiles
                    if qmin <= Q - 1e-12:
                        assert kept, (i, tx, ty, qmin, Q)
                    elif qmin - slack > Q:
                        assert not kept, (i, tx, ty, qmin, Q)
                    checked += 1
        assert checked > 50


def pin_ellipse_lossless_plain(orc):
    """Plain mode with the ellipse test renders exactly the square-footprint
    image (a dropped tile holds only pixels with alpha < tau), with a subset of
    its pairs; with AdaGScale every pixel centre of a dropped tile has
    alpha < Th; brute force and tiled agree."""
    scene, cam = tiny_scene(220, 81, W=80, H=64)
    W, H = cam["width"], cam["height"]
    sq = orc.render(scene, cam, oracle.params(cam))
    el = orc.render(scene, cam, oracle.params(cam, tile_test=oracle.TILE_ELLIPSE))
    np.testing.assert_array_equal(el["image"], sq["image"])
    Ps, Pe = _pairs(sq, W), _pairs(el, W)
    assert Pe <= Ps and len(Pe) < len(Ps)
    par = oracle.params(cam, scale_mode=1, K=0.2, tile_test=oracle.TILE_ELLIPSE)
    ada = orc.render(scene, cam, par)
    ada_sq = orc.render(scene, cam, oracle.params(cam, scale_mode=1, K=0.2))
    Pa, Pas = _pairs(ada, W), _pairs(ada_sq, W)
    assert Pa <= Pas
    gx = (W + 15) // 16
    px, py = np.meshgrid(np.arange(W), np.arange(H))
    for (t, i) in Pas - Pa:
        g = ada["dbl"][i]
        tx, ty = t % gx, t // gx
        sel = (px // 16 == tx) & (py // 16 == ty)
        dx, dy = px[sel] - g[oracle.F_U], py[sel] - g[oracle.F_V]
        q = g[oracle.F_A] * dx * dx + 2 * g[oracle.F_B] * dx * dy + g[oracle.F_C] * dy * dy
        assert np.all(g[oracle.F_OPAC] * np.exp(-0.5 * q) < g[oracle.F_TH] * (1 + 1e-12))
    np.testing.assert_array_equal(ada["image"], orc.render_bruteforce(scene, cam, par))


# --------------------------------------------------------------------------
# Peripheral-score diagnostics: Eq. 3-4 contributions, Eq. 6-9 estimates and
# the contribution-skip render of Fig. 4a / Fig. 5
# --------------------------------------------------------------------------
def _two_layers(back_px=0):
    """A wide front Gaussian (opacity 0.5, depth 2, on the axis) over a small
    back one (opacity 0.9, depth 3, back_px pixels right of the centre) seen by
    a 65x65 camera, with the closed-form alpha of each at every pixel: an
    isotropic Gaussian of scale s at (x, 0, z) projects to the diagonal
    covariance ((f s/z)^2 (1 + x^2/z^2) + 0.3, (f s/z)^2 + 0.3).  Both
    footprints cover their alpha >= tau pixels; the transmittance never
    reaches the stop."""
    W = H = 65
    f = 80.0
    cam = axis_camera(W, H, f)
    lam_f = (f * 0.3 / 2.0) ** 2 + 0.3
    s_b, z_b = 0.02, 3.0
    x_b = back_px * z_b / f
    lam_bx = (f * s_b / z_b) ** 2 * (1 + (x_b / z_b) ** 2) + 0.3
    lam_by = (f * s_b / z_b) ** 2 + 0.3
    sc = concat(one_gaussian((0, 0, 2.0), (0.3, 0.3, 0.3), opacity=0.5),
                one_gaussian((x_b, 0, z_b), (s_b, s_b, s_b), opacity=0.9, dc=(0.9, 0.1, -0.4)))
    k = np.arange(-32, 33)
    dx, dy = np.meshgrid(k, k)
    af = np.minimum(0.99, 0.5 * np.exp(-(dx * dx + dy * dy) / (2 * lam_f)))
    ab = np.minimum(0.99, 0.9 * np.exp(-(dx - back_px) ** 2 / (2 * lam_bx) - dy * dy / (2 * lam_by)))
    return cam, sc, af, ab


def pin_peripheral_two_layers(orc):
    """Eq. 4 per Gaussian against a direct per-pixel sum: the back Gaussian
    sees T = 1 - alpha_front wherever the front one blends."""
    cam, sc, af, ab = _two_layers()
    par = oracle.params(cam)
    dbl, irec = orc.preprocess(sc, cam, par)
    ts, ids = orc.tile_lists(dbl, irec, cam["width"], cam["height"])
    bf, bb = af >= TAU, ab >= TAU
    Tb = np.where(bf, 1.0 - af, 1.0)
    for x in (0.02, 0.3, 0.95, np.inf):
        out = orc.peripheral(dbl, ts, ids, cam["width"], cam["height"], par, np.array([x, x]))
        exp_ps = [af[bf & (af < x)].sum(), (ab * Tb)[bb & (ab < x)].sum()]
        exp_sa = [af[bf & (af < x)].sum(), ab[bb & (ab < x)].sum()]
        np.testing.assert_allclose(out["ps"], exp_ps, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(out["sum_alpha"], exp_sa, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(out["max_T"], [1.0, Tb[bb].max()], rtol=1e-12)
    assert out["ps"][1] < out["sum_alpha"][1]


def pin_peripheral_closed_form(orc):
    """A lone large Gaussian (T = 1 everywhere): Eq. 4 equals the pixel sum of
    alpha and lies within 1% of Eq. 9's annulus integral 2 pi sqrt(det) (x - tau),
    the band ending at the opacity."""
    W = H = 161
    f, d, sig = 200.0, 2.0, 0.3
    cam = axis_camera(W, H, f)
    sc = one_gaussian((0.013, -0.007, d), (0.2, 0.11, 0.05), quat=(0.8, 0.0, 0.0, 0.6), opacity=sig)
    par = oracle.params(cam)
    dbl, irec = orc.preprocess(sc, cam, par)
    ts, ids = orc.tile_lists(dbl, irec, W, H)
    det = dbl[0, oracle.F_DET]
    for x in (0.02, 0.1, 0.2, 0.5):
        out = orc.peripheral(dbl, ts, ids, W, H, par, np.array([x]))
        np.testing.assert_allclose(out["ps"], out["sum_alpha"], rtol=1e-13)
        np.testing.assert_allclose(out["ps"][0], 2 * math.pi * math.sqrt(det) * (min(x, sig) - TAU), rtol=1e-2)
        assert out["max_T"][0] == 1.0


def pin_peripheral_invariants(orc):
    """On a random scene: with no level the scores telescope to the covered
    fraction of every pixel (sum_i alpha_i T_i = 1 - T_final); Eq. 6 bounds
    Eq. 4 from above; Eq. 4 grows with the level; at each Gaussian's own Th
    (Eq. 10), Eq. 9 returns K wherever Th <= opacity."""
    scene, cams, _ = synth.workload("c1_cube16k_256", n=400, width=64, height=48, views=1)
    cam = cams[0]
    lut = np.linspace(1.0, 0.5, 20)
    par = oracle.params(cam, lut=lut)
    dbl, irec = orc.preprocess(scene, cam, par)
    ts, ids = orc.tile_lists(dbl, irec, 64, 48)
    n = dbl.shape[0]
    full = orc.peripheral(dbl, ts, ids, 64, 48, par, np.full(n, np.inf))
    ref = orc.rasterize(dbl, ts, ids, 64, 48, par)
    np.testing.assert_allclose(full["ps"].sum(), (1.0 - ref["final_T"]).sum(), rtol=1e-10)
    assert np.all(full["max_T"] * full["sum_alpha"] >= full["ps"] * (1 - 1e-12))
    half = orc.peripheral(dbl, ts, ids, 64, 48, par, np.full(n, 0.2))
    assert np.all(half["ps"] <= full["ps"] * (1 + 1e-12)) and half["ps"].sum() < full["ps"].sum()
    K = 0.5
    sc = orc.peripheral_scores(scene, cam, K, lut)
    live = irec[:, oracle.I_TOUCHED] > 0
    ok = live & np.isfinite(sc["th"]) & (sc["th"] <= dbl[:, oracle.F_OPAC])
    assert ok.sum() > 20
    np.testing.assert_allclose(sc["eq9"][ok], K, rtol=1e-9)
    over = live & (sc["th"] > dbl[:, oracle.F_OPAC])
    assert over.any() and np.all(sc["eq9"][over] < K)


def pin_skip_render(orc):
    """Contribution-skip render: no threshold gives the plain image bit for bit,
    a threshold above every contribution leaves the background, and on two
    layers each ranking skips exactly the blends a per-pixel restatement
    predicts (rule 0 ranks by the unskipped T, the image uses the kept blends)."""
    W = H = 65
    bg = (0.2, 0.4, 0.6)
    cases = ((0, 0, None, 0.05), (0, 0, None, 0.3), (0, 1, np.array([1.0, 0.5]), 0.2), (20, 0, None, 0.36),
             (20, 2, np.array([0.7, 0.9]), 0.3))
    for back_px, rule, weight, thr in cases:
        cam, sc, af, ab = _two_layers(back_px)
        par = oracle.params(cam, bg=bg)
        dbl, irec = orc.preprocess(sc, cam, par)
        ts, ids = orc.tile_lists(dbl, irec, W, H)
        if thr == 0.05:
            ref = orc.rasterize(dbl, ts, ids, W, H, par, want_state=True)
            out = orc.render_skip(dbl, ts, ids, W, H, par, 0, None, 0.0)
            np.testing.assert_array_equal(out["image"], ref["image"])
            assert out["skipped"] == 0 and out["blends"] == int(ref["state"][..., 0].sum())
            out = orc.render_skip(dbl, ts, ids, W, H, par, 0, None, 2.0)
            np.testing.assert_allclose(out["image"], np.broadcast_to(np.array(bg)[:, None, None], (3, H, W)),
                                       rtol=1e-15)
            assert out["skipped"] == out["blends"]
        bf, bb = af >= TAU, ab >= TAU
        cf, cb = dbl[0, oracle.F_R:oracle.F_BL + 1], dbl[1, oracle.F_R:oracle.F_BL + 1]
        w = np.ones(2) if weight is None else weight
        kf = bf & (w[0] * af >= thr)
        rank_b = ab * np.where(bf, 1.0 - af, 1.0) if rule == 0 else w[1] * ab
        kb = bb & (rank_b >= thr)
        Ts_b = np.where(kf, 1.0 - af, 1.0)
        Ts = Ts_b * np.where(kb, 1.0 - ab, 1.0)
        img = (cf[:, None, None] * np.where(kf, af, 0.0) + cb[:, None, None] * np.where(kb, ab * Ts_b, 0.0)
               + np.array(bg)[:, None, None] * Ts)
        out = orc.render_skip(dbl, ts, ids, W, H, par, rule, weight, thr)
        np.testing.assert_allclose(out["image"], img, rtol=1e-12, atol=1e-15)
        assert out["skipped"] == int((bf & ~kf).sum() + (bb & ~kb).sum())
        assert 0 < out["skipped"] < out["blends"]



# --------------------------------------------------------------------------
# Edge classes: every discrete decision of the preprocess and the blend is
# flagged when its decision variable lies within the documented band of its
# threshold, and only then.  Each pin places one Gaussian (or pixel) at a
# chosen distance from one threshold -- half the band (flag expected) and
# twice the band (no flag) on both sides -- with the position computed from
# the closed forms of an on-axis Gaussian, independently of the oracle.
# The bands (relative width eps = 1e-5, the oracle's default edge_rel):
#   near plane  |t_z - near| <= eps * max(t_z, near)
#   det guard   det <= eps * (|a c| + b^2) of the dilated 2D covariance
#   Th vs sigma |Th - sigma| <= eps * max(Th, sigma)
#   radius ceil the ceil changes when lambda_max moves by +-eps relative
#   rectangle   a tile index changes when u (v) moves by +-eps * (|fx tx/tz| +
#               |cx|) (the view-space mean taken exactly: no term for the
#               magnitudes that cancel in R m + t_cam)
#   LUT bin     |depth/width - edge| <= eps * max(depth/width, 1) at an inner
#               bin edge (the last bin is open-ended: no decision)
#   ellipse     |min q over the tile - Q| <= eps max(Q, 1) + 2 pos_err
#               sqrt((A + C) max(Q, m)) + 2e-6 S (S: the size of q's terms
#               over the row's part of the square)
#   pixel alpha |ln(alpha / tau)| <= eps + pos_err |grad ln alpha|, and
#               |p| <= eps; each adds 2 tau T c_max (2 sigma T c_max) to the
#               pixel's flip budget
# --------------------------------------------------------------------------
EPS = 1e-5
NEAR32 = float(np.float32(0.2))          # the camera's near plane as the GPU receives it


def _edge_bits(orc, sc, cam, **pkw):
    dbl, irec = orc.preprocess(sc, cam, oracle.params(cam, **pkw))
    return dbl[0], irec[0]


def _iso_scale(lam, f, d):
    """World scale of an isotropic Gaussian at depth d on the optical axis whose
    dilated 2D covariance is lam * I: lam = (f s / d)^2 + 0.3."""
    return d * math.sqrt(lam - 0.3) / f


def pin_edge_near_plane(orc):
    for ctrans in (0.0, 5.0):            # camera at the origin, and 5 units behind it
        cam = axis_camera(64, 64, 60.0, campos=(0.0, 0.0, -ctrans))
        for sgn in (1.0, -1.0):
            for k, want in ((0.5, True), (2.0, False)):
                tz = NEAR32 * (1.0 + sgn * k * EPS)   # the band's scale is max(t_z, near)
                sc = one_gaussian((0.0, 0.0, tz - ctrans), (0.01, 0.01, 0.01))
                _, ir = _edge_bits(orc, sc, cam)
                got = bool(ir[oracle.I_EDGE] & oracle.EDGE_NEAR)
                assert got == want, ("near", ctrans, sgn, k, got)
                assert (ir[oracle.I_CULL] == oracle.CULL_NEAR) == (sgn < 0), ("near cull", ctrans, sgn, k)


def pin_edge_det_guard(orc):
    """A needle at 45 degrees on the optical axis: Sigma2D = k R diag(s1^2, s2^2) R^T
    + 0.3 I with k = (f/d)^2, so det = (k s1^2 + 0.3)(k s2^2 + 0.3) and
    a c + b^2 = ((a' + b')/2 + 0.3)^2 + ((a' - b')/2)^2 with a' = k s1^2, b' = k s2^2."""
    f, d, s2 = 80.0, 2.0, 1e-7
    kk = (f / d) ** 2
    cam = axis_camera(65, 65, f)
    qz = (math.cos(math.pi / 8), 0.0, 0.0, math.sin(math.pi / 8))

    def ratio(s1):
        a, b = kk * s1 * s1, kk * s2 * s2
        return (a + 0.3) * (b + 0.3) / (((a + b) / 2 + 0.3) ** 2 + ((a - b) / 2) ** 2)

    for k, want in ((0.5, True), (2.0, False)):
        lo, hi = 1e-3, 1e3               # ratio falls with s1: bisect for ratio = k eps
        for _ in range(200):
            mid = math.sqrt(lo * hi)
            if ratio(mid) > k * EPS:
                lo = mid
            else:
                hi = mid
        sc = one_gaussian((0.0, 0.0, d), (lo, s2, s2), quat=qz)
        g, ir = _edge_bits(orc, sc, cam)
        np.testing.assert_allclose(g[oracle.F_DET], (kk * lo * lo + 0.3) * (kk * s2 * s2 + 0.3), rtol=1e-9)
        assert bool(ir[oracle.I_EDGE] & oracle.EDGE_DET) == want, ("det", k)


def pin_edge_th_vs_opacity(orc):
    f, d, lam, sig = 80.0, 2.0, 6.0, 0.6
    cam = axis_camera(65, 65, f)
    sc = one_gaussian((0.0, 0.0, d), (_iso_scale(lam, f, d),) * 3, opacity=sig)
    for sgn in (1.0, -1.0):
        for k, want in ((0.5, True), (2.0, False)):
            th = sig * (1.0 + sgn * k * EPS)
            K = (th - TAU) * 2.0 * math.pi * lam        # Eq. 10 with T_up = 1, sqrt(det) = lam
            g, ir = _edge_bits(orc, sc, cam, scale_mode=1, K=K)
            np.testing.assert_allclose(g[oracle.F_TH], th, rtol=1e-12)
            assert bool(ir[oracle.I_EDGE] & oracle.EDGE_TH) == want, ("th", sgn, k)
            assert (ir[oracle.I_CULL] == oracle.CULL_TH) == (sgn > 0), ("th cull", sgn, k)


def pin_edge_radius_ceil(orc):
    """Isotropic on axis: lambda_max = lam + sqrt(0.1) (the eigenvalue guard), the
    plain radius ceil(3 sqrt(lambda_max)); AdaGScale with K -> 0 and opacity 0.9
    keeps the factor 3 (sqrt(2 ln(0.9 / tau)) > 3)."""
    f, d, R = 80.0, 2.0, 7
    cam = axis_camera(65, 65, f)
    for mode, K in ((0, 0.0), (1, 1e-9)):
        for sgn in (1.0, -1.0):
            for k, want in ((0.5, True), (2.0, False)):
                lam1 = (R / 3.0) ** 2 * (1.0 + sgn * k * EPS)
                lam = lam1 - math.sqrt(0.1)
                sc = one_gaussian((0.0, 0.0, d), (_iso_scale(lam, f, d),) * 3, opacity=0.9)
                g, ir = _edge_bits(orc, sc, cam, scale_mode=mode, K=K)
                np.testing.assert_allclose(g[oracle.F_LAMBDA], lam1, rtol=1e-12)
                assert ir[oracle.I_RADIUS] == (R if sgn < 0 else R + 1)
                assert bool(ir[oracle.I_EDGE] & oracle.EDGE_CEIL) == want, ("ceil", mode, sgn, k)


def pin_edge_rect(orc):
    """On-axis Gaussian with the principal point moved: u = cx exactly, and the
    band's scale is |cx| (t_x = 0) -- also when t_x = 0 is the difference of two
    large terms (camera and Gaussian 300 units off the origin along x).  Radius 5
    (3 sqrt(lambda_max) = 4.5).  The tile index of the left end changes where
    u - r crosses 16 j - 1 (the first pixel centre moves to the next tile), of
    the right end where u + r crosses 16 j."""
    f, d = 60.0, 2.0
    lam = 2.25 - math.sqrt(0.1)
    s = _iso_scale(lam, f, d)
    for off in (0.0, 300.0):
        for side in ("left", "right", "top"):
            for sgn in (1.0, -1.0):
                for k, want in ((0.5, True), (2.0, False)):
                    cam = axis_camera(80, 80, f, campos=(off, 0.0, 0.0))
                    base = 31.0 + 5.0 if side != "right" else 48.0 - 5.0     # u - 5 = 31, or u + 5 = 48
                    c = base
                    for _ in range(3):
                        c = base + sgn * k * EPS * abs(c)
                    if side == "top":
                        cam["cy"], cam["cx"] = c, 40.0
                    else:
                        cam["cx"], cam["cy"] = c, 40.0
                    sc = one_gaussian((off, 0.0, d), (s, s, s))
                    g, ir = _edge_bits(orc, sc, cam)
                    assert ir[oracle.I_RADIUS] == 5
                    got = bool(ir[oracle.I_EDGE] & oracle.EDGE_RECT)
                    assert got == want, ("rect", off, side, sgn, k, got)
                    if side == "top":
                        lo_t, hi_t = ir[oracle.I_Y0], ir[oracle.I_Y1]
                    else:
                        lo_t, hi_t = ir[oracle.I_X0], ir[oracle.I_X1]
                    if side == "right":
                        assert hi_t == (4 if sgn > 0 else 3)
                    else:
                        assert lo_t == (2 if sgn > 0 else 1)


def pin_edge_lut_bin(orc):
    f = 200.0
    cam = axis_camera(65, 65, f)
    for edge_depth, decision in ((5.0, True), (10.0, True), (95.0, True), (100.0, False)):
        for sgn in (1.0, -1.0):
            for k in (0.5, 2.0):
                d = edge_depth * (1.0 + sgn * k * EPS)
                sc = one_gaussian((0.0, 0.0, d), (_iso_scale(9.0, f, d),) * 3, opacity=0.8)
                _, ir = _edge_bits(orc, sc, cam, scale_mode=1, K=0.01)
                want = decision and k < 1.0
                assert bool(ir[oracle.I_EDGE] & oracle.EDGE_LUT) == want, ("lut", edge_depth, sgn, k)


def pin_edge_ellipse(orc):
    """Isotropic conic (A = C = 1/lam, B = 0), v = 40 mid-row: the tile right of
    the centre in its row has min q = (48 - u)^2 / lam; every other tile of the
    square is far from Q = 2 ln(sigma / tau).  pos_err = 0 isolates the other
    two terms of the band."""
    f, d, lam, sig, W, H = 60.0, 2.0, 9.0, 0.8, 80, 80
    Q = 2.0 * math.log(sig / TAU)
    s = _iso_scale(lam, f, d)
    for pe in (0.0, 2e-3):
        for sgn in (1.0, -1.0):
            for k, want in ((0.5, True), (2.0, False)):
                u = 48.0 - math.sqrt(lam * Q)
                for _ in range(4):       # the band depends (weakly) on u through S
                    r = math.ceil(3.0 * math.sqrt(lam + math.sqrt(0.1)))
                    x0 = int(math.ceil(u - r)) // 16
                    x1 = int(math.floor(u + r)) // 16 + 1
                    X = max(abs(16 * x0 - u), abs(min(16 * x1 - 1, W - 1) - u))
                    S = (X * X + 8.0 * 8.0) / lam
                    band = EPS * max(Q, 1.0) + 2.0 * pe * math.sqrt((2.0 / lam) * Q) + 2e-6 * S
                    m = Q + sgn * k * band
                    u = 48.0 - math.sqrt(lam * m)
                cam = axis_camera(W, H, f)
                cam["cx"], cam["cy"] = u, 40.0
                sc = one_gaussian((0.0, 0.0, d), (s, s, s), opacity=sig)
                _, ir = _edge_bits(orc, sc, cam, tile_test=oracle.TILE_ELLIPSE, pos_err=pe)
                assert bool(ir[oracle.I_EDGE] & oracle.EDGE_ELLIPSE) == want, ("ellipse", pe, sgn, k)


def pin_edge_pixel_budget(orc):
    """One isotropic Gaussian at a pixel centre, alpha = sigma exp(-r^2 / (2 lam)):
    lam is chosen so that the 4 pixels at distance 4 have ln(alpha / tau) = delta.
    The flip budget is 2 tau T c_max = 2 tau there (T = 1, colours < 1) when
    |delta| is within the band and zero there when it is outside (the centre
    pixel, p = 0 exactly, always carries 2 sigma; every other pixel nothing).  Then the
    centre moved by e from the pixel: p = -e^2 / (2 lam) against the p <= 0 test."""
    f, d, sig, W = 80.0, 2.0, 0.7, 65
    cam = axis_camera(W, W, f)
    ring = [(32 + 4, 32), (32 - 4, 32), (32, 32 + 4), (32, 32 - 4)]
    for pe in (0.0, 1e-3):
        for sgn in (1.0, -1.0):
            for k, want in ((0.5, True), (2.0, False)):
                lam = 8.0 / math.log(sig / TAU)
                for _ in range(4):       # the band's gradient term depends on lam
                    band = EPS + pe * 4.0 / lam          # |grad ln alpha| = (|A dx| + |C dy|) = 4 / lam
                    lam = 8.0 / (math.log(sig / TAU) - sgn * k * band)
                sc = one_gaussian((0.0, 0.0, d), (_iso_scale(lam, f, d),) * 3, opacity=sig)
                out = orc.render(sc, cam, oracle.params(cam, pos_err=pe))
                bud = out["budget"]
                expect = np.zeros_like(bud)
                expect[32, 32] = 2.0 * sig       # the centre pixel has p = 0 exactly: always in its band
                if want:
                    for (x, y) in ring:
                        expect[y, x] = 2.0 * TAU
                np.testing.assert_allclose(bud, expect, rtol=1e-12, atol=0, err_msg="alpha-tau %g %g %g" % (pe, sgn, k))
    lam = 4.0
    for k, want in ((0.5, True), (2.0, False)):
        e = math.sqrt(2.0 * lam * k * EPS)
        cam["cx"] = 32.0 + e
        sc = one_gaussian((0.0, 0.0, d), (_iso_scale(lam, f, d),) * 3, opacity=sig)
        out = orc.render(sc, cam, oracle.params(cam, pos_err=0.0))
        bud = out["budget"]
        assert (bud[32, 32] == 2.0 * sig) == want and np.count_nonzero(bud) == int(want), ("p", k)


def pin_gradient_edges(orc):
    """Decisions that move only the derivatives are flagged within their bands:
    a colour channel at the clamp at 0 (|0.5 + C0 dc| <= eps (0.5 + |C0 dc|)),
    x/z at the 1.3 tan(fov/2) frustum clamp, and per pixel of the backward the
    alpha-tau ring and the transmittance stop T (1 - alpha) vs 1e-4."""
    f, d = 80.0, 2.0
    cam = axis_camera(65, 65, f)
    for sgn in (1.0, -1.0):
        for k, want in ((0.5, True), (2.0, False)):
            # colour: 0.5 + C0 dc = sgn k eps (0.5 + C0 |dc|), dc < 0
            dc = -(0.5 - sgn * k * EPS * 1.0) / (C0 * (1.0 + sgn * k * EPS))
            sc = one_gaussian((0.0, 0.0, d), (0.05, 0.05, 0.05), dc=(dc, 0.2, 0.2))
            _, ir = _edge_bits(orc, sc, cam)
            assert bool(ir[oracle.I_GEDGE] & oracle.GEDGE_COLOUR) == want, ("colour", sgn, k)
            assert bool(ir[oracle.I_CLAMP] & 1) == (sgn < 0)
            # frustum: x/z = lim (1 + sgn k eps), lim = 1.3 W / (2 f)
            lim = 1.3 * 0.5 * 65 / f
            x = d * lim * (1.0 + sgn * k * EPS)
            sc = one_gaussian((x, 0.0, d), (0.05, 0.05, 0.05))
            _, ir = _edge_bits(orc, sc, cam)
            assert bool(ir[oracle.I_GEDGE] & oracle.GEDGE_FRUSTUM) == want, ("frustum", sgn, k)
    # the alpha-tau ring of pin_edge_pixel_budget: 4 ring pixels + the centre (p = 0)
    sig, W = 0.7, 65
    for k, want in ((0.5, 5), (2.0, 1)):
        lam = 8.0 / (math.log(sig / TAU) - k * EPS)
        sc = one_gaussian((0.0, 0.0, d), (_iso_scale(lam, f, d),) * 3, opacity=sig)
        par = oracle.params(cam, pos_err=0.0)
        out = orc.render(sc, cam, par)
        g = orc.backward(sc, cam, par, out["tile_start"], out["ids"], np.ones((3, W, W)))
        assert g["edge"][0] == want, ("ring", k, g["edge"][0])
    # the stop: three isotropic Gaussians stacked on the axis, 0.3 px off the
    # centre of pixel (32, 32); the third's opacity puts T (1 - alpha_3) at
    # 1e-4 (1 + delta) there (alpha_i = sigma_i exp(-e^2 / (2 lam_i)))
    e, s_w = 0.3, 0.05
    camo = axis_camera(W, W, f)
    camo["cx"] = 32.0 + e
    lam_at = lambda dd: (f * s_w / dd) ** 2 + 0.3
    a_front = [0.95 * math.exp(-e * e / (2 * lam_at(dd))) for dd in (2.0, 2.5)]
    T2 = (1.0 - a_front[0]) * (1.0 - a_front[1])
    for k, want in ((0.5, 1), (2.0, 0)):
        band = EPS + 3 * 1.2e-7
        a3 = 1.0 - 1e-4 * (1.0 + k * band) / T2
        sig3 = a3 / math.exp(-e * e / (2 * lam_at(3.0)))
        sc = concat(one_gaussian((0.0, 0.0, 2.0), (s_w,) * 3, opacity=0.95),
                    one_gaussian((0.0, 0.0, 2.5), (s_w,) * 3, opacity=0.95),
                    one_gaussian((0.0, 0.0, 3.0), (s_w,) * 3, opacity=sig3))
        par = oracle.params(camo, pos_err=0.0)
        out = orc.render(sc, camo, par)
        g = orc.backward(sc, camo, par, out["tile_start"], out["ids"], np.ones((3, W, W)))
        assert g["edge"][2] == want, ("stop", k, g["edge"][2])
        if want == 0:   # nothing near a threshold anywhere: no budget
            assert all(not np.any(v) for v in g["budget"].values())
    # the flip budget bounds what the stop flip does to the two front Gaussians
    rng = np.random.default_rng(3)
    wr = rng.normal(size=(3, W, W))
    gs = []
    for sgn in (1.0, -1.0):         # third Gaussian blended (+), or the pixel stops before it (-)
        band = EPS + 3 * 1.2e-7
        a3 = 1.0 - 1e-4 * (1.0 + sgn * 0.5 * band) / T2
        sig3 = a3 / math.exp(-e * e / (2 * lam_at(3.0)))
        sc = concat(one_gaussian((0.0, 0.0, 2.0), (s_w,) * 3, opacity=0.95),
                    one_gaussian((0.0, 0.0, 2.5), (s_w,) * 3, opacity=0.95),
                    one_gaussian((0.0, 0.0, 3.0), (s_w,) * 3, opacity=sig3))
        par = oracle.params(camo, pos_err=0.0)
        out = orc.render(sc, camo, par)
        gs.append(orc.backward(sc, camo, par, out["tile_start"], out["ids"], wr))
    # (the two scenes also differ smoothly: the third opacity by ~1e-5 relative)
    for key in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
        for gg in gs:
            assert np.all(gg["budget"][key][..., :2] >= 0)
        diff = np.abs(gs[0][key][..., :2] - gs[1][key][..., :2])
        bound = np.minimum(gs[0]["budget"][key][..., :2], gs[1]["budget"][key][..., :2])
        smooth = 1e-4 * np.maximum(np.abs(gs[0][key][..., :2]), np.abs(gs[1][key][..., :2]))
        assert np.all(diff <= bound + smooth + 1e-10 * np.abs(gs[0][key]).max()), key
    # the flip itself moves the front Gaussians' x-gradient far beyond the smooth part
    dmx = np.abs(gs[0]["mean"][0, :2] - gs[1]["mean"][0, :2])
    assert np.all(dmx > 1e-3 * np.abs(gs[0]["mean"][0, :2]))
    # an alpha-tau flip of a small back Gaussian (its ring of pin_edge_pixel_budget)
    # under a wide front Gaussian whose colour equals the background: the front's
    # colour-behind changes by about tau |c_back - bg| at the ring although
    # c_front - R is nearly zero there.  The smooth part is measured between two
    # scenes on the same side of the flip (0.5 and 0.6 of the band).
    cam = axis_camera(W, W, f)
    dc_f = np.array([0.3, -0.2, 0.1])
    bg = tuple(float(x) for x in dc_f * C0 + 0.5)
    gs = {}
    for frac in (0.5, 0.6, -0.5):
        lam = 8.0 / (math.log(sig / TAU) - frac * EPS)
        sc = concat(one_gaussian((0.0, 0.0, 1.5), (0.4, 0.4, 0.4), opacity=0.3, dc=dc_f),
                    one_gaussian((0.0, 0.0, d), (_iso_scale(lam, f, d),) * 3, opacity=sig, dc=(-0.4, 0.6, 0.2)))
        par = oracle.params(cam, pos_err=0.0, bg=bg)
        out = orc.render(sc, cam, par)
        gs[frac] = orc.backward(sc, cam, par, out["tile_start"], out["ids"], wr)
    assert gs[0.5]["edge"][1] > 0 and gs[-0.5]["edge"][1] > 0
    moved = 0
    for key in ("mean", "log_scale", "opacity_logit", "sh"):
        diff = np.abs(gs[0.5][key][..., 0] - gs[-0.5][key][..., 0])
        smooth = 20.0 * np.abs(gs[0.5][key][..., 0] - gs[0.6][key][..., 0])
        noise = 1e-10 * np.abs(gs[0.5][key]).max()      # the order of the parallel sums
        bound = np.minimum(gs[0.5]["budget"][key][..., 0], gs[-0.5]["budget"][key][..., 0])
        assert np.all(diff <= bound + smooth + noise), ("ring", key)
        moved += int(np.count_nonzero(diff > 10 * smooth + 1e3 * noise))
    assert moved > 0


def pin_eval_count(orc):
    """Evaluations of Eq. 1-2 per pixel: the entries of its tile list up to and
    including the one at which it stops, else the whole list.  Four Gaussians
    centred on pixel (32, 32): three of opacity 0.98 take T to 0.02^2 there and
    the third's T (1 - alpha) = 8e-6 < 1e-4 stops the pixel, so it evaluates 3
    of the 4 entries; at pixel (36, 36) no alpha comes near and all 4 count."""
    cam = axis_camera(65, 65, 80.0)
    sc = concat(*[one_gaussian((0.0, 0.0, d), (0.05, 0.05, 0.05), opacity=0.98) for d in (2.0, 2.1, 2.2)],
                one_gaussian((0.0, 0.0, 2.3), (0.05, 0.05, 0.05), opacity=0.5))
    out = orc.render(sc, cam, oracle.params(cam), want_state=True)
    assert len(out["ids"]) >= 4 and out["tile_start"][-1] == len(out["ids"])
    st = out["state"]
    assert st[32, 32, 2] == 3 and st[32, 32, 0] == 2          # two blended, the third stops it
    np.testing.assert_allclose(out["final_T"][32, 32], 0.02 * 0.02, rtol=1e-12)
    assert st[36, 36, 2] == 4

ALL_PINS = [pin_isotropic_on_axis, pin_off_axis_jacobian, pin_rotation_conventions, pin_eq9_quadrature,
            pin_eq8_riemann_pixels, pin_sh_basis, pin_sh_colour, pin_rect_enumeration, pin_bruteforce,
            pin_ideal_render, pin_invariants, pin_low_opacity_invisible, pin_max_T, pin_backward_fd,
            pin_ellipse_tiles, pin_ellipse_lossless_plain, pin_peripheral_two_layers, pin_peripheral_closed_form,
            pin_peripheral_invariants, pin_skip_render, pin_edge_near_plane, pin_edge_det_guard,
            pin_edge_th_vs_opacity, pin_edge_radius_ceil, pin_edge_rect, pin_edge_lut_bin, pin_edge_ellipse,
            pin_edge_pixel_budget, pin_gradient_edges, pin_eval_count]
