"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to a closed form, a library routine, a
finite difference, brute force or an invariant that the paper states, so that
a dropped term, a wrong sign or index, or a transposed operand anywhere in
the oracle fails at least one of them.  CPU only.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
import scipy.special as sp

import oracle
from paper_2603_11531_gb300 import synth

SH_C0 = 0.5 / math.sqrt(math.pi)


class Cam:
    def __init__(self, R, t, f, W, H, cx=None, cy=None, znear=0.2):
        self.R = np.asarray(R, np.float32)
        self.t = np.asarray(t, np.float32)
        self.fx = self.fy = float(np.float32(f))
        self.cx = float(np.float32(W / 2 if cx is None else cx))
        self.cy = float(np.float32(H / 2 if cy is None else cy))
        self.width, self.height, self.znear = W, H, znear


def _rec(mu, s, q=(1, 0, 0, 0), o=0.8, Y=None):
    r = np.zeros(24, np.float64)
    r[0:3], r[3:6], r[6:10], r[10] = mu, s, q, o
    if Y is not None:
        r[11:23] = np.asarray(Y, np.float64).reshape(12)
    return r


def _const_colour_Y(c):
    """SH coefficients whose colour is c for every viewing direction."""
    Y = np.zeros((4, 3))
    Y[0] = (np.asarray(c, np.float64) - 0.5) / SH_C0
    return Y


def _f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Closed forms for projection + EWA + alpha + Eq. 2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("o,sigma,z", [(0.8, 0.05, 3.0), (0.35, 0.02, 2.0), (1.0, 0.1, 4.0), (1.0, 0.4, 2.0)])
def test_single_isotropic_gaussian_closed_form(oracle_lib, o, sigma, z):
    """One isotropic Gaussian on the optical axis: Sigma_2D = ((f s / z)^2 + 0.3) I,
    so C(p) = a(p) c + (1 - a(p)) c_bg with a = min(0.99, o exp(-|p - c_pix|^2 / (2 v)))
    inside q <= 9 and c_bg outside (Eq. 2 with a single term; any rotation)."""
    W = H = 64
    f = 100.0
    c = np.array([0.9, 0.3, 0.6])
    bg = np.array([0.1, 0.2, 0.05])
    rng = np.random.default_rng(0)
    q = rng.normal(size=4)
    rec = _rec(_f32([0, 0, z]), _f32([sigma] * 3), _f32(q), float(np.float32(o)),
               _f32(_const_colour_Y(c)))
    cam = Cam(np.eye(3), [0, 0, 0], f, W, H)
    out = oracle.render(rec[None], cam, bg=bg, want_aux=True, want_count=True)
    s32 = float(np.float32(sigma))
    v = (cam.fx * s32 / float(np.float32(z))) ** 2 + 0.3
    g = out["gauss"][0]
    assert g["visible"] == 1
    np.testing.assert_allclose(g["cov"], [v, 0.0, v], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g["mean"], [W / 2, H / 2], rtol=0, atol=1e-12)
    cf = _f32(_const_colour_Y(c))[0] * SH_C0 + 0.5
    ys, xs = np.mgrid[0:H, 0:W]
    d2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
    qq = d2 / v
    alpha = np.minimum(0.99, float(np.float32(o)) * np.exp(-0.5 * qq))
    inside = qq <= 9.0
    band = np.abs(qq - 9.0) < 1e-4
    exp_rgb = np.where(inside[..., None], alpha[..., None] * cf + (1 - alpha[..., None]) * bg, bg)
    ok = ~band
    np.testing.assert_allclose(out["rgb"][ok], exp_rgb[ok], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(out["count"][ok], inside[ok].astype(np.int32))
    # T = 1 - a inside (a single factor of Eq. 2's transmittance)
    np.testing.assert_allclose(out["aux"][4][ok], np.where(inside, 1 - alpha, 1.0)[ok], atol=1e-12)


def _proj(t, f, cx, cy):
    return np.array([f * t[0] / t[2] + cx, f * t[1] / t[2] + cy])


def _fd_jacobian(t, f, cx, cy, h=1e-6):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (_proj(t + e, f, cx, cy) - _proj(t - e, f, cx, cy)) / (2 * h)
    return J


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ewa_covariance_matches_fd_jacobian_and_scipy_rotation(oracle_lib, seed):
    """Sigma_2D = J W R S^2 R^T W^T J^T + 0.3 I with J the derivative of the
    pinhole projection (central differences here) and R from scipy."""
    rng = np.random.default_rng(seed)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 320, 240, 60.0)[seed + 1]
    mu = _f32(rng.uniform(-1, 1, 3))
    s = _f32(np.exp(rng.normal(-3, 0.5, 3)))
    q = _f32(rng.normal(size=4))
    g = oracle.preprocess(_rec(mu, s, q)[None], cam)[0]
    Wm = np.asarray(cam.R, np.float64)
    t = Wm @ mu + np.asarray(cam.t, np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    J = _fd_jacobian(t, cam.fx, cam.cx, cam.cy)
    S = J @ Wm @ R @ np.diag(s ** 2) @ R.T @ Wm.T @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(g["cov"], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-6)
    np.testing.assert_allclose(g["mean"], _proj(t, cam.fx, cam.cx, cam.cy), rtol=1e-12)
    np.testing.assert_allclose(g["depth"], t[2], rtol=1e-12)
    inv = np.linalg.inv(S)
    np.testing.assert_allclose(g["conic"], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-5)


def test_jacobian_frustum_clamp(oracle_lib):
    """Outside 1.3 x the half field of view the Jacobian is taken at the
    clamped direction (3DGS reading); the mean itself is not clamped."""
    W, H, f = 100, 80, 50.0
    cam = Cam(np.eye(3), [0, 0, 0], f, W, H)
    z = 2.0
    limx = 1.3 * (0.5 * W / f)
    x = 3.0 * limx * z          # far outside the limit
    s = 0.05
    g = oracle.preprocess(_rec(_f32([x, 0.0, z]), _f32([s] * 3))[None], cam)[0]
    tc = np.array([limx * z, 0.0, z])
    J = _fd_jacobian(tc, f, cam.cx, cam.cy)
    S = J @ (float(np.float32(s)) ** 2 * np.eye(3)) @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(g["cov"], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-6)
    np.testing.assert_allclose(g["mean"][0], f * float(np.float32(x)) / z + W / 2, rtol=1e-12)


def test_rotation_matches_scipy(oracle_lib):
    rng = np.random.default_rng(3)
    for _ in range(50):
        q = rng.normal(size=4)
        R = oracle.rotation(q)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-13)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1) < 1e-13
        np.testing.assert_allclose(oracle.rotation(-q), R, atol=1e-13)
        np.testing.assert_allclose(oracle.rotation(2.5 * q), R, atol=1e-13)


def test_rotation_about_z_covariance_sign(oracle_lib):
    """A rotation by theta about the optical axis gives an off-diagonal
    Sigma_xy = (sx^2 - sy^2) cos(theta) sin(theta) (f/z)^2: pins the quaternion
    order (w, x, y, z) and the handedness."""
    f, z, th = 100.0, 3.0, 0.5
    sx, sy = 0.08, 0.02
    q = [math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)]
    cam = Cam(np.eye(3), [0, 0, 0], f, 64, 64)
    g = oracle.preprocess(_rec(_f32([0, 0, z]), _f32([sx, sy, 0.01]), _f32(q))[None], cam)[0]
    sx32, sy32 = float(np.float32(sx)), float(np.float32(sy))
    k = (cam.fx / float(np.float32(z))) ** 2
    exp_b = (sx32 ** 2 - sy32 ** 2) * math.cos(th) * math.sin(th) * k
    assert g["cov"][1] == pytest.approx(exp_b, rel=1e-6)
    assert g["cov"][0] == pytest.approx((sx32 ** 2 * math.cos(th) ** 2 + sy32 ** 2 * math.sin(th) ** 2) * k + 0.3, rel=1e-6)


# ---------------------------------------------------------------------------
# Degree-1 SH colour (Sec. 3.2) against scipy's spherical harmonics
# ---------------------------------------------------------------------------

def _sh_basis_scipy(P):
    """Real degree-<=1 basis in the 3DGS ordering, from scipy's complex SH
    (Condon-Shortley phase included): [Y00, sqrt2 Im Y11, Y10, sqrt2 Re Y11]."""
    x, y, z = P
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    y00 = sp.sph_harm_y(0, 0, theta, phi).real
    y10 = sp.sph_harm_y(1, 0, theta, phi).real
    y11 = sp.sph_harm_y(1, 1, theta, phi)
    return np.array([y00, math.sqrt(2) * y11.imag, y10, math.sqrt(2) * y11.real])


def test_sh_degree1_colour_matches_scipy_basis(oracle_lib):
    rng = np.random.default_rng(5)
    cam = synth.orbit_cameras(8, 8.0, 1.0, 200, 150, 60.0)[3]
    n = 40
    mu = rng.uniform(-1, 1, (n, 3))
    recs = []
    for i in range(n):
        Y = rng.normal(0, 0.3, (4, 3))
        recs.append(_rec(_f32(mu[i]), _f32([0.05] * 3), Y=_f32(Y)))
    A = np.stack(recs)
    g = oracle.preprocess(A, cam)
    centre = -np.asarray(cam.R, np.float64).T @ np.asarray(cam.t, np.float64)
    for i in range(n):
        d = A[i, 0:3] - centre
        P = d / np.linalg.norm(d)
        np.testing.assert_allclose(g[i]["dir"], P, atol=1e-12)
        basis = _sh_basis_scipy(P)
        Y = A[i, 11:23].reshape(4, 3)
        exp = np.maximum(0.0, basis @ Y + 0.5)
        np.testing.assert_allclose(g[i]["rgb"], exp, atol=1e-12)


def test_sh_constant_term_is_view_independent(oracle_lib):
    cams = synth.orbit_cameras(6, 8.0, 1.0, 64, 64, 60.0)
    rec = _rec([0.2, -0.1, 0.3], [0.05] * 3, Y=_const_colour_Y([0.7, 0.2, 0.4]))
    cols = [oracle.preprocess(rec[None], c)[0]["rgb"] for c in cams]
    for c in cols:
        np.testing.assert_allclose(c, [0.7, 0.2, 0.4], atol=1e-12)


# ---------------------------------------------------------------------------
# Invariants of Eq. 2 (order independence, weight scale, same colour)
# ---------------------------------------------------------------------------

def _small_scene(n=300, seed=11):
    s = synth.uniform_scene(n, seed=seed, precision="fp32")
    return s.attrs


def test_permutation_invariance(oracle_lib):
    """Sec. 2 / Sec. 3.1: numerator and denominator are sums (and T a
    product), so shuffling the Gaussians leaves the image unchanged."""
    attrs = _small_scene()
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 80, 72, 60.0)
    a = oracle.render(attrs, cam, bg=(0.2, 0.1, 0.3), want_count=True)
    perm = np.random.default_rng(1).permutation(len(attrs))
    b = oracle.render(attrs[perm], cam, bg=(0.2, 0.1, 0.3), want_count=True)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(a["count"], b["count"])


def test_weight_scale_invariance(oracle_lib):
    attrs = _small_scene()
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 64, 64, 60.0)
    g = oracle.preprocess(attrs, cam)
    off, gids = oracle.bin_tiles(g, 64, 64)
    a, _, _ = oracle.rasterize(g, off, gids, 64, 64, (0.3, 0.3, 0.3))
    g2 = g.copy()
    g2["weight"] *= 7.3
    b, _, _ = oracle.rasterize(g2, off, gids, 64, 64, (0.3, 0.3, 0.3))
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_same_colour_invariant(oracle_lib):
    """If every c_i = c then C = (1 - T) c + T c_bg whatever the weights."""
    mlp = synth.random_mlp(7)
    rng = np.random.default_rng(2)
    n = 200
    attrs = _small_scene(n).astype(np.float64)
    attrs[:, 11:23] = _const_colour_Y([0.25, 0.75, 0.5]).reshape(12)
    cam = synth.look_at((0.3, -0.2, -3), (0, 0, 0), 64, 48, 60.0)
    bg = np.array([0.9, 0.05, 0.1])
    for use_mlp in (False, True):
        out = oracle.render(attrs, cam, mlp=mlp, use_mlp=use_mlp, bg=bg, want_aux=True)
        T = out["aux"][4]
        exp = (1 - T)[..., None] * np.array([0.25, 0.75, 0.5]) + T[..., None] * bg
        np.testing.assert_allclose(out["rgb"], exp, atol=1e-12)
    assert rng is not None


# ---------------------------------------------------------------------------
# Brute force on tiny scenes: tile lists and per-pixel sums
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("W,H,n,seed", [(32, 32, 64, 0), (37, 29, 48, 1), (50, 17, 30, 2)])
def test_bruteforce_tiles_and_pixels(oracle_lib, W, H, n, seed):
    attrs = synth.uniform_scene(n, seed=seed + 100).attrs
    cam = synth.look_at((0.1, 0.0, -2.5), (0, 0, 0), W, H, 60.0)
    bg = np.array([0.05, 0.1, 0.2])
    out = oracle.render(attrs, cam, bg=bg, want_aux=True, want_count=True)
    g = out["gauss"]
    tx, ty = oracle.tiles(W, H)
    # tile lists: the visible Gaussians whose rectangle overlaps the tile,
    # minus those the tile test rules out -- and a Gaussian ruled out
    # includes no pixel of the tile (brute force over the tile's pixels)
    for t in range(tx * ty):
        i, j = t % tx, t // tx
        in_rect = [k for k in range(n) if g[k]["visible"] and g[k]["rect"][0] <= i < g[k]["rect"][2]
                   and g[k]["rect"][1] <= j < g[k]["rect"][3]]
        got = list(out["gids"][out["offsets"][t]:out["offsets"][t + 1]])
        assert got == [k for k in in_rect if k in got]
        for k in set(in_rect) - set(got):
            assert not any(oracle.includes(g[k], px, py)
                           for py in range(16 * j, min(16 * j + 16, H))
                           for px in range(16 * i, min(16 * i + 16, W)))
    # pixels: loop over ALL Gaussians with the same membership rule
    for py in range(H):
        for px in range(W):
            i, j = px // 16, py // 16
            A = np.zeros(3)
            B, T, cnt = 0.0, 1.0, 0
            for k in range(n):
                gk = g[k]
                if not gk["visible"]:
                    continue
                if not (gk["rect"][0] <= i < gk["rect"][2] and gk["rect"][1] <= j < gk["rect"][3]):
                    continue
                if not oracle.includes(gk, px, py):
                    continue
                dx, dy = px + 0.5 - gk["mean"][0], py + 0.5 - gk["mean"][1]
                qq = gk["conic"][0] * dx * dx + 2 * gk["conic"][1] * dx * dy + gk["conic"][2] * dy * dy
                a = min(0.99, gk["opacity"] * math.exp(-0.5 * qq))
                A += gk["rgb"] * a * gk["weight"]
                B += a * gk["weight"]
                T *= 1 - a
                cnt += 1
            C = ((1 - T) * A / B if B > 0 else 0.0) + T * bg
            np.testing.assert_allclose(out["rgb"][py, px], C, rtol=0, atol=1e-12)
            assert out["count"][py, px] == cnt


def test_two_gaussians_at_a_pixel(oracle_lib):
    """Two on-axis isotropic Gaussians at depths 2 and 3 seen at the centre
    pixel: Eq. 2 and Eq. 3 written out by hand (a second transcription of the
    formulas, kept for the arithmetic, not as an independent source)."""
    f, W, H = 80.0, 16, 16
    cam = Cam(np.eye(3), [0, 0, 0], f, W, H)
    z = [2.0, 3.0]
    s = [0.04, 0.06]
    o = [0.6, 0.7]
    cols = [np.array([1.0, 0.2, 0.1]), np.array([0.1, 0.3, 0.9])]
    recs = np.stack([_rec(_f32([0, 0, z[k]]), _f32([s[k]] * 3), o=float(np.float32(o[k])),
                          Y=_f32(_const_colour_Y(cols[k]))) for k in range(2)])
    bg = np.array([0.0, 0.5, 0.0])
    out = oracle.render(recs, cam, bg=bg)
    px = py = 8       # centre (8.5, 8.5); principal point (8, 8)
    al, ws, cs = [], [], []
    for k in range(2):
        s32 = float(np.float32(s[k]))
        v = (f * s32 / z[k]) ** 2 + 0.3
        al.append(min(0.99, float(np.float32(o[k])) * math.exp(-0.5 * (0.5 ** 2 + 0.5 ** 2) / v)))
        ws.append(1.0 + 1.0 / z[k] ** 2 + math.exp(s32 / z[k]))
        cs.append(_f32(_const_colour_Y(cols[k]))[0] * SH_C0 + 0.5)
    T = (1 - al[0]) * (1 - al[1])
    num = cs[0] * al[0] * ws[0] + cs[1] * al[1] * ws[1]
    den = al[0] * ws[0] + al[1] * ws[1]
    np.testing.assert_allclose(out["rgb"][py, px], (1 - T) * num / den + T * bg, atol=1e-12)


# ---------------------------------------------------------------------------
# Eq. 3 properties the paper states in words
# ---------------------------------------------------------------------------

def test_weight_decreases_with_depth_increases_with_scale(oracle_lib):
    """Sec. 3.1: inverse depth lowers the weight of distant Gaussians; larger
    scale raises it; it depends only on the largest scale (so not on the
    rotation)."""
    cam = Cam(np.eye(3), [0, 0, 0], 100.0, 64, 64)
    zs = [0.5, 1.0, 2.0, 4.0, 8.0]
    w_z = [oracle.preprocess(_rec([0, 0, z], [0.1, 0.05, 0.02])[None], cam)[0]["weight"] for z in zs]
    assert all(a > b for a, b in zip(w_z, w_z[1:]))
    ss = [0.01, 0.05, 0.1, 0.3]
    w_s = [oracle.preprocess(_rec([0, 0, 2.0], [s, 0.01, 0.01])[None], cam)[0]["weight"] for s in ss]
    assert all(a < b for a, b in zip(w_s, w_s[1:]))
    w_a = oracle.preprocess(_rec([0, 0, 2.0], [0.01, 0.3, 0.01], q=(0.3, 0.4, -0.2, 0.8))[None], cam)[0]["weight"]
    w_b = oracle.preprocess(_rec([0, 0, 2.0], [0.3, 0.01, 0.01])[None], cam)[0]["weight"]
    assert w_a == pytest.approx(w_b, rel=1e-14)


def _zero_mlp(b_phi, b_o):
    z64 = np.zeros((64, 22), np.uint16)
    return synth.MLPWeights(z64, np.zeros(64, np.float32), np.zeros((64, 64), np.uint16),
                            np.zeros(64, np.float32), np.zeros((5, 64), np.uint16),
                            np.array([b_phi, b_o, 0, 0, 0], np.float32))


def test_weight_with_phi_zero_and_large_phi(oracle_lib):
    cam = Cam(np.eye(3), [0, 0, 0], 100.0, 64, 64)
    rec = _rec([0, 0, 2.0], [0.1, 0.05, 0.02])[None]
    g0 = oracle.preprocess(rec, cam, mlp=_zero_mlp(-1.0, 0.0), use_mlp=True)[0]
    assert g0["phi"] == 0.0
    assert g0["weight"] == pytest.approx(math.exp(0.1 / 2.0), rel=1e-14)
    g1 = oracle.preprocess(rec, cam, mlp=_zero_mlp(1000.0, 0.0), use_mlp=True)[0]
    assert g1["weight"] / 1000.0 ** 2 == pytest.approx(1.0, rel=1e-3)


# ---------------------------------------------------------------------------
# Eq. 4 MLP against torch (library special case) and its degenerate case
# ---------------------------------------------------------------------------

def test_bf16_round_matches_torch(oracle_lib):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    v = rng.normal(0, 3, 2000).astype(np.float32)
    v[:10] = [0.0, 1.0, -1.0, 1.00390625, 1.01171875, 3.0e-5, 65504.0, 1.0078125, -2.5, 1e20]
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.bf16_round(float(x)) for x in v])
    np.testing.assert_array_equal(got, ref)


def test_mlp_matches_torch_linear(oracle_lib):
    torch = pytest.importorskip("torch")
    mlp = synth.random_mlp(9)
    rng = np.random.default_rng(6)

    def w(bits):
        return torch.from_numpy(synth.bf16_bits_to_f32(bits).astype(np.float64))

    def bf(t):
        return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)

    l1 = torch.nn.Linear(22, 64, dtype=torch.float64)
    l2 = torch.nn.Linear(64, 64, dtype=torch.float64)
    l3 = torch.nn.Linear(64, 5, dtype=torch.float64)
    with torch.no_grad():
        l1.weight.copy_(w(mlp.w1)); l1.bias.copy_(torch.from_numpy(mlp.b1.astype(np.float64)))
        l2.weight.copy_(w(mlp.w2)); l2.bias.copy_(torch.from_numpy(mlp.b2.astype(np.float64)))
        l3.weight.copy_(w(mlp.w3)); l3.bias.copy_(torch.from_numpy(mlp.b3.astype(np.float64)))
        for _ in range(64):
            x = rng.normal(0, 0.6, 22).astype(np.float32).astype(np.float64)
            xt = bf(torch.from_numpy(x))
            h1 = bf(torch.relu(l1(xt)))
            h2 = bf(torch.relu(l2(h1)))
            y = l3(h2)
            exp = np.array([max(0.0, y[0].item()), torch.sigmoid(y[1]).item(), y[2].item(),
                            y[3].item(), y[4].item()])
            np.testing.assert_allclose(oracle.mlp_eval(mlp, x), exp, rtol=1e-12, atol=1e-12)


def test_paper_width_mlp_matches_torch_linear(oracle_lib):
    """App. C's MLP_f (22 -> 256 -> 128 -> 64, then the phi / o heads):
    the oracle's generic layers against a torch nn.Linear chain in FP64 with
    the same BF16 rounding of every layer input."""
    torch = pytest.importorskip("torch")
    mlp = synth.random_mlp_paper(19)
    assert mlp.hidden == (256, 128, 64)
    rng = np.random.default_rng(16)

    def lin(bits, b):
        wt = torch.from_numpy(synth.bf16_bits_to_f32(bits).astype(np.float64))
        m = torch.nn.Linear(wt.shape[1], wt.shape[0], dtype=torch.float64)
        with torch.no_grad():
            m.weight.copy_(wt)
            m.bias.copy_(torch.from_numpy(np.asarray(b, np.float64)))
        return m

    def bf(t):
        return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)

    layers = [lin(mlp.w1, mlp.b1), lin(mlp.w2, mlp.b2), lin(mlp.w3, mlp.b3)]
    head = lin(mlp.w4, mlp.b4)
    with torch.no_grad():
        for _ in range(32):
            x = rng.normal(0, 0.6, 22).astype(np.float32).astype(np.float64)
            h = bf(torch.from_numpy(x))
            for l in layers:
                h = bf(torch.relu(l(h)))
            y = head(h)
            exp = np.array([max(0.0, y[0].item()), torch.sigmoid(y[1]).item(), y[2].item(),
                            y[3].item(), y[4].item()])
            np.testing.assert_allclose(oracle.mlp_eval(mlp, x), exp, rtol=1e-12, atol=1e-12)


def test_paper_width_mlp_zero_weights_reduce_to_plain(oracle_lib):
    """Zero weights in every layer of the paper-width MLP: the render equals
    the plain render with phi = ReLU(b_phi), o = sigmoid(b_o)."""
    mlp = synth.random_mlp_paper(3)
    for k in ("w1", "w2", "w3", "w4"):
        setattr(mlp, k, np.zeros_like(getattr(mlp, k)))
    b_o = -0.3
    mlp.b4 = np.array([1.0, b_o, 0.0, 0.0, 0.0], np.float32)
    attrs = _small_scene(120).astype(np.float64)
    attrs[:, 10] = 1.0 / (1.0 + math.exp(-b_o))
    cam = synth.look_at((0, 0.2, -3), (0, 0, 0), 40, 40, 60.0)
    a = oracle.render(attrs, cam, mlp=mlp, use_mlp=True)
    b = oracle.render(attrs, cam)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)


def test_mlp_zero_weights_reduce_to_plain(oracle_lib):
    """Zero weights: phi = ReLU(b_phi), o = sigmoid(b_o), so the MLP render
    equals the plain render of a scene whose stored opacities are sigmoid(b_o)."""
    attrs = _small_scene(150).astype(np.float64)
    b_o = 0.4
    o = 1.0 / (1.0 + math.exp(-b_o))
    attrs[:, 10] = o
    cam = synth.look_at((0, 0.2, -3), (0, 0, 0), 48, 48, 60.0)
    a = oracle.render(attrs, cam, mlp=_zero_mlp(1.0, b_o), use_mlp=True)
    b = oracle.render(attrs, cam)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)


# ---------------------------------------------------------------------------
# The FP32 contract agrees with the FP64 values it stands in for
# ---------------------------------------------------------------------------

def test_fp32_contract_consistent_with_fp64(oracle_lib):
    attrs = synth.unbounded_scene(3000, seed=8, precision="fp16").attrs
    cam = synth.orbit_cameras(4, 8.0, 1.0, 320, 212, 60.0)[1]
    g = oracle.preprocess(attrs, cam)
    v = g[g["visible"] == 1]
    assert len(v) > 500
    np.testing.assert_allclose(v["m32"], v["mean"], rtol=2e-5, atol=1e-3)
    l = v["l32"].astype(np.float64)
    A, B, C = v["conic"][:, 0], v["conic"][:, 1], v["conic"][:, 2]
    np.testing.assert_allclose(l[:, 0] ** 2, A, rtol=1e-3)
    np.testing.assert_allclose(l[:, 0] * l[:, 1], B, rtol=1e-3, atol=1e-5 * np.abs(A).max())
    np.testing.assert_allclose(l[:, 1] ** 2 + l[:, 2] ** 2, C, rtol=1e-3)
    # the rectangle is the 3-sigma square of the largest eigenvalue (numpy eig)
    checked = 0
    for gi in v[:400]:
        a, b, c = gi["cov"]
        lam = np.linalg.eigvalsh(np.array([[a, b], [b, c]])).max()
        r_exact = 3 * math.sqrt(lam)
        if abs(r_exact - round(r_exact)) < 1e-3:
            continue
        r = math.ceil(r_exact)
        mx, my = gi["mean"]
        lo = [math.floor((mx - r) / 16), math.floor((my - r) / 16)]
        hi = [math.floor((mx + r) / 16) + 1, math.floor((my + r) / 16) + 1]
        if any(abs((m + d) / 16 - round((m + d) / 16)) < 1e-3 for m in (mx, my) for d in (-r, r)):
            continue
        exp = [min(max(lo[0], 0), 20), min(max(lo[1], 0), 14), min(max(hi[0], 0), 20), min(max(hi[1], 0), 14)]
        assert list(gi["rect"]) == exp
        checked += 1
    assert checked > 300


def test_predicate_matches_fp64_ellipse_away_from_boundary(oracle_lib):
    attrs = synth.uniform_scene(200, seed=12).attrs
    cam = synth.look_at((0, 0, -3), (0, 0, 0), 96, 96, 60.0)
    g = oracle.preprocess(attrs, cam)
    rng = np.random.default_rng(0)
    n_in = n_tot = 0
    for gi in g[g["visible"] == 1][:60]:
        for _ in range(60):
            r = 3.5 * math.sqrt(max(gi["cov"][0], gi["cov"][2]))
            px = int(np.clip(math.floor(gi["mean"][0] + rng.uniform(-r, r)), 0, 95))
            py = int(np.clip(math.floor(gi["mean"][1] + rng.uniform(-r, r)), 0, 95))
            dx, dy = px + 0.5 - gi["mean"][0], py + 0.5 - gi["mean"][1]
            A, B, C = gi["conic"]
            qq = A * dx * dx + 2 * B * dx * dy + C * dy * dy
            if abs(qq - 9) < 1e-3:
                continue
            assert oracle.includes(gi, px, py) == (qq <= 9)
            n_in += qq <= 9
            n_tot += 1
    assert n_in > 500 and n_tot > 2000


def test_tile_lists_are_the_rectangle_set_minus_tiles_without_pixels(oracle_lib):
    """On a larger unbounded scene: every listed (tile, Gaussian) pair lies in
    the Gaussian's 3-sigma rectangle (the tile test only removes pairs), and
    every rectangle pair left out has no pixel centre strictly inside the
    ellipse q <= 9 (evaluated in FP64 with a 1e-3 margin, so that a pair the
    FP32 predicate could include is never missing)."""
    scene = synth.unbounded_scene(20000, seed=9, precision="fp16")
    cam = synth.orbit_cameras(8, 8.0, 1.0, 320, 213, 60.0)[2]
    g = oracle.preprocess(scene.attrs, cam)
    off, gids = oracle.bin_tiles(g, cam.width, cam.height)
    tx, ty = oracle.tiles(cam.width, cam.height)
    tile = np.repeat(np.arange(tx * ty), np.diff(off))
    rect = g["rect"][gids]
    i, j = tile % tx, tile // tx
    assert np.all(g["visible"][gids] == 1)
    assert np.all((rect[:, 0] <= i) & (i < rect[:, 2]) & (rect[:, 1] <= j) & (j < rect[:, 3]))
    listed = set(zip(tile.tolist(), gids.tolist()))
    dropped = 0
    for k in np.flatnonzero(g["visible"]):
        x0, y0, x1, y1 = g["rect"][k]
        c = g["conic"][k]
        m = g["mean"][k]
        for tj in range(y0, y1):
            for ti in range(x0, x1):
                if (tj * tx + ti, int(k)) in listed:
                    continue
                dropped += 1
                px = np.arange(16 * ti, min(16 * ti + 16, cam.width)) + 0.5 - m[0]
                py = np.arange(16 * tj, min(16 * tj + 16, cam.height)) + 0.5 - m[1]
                dx, dy = np.meshgrid(px, py)
                q = c[0] * dx * dx + 2 * c[1] * dx * dy + c[2] * dy * dy
                assert q.min() > 9.0 - 1e-3, (k, ti, tj)
    assert dropped > 0 and len(listed) > 0
