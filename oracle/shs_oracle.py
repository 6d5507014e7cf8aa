"""FP64 CPU oracle for SH soft-shadow shading (Lyu et al., "Efficient and
Differentiable Shadow Computation for Inverse Problems", arXiv 2104.00359).

TEST INFRASTRUCTURE.  This module exists to check the CUDA library.  Only the
test suite, the package smoke check and the CPU-baseline leg of the benchmark
may import it; the shading library itself never calls it and has no CPU
fallback.  It shares no code with the CUDA path.

Everything here is plain float64 numpy, written step by step in the paper's
order so it can be read against the paper:

* real orthonormal SH basis, linear index i = l^2 + l + m      (Sec. 3.2, Eq. 3)
* SH triple-product tensor C_ijk = int y_i y_j y_k            (Sec. 3.2, Eq. 6-7)
* clamped-cosine lobe H as a rotated zonal function           (Sec. 3.3, Eq. 10-11)
* per-sphere log of the softened blocker, e^-eps when blocked (Sec. 3.3.2, Eq. 13)
  projected along z (ZH) and rotated toward the sphere centre
* log-visibility = sum over spheres, then SH exponential      (Sec. 3.3.2, Eq. 12)
* shading B = a * (L . (V * H))                               (Sec. 3.2, Eq. 8)
* lighting projected from an equirectangular map              (Sec. 3.3, Eq. 9)
* reverse-mode adjoint of all of the above (for d/d lighting, albedo, sphere
  centres and radii, point positions and normals; Sec. 3.5)

Readings where the paper is silent (each is also a configuration field):

* Real SH without the Condon-Shortley phase; m > 0 <-> cos(m phi),
  m < 0 <-> sin(|m| phi).  Indices are 0-based.
* The triple product is truncated to the same n bands as its inputs.
* A shading point inside or on a sphere (D <= r) sees a hemisphere cap
  (sin(alpha) clamped to 1, cos(alpha) = 0); no gradient flows through the
  clamped cap angle.  A sphere whose centre coincides with the point (D = 0)
  is skipped.  By default every sphere contributes (the paper sums all
  blockers); with ``horizon_cull`` a sphere lying entirely below the tangent
  plane at x, (c - x) . n_hat < -r, is dropped for that point (no gradient
  flows through that selection).
* SH exponential (the paper defers to Ren et al. 2006 "scaling, squaring and
  optimal linear approximation" without giving constants):
    1. DC isolation  e0 = exp(f_0 / sqrt(4 pi)),  fh = f with fh_0 = 0
    2. scaling       k = smallest integer >= 0 with |fh| <= tau * 2^k,
                     capped at kmax (or a fixed k), g = fh / 2^k
    3. optimal linear approximation of exp on span{1, g}: least squares with
       the values of g over the sphere taken as N(0, s^2), s^2 = |g|^2/(4 pi),
       which gives a = b = exp(|g|^2 / (8 pi));  V0 = a * sqrt(4 pi) e_0 + b g
    4. k squarings V <- V * V (truncated triple product)
    5. V <- e0 * V
  Parity of these constants is unpinned against the paper (it prints none);
  they are pinned to the definitions stated above.  Variants: exp_mode 1
  replaces steps 2-4 by the projection of exp(fh~) by a quadrature rule;
  exp_mode 2 takes a and b in step 3 from a table a(s), b(s), s = |g|,
  linear between its nodes and constant past the last (``ol_table``; the
  fitted tables come from oracle/fit_ol_table.py).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from numpy.polynomial import legendre as _leg
from numpy.polynomial import polynomial as _poly

FOUR_PI = 4.0 * math.pi
SQRT_FOUR_PI = math.sqrt(FOUR_PI)


@dataclass
class Config:
    """Method constants.  ``epsilon`` = 3 is the paper's softened-blocker
    exponent (Sec. 3.3.2, Eq. 13); the others are the readings above."""
    n_bands: int = 4
    epsilon: float = 3.0
    exp_tau: float = 1.0
    exp_kmax: int = 16
    fixed_k: int = -1
    horizon_cull: bool = False
    exp_mode: int = 0          # 0: scaling + optimal linear + squarings; 1: projected exponential
    exp_rule: tuple | None = None   # (n_theta, n_phi) of the projected exponential; None: (2n, 4n)
    ol_table: tuple | None = None   # exp_mode 2: (a [M], b [M], s_max), a(s), b(s) on s_m = m s_max / (M-1)


def sh_index(l, m):
    """Linear SH index i = l^2 + l + m (Sec. 3.2)."""
    return l * l + l + m


def band_of(K):
    """Band l of each linear index 0..K-1."""
    return np.floor(np.sqrt(np.arange(K))).astype(np.int64)


# ----------------------------------------------------------------------------
# O1: real SH basis (Sec. 3.2, Eq. 3-4)
# ----------------------------------------------------------------------------

def sh_normalisation(l, m):
    am = abs(m)
    return math.sqrt((2 * l + 1) / FOUR_PI * math.factorial(l - am) / math.factorial(l + am))


def _legendre_derivative_power(l, order):
    """Power-basis coefficients (in z) of d^order/dz^order P_l(z)."""
    c = np.zeros(l + 1)
    c[l] = 1.0
    return _poly.polyder(_leg.leg2poly(c), order) if order > 0 else _leg.leg2poly(c)


def real_sh(n_bands, dirs):
    """y_i(dirs) for i < n_bands^2; dirs [..., 3] unit vectors.

    Textbook Cartesian form of the real orthonormal SH: with
    P_l^m(z) = (1 - z^2)^{m/2} d^m P_l / dz^m (no Condon-Shortley phase) and
    (1 - z^2)^{m/2} e^{i m phi} = (x + i y)^m on the unit sphere,
      y_l0        = N_l0 P_l(z)
      y_l,+m      = sqrt(2) N_lm d^mP_l/dz^m (z) Re (x + i y)^m
      y_l,-m      = sqrt(2) N_lm d^mP_l/dz^m (z) Im (x + i y)^m
    """
    dirs = np.asarray(dirs, dtype=np.float64)
    x, y, z = dirs[..., 0], dirs[..., 1], dirs[..., 2]
    out = np.empty(dirs.shape[:-1] + (n_bands * n_bands,))
    w = x + 1j * y
    for l in range(n_bands):
        for am in range(l + 1):
            pz = _poly.polyval(z, _legendre_derivative_power(l, am))
            N = sh_normalisation(l, am)
            if am == 0:
                out[..., sh_index(l, 0)] = N * pz
            else:
                wm = w ** am
                out[..., sh_index(l, am)] = math.sqrt(2) * N * pz * wm.real
                out[..., sh_index(l, -am)] = math.sqrt(2) * N * pz * wm.imag
    return out


def real_sh_grad(n_bands, dirs):
    """Gradient of the Cartesian polynomial extension of y_i: [..., K, 3].
    The gradient on the sphere is its tangential part."""
    dirs = np.asarray(dirs, dtype=np.float64)
    x, y, z = dirs[..., 0], dirs[..., 1], dirs[..., 2]
    K = n_bands * n_bands
    out = np.zeros(dirs.shape[:-1] + (K, 3))
    w = x + 1j * y
    for l in range(n_bands):
        for am in range(l + 1):
            pz = _poly.polyval(z, _legendre_derivative_power(l, am))
            dpz = _poly.polyval(z, _legendre_derivative_power(l, am + 1)) if am + 1 <= l else 0.0 * z
            N = sh_normalisation(l, am)
            if am == 0:
                out[..., sh_index(l, 0), 2] = N * dpz
                continue
            s2N = math.sqrt(2) * N
            wm = w ** am
            dw = am * w ** (am - 1)          # d/dx (x+iy)^m ; d/dy = i * dw
            ip, im_ = sh_index(l, am), sh_index(l, -am)
            out[..., ip, 0] = s2N * pz * dw.real
            out[..., ip, 1] = s2N * pz * (-dw.imag)
            out[..., ip, 2] = s2N * dpz * wm.real
            out[..., im_, 0] = s2N * pz * dw.imag
            out[..., im_, 1] = s2N * pz * dw.real
            out[..., im_, 2] = s2N * dpz * wm.imag
    return out


def sphere_quadrature(n_theta, n_phi):
    """Gauss-Legendre nodes in z = cos(theta) times uniform nodes in phi.
    Exact for polynomials in (x, y, z) of degree < min(2 n_theta, n_phi)."""
    zt, wt = _leg.leggauss(n_theta)
    phi = 2.0 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    Z, PHI = np.meshgrid(zt, phi, indexing="ij")
    S = np.sqrt(1.0 - Z * Z)
    dirs = np.stack([S * np.cos(PHI), S * np.sin(PHI), Z], axis=-1).reshape(-1, 3)
    w = (wt[:, None] * np.full(n_phi, 2.0 * math.pi / n_phi)[None, :]).reshape(-1)
    return dirs, w


# ----------------------------------------------------------------------------
# O2: triple-product tensor (Sec. 3.2, Eq. 6-7)
# ----------------------------------------------------------------------------

_GAUNT_CACHE = {}


def gaunt_tensor(n_bands):
    """C_ijk = int y_i y_j y_k d omega for i, j, k < n_bands^2, by a
    quadrature exact for the degree-3(n-1) integrand."""
    if n_bands in _GAUNT_CACHE:
        return _GAUNT_CACHE[n_bands]
    deg = 3 * (n_bands - 1)
    dirs, w = sphere_quadrature(deg // 2 + 2, deg + 2)
    Y = real_sh(n_bands, dirs)
    C = np.einsum("q,qi,qj,qk->ijk", w, Y, Y, Y, optimize=True)
    C[np.abs(C) < 1e-13] = 0.0
    _GAUNT_CACHE[n_bands] = C
    return C


def sh_product(C, a, b):
    """(a * b)_i = sum_jk C_ijk a_j b_k (Eq. 7), batched over leading axes."""
    return np.einsum("ijk,...j,...k->...i", C, a, b, optimize=True)


# ----------------------------------------------------------------------------
# O3: clamped-cosine lobe (Sec. 3.3, Eq. 10-11)
# ----------------------------------------------------------------------------

def _gauss_on_interval(lo, hi, n=32):
    t, w = _leg.leggauss(n)
    return 0.5 * (hi - lo) * t + 0.5 * (hi + lo), 0.5 * (hi - lo) * w


def clamped_cosine_zh(n_bands):
    """ZH coefficients of max(i_z . omega, 0): 2 pi N_l0 int_0^1 t P_l(t) dt."""
    t, w = _gauss_on_interval(0.0, 1.0)
    out = np.empty(n_bands)
    for l in range(n_bands):
        pl = _leg.legval(t, np.eye(l + 1)[l])
        out[l] = 2.0 * math.pi * sh_normalisation(l, 0) * np.sum(w * t * pl)
    return out


def zh_rotation_scale(n_bands):
    """sqrt(4 pi / (2l + 1)) per coefficient: rotating a zonal function with
    ZH coefficients z_l to direction d gives z_l sqrt(4pi/(2l+1)) y_lm(d)."""
    l = band_of(n_bands * n_bands)
    return np.sqrt(FOUR_PI / (2.0 * l + 1.0))


def cosine_lobe(n_bands, normals):
    """H(x) = phi_SH(n(x)) applied to the clamped-cosine ZH (Eq. 11)."""
    nrm = np.asarray(normals, np.float64)
    nh = nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)
    zh = clamped_cosine_zh(n_bands)[band_of(n_bands * n_bands)]
    return zh_rotation_scale(n_bands) * zh * real_sh(n_bands, nh)


# ----------------------------------------------------------------------------
# O4: per-sphere log-visibility (Sec. 3.3.2, Eq. 13 and the text after it)
# ----------------------------------------------------------------------------

def cap_cosine(points, center, radius):
    """d = c - x, D = |d|, s = sin(alpha) = min(r / D, 1), cos(alpha)."""
    d = center[None, :] - points
    D = np.linalg.norm(d, axis=-1)
    valid = D > 0.0
    Ds = np.where(valid, D, 1.0)
    s = np.minimum(radius / Ds, 1.0)
    cos_a = np.sqrt(np.maximum(1.0 - s * s, 0.0))
    return d, Ds, valid, s, cos_a


def log_cap_zh(n_bands, epsilon, cos_a):
    """ZH (along z) of log V'(omega) = -eps on the cap omega_z >= cos(alpha),
    0 elsewhere: -eps 2 pi N_l0 int_{cos alpha}^1 P_l(t) dt.  [..., n_bands]"""
    out = np.empty(np.shape(cos_a) + (n_bands,))
    for l in range(n_bands):
        t, w = _gauss_on_interval(np.asarray(cos_a)[..., None], 1.0)
        pl = _leg.legval(t, np.eye(l + 1)[l])
        out[..., l] = -epsilon * 2.0 * math.pi * sh_normalisation(l, 0) * np.sum(w * pl, axis=-1)
    return out


def horizon_keep(cfg, d, radius, normals):
    """Pairs that contribute: all of them, or with horizon culling those whose
    sphere reaches the upper half-space of the normal, (c - x) . n_hat >= -r."""
    if not cfg.horizon_cull:
        return np.ones(d.shape[0], dtype=bool)
    nrm = np.asarray(normals, np.float64)
    nh = nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)
    return np.sum(d * nh, axis=-1) >= -radius


def log_visibility(cfg, points, centers, radii, normals=None):
    """f(x) = sum_j rotate(ZH of log V'_j, (c_j - x)/|c_j - x|)  [P, K]."""
    n = cfg.n_bands
    K = n * n
    P = points.shape[0]
    pts = np.asarray(points, np.float64)
    f = np.zeros((P, K))
    lvec = band_of(K)
    R = zh_rotation_scale(n)
    if cfg.horizon_cull and normals is None:
        raise ValueError("horizon culling needs the normals")
    for j in range(np.shape(centers)[0]):
        d, D, valid, s, ca = cap_cosine(pts, np.asarray(centers[j], np.float64), float(radii[j]))
        valid = valid & horizon_keep(cfg, d, float(radii[j]), normals)
        zh = log_cap_zh(n, cfg.epsilon, ca)
        sh = d / D[:, None]
        Fj = R[None, :] * zh[:, lvec] * real_sh(n, sh)
        f += np.where(valid[:, None], Fj, 0.0)
    return f


# ----------------------------------------------------------------------------
# O6: SH exponential (Sec. 3.3.2; scaling, squaring, optimal linear approx.)
# ----------------------------------------------------------------------------

def exp_scaling_k(cfg, f):
    """Number of squarings per point (reading stated in the module header)."""
    fh = f[:, 1:]
    norm = np.sqrt(np.sum(fh * fh, axis=-1))
    if cfg.fixed_k >= 0:
        return np.full(f.shape[0], cfg.fixed_k, dtype=np.int64)
    # |fh| > tau 2^j holds for exactly the j < k, so counting them gives k.
    k = np.zeros(f.shape[0], dtype=np.int64)
    for j in range(cfg.exp_kmax):
        k += norm > cfg.exp_tau * (2.0 ** j)
    return k


def ol_coefficients(cfg, s):
    """Optimal-linear coefficients a(s), b(s) and their derivatives at the
    norms s of the scaled exponents.  exp_mode 0/1: the Gaussian reading
    a = b = exp(s^2 / 8 pi).  exp_mode 2: a fitted table, linear between its
    nodes s_m = m s_max / (M - 1) and constant beyond s_max."""
    s = np.asarray(s, np.float64)
    if cfg.exp_mode != 2:
        a = np.exp(s * s / (2.0 * FOUR_PI))
        return a, a.copy(), a * s / FOUR_PI, a * s / FOUR_PI
    ta, tb, s_max = cfg.ol_table
    ta, tb = np.asarray(ta, np.float64), np.asarray(tb, np.float64)
    M = ta.shape[0]
    h = s_max / (M - 1)
    x = np.clip(s / h, 0.0, M - 1.0)
    i = np.minimum(np.floor(x).astype(np.int64), M - 2)
    t = x - i
    a = ta[i] + t * (ta[i + 1] - ta[i])
    b = tb[i] + t * (tb[i + 1] - tb[i])
    inside = s < s_max
    da = np.where(inside, (ta[i + 1] - ta[i]) / h, 0.0)
    db = np.where(inside, (tb[i + 1] - tb[i]) / h, 0.0)
    return a, b, da, db


def sh_exp(cfg, C, f, k=None):
    """V = exp*(f) with the steps of the module header.  Returns V and the
    per-point intermediates the adjoint needs."""
    P, K = f.shape
    if k is None:
        k = exp_scaling_k(cfg, f)
    k = np.asarray(k, dtype=np.int64)
    if P and (k.min() < 0 or k.max() > 64):
        raise ValueError("squaring count out of range")
    e0 = np.exp(f[:, 0] / SQRT_FOUR_PI)
    fh = f.copy()
    fh[:, 0] = 0.0
    g = fh / (2.0 ** k)[:, None]
    sn = np.sqrt(np.sum(g * g, axis=-1))
    a, b, da_ds, db_ds = ol_coefficients(cfg, sn)
    S = b[:, None] * g
    S[:, 0] = a * SQRT_FOUR_PI
    levels = [S]
    for t in range(int(k.max()) if P else 0):
        act = (k > t)[:, None]
        S = np.where(act, sh_product(C, S, S), S)
        levels.append(S)
    V = e0[:, None] * S
    return V, dict(k=k, e0=e0, g=g, a=a, b=b, da_ds=da_ds, db_ds=db_ds, s=sn, levels=levels)


def projected_exp_rule(n_bands):
    """Quadrature of the projected-exponential variant: 2n Gauss-Legendre nodes
    in cos(theta) x 4n uniform azimuths (exact for polynomial integrands of
    degree < 4n; exp of the log-visibility is not one, so the rule is part of
    the variant's definition)."""
    return sphere_quadrature(2 * n_bands, 4 * n_bands)


def sh_exp_projected(n_bands, f, rule=None):
    """Variant of the SH exponential (the next-step alternative to Ren et
    al.'s scaling and squaring): the projection onto n bands of the pointwise
    exponential of the band-limited log-visibility,
        V_i = sum_q w_q exp(f~(w_q)) y_i(w_q),   f~ = sum_j f_j y_j,
    with the constant term isolated (exp(f~) = e0 exp(f^), e0 = exp(f_0 y_0)).
    Returns V and the intermediates of its adjoint."""
    dirs, w = rule if rule is not None else projected_exp_rule(n_bands)
    Y = real_sh(n_bands, dirs)                     # [Q, K]
    e0 = np.exp(f[:, 0] / SQRT_FOUR_PI)
    fh = f.copy()
    fh[:, 0] = 0.0
    E = np.exp(fh @ Y.T)                           # [P, Q]
    U = (E * w[None, :]) @ Y
    V = e0[:, None] * U
    return V, dict(k=np.zeros(f.shape[0], dtype=np.int64), e0=e0, E=E, Y=Y, w=w, U=U)


# ----------------------------------------------------------------------------
# Forward shading (Eq. 8)
# ----------------------------------------------------------------------------

def shade_forward(cfg, points, normals, albedo, centers, radii, light, k=None):
    """B_c(x) = a_c(x) * (L_c . (V(x) * H(x))) for c in RGB.

    All arrays are upcast to float64.  ``k`` optionally overrides the number
    of squarings per point.  Returns a dict with ``radiance`` [P, 3] and the
    intermediates ``f``, ``V``, ``H``, ``W`` = V*H and ``k``."""
    n = cfg.n_bands
    C = gaunt_tensor(n)
    pts = np.asarray(points, np.float64)
    alb = np.asarray(albedo, np.float64)
    L = np.asarray(light, np.float64).reshape(3, n * n)
    f = log_visibility(cfg, pts, np.asarray(centers, np.float64).reshape(-1, 3),
                       np.asarray(radii, np.float64).reshape(-1), normals)
    if cfg.exp_mode == 1:
        V, ex = sh_exp_projected(n, f, None if cfg.exp_rule is None else sphere_quadrature(*cfg.exp_rule))
    else:
        V, ex = sh_exp(cfg, C, f, k)
    H = cosine_lobe(n, normals)
    W = sh_product(C, V, H)
    B = alb * (W @ L.T)
    return dict(radiance=B, f=f, V=V, H=H, W=W, k=ex["k"], _exp=ex)


# ----------------------------------------------------------------------------
# Lighting from an environment map (Eq. 9)
# ----------------------------------------------------------------------------

def envmap_directions(height, width):
    """Pixel-centre directions and exact pixel solid angles of an
    equirectangular map: row r spans polar angles [r, r+1] pi / H from +z,
    column c spans azimuths [c, c+1] 2 pi / W; the pixel's solid angle is
    (cos theta_r - cos theta_{r+1}) 2 pi / W.  Returns dirs [H, W, 3] and
    d_omega [H]."""
    H, W = int(height), int(width)
    theta = (np.arange(H) + 0.5) * math.pi / H
    phi = (np.arange(W) + 0.5) * 2.0 * math.pi / W
    edges = np.cos(np.arange(H + 1) * math.pi / H)
    d_omega = (edges[:-1] - edges[1:]) * 2.0 * math.pi / W
    st, ct = np.sin(theta)[:, None], np.cos(theta)[:, None]
    dirs = np.stack([st * np.cos(phi)[None, :], st * np.sin(phi)[None, :],
                     np.broadcast_to(ct, (H, W))], axis=-1)
    return dirs, d_omega


def project_envmap(n_bands, env):
    """L_c,i = int L_c(omega) y_i(omega) d omega (Eq. 9) for an
    equirectangular radiance map env [H, W, 3]: the sum over pixels of the
    pixel value times y_i at the pixel centre times the pixel's solid angle.
    Returns [3, K].  Processed a band of rows at a time."""
    env = np.asarray(env, np.float64)
    H, W = env.shape[:2]
    dirs, d_omega = envmap_directions(H, W)
    out = np.zeros((3, n_bands * n_bands))
    step = max(1, 65536 // max(W, 1))
    for r0 in range(0, H, step):
        Y = real_sh(n_bands, dirs[r0:r0 + step])                 # [h, W, K]
        w = env[r0:r0 + step] * d_omega[r0:r0 + step, None, None]  # [h, W, 3]
        out += np.einsum("hwc,hwk->ck", w, Y)
    return out


# ----------------------------------------------------------------------------
# Reverse-mode adjoint (Sec. 3.5: B is differentiable w.r.t. theta, L and a)
# ----------------------------------------------------------------------------

def _sh_exp_adjoint(C, ex, dV):
    """df from dV through the scaling, optimal linear step and squarings."""
    # V = e0 * S_k ;  S_{t+1} = S_t * S_t ;  S_0 = a (sqrt(4pi) e_0 + g)
    k_pt, e0, g, a, levels = ex["k"], ex["e0"], ex["g"], ex["a"], ex["levels"]
    Sk = levels[-1]
    de0 = np.sum(dV * Sk, axis=-1)
    dS = e0[:, None] * dV
    for t in reversed(range(len(levels) - 1)):
        act = (k_pt > t)[:, None]
        back = 2.0 * np.einsum("ijk,pi,pk->pj", C, dS, levels[t], optimize=True)
        dS = np.where(act, back, dS)
    # S_0 = a(s) sqrt(4 pi), S_i = b(s) g_i (i >= 1), s = |g|
    b, da_ds, db_ds, sn = ex["b"], ex["da_ds"], ex["db_ds"], ex["s"]
    dA = dS[:, 0] * SQRT_FOUR_PI
    dB = np.sum(dS[:, 1:] * g[:, 1:], axis=-1)
    coef = np.where(sn > 0, (dA * da_ds + dB * db_ds) / np.where(sn > 0, sn, 1.0), 0.0)
    dg = b[:, None] * dS + coef[:, None] * g
    dg[:, 0] = 0.0
    df = dg / (2.0 ** k_pt)[:, None]
    df[:, 0] = de0 * e0 / SQRT_FOUR_PI
    return df


def _sh_exp_projected_adjoint(ex, dV):
    """df from dV through V = e0 (E w) Y, E = exp(f^ Y^T), e0 = exp(f_0 y_0)."""
    e0, E, Y, w, U = ex["e0"], ex["E"], ex["Y"], ex["w"], ex["U"]
    de0 = np.sum(dV * U, axis=-1)
    dE = (e0[:, None] * dV) @ Y.T * w[None, :]        # [P, Q]
    df = (dE * E) @ Y
    df[:, 0] = de0 * e0 / SQRT_FOUR_PI
    return df


def shade_backward(cfg, points, normals, albedo, centers, radii, light, d_radiance, k=None):
    """Gradients of sum(d_radiance * B) w.r.t. every input, in float64.

    Returns dict with d_light [3,K], d_albedo [P,3], d_centers [N,3],
    d_radii [N], d_points [P,3], d_normals [P,3] and the forward dict.  For the
    outputs that are sums (lighting, centres and radii over points; point
    positions over spheres; normals over the K lobe coefficients) it also
    returns ``abs_<name>``: the same sum of the
    absolute terms, the scale that bounds rounding error in any evaluation
    order."""
    n = cfg.n_bands
    K = n * n
    C = gaunt_tensor(n)
    pts = np.asarray(points, np.float64)
    nrm = np.asarray(normals, np.float64)
    alb = np.asarray(albedo, np.float64)
    ctr = np.asarray(centers, np.float64).reshape(-1, 3)
    rad = np.asarray(radii, np.float64).reshape(-1)
    L = np.asarray(light, np.float64).reshape(3, K)
    dB = np.asarray(d_radiance, np.float64)
    fw = shade_forward(cfg, pts, nrm, alb, ctr, rad, L, k)
    V, H, W, ex = fw["V"], fw["H"], fw["W"], fw["_exp"]

    # B_c = a_c (L_c . W)
    LW = W @ L.T                                   # [P, 3]
    d_albedo = dB * LW
    d_light = (alb * dB).T @ W                     # [3, K]
    abs_d_light = np.abs(alb * dB).T @ np.abs(W)
    dW = (alb * dB) @ L                            # [P, K]

    # W = V * H
    dV = np.einsum("ijk,pi,pk->pj", C, dW, H, optimize=True)
    dH = np.einsum("ijk,pi,pj->pk", C, dW, V, optimize=True)

    # H = R_l zh_l y(n / |n|)
    nlen = np.linalg.norm(nrm, axis=-1, keepdims=True)
    nh = nrm / nlen
    coef = zh_rotation_scale(n) * clamped_cosine_zh(n)[band_of(K)]
    Yg = real_sh_grad(n, nh)                       # [P, K, 3]
    dnh = np.einsum("pk,pkc->pc", dH * coef, Yg)
    d_normals = (dnh - nh * np.sum(nh * dnh, axis=-1, keepdims=True)) / nlen
    # each component is a sum over the K coefficients of tangential terms
    Yt = Yg - nh[:, None, :] * np.sum(nh[:, None, :] * Yg, axis=-1, keepdims=True)
    abs_d_normals = np.einsum("pk,pkc->pc", np.abs(dH * coef), np.abs(Yt)) / nlen

    if cfg.exp_mode == 1:
        df = _sh_exp_projected_adjoint(ex, dV)
    else:
        df = _sh_exp_adjoint(C, ex, dV)

    # f = sum_j R_l zh_l(cos a_j) y(s_j),  s_j = d_j / D_j,  d_j = c_j - x
    lvec = band_of(K)
    R = zh_rotation_scale(n)
    d_points = np.zeros_like(pts)
    d_centers = np.zeros_like(ctr)
    d_radii = np.zeros_like(rad)
    abs_d_centers = np.zeros_like(ctr)
    abs_d_radii = np.zeros_like(rad)
    abs_d_points = np.zeros_like(pts)
    for j in range(ctr.shape[0]):
        d, D, valid, s, ca = cap_cosine(pts, ctr[j], rad[j])
        valid = valid & horizon_keep(cfg, d, rad[j], nrm)
        sh = d / D[:, None]
        Y = real_sh(n, sh)
        zh = log_cap_zh(n, cfg.epsilon, ca)
        dzh = np.zeros((pts.shape[0], n))
        for l in range(n):
            sel = lvec == l
            dzh[:, l] = np.sum(df[:, sel] * R[sel] * Y[:, sel], axis=-1)
        dY = df * R[None, :] * zh[:, lvec]
        dsh = np.einsum("pk,pkc->pc", dY, real_sh_grad(n, sh))
        # d zh_l / d cos(alpha) = +eps 2 pi N_l0 P_l(cos alpha)
        dca = np.zeros(pts.shape[0])
        for l in range(n):
            dca += dzh[:, l] * cfg.epsilon * 2.0 * math.pi * sh_normalisation(l, 0) \
                * _leg.legval(ca, np.eye(l + 1)[l])
        open_cap = s < 1.0
        ca_safe = np.where(open_cap, ca, 1.0)
        ds = np.where(open_cap, -dca * s / ca_safe, 0.0)   # cos a = sqrt(1 - s^2)
        dr = ds / D                                          # s = r / D
        dD = -ds * rad[j] / (D * D)
        dd = (dsh - sh * np.sum(sh * dsh, axis=-1, keepdims=True)) / D[:, None] + dD[:, None] * sh
        dd = np.where(valid[:, None], dd, 0.0)
        dr = np.where(valid, dr, 0.0)
        d_centers[j] = dd.sum(axis=0)
        d_radii[j] = dr.sum()
        abs_d_centers[j] = np.abs(dd).sum(axis=0)
        abs_d_radii[j] = np.abs(dr).sum()
        abs_d_points += np.abs(dd)
        d_points -= dd
    return dict(d_light=d_light, d_albedo=d_albedo, d_centers=d_centers, d_radii=d_radii,
                d_points=d_points, d_normals=d_normals, df=df, forward=fw,
                abs_d_light=abs_d_light, abs_d_centers=abs_d_centers, abs_d_radii=abs_d_radii,
                abs_d_points=abs_d_points, abs_d_normals=abs_d_normals)
