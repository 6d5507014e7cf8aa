"""Algebraic identities the kernels rely on, checked in numpy (no GPU).

1. The env-map kernel's four-fold azimuthal grouping (Eq. 9 moments): the
   columns at phi, pi - phi, pi + phi and -phi share cos(m phi), sin(m phi),
   with even-m terms taking v1 + v3 + (v2 + v4) and odd-m terms
   v1 + v3 - (v2 + v4) (sine terms: v1 - v3 +- (v2 - v4)).
2. Its three-term recurrence for cos(m phi), sin(m phi), m < 8, in float32.
3. The chain reduction's closed form of dL/dw from dL/dR for
   R(w) = I + A K + B K^2 (K = [w]x): with K_a = [e_a]x,
   sum (A K_a + B (K_a K + K K_a) + A' w_a K + B' w_a K^2) o X
   = A (X[a2][a1] - X[a1][a2]) + B ((X^T w)_a + (X w)_a - 2 w_a tr X)
     + A' w_a (w . vee(X - X^T)) + B' w_a (w^T X w - |w|^2 tr X)."""

import numpy as np
import pytest


def _moments_direct(row, nb):
    W = row.shape[0]
    phi = 2.0 * np.pi * (np.arange(W) + 0.5) / W
    out = np.zeros((nb, 3, 2))
    for m in range(nb):
        out[m, :, 0] = (row * np.cos(m * phi)[:, None]).sum(0)
        out[m, :, 1] = (row * np.sin(m * phi)[:, None]).sum(0)
    return out


def _moments_grouped(row, nb):
    """The kernel's order: 4-column group g of the first quarter and its
    mirror groups; pixel j of a group pairs with pixel 3 - j of the mirrors
    at pi - phi and -phi."""
    W = row.shape[0]
    phi = 2.0 * np.pi * (np.arange(W) + 0.5) / W
    out = np.zeros((nb, 3, 2))
    q4, w8, w4 = W >> 4, W >> 3, W >> 2
    for g in range(q4):
        A, B, C, D = (row[4 * x:4 * x + 4] for x in (g, w8 - 1 - g, w8 + g, w4 - 1 - g))
        for j in range(4):
            v1, v2, v3, v4 = A[j], C[j], D[3 - j], B[3 - j]
            ep, em = (v1 + v3) + (v2 + v4), (v1 + v3) - (v2 + v4)
            sp, sm = (v1 - v3) + (v2 - v4), (v1 - v3) - (v2 - v4)
            out[0, :, 0] += ep
            c1, s1 = np.cos(phi[4 * g + j]), np.sin(phi[4 * g + j])
            cp, spv, cm, smv = 1.0, 0.0, c1, s1
            for m in range(1, nb):
                out[m, :, 0] += (em if m & 1 else ep) * cm
                out[m, :, 1] += (sm if m & 1 else sp) * smv
                cp, spv, cm, smv = cm, smv, 2 * c1 * cm - cp, 2 * c1 * smv - spv
    return out


@pytest.mark.parametrize("W", [16, 48, 96, 2048])
def test_envmap_fourfold_grouping(W):
    row = np.random.default_rng(W).normal(size=(W, 3))
    ref = _moments_direct(row, 8)
    got = _moments_grouped(row, 8)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(row).sum()


def test_harmonic_recurrence_float32():
    """cos(m phi), sin(m phi) by x_{m+1} = 2 cos(phi) x_m - x_{m-1} from a
    float32 (cos phi, sin phi): within 64 float32 ulps of 1 for m < 8 at
    every column centre of an 8192-wide map."""
    W = 8192
    phi = 2.0 * np.pi * (np.arange(W // 4) + 0.5) / W
    c1, s1 = np.cos(phi).astype(np.float32), np.sin(phi).astype(np.float32)
    two = (c1 + c1).astype(np.float32)
    cp, sp = np.ones_like(c1), np.zeros_like(s1)
    cm, sm = c1, s1
    worst = 0.0
    for m in range(1, 8):
        worst = max(worst, np.abs(cm - np.cos(m * phi)).max(), np.abs(sm - np.sin(m * phi)).max())
        cn = (two * cm - cp).astype(np.float32)
        sn = (two * sm - sp).astype(np.float32)
        cp, sp, cm, sm = cm, sm, cn, sn
    assert worst <= 64 * np.finfo(np.float32).eps


def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def test_pose_gradient_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(20):
        w = rng.normal(size=3)
        X = rng.normal(size=(3, 3))
        A, B, dA, dB = rng.normal(size=4)
        K = _skew(w)
        t2 = w @ w
        K2 = np.outer(w, w) - t2 * np.eye(3)
        for a in range(3):
            Ka = _skew(np.eye(3)[a])
            G = A * Ka + B * (Ka @ K + K @ Ka) + dA * w[a] * K + dB * w[a] * K2
            ref = (G * X).sum()
            a1, a2 = (a + 1) % 3, (a + 2) % 3
            tr = np.trace(X)
            kx = w[0] * (X[2, 1] - X[1, 2]) + w[1] * (X[0, 2] - X[2, 0]) + w[2] * (X[1, 0] - X[0, 1])
            got = (A * (X[a2, a1] - X[a1, a2]) + B * (X[:, a] @ w + X[a] @ w - 2 * w[a] * tr)
                   + dA * w[a] * kx + dB * w[a] * (w @ X @ w - t2 * tr))
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))
