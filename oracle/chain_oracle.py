"""FP64 oracle of the scene chain above the shading path (Sec. 3.3.1, Sec.
3.5): a linear deformation model and a rigid 6-DoF pose per view.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
legs use this module; the library never does.

The chain, per array of M rows (vertices, normals or sphere centres):

    x_rest[m] = base[m] + basis[m] p            (basis[m]: 3 x D, p: D)
    x[m]      = R(w) x_rest[m] + t              (t dropped for directions)

with R(w) = exp([w]x) the rotation of the axis-angle vector w (Rodrigues'
formula).  The adjoint, for an upstream gradient g[m] = dL/dx[m]:

    dL/dp  = sum_m basis[m]^T R^T g[m]
    dL/dt  = sum_m g[m]                         (points and centres only)
    dL/dR  = sum_m g[m] x_rest[m]^T,   dL/dw_a = <dL/dR, dR/dw_a>

dR/dw_a is written out from R = I + A(th) K + B(th) K^2 (K = [w]x,
A = sin th / th, B = (1 - cos th) / th^2):
dR/dw_a = A K_a + B (K_a K + K K_a) + (A'/th) w_a K + (B'/th) w_a K^2,
K_a = [e_a]x.
"""

import numpy as np


def skew(w):
    """[w]x, the matrix of the cross product with w."""
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def _coeffs(th):
    """A, B and A'/th, B'/th at angle th (series below 1e-3 rad)."""
    if th < 1e-3:
        t2 = th * th
        A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0
        B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0
        dA = -1.0 / 3.0 + t2 / 30.0
        dB = -1.0 / 12.0 + t2 / 180.0
        return A, B, dA, dB
    s, c = np.sin(th), np.cos(th)
    A = s / th
    B = (1.0 - c) / (th * th)
    dA = (th * c - s) / th ** 3
    dB = (th * s - 2.0 * (1.0 - c)) / th ** 4
    return A, B, dA, dB


def rodrigues(w):
    """R(w) = exp([w]x)."""
    w = np.asarray(w, np.float64)
    K = skew(w)
    A, B, _, _ = _coeffs(float(np.linalg.norm(w)))
    return np.eye(3) + A * K + B * (K @ K)


def rodrigues_grad(w):
    """[3, 3, 3]: dR/dw_a for a = 0, 1, 2."""
    w = np.asarray(w, np.float64)
    K = skew(w)
    K2 = K @ K
    A, B, dA, dB = _coeffs(float(np.linalg.norm(w)))
    out = np.zeros((3, 3, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        Ka = skew(e)
        out[a] = A * Ka + B * (Ka @ K + K @ Ka) + dA * w[a] * K + dB * w[a] * K2
    return out


def deform_pose(base, basis, p, pose, direction=False):
    """x [M, 3] and x_rest [M, 3] for base [M, 3], basis [M, 3, D], p [D],
    pose (w, t) [6]."""
    base = np.asarray(base, np.float64)
    basis = np.asarray(basis, np.float64)
    p = np.asarray(p, np.float64)
    pose = np.asarray(pose, np.float64)
    x_rest = base + basis @ p
    R = rodrigues(pose[:3])
    x = x_rest @ R.T
    if not direction:
        x = x + pose[3:]
    return x, x_rest


def deform_pose_backward(base, basis, p, pose, g, direction=False):
    """dL/dp [D] and dL/dpose [6] for an upstream gradient g [M, 3], with the
    sums of absolute terms (the scale of float32 summation error)."""
    basis = np.asarray(basis, np.float64)
    g = np.asarray(g, np.float64)
    pose = np.asarray(pose, np.float64)
    _, x_rest = deform_pose(base, basis, p, pose, direction)
    R = rodrigues(pose[:3])
    gr = g @ R                                   # rows R^T g[m]
    terms = basis * gr[:, :, None]               # [M, 3, D]
    dp = terms.sum(axis=(0, 1))
    abs_dp = np.abs(terms).sum(axis=(0, 1))
    dR = g.T @ x_rest
    abs_dR = np.abs(g).T @ np.abs(x_rest)
    G = rodrigues_grad(pose[:3])
    dw = np.array([np.sum(dR * G[a]) for a in range(3)])
    abs_dw = np.array([np.sum(abs_dR * np.abs(G[a])) for a in range(3)])
    if direction:
        dt, abs_dt = np.zeros(3), np.zeros(3)
    else:
        dt, abs_dt = g.sum(axis=0), np.abs(g).sum(axis=0)
    return dict(d_p=dp, abs_d_p=abs_dp, d_pose=np.concatenate([dw, dt]),
                abs_d_pose=np.concatenate([abs_dw, abs_dt]))
