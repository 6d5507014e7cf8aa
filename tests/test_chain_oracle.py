"""Pins of the chain oracle (oracle/chain_oracle.py): Rodrigues' rotation
against scipy's matrix exponential and its defining properties, and the
adjoint against central differences."""

import numpy as np
import pytest

from oracle import chain_oracle as C


@pytest.mark.parametrize("scale", [0.0, 1e-5, 0.3, 2.0, 3.1])
def test_rodrigues_is_the_exponential_of_the_skew_matrix(scale):
    from scipy.linalg import expm
    rng = np.random.default_rng(int(scale * 10))
    w = rng.normal(size=3)
    w = w / np.linalg.norm(w) * scale
    R = C.rodrigues(w)
    np.testing.assert_allclose(R, expm(C.skew(w)), atol=1e-13)
    np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-13)
    np.testing.assert_allclose(R @ w, w, atol=1e-13)          # the axis is fixed
    assert abs(np.linalg.det(R) - 1.0) < 1e-13


@pytest.mark.parametrize("scale", [0.0, 1e-4, 0.7, 2.9])
def test_rodrigues_grad_central_differences(scale):
    from scipy.linalg import expm
    rng = np.random.default_rng(5)
    w = rng.normal(size=3)
    w = w / np.linalg.norm(w) * scale
    G = C.rodrigues_grad(w)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (expm(C.skew(w + e)) - expm(C.skew(w - e))) / (2 * h)
        np.testing.assert_allclose(G[a], fd, atol=1e-8)


@pytest.mark.parametrize("direction", [False, True])
def test_chain_adjoint_central_differences(direction):
    rng = np.random.default_rng(7)
    M, D = 9, 5
    base, basis = rng.normal(size=(M, 3)), rng.normal(size=(M, 3, D))
    p, pose, g = rng.normal(size=D), np.concatenate([rng.normal(size=3), rng.normal(size=3)]), rng.normal(size=(M, 3))
    out = C.deform_pose_backward(base, basis, p, pose, g, direction)
    h = 1e-6

    def L(pp, qq):
        return np.sum(g * C.deform_pose(base, basis, pp, qq, direction)[0])

    for i in range(D):
        e = np.zeros(D)
        e[i] = h
        assert abs((L(p + e, pose) - L(p - e, pose)) / (2 * h) - out["d_p"][i]) < 1e-7
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        assert abs((L(p, pose + e) - L(p, pose - e)) / (2 * h) - out["d_pose"][i]) < 1e-7
    if direction:
        assert np.all(out["d_pose"][3:] == 0)


def test_identity_pose_and_zero_parameters():
    rng = np.random.default_rng(8)
    base, basis = rng.normal(size=(4, 3)), rng.normal(size=(4, 3, 3))
    x, xr = C.deform_pose(base, basis, np.zeros(3), np.zeros(6))
    np.testing.assert_array_equal(x, base)
    np.testing.assert_array_equal(xr, base)
