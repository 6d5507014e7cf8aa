"""Fitted coefficients a(s), b(s) of the optimal linear step of the SH
exponential (Sec. 3.3.2, which adopts Ren et al.'s scaling, squaring and
optimal linear setting; the paper prints no table of its own).

TEST INFRASTRUCTURE, like the rest of this package: it is run by hand (and by
tests on small ensembles) and writes tests/golden/ol_table_n<n>.txt, which
the tests feed to the oracle and to the library alike.

The step.  With g = f^ / 2^k the scaled exponent (zero DC) and s = |g| its
coefficient norm, the step is exp*(g) ~ a(s) sqrt(4 pi) e_0 + b(s) g, followed
by the k truncated squarings.  The fit chooses the node values of a and b
(linear between M nodes s_m = m s_max / (M - 1), constant past s_max) that
minimise, over an ensemble of log-visibility vectors f, the error of the
whole method against the projected exponential of the same function:

    J(a, b) = sum_f | S_k(a, b; f^) - P_n[exp(f^~)] |^2

(S_k: the step and k squarings; the DC factor e^{f_0 y_0} is common to both
sides and left out).  J is nonlinear in the nodes through the squarings; the
fit runs Levenberg-Marquardt from the Gaussian reading a = b = exp(s^2/8 pi),
with a small pull towards that reading so nodes no sample reaches keep it.
Fitting the step alone (least squares of the one-step error) was tried and
gives a worse method: the squarings of a truncated expansion do not commute
with the projection, so the best single step is not the best start.

The ensemble: log-visibility vectors f of points of three synthetic scene
families (random cube scenes, a height field under hovering spheres, a
capsule body above a ground plane), with the scaling count k of the method.
"""

import argparse
import os

import numpy as np

from . import shs_oracle as O


def ensemble(n_bands, n_points, seed=0):
    """[n_points, K] log-visibility vectors f of synthetic scene points."""
    from paper_2104_00359_gb300 import synthetic as S
    cfg = O.Config(n_bands=n_bands)
    rng = np.random.default_rng(seed)
    per = -(-n_points // 3)
    sources = [
        S.random_scene(seed + 11, 4 * per, 24, n_bands),
        S.height_field_scene(seed=seed + 12, res=64, n_spheres=60, n_bands=n_bands, n_bumps=6),
        S.capsule_body_scene(seed=seed + 13, res=64, n_bones=6, spheres_per_bone=4, n_bands=n_bands),
    ]
    out = []
    for sc in sources:
        P = sc["points"].shape[0]
        idx = rng.choice(P, size=min(P, per), replace=False)
        out.append(O.log_visibility(cfg, sc["points"][idx].astype(np.float64),
                                    sc["centers"].astype(np.float64), sc["radii"].astype(np.float64)))
    return np.concatenate(out)[:n_points]


def projected_exp_targets(n_bands, G, rule=None, chunk=2048):
    """T = P_n[exp(g~)] for each row g of G, by a fine quadrature."""
    dirs, w = rule if rule is not None else O.sphere_quadrature(8 * n_bands, 16 * n_bands)
    Y = O.real_sh(n_bands, dirs)
    T = np.empty_like(G)
    for i in range(0, G.shape[0], chunk):
        X = G[i:i + chunk] @ Y.T
        T[i:i + chunk] = (np.exp(X) * w) @ Y
    return T


def hat_basis(s, M, s_max):
    """[len(s), M] weights of the piecewise-linear interpolant at s (constant
    beyond s_max), the form the library evaluates."""
    h = s_max / (M - 1)
    x = np.clip(np.asarray(s, np.float64) / h, 0.0, M - 1.0)
    i = np.minimum(np.floor(x).astype(np.int64), M - 2)
    t = x - i
    B = np.zeros((x.shape[0], M))
    r = np.arange(x.shape[0])
    B[r, i] = 1.0 - t
    B[r, i + 1] += t
    return B


class Problem:
    """The fit's data: the scaled exponents g, their counts k and norms s, and
    the targets T, for an ensemble of f at n_bands."""

    def __init__(self, n_bands, f, rule=None):
        cfg = O.Config(n_bands=n_bands)
        self.C = O.gaunt_tensor(n_bands)
        self.k = O.exp_scaling_k(cfg, f)
        fh = f.copy()
        fh[:, 0] = 0.0
        self.g = fh / (2.0 ** self.k)[:, None]
        self.s = np.sqrt(np.sum(self.g * self.g, axis=1))
        self.T = projected_exp_targets(n_bands, fh, rule)
        self.w = 1.0 / np.sum(self.T * self.T, axis=1)      # relative error per point

    def run(self, A, B):
        """S_k for per-sample step coefficients A, B."""
        S = B[:, None] * self.g
        S[:, 0] = A * O.SQRT_FOUR_PI
        for t in range(int(self.k.max()) if S.shape[0] else 0):
            S = np.where((self.k > t)[:, None], O.sh_product(self.C, S, S), S)
        return S

    def objective(self, a, b, s_max):
        H = hat_basis(self.s, a.shape[0], s_max)
        R = self.run(H @ a, H @ b) - self.T
        return float(np.sum(self.w[:, None] * R * R))


def gaussian_table(M, s_max):
    s = np.linspace(0.0, s_max, M)
    a = np.exp(s * s / (2.0 * O.FOUR_PI))
    return a, a.copy()


def fit(prob, M, s_max, iters=12, pull=1e-3, smooth=1.0):
    """Levenberg-Marquardt node values (a [M], b [M]) from the Gaussian
    reading, minimising the relative error J plus `pull` times the squared
    distance to the Gaussian table and `smooth` times the squared second
    differences of a and b (both per point of the ensemble)."""
    a0, b0 = gaussian_table(M, s_max)
    a, b = a0.copy(), b0.copy()
    H = hat_basis(prob.s, M, s_max)
    N, K = prob.g.shape
    sw = np.sqrt(prob.w)[:, None]
    D2 = np.diff(np.eye(M), 2, axis=0)
    Reg = pull * np.eye(2 * M) + smooth * np.kron(np.eye(2), D2.T @ D2)
    lam = 1e-3

    def cost(a, b):
        R = (prob.run(H @ a, H @ b) - prob.T) * sw
        d = np.concatenate([a - a0, b - b0])
        return float(np.sum(R * R) + N * d @ Reg @ d), R

    J0, R = cost(a, b)
    for _ in range(iters):
        A, B = H @ a, H @ b
        d = 1e-6
        JA = (prob.run(A + d, B) - prob.run(A - d, B)) / (2 * d) * sw   # [N, K]
        JB = (prob.run(A, B + d) - prob.run(A, B - d)) / (2 * d) * sw
        Jm = np.concatenate([(JA[:, :, None] * H[:, None, :]).reshape(N * K, M),
                             (JB[:, :, None] * H[:, None, :]).reshape(N * K, M)], axis=1)
        gvec = Jm.T @ R.reshape(-1) + N * Reg @ np.concatenate([a - a0, b - b0])
        JtJ = Jm.T @ Jm + N * Reg
        while True:
            step = np.linalg.solve(JtJ + lam * np.diag(np.diag(JtJ)), -gvec)
            an, bn = a + step[:M], b + step[M:]
            J1, R1 = cost(an, bn)
            if J1 < J0:
                a, b, J0, R = an, bn, J1, R1
                lam = max(lam / 3.0, 1e-9)
                break
            lam *= 10.0
            if lam > 1e6:
                return a, b
    return a, b


def write_table(path, n_bands, a, b, s_max, n_dirs, seed):
    with open(path, "w") as fh:
        fh.write("# Optimal linear coefficients a(s), b(s) of the SH exponential's scaled step\n")
        fh.write("# (Sec. 3.3.2), fitted end to end against the projected exponential over\n")
        fh.write("# synthetic log-visibility ensembles.\n")
        fh.write(f"# Written by: python -m oracle.fit_ol_table --n-bands {n_bands} --nodes {a.shape[0]} "
                 f"--s-max {s_max} --dirs {n_dirs} --seed {seed}\n")
        fh.write(f"# n_bands {n_bands} s_max {s_max!r} nodes {a.shape[0]}\n")
        fh.write("# columns: s a b\n")
        h = s_max / (a.shape[0] - 1)
        for m in range(a.shape[0]):
            fh.write(f"{m * h:.17g} {a[m]:.17g} {b[m]:.17g}\n")


def read_table(path):
    """(a [M], b [M], s_max) from a file write_table made."""
    s_max = None
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("# n_bands"):
                s_max = float(line.split()[4])
            elif line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    rows = np.array(rows)
    return rows[:, 1].copy(), rows[:, 2].copy(), s_max


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-bands", type=int, default=4)
    ap.add_argument("--nodes", type=int, default=33)
    ap.add_argument("--s-max", type=float, default=1.0)
    ap.add_argument("--dirs", type=int, default=1500, help="ensemble size (points)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    prob = Problem(args.n_bands, ensemble(args.n_bands, args.dirs, args.seed))
    a, b = fit(prob, args.nodes, args.s_max)
    ga, gb = gaussian_table(args.nodes, args.s_max)
    print("J gaussian", prob.objective(ga, gb, args.s_max), "J fitted", prob.objective(a, b, args.s_max))
    out = args.out or os.path.join(os.path.dirname(__file__), "..", "tests", "golden",
                                   f"ol_table_n{args.n_bands}.txt")
    write_table(out, args.n_bands, a, b, args.s_max, args.dirs, args.seed)
    print(out, "a(s_max)", a[-1], "b(s_max)", b[-1])


if __name__ == "__main__":
    main()
