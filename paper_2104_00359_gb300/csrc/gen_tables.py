#!/usr/bin/env python3
"""Generate the unrolled spherical-harmonics device code used by the CUDA
kernels (``generated/shs_sh_gen.cuh``).

For each supported band count n (K = n^2 coefficients) it emits:

* ``ybar(x, y, z, Y)``: the un-normalised real SH polynomials
  Ybar_lm = Pbar_l^|m|(z) * {C_m, S_m}(x, y) where C_m + i S_m = (x + i y)^m and
  Pbar_l^m = d^m P_l / dz^m (no Condon-Shortley phase).  The normalised basis
  (Sec. 3.2, Eq. 3) is y_i = NORM[i] * Ybar_i.
* ``ybar_vjp(x, y, z, w, gx, gy, gz)``: the gradient of sum_i w_i Ybar_i with
  respect to (x, y, z), emitted by reverse-mode differentiation of the
  straight-line code above.
* ``mul(a, b, o)``: the truncated SH triple product o = a * b,
  o_i = sum_jk C_ijk a_j b_k (Eq. 7), unrolled over the nonzero C_ijk.
* ``sqr(a, o)``: o = a * a using the j <-> k symmetry of C.
* the monomial-basis pair terms (``accumulate``, ``mono_to_f``) and the
  per-band gradient polynomials of the pair adjoint (``grad_coeffs``,
  ``grad_eval``), from the homogeneous form of Ybar (equal on the unit sphere).
* tables: NORM[i], AHAT[l] (clamped-cosine convolution constants, Eq. 10-11).

C_ijk is computed here by exact integration of monomials over the sphere,
  int x^a y^b z^c dw = 4 pi (a-1)!! (b-1)!! (c-1)!! / (a+b+c+1)!!  (a, b, c even),
applied to the products of the SH polynomials -- a different route from any
quadrature.  Run ``python gen_tables.py`` to rewrite the header; the build
checks that the committed header is current.
"""

from __future__ import annotations

import math
import re
import os
import sys
from fractions import Fraction

import numpy as np

BANDS = (1, 2, 3, 4, 5, 6, 7, 8)
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "generated", "shs_sh_gen.cuh")


# ---------------------------------------------------------------------------
# exact polynomials: dict {(a, b, c): Fraction} for x^a y^b z^c
# ---------------------------------------------------------------------------

def p_add(p, q, s=1):
    r = dict(p)
    for k, v in q.items():
        r[k] = r.get(k, 0) + s * v
        if r[k] == 0:
            del r[k]
    return r


def p_mul(p, q):
    r = {}
    for (a1, b1, c1), v1 in p.items():
        for (a2, b2, c2), v2 in q.items():
            k = (a1 + a2, b1 + b2, c1 + c2)
            r[k] = r.get(k, 0) + v1 * v2
    return {k: v for k, v in r.items() if v != 0}


def p_scale(p, s):
    return {k: v * s for k, v in p.items() if v * s != 0}


X = {(1, 0, 0): Fraction(1)}
Y = {(0, 1, 0): Fraction(1)}
Z = {(0, 0, 1): Fraction(1)}
ONE = {(0, 0, 0): Fraction(1)}


def ybar_polys(n):
    """Exact Ybar_i polynomials (index i = l^2 + l + m) by the same recurrences
    the emitted code uses."""
    Cm, Sm = [ONE], [{}]
    for m in range(1, n):
        Cm.append(p_add(p_mul(X, Cm[-1]), p_mul(Y, Sm[-1]), -1))
        Sm.append(p_add(p_mul(X, Sm[-1]), p_mul(Y, Cm[-2])))
    Pb = {}
    for m in range(n):
        Pb[(m, m)] = {(0, 0, 0): Fraction(math.prod(range(1, 2 * m, 2)))}
        if m + 1 < n:
            Pb[(m + 1, m)] = p_scale(p_mul(Z, Pb[(m, m)]), 2 * m + 1)
        for l in range(m + 2, n):
            t = p_add(p_scale(p_mul(Z, Pb[(l - 1, m)]), 2 * l - 1),
                      p_scale(Pb[(l - 2, m)], l + m - 1), -1)
            Pb[(l, m)] = p_scale(t, Fraction(1, l - m))
    out = [None] * (n * n)
    for l in range(n):
        out[l * l + l] = Pb[(l, 0)]
        for m in range(1, l + 1):
            out[l * l + l + m] = p_mul(Pb[(l, m)], Cm[m])
            out[l * l + l - m] = p_mul(Pb[(l, m)], Sm[m])
    return out


def monomials(deg):
    """Exponent triples (a, b, c) with a + b + c = deg, in emission order."""
    return [(a, b, deg - a - b) for a in range(deg, -1, -1) for b in range(deg - a, -1, -1)]


def homogeneous_polys(n):
    """Ybar_i made homogeneous of degree l_i by multiplying each lower-degree
    term by (x^2 + y^2 + z^2)^j (equal on the unit sphere).  Returns a list of
    dicts {(a, b, c): Fraction}."""
    R2 = p_add(p_add(p_mul(X, X), p_mul(Y, Y)), p_mul(Z, Z))
    out = []
    for i, p in enumerate(ybar_polys(n)):
        l = int(math.isqrt(i))
        h = {}
        for (a, b, c), v in p.items():
            t = {(a, b, c): v}
            for _ in range((l - a - b - c) // 2):
                t = p_mul(t, R2)
            h = p_add(h, t)
        assert all(sum(k) == l for k in h)
        out.append(h)
    return out


def dfact(k):
    return math.prod(range(k, 0, -2)) if k > 0 else 1


def sphere_moment(a, b, c):
    """int_{S^2} x^a y^b z^c dw / (4 pi), exact."""
    if a % 2 or b % 2 or c % 2:
        return Fraction(0)
    return Fraction(dfact(a - 1) * dfact(b - 1) * dfact(c - 1), dfact(a + b + c + 1))


def norms(n):
    """NORM[i] with y_i = NORM[i] * Ybar_i."""
    out = []
    for l in range(n):
        for m in range(-l, l + 1):
            am = abs(m)
            N = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            out.append(N * (math.sqrt(2.0) if am else 1.0))
    return out


def gaunt_monomial(n):
    """C_ijk = NORM_i NORM_j NORM_k int Ybar_i Ybar_j Ybar_k dw, with the
    integral taken monomial by monomial from the closed form above.

    Dense float64 arrays over exponent triples: Q_jk = Ybar_j Ybar_k (exponents
    < 2n-1), R_i[b] = sum_a Ybar_i[a] M[a + b] (M the sphere moments), and
    C_ijk = <R_i, Q_jk>.  Returns {(i, j, k): value} for j <= k, value != 0."""
    K = n * n
    P = ybar_polys(n)
    N = norms(n)
    e2, e3 = 2 * n - 1, 3 * n - 2
    M = np.zeros((e3, e3, e3))
    for a in range(0, e3, 2):
        for b in range(0, e3, 2):
            for c in range(0, e3, 2):
                M[a, b, c] = 4.0 * math.pi * float(sphere_moment(a, b, c))
    dense = np.zeros((K, n, n, n))
    for i, p in enumerate(P):
        for (a, b, c), v in p.items():
            dense[i, a, b, c] = float(v)
    R = np.zeros((K, e2, e2, e2))
    for i, p in enumerate(P):
        for (a, b, c), v in p.items():
            R[i] += float(v) * M[a:a + e2, b:b + e2, c:c + e2]
    pairs = [(j, k) for j in range(K) for k in range(j, K)]
    Q = np.zeros((len(pairs), e2, e2, e2))
    for q, (j, k) in enumerate(pairs):
        for (a, b, c), v in P[j].items():
            Q[q, a:a + n, b:b + n, c:c + n] += float(v) * dense[k]
    G = R.reshape(K, -1) @ Q.reshape(len(pairs), -1).T
    lb = [int(math.isqrt(i)) for i in range(K)]
    out = {}
    for i in range(K):
        for q, (j, k) in enumerate(pairs):
            li, lj, lk = lb[i], lb[j], lb[k]
            if (li + lj + lk) % 2 or li > lj + lk or lj > li + lk or lk > li + lj:
                continue
            v = N[i] * N[j] * N[k] * G[i, q]
            if abs(v) > 1e-12:
                out[(i, j, k)] = v
    return out


def ahat(n):
    """A_hat_l = 2 pi int_0^1 t P_l(t) dt, exact from P_l's coefficients."""
    out = []
    for l in range(n):
        # P_l power coefficients via Bonnet recurrence in Fractions
        p0, p1 = [Fraction(1)], [Fraction(0), Fraction(1)]
        if l == 0:
            c = p0
        elif l == 1:
            c = p1
        else:
            for ll in range(1, l):
                nxt = [Fraction(0)] * (ll + 2)
                for i, v in enumerate(p1):
                    nxt[i + 1] += Fraction(2 * ll + 1, ll + 1) * v
                for i, v in enumerate(p0):
                    nxt[i] -= Fraction(ll, ll + 1) * v
                p0, p1 = p1, nxt
            c = p1
        integ = sum(v / (i + 2) for i, v in enumerate(c))
        out.append(2.0 * math.pi * float(integ))
    return out


# ---------------------------------------------------------------------------
# straight-line code builder with constant folding and reverse mode
# ---------------------------------------------------------------------------

class Code:
    def __init__(self, prefix):
        self.ops = []          # (name, kind, args)
        self.prefix = prefix
        self.count = 0

    def _new(self, kind, args):
        name = f"{self.prefix}{self.count}"
        self.count += 1
        self.ops.append((name, kind, args))
        return ("v", name)

    @staticmethod
    def const(v):
        return ("c", float(v))

    def mul(self, a, b):
        if a[0] == "c" and b[0] == "c":
            return self.const(a[1] * b[1])
        if a[0] == "c":
            a, b = b, a
        if b[0] == "c":
            if b[1] == 0.0:
                return self.const(0.0)
            if b[1] == 1.0:
                return a
        return self._new("mul", (a, b))

    def add(self, a, b, sb=1.0):
        if b[0] == "c" and b[1] == 0.0:
            return a
        if a[0] == "c" and a[1] == 0.0:
            return b if sb == 1.0 else self.mul(b, self.const(sb))
        if a[0] == "c" and b[0] == "c":
            return self.const(a[1] + sb * b[1])
        return self._new("add", (a, b, sb))


def fmt(v):
    if v[0] == "c":
        r = repr(float(np.float32(v[1])))
        if "e" not in r and "." not in r and "inf" not in r and "nan" not in r:
            r += ".0"
        return r + "f"
    return v[1]


def build_ybar(n):
    code = Code("t")
    x, y, z = ("v", "x"), ("v", "y"), ("v", "z")
    C = [code.const(1.0)]
    S = [code.const(0.0)]
    for m in range(1, n):
        C.append(code.add(code.mul(x, C[-1]), code.mul(y, S[-1]), -1.0))
        S.append(code.add(code.mul(x, S[-1]), code.mul(y, C[-2])))
    Pb = {}
    for m in range(n):
        Pb[(m, m)] = code.const(math.prod(range(1, 2 * m, 2)))
        if m + 1 < n:
            Pb[(m + 1, m)] = code.mul(code.mul(z, Pb[(m, m)]), code.const(2 * m + 1))
        for l in range(m + 2, n):
            a = code.mul(code.mul(z, Pb[(l - 1, m)]), code.const((2 * l - 1) / (l - m)))
            b = code.mul(Pb[(l - 2, m)], code.const((l + m - 1) / (l - m)))
            Pb[(l, m)] = code.add(a, b, -1.0)
    outs = [None] * (n * n)
    for l in range(n):
        outs[l * l + l] = Pb[(l, 0)]
        for m in range(1, l + 1):
            outs[l * l + l + m] = code.mul(Pb[(l, m)], C[m])
            outs[l * l + l - m] = code.mul(Pb[(l, m)], S[m])
    return code, outs


def emit_forward(code, outs, target):
    lines = []
    for name, kind, args in code.ops:
        if kind == "mul":
            lines.append(f"const float {name} = {fmt(args[0])} * {fmt(args[1])};")
        else:
            a, b, sb = args
            op = "+" if sb > 0 else "-"
            if abs(sb) == 1.0:
                lines.append(f"const float {name} = {fmt(a)} {op} {fmt(b)};")
            else:
                lines.append(f"const float {name} = fmaf({fmt(code.const(sb))}, {fmt(b)}, {fmt(a)});")
    for i, o in enumerate(outs):
        lines.append(f"{target}[{i}] = {fmt(o)};")
    return lines


def emit_vjp(code, outs):
    """Reverse sweep: adjoints of x, y, z for the scalar sum_i w[i] * out_i."""
    adj = {}      # var name -> list of terms (strings)

    def acc(var, term):
        if var[0] == "c":
            return
        adj.setdefault(var[1], []).append(term)

    for i, o in enumerate(outs):
        acc(o, f"w[{i}]")
    lines = []
    for name, kind, args in reversed(code.ops):
        terms = adj.get(name)
        if not terms:
            continue
        g = f"a_{name}"
        lines.append(f"const float {g} = {' + '.join(terms)};")
        if kind == "mul":
            a, b = args
            if b[0] == "c":
                acc(a, f"{fmt(b)} * {g}")
            elif a[0] == "c":
                acc(b, f"{fmt(a)} * {g}")
            else:
                acc(a, f"{fmt(b)} * {g}")
                acc(b, f"{fmt(a)} * {g}")
        else:
            a, b, sb = args
            acc(a, g)
            if sb == 1.0:
                acc(b, g)
            elif sb == -1.0:
                acc(b, f"-{g}")
            else:
                acc(b, f"{fmt(code.const(sb))} * {g}")
    for v, nm in (("x", "gx"), ("y", "gy"), ("z", "gz")):
        terms = adj.get(v)
        lines.append(f"{nm} = {' + '.join(terms) if terms else '0.0f'};")
    return lines


def emit_gaunt(n, C):
    K = n * n
    mul_lines, sqr_lines = [], []
    by_i = {i: [] for i in range(K)}
    for (i, j, k), v in sorted(C.items()):
        by_i[i].append((j, k, v))
    for i in range(K):
        terms_m, terms_s = [], []
        for j, k, v in by_i[i]:
            c = fmt(("c", v))
            if j == k:
                terms_m.append((c, f"a[{j}] * b[{j}]"))
                terms_s.append((c, f"a[{j}] * a[{j}]"))
            else:
                terms_m.append((c, f"(a[{j}] * b[{k}] + a[{k}] * b[{j}])"))
                terms_s.append((fmt(("c", 2 * v)), f"a[{j}] * a[{k}]"))
        for lines, terms in ((mul_lines, terms_m), (sqr_lines, terms_s)):
            if not terms:
                lines.append(f"o[{i}] = 0.0f;")
                continue
            lines.append(f"o[{i}] = {balanced_sum(terms)};")
    return mul_lines, sqr_lines


def balanced_sum(terms, chains=4):
    """sum of c * t over (c, t) as up to ``chains`` interleaved FMA chains added
    pairwise: rounding error grows with len/chains instead of len, and the
    chains are independent instructions."""
    groups = [terms[g::chains] for g in range(min(chains, len(terms)))]
    exprs = []
    for grp in groups:
        e = f"{grp[0][0]} * {grp[0][1]}"
        for c, t in grp[1:]:
            e = f"fmaf({c}, {t}, {e})"
        exprs.append(e)
    while len(exprs) > 1:
        nxt = [f"({exprs[k]} + {exprs[k + 1]})" for k in range(0, len(exprs) - 1, 2)]
        if len(exprs) % 2:
            nxt.append(exprs[-1])
        exprs = nxt
    return exprs[0]


def _mono_lines(maxdeg, prefix="m"):
    """Straight-line products for every monomial of degree 1..maxdeg in x, y, z."""
    name = {(0, 0, 0): "1.0f"}
    lines = []
    for deg in range(1, maxdeg + 1):
        for (a, b, c) in monomials(deg):
            if a > 0:
                src, f = (a - 1, b, c), "x"
            elif b > 0:
                src, f = (a, b - 1, c), "y"
            else:
                src, f = (a, b, c - 1), "z"
            nm = f"{prefix}{a}_{b}_{c}"
            lines.append(f"const float {nm} = {f}" + ("" if src == (0, 0, 0) else f" * {name[src]}") + ";")
            name[(a, b, c)] = nm
    return lines, name


def emit_monomial_route(n):
    """Code for the monomial-basis pair terms (used for n <= 5).

    accumulate(G, x, y, z, acc): acc[off_l + a] += G[l] * x^a1 y^a2 z^a3 for
      every monomial of degree l < n (forward pair term in monomial form).
    mono_to_f(acc, f): f_i = sum_a Hbar_i[a] acc[off_l + a], Hbar_i the
      homogeneous Ybar_i, i.e. the un-normalised log-visibility coefficients.
    grad_coeffs(w, gq): for bands l >= 1, the coefficients over monomials of
      degree l-1 of the three partial derivatives of Phi_l = sum_m w_lm Hbar_lm.
    grad_eval(x, y, z, gq, gx, gy, gz): (gx, gy, gz)[l-1] = grad Phi_l(x, y, z).
    """
    H = homogeneous_polys(n)
    offs, na = [], 0
    for l in range(n):
        offs.append(na)
        na += len(monomials(l))
    # Monomials are built up to degree n-2; the top band's terms are
    # G_{n-1} x^a y^b z^c = (G_{n-1} v) m' with v the first variable of the
    # monomial and m' of degree n-2, so its monomials are never formed.
    top = n - 1
    ml, name = _mono_lines(max(top - 1, 1) if top >= 1 else 0)
    if top >= 2:
        ml += [f"const float gt{v} = G[{top}] * {v};" for v in "xyz"]
    acc = []
    for l in range(n):
        for ai, mono in enumerate(monomials(l)):
            o = offs[l] + ai
            if l == top and l >= 2:
                v = next(i for i in range(3) if mono[i] > 0)
                low = list(mono)
                low[v] -= 1
                acc.append(f"acc[{o}] = fmaf(gt{'xyz'[v]}, {name[tuple(low)]}, acc[{o}]);")
            else:
                m = "1.0f" if mono == (0, 0, 0) else name[mono]
                acc.append(f"acc[{o}] = fmaf(G[{l}], {m}, acc[{o}]);")
    m2f = []
    for i in range(n * n):
        l = int(math.isqrt(i))
        terms = [(fmt(("c", float(v))), f"acc[{offs[l] + monomials(l).index(mono)}]")
                 for mono, v in sorted(H[i].items()) if v != 0]
        m2f.append(f"f[{i}] = {balanced_sum(terms)};")
    goffs, ng = [], 0
    for l in range(1, n):
        goffs.append(ng)
        ng += 3 * len(monomials(l - 1))
    gc = []
    for l in range(1, n):
        lower = monomials(l - 1)
        for comp in range(3):
            for bi, beta in enumerate(lower):
                up = list(beta)
                up[comp] += 1
                up = tuple(up)
                factor = up[comp]
                terms = []
                for m in range(-l, l + 1):
                    i = l * l + l + m
                    v = H[i].get(up, 0)
                    if v != 0:
                        terms.append((fmt(("c", float(v) * factor)), f"w[{i}]"))
                o = goffs[l - 1] + comp * len(lower) + bi
                gc.append(f"gq[{o}] = {balanced_sum(terms) if terms else '0.0f'};")
    ge_m, gname = _mono_lines(max(n - 2, 0), prefix="u")
    ge = list(ge_m)
    for l in range(1, n):
        lower = monomials(l - 1)
        for comp, g in ((0, "gx"), (1, "gy"), (2, "gz")):
            terms = []
            for bi, beta in enumerate(lower):
                o = goffs[l - 1] + comp * len(lower) + bi
                terms.append(f"gq[{o}]" + ("" if beta == (0, 0, 0) else f" * {gname[beta]}"))
            ge.append(f"{g}[{l - 1}] = {' + '.join(terms)};")
    return na, ng, ml, acc, m2f, gc, ge


def packed_lines(lines):
    """The float2 form of straight-line scalar code made of 'const float a =
    b;', 'const float a = b * c;' and 'acc[i] = fmaf(b, c, acc[i]);' lines,
    with the packed sm_100 float32x2 intrinsics."""
    out = []
    for ln in lines:
        m = re.fullmatch(r"const float (\w+) = (\S+) \* (\S+);", ln)
        if m:
            out.append(f"const float2 {m[1]} = __fmul2_rn({m[2]}, {m[3]});")
            continue
        m = re.fullmatch(r"const float (\w+) = (\w+);", ln)
        if m:
            out.append(f"const float2 {m[1]} = {m[2]};")
            continue
        m = re.fullmatch(r"(acc\[\d+\]) = fmaf\((\S+), (\S+), (acc\[\d+\])\);", ln)
        if m and m[1] == m[4]:
            if m[3] == "1.0f":
                out.append(f"{m[1]} = __fadd2_rn({m[2]}, {m[1]});")
            else:
                out.append(f"{m[1]} = __ffma2_rn({m[2]}, {m[3]}, {m[1]});")
            continue
        raise ValueError(f"cannot pack: {ln}")
    return out


QUAD_FROM = 7   # band counts from which the triple product runs by quadrature


def quadrature_tables(n):
    """Separable quadrature for the truncated triple product at n bands.

    y_i(theta, phi) = Leg_i(theta) T_f(i)(phi) with T_0 = 1, T_{2m-1} =
    cos(m phi), T_{2m} = sin(m phi).  The product of three SH of degree < n is
    a polynomial of degree <= 3(n-1) on the sphere, so NZ = 3(n-1)/2 + 1
    Gauss-Legendre nodes in z = cos(theta) and NP = 3(n-1) + 1 uniform azimuths
    integrate it exactly:  (a * b)_i = sum_{za, pb} w_za A B y_i.
    Returns (leg [NZ][K], trig [NP][2n-1], w [NZ]) in float64 and checks the
    factorisation and the exactness against the Gaunt tensor."""
    K = n * n
    D = 3 * (n - 1)
    NZ, NP = D // 2 + 1, D + 1
    z, wz = np.polynomial.legendre.leggauss(NZ)
    H = homogeneous_polys(n)
    N = norms(n)

    def ysh(i, x, y, zz):
        return N[i] * sum(float(v) * x ** a * y ** b * zz ** c for (a, b, c), v in H[i].items())

    def f_of(m):
        return 0 if m == 0 else (2 * m - 1 if m > 0 else 2 * (-m))

    leg = np.zeros((NZ, K))
    for za in range(NZ):
        st = math.sqrt(1.0 - z[za] ** 2)
        for i in range(K):
            l = int(math.isqrt(i))
            m = i - l * l - l
            ph = 0.0 if m >= 0 else math.pi / (2 * (-m))
            leg[za, i] = ysh(i, st * math.cos(ph), st * math.sin(ph), z[za])
    phis = 2.0 * math.pi * (np.arange(NP) + 0.5) / NP
    trig = np.zeros((NP, 2 * n - 1))
    trig[:, 0] = 1.0
    for m in range(1, n):
        trig[:, 2 * m - 1] = np.cos(m * phis)
        trig[:, 2 * m] = np.sin(m * phis)
    w = wz * 2.0 * math.pi / NP
    # checks: separation at an arbitrary azimuth, exactness against C_ijk
    rng = np.random.default_rng(0)
    for za in range(NZ):
        st = math.sqrt(1.0 - z[za] ** 2)
        ph = 0.731
        for i in range(K):
            l = int(math.isqrt(i))
            m = i - l * l - l
            t = 1.0 if m == 0 else (math.cos(m * ph) if m > 0 else math.sin(-m * ph))
            assert abs(ysh(i, st * math.cos(ph), st * math.sin(ph), z[za]) - leg[za, i] * t) < 1e-12
    fidx = [f_of(i - int(math.isqrt(i)) ** 2 - int(math.isqrt(i))) for i in range(K)]
    Y = np.einsum("ai,bi->abi", leg, trig[:, fidx])          # [NZ, NP, K]
    a, bb = rng.normal(size=K), rng.normal(size=K)
    prod = np.einsum("ab,ab,abi->i", w[:, None] * (Y @ a), Y @ bb, Y)
    ref = np.zeros(K)
    for (i, j, k), v in gaunt_monomial(n).items():
        ref[i] += float(v) * (a[j] * bb[k] + (a[k] * bb[j] if j != k else 0.0))
    assert np.abs(prod - ref).max() < 1e-10 * max(1.0, np.abs(ref).max()), np.abs(prod - ref).max()
    return leg, trig, w


def exp_rule_tables(n):
    """Rule of the projected-exponential variant: 2n Gauss-Legendre nodes in
    cos(theta) x 4n uniform azimuths, in the separable form of
    quadrature_tables (leg [2n][K], trig [4n][2n-1], w [2n]).  Checked:
    the factorisation, and sum_q w y_i y_j = delta_ij (exact at this degree)."""
    K = n * n
    NZ, NP = 2 * n, 4 * n
    z, wz = np.polynomial.legendre.leggauss(NZ)
    H = homogeneous_polys(n)
    N = norms(n)

    def ysh(i, x, y, zz):
        return N[i] * sum(float(v) * x ** a * y ** b * zz ** c for (a, b, c), v in H[i].items())

    leg = np.zeros((NZ, K))
    for za in range(NZ):
        st = math.sqrt(1.0 - z[za] ** 2)
        for i in range(K):
            l = int(math.isqrt(i))
            m = i - l * l - l
            ph = 0.0 if m >= 0 else math.pi / (2 * (-m))
            leg[za, i] = ysh(i, st * math.cos(ph), st * math.sin(ph), z[za])
    phis = 2.0 * math.pi * (np.arange(NP) + 0.5) / NP
    trig = np.zeros((NP, 2 * n - 1))
    trig[:, 0] = 1.0
    for m in range(1, n):
        trig[:, 2 * m - 1] = np.cos(m * phis)
        trig[:, 2 * m] = np.sin(m * phis)
    w = wz * 2.0 * math.pi / NP

    def f_of(i):
        l = int(math.isqrt(i))
        m = i - l * l - l
        return 0 if m == 0 else (2 * m - 1 if m > 0 else 2 * (-m))
    Y = np.einsum("ai,bi->abi", leg, trig[:, [f_of(i) for i in range(K)]])
    gram = np.einsum("a,abi,abj->ij", w, Y, Y)
    assert np.abs(gram - np.eye(K)).max() < 1e-12
    for za in range(NZ):
        st = math.sqrt(1.0 - z[za] ** 2)
        for i in range(K):
            l = int(math.isqrt(i))
            m = i - l * l - l
            t = 1.0 if m == 0 else (math.cos(m * 0.4) if m > 0 else math.sin(-m * 0.4))
            assert abs(ysh(i, st * math.cos(0.4), st * math.sin(0.4), z[za]) - leg[za, i] * t) < 1e-12
    return leg, trig, w


def emit_exp_rule(n):
    leg, trig, w = exp_rule_tables(n)

    def arr(name, a):
        vals = ", ".join(fmt(("c", float(v))) for v in np.asarray(a).ravel())
        return f"static __constant__ float {name}[{np.asarray(a).size}] = {{{vals}}};"
    return [f"#if defined(SHS_NB) && SHS_NB == {n}",
            arr(f"kExpLeg{n}", leg), arr(f"kExpTrig{n}", trig), arr(f"kExpW{n}", w),
            "#endif"]


def emit_quadrature(n):
    leg, trig, w = quadrature_tables(n)

    def arr(name, a):
        vals = ", ".join(fmt(("c", float(v))) for v in np.asarray(a).ravel())
        return f"static __constant__ float {name}[{np.asarray(a).size}] = {{{vals}}};"
    return [f"#if defined(SHS_NB) && SHS_NB == {n}",
            arr(f"kQuadLeg{n}", leg), arr(f"kQuadTrig{n}", trig), arr(f"kQuadW{n}", w),
            "#endif"], leg.shape[0], trig.shape[0]


def indent(lines, k=8):
    return "\n".join(" " * k + ln for ln in lines)


def generate():
    parts = [
        "// Generated by gen_tables.py -- do not edit.",
        "// Real SH polynomials, their reverse-mode gradients, and the truncated",
        "// SH triple product (Sec. 3.2, Eq. 3 and Eq. 6-7), unrolled per band count",
        "// (from 7 bands, quadrature tables for the triple product instead).",
        "#pragma once",
        "",
        "namespace shsgen {",
        "",
        "template <int NB> struct SH;",
        "",
    ]
    for n in BANDS:
        K = n * n
        C = gaunt_monomial(n)
        code, outs = build_ybar(n)
        fwd = emit_forward(code, outs, "Y")
        vjp = emit_forward(code, [], "Y") + emit_vjp(code, outs)
        mul_l, sqr_l = emit_gaunt(n, C) if n < QUAD_FROM else ([], [])
        N = norms(n)
        A = ahat(n)
        if n >= QUAD_FROM:
            parts.extend(emit_quadrature(n)[0])
        parts.extend(emit_exp_rule(n))
        parts.append(f"template <> struct SH<{n}> {{")
        parts.append(f"    static constexpr int K = {K};")
        parts.append(f"    static constexpr int NNZ_SYM = {len(C)};   // entries (i, j <= k)")
        parts.append(f"    static constexpr int EZ = {2 * n};    // projected-exponential rule: Gauss-Legendre nodes")
        parts.append(f"    static constexpr int EP = {4 * n};    // projected-exponential rule: uniform azimuths")
        parts.append("#if defined(SHS_NB) && SHS_NB == " + str(n))
        parts.append(f"    __device__ __forceinline__ static const float* eleg() {{ return kExpLeg{n}; }}")
        parts.append(f"    __device__ __forceinline__ static const float* etrig() {{ return kExpTrig{n}; }}")
        parts.append(f"    __device__ __forceinline__ static const float* ew() {{ return kExpW{n}; }}")
        parts.append("#endif")
        parts.append("    __device__ __forceinline__ static float norm(int i) {")
        parts.append("        switch (i) {")
        for i, v in enumerate(N):
            parts.append(f"            case {i}: return {fmt(('c', v))};")
        parts.append("            default: return 0.0f;")
        parts.append("        }")
        parts.append("    }")
        parts.append("    __device__ __forceinline__ static float ahat(int l) {")
        parts.append("        switch (l) {")
        for l, v in enumerate(A):
            parts.append(f"            case {l}: return {fmt(('c', v))};")
        parts.append("            default: return 0.0f;")
        parts.append("        }")
        parts.append("    }")
        parts.append("    __device__ __forceinline__ static void ybar(float x, float y, float z, float* Y) {")
        parts.append("        (void)x; (void)y; (void)z;")
        parts.append(indent(fwd))
        parts.append("    }")
        parts.append("    __device__ __forceinline__ static void ybar_vjp(float x, float y, float z, const float* w,")
        parts.append("                                                    float& gx, float& gy, float& gz) {")
        parts.append("        (void)x; (void)y; (void)z; (void)w;")
        parts.append(indent([ln for ln in vjp if not ln.startswith("Y[")]))
        parts.append("    }")
        na, ng, ml, acc_l, m2f_l, gc_l, ge_l = emit_monomial_route(n)
        parts.append(f"    static constexpr int NA = {na};   // monomials of degree < n")
        parts.append(f"    static constexpr int NG = {max(ng, 1)};   // gradient coefficients, bands >= 1")
        parts.append("    __device__ __forceinline__ static void accumulate(const float* G, float x, float y, float z, float* acc) {")
        parts.append("        (void)x; (void)y; (void)z;")
        parts.append(indent(ml + acc_l))
        parts.append("    }")
        parts.append("    // the same for two pairs at once, one per half of each float2")
        parts.append("    __device__ __forceinline__ static void accumulate2(const float2* G, float2 x, float2 y, float2 z,")
        parts.append("                                                       float2* acc) {")
        parts.append("        (void)x; (void)y; (void)z;")
        parts.append(indent(packed_lines(ml + acc_l)))
        parts.append("    }")
        parts.append("    __device__ __forceinline__ static void mono_to_f(const float* acc, float* f) {")
        parts.append(indent(m2f_l))
        parts.append("    }")
        parts.append("    __device__ __forceinline__ static void grad_coeffs(const float* w, float* gq) {")
        parts.append("        (void)w; (void)gq;")
        parts.append(indent(gc_l))
        parts.append("    }")
        parts.append("    __device__ __forceinline__ static void grad_eval(float x, float y, float z, const float* gq,")
        parts.append("                                                     float* gx, float* gy, float* gz) {")
        parts.append("        (void)x; (void)y; (void)z; (void)gq; (void)gx; (void)gy; (void)gz;")
        parts.append(indent(ge_l))
        parts.append("    }")
        # From 7 bands on the products are tens of thousands of FMAs each:
        # one out-of-line copy per translation unit instead of one per call
        # site keeps compile time and the instruction footprint bounded (the
        # operands of an out-of-line call live in local memory, a few hundred
        # bytes against ~10^4 FMAs per call; the operands never alias, which
        # lets every input stay in a register while the outputs are stored).
        if n < QUAD_FROM:
            parts.append("    __device__ __forceinline__ static void mul(const float* __restrict__ a, const float* __restrict__ b,")
            parts.append("                                               float* __restrict__ o) {")
            parts.append(indent(mul_l))
            parts.append("    }")
            parts.append("    __device__ __forceinline__ static void sqr(const float* __restrict__ a, float* __restrict__ o) {")
            parts.append(indent(sqr_l))
            parts.append("    }")
        else:
            # The unrolled products would be 10^4 FMAs of straight-line code
            # each (instruction-fetch bound); these band counts use the
            # separable quadrature of quadrature_tables() instead.
            _, nz, npp = emit_quadrature(n)
            parts.append(f"    static constexpr int QZ = {nz};    // Gauss-Legendre nodes in cos(theta)")
            parts.append(f"    static constexpr int QP = {npp};    // uniform azimuths")
            parts.append(f"    static constexpr int QF = {2 * n - 1};    // azimuthal harmonics 1, cos m phi, sin m phi")
            parts.append("#if defined(SHS_NB) && SHS_NB == " + str(n))
            parts.append(f"    __device__ __forceinline__ static const float* qleg() {{ return kQuadLeg{n}; }}")
            parts.append(f"    __device__ __forceinline__ static const float* qtrig() {{ return kQuadTrig{n}; }}")
            parts.append(f"    __device__ __forceinline__ static const float* qw() {{ return kQuadW{n}; }}")
            parts.append("#endif")
        parts.append("};")
        parts.append("")
    parts.append("}  // namespace shsgen")
    parts.append("")
    return "\n".join(parts)


def main(argv):
    text = generate()
    if "--check" in argv:
        cur = open(OUT).read() if os.path.exists(OUT) else ""
        if cur != text:
            print("generated header is stale; run gen_tables.py", file=sys.stderr)
            return 1
        return 0
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as fh:
        fh.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
