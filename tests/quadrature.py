"""Brute-force numerical evaluation of contracted Cartesian-Gaussian ERIs.

Independent of every recursion and of the Boys function: the kernel is
written as a Gaussian transform,

    1/r           = (2/sqrt(pi)) int_0^inf   exp(-t^2 r^2) dt
    erf(w r)/r    = (2/sqrt(pi)) int_0^w     exp(-t^2 r^2) dt
    erfc(w r)/r   = (2/sqrt(pi)) int_w^inf   exp(-t^2 r^2) dt

so that for fixed t the six-dimensional integral factorises into three
two-dimensional Gaussian-times-polynomial integrals, one per Cartesian axis.
Each is done with a tensor Gauss-Hermite rule after a Cholesky change of
variables (exact for the polynomial degrees involved, <= 8 per axis), and the
remaining one-dimensional t integral with adaptive quadrature.

Normalisation is also done numerically (Gauss-Hermite moments), so the
oracle's closed-form normalisation is checked too.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.hermite import hermgauss
from scipy.integrate import quad_vec

GH_X, GH_W = hermgauss(12)


def cart_components(l: int):
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def _moment(n: int, g):
    """int x^n exp(-g x^2) dx by Gauss-Hermite."""
    g = np.asarray(g, dtype=np.float64)
    s = np.sqrt(g)
    return np.sum(GH_W[None, :] * (GH_X[None, :] / s[..., None]) ** n, axis=-1) / s


def normalized_coefs(l: int, alpha, raw):
    """Primitive x^l exp(-a r^2) scaled to unit norm, then the contracted axial
    component scaled to unit self-overlap."""
    alpha = np.asarray(alpha, dtype=np.float64)
    raw = np.asarray(raw, dtype=np.float64)
    g = 2.0 * alpha
    nrm = 1.0 / np.sqrt(_moment(2 * l, g) * _moment(0, g) ** 2)
    c = raw * nrm
    G = alpha[:, None] + alpha[None, :]
    S = np.sum(c[:, None] * c[None, :] * _moment(2 * l, G) * _moment(0, G) ** 2)
    return c / math.sqrt(S)


def _axis_table(t, A, B, C, D, al, be, ga, de, lmax):
    """T[p, ea, eb, ec, ed] = int int (x1-A)^ea (x1-B)^eb (x2-C)^ec (x2-D)^ed
    exp(-al(x1-A)^2 - be(x1-B)^2 - ga(x2-C)^2 - de(x2-D)^2 - t^2 (x1-x2)^2)."""
    p = al + be
    q = ga + de
    t2 = t * t
    M11 = p + t2
    M22 = q + t2
    M12 = -t2 * np.ones_like(p)
    r1 = al * A + be * B
    r2 = ga * C + de * D
    det = M11 * M22 - M12 * M12
    m1 = (M22 * r1 - M12 * r2) / det
    m2 = (M11 * r2 - M12 * r1) / det
    c0 = (M11 * m1 * m1 + 2 * M12 * m1 * m2 + M22 * m2 * m2) - (al * A * A + be * B * B + ga * C * C + de * D * D)
    l11 = np.sqrt(M11)
    l21 = M12 / l11
    l22 = np.sqrt(M22 - l21 * l21)
    y1 = GH_X[:, None] * np.ones_like(GH_X)[None, :]
    y2 = GH_X[None, :] * np.ones_like(GH_X)[:, None]
    w = (GH_W[:, None] * GH_W[None, :]).reshape(-1)
    y1 = y1.reshape(-1)
    y2 = y2.reshape(-1)
    x1 = m1[:, None] + y1[None, :] / l11[:, None] - y2[None, :] * (l21 / (l11 * l22))[:, None]
    x2 = m2[:, None] + y2[None, :] / l22[:, None]
    pw = lambda x, c: np.stack([(x - c) ** e for e in range(lmax + 1)], axis=1)  # (p, e, n)
    ua, ub, uc, ud = pw(x1, A), pw(x1, B), pw(x2, C), pw(x2, D)
    T = np.einsum("pan,pbn,pcn,pdn,n->pabcd", ua, ub, uc, ud, w, optimize=True)
    scale = np.exp(c0) / (l11 * l22)
    return T * scale[:, None, None, None, None]


def eri_quadrature(shells, kernel: str = "coulomb", omega: float = 0.11, epsrel: float = 1e-12,
                   epsabs: float = 1e-14):
    """shells: four tuples (center(3), l, alphas, normalised coefs).
    Returns the contracted integrals shaped (nA, nB, nC, nD)."""
    (A, la, aa, ca), (B, lb, ab, cb), (C, lc, ac, cc), (D, ld, ad, cd) = shells
    A, B, C, D = (np.asarray(x, dtype=np.float64) for x in (A, B, C, D))
    g = np.meshgrid(np.arange(len(aa)), np.arange(len(ab)), np.arange(len(ac)), np.arange(len(ad)),
                    indexing="ij")
    i, j, k, m = (x.reshape(-1) for x in g)
    al, be, ga, de = np.asarray(aa)[i], np.asarray(ab)[j], np.asarray(ac)[k], np.asarray(ad)[m]
    coef = np.asarray(ca)[i] * np.asarray(cb)[j] * np.asarray(cc)[k] * np.asarray(cd)[m]
    comps = [cart_components(x) for x in (la, lb, lc, ld)]
    tuples = [(a, b, c, d) for a in comps[0] for b in comps[1] for c in comps[2] for d in comps[3]]
    idx = np.array([[[a[x], b[x], c[x], d[x]] for x in range(3)] for (a, b, c, d) in tuples])
    lmax = 2

    def integrand(t):
        tabs = [_axis_table(t, A[x], B[x], C[x], D[x], al, be, ga, de, lmax) for x in range(3)]
        vals = np.ones((len(tuples), coef.shape[0]))
        for x in range(3):
            e = idx[:, x, :]
            vals = vals * tabs[x][:, e[:, 0], e[:, 1], e[:, 2], e[:, 3]].T
        return (2.0 / math.sqrt(math.pi)) * (vals @ coef)

    if kernel == "coulomb":
        lo, hi = 0.0, np.inf
    elif kernel == "erf":
        lo, hi = 0.0, omega
    elif kernel == "erfc":
        lo, hi = omega, np.inf
    else:
        raise ValueError(kernel)
    res, _err = quad_vec(integrand, lo, hi, epsrel=epsrel, epsabs=epsabs, limit=2000)
    return np.asarray(res).reshape(len(comps[0]), len(comps[1]), len(comps[2]), len(comps[3]))
