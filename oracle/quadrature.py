"""Consistent loads, the L2 projection P_h and the L2 error, by Gauss-Legendre quadrature.

Test infrastructure only (see ``oracle/__init__``).

P_h is the L2-orthogonal projection onto V_h (Sec. 2.1, Eq. (3-11) and
Eq. (1-5)): its nodal coefficients solve M u = F with the consistent load
F_k = (g, phi_k).  The paper's error ||U - u(T)||_0 (Sec. 5) is the
continuous L2 norm, evaluated here per element with a tensor Gauss rule.

Descriptor evaluation (the source terms and initial data given by
``paper_2412_01138_gb300.inputs``) is also written out here.
"""
from __future__ import annotations

import numpy as np

from paper_2412_01138_gb300 import inputs as _in

from .fem import axis_grid


def gauss_legendre(npts: int):
    """Nodes in [0,1] and weights summing to 1 (numpy's Legendre rule, mapped)."""
    xi, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (xi + 1.0), 0.5 * w


def is_time_dependent(f: "_in.Factor") -> bool:
    return f.kind == _in.S_MOVING_HAT


def eval_factor(f: "_in.Factor", x: np.ndarray, t=None) -> np.ndarray:
    """One spatial factor at points x (time t for the factors that move)."""
    p = f.params4()
    if f.kind == _in.S_ONE:
        return np.ones_like(x)
    if f.kind == _in.S_SIN:
        return np.sin(p[0] * x + p[1])
    if f.kind == _in.S_GAUSS:
        return np.exp(-((x - p[0]) ** 2) / (2.0 * p[1] ** 2))
    if f.kind == _in.S_POLY:
        return p[0] + x * (p[1] + x * (p[2] + x * p[3]))
    if f.kind == _in.S_MOVING_HAT:
        if t is None:
            raise ValueError("a moving hat needs the time (general forcing path only)")
        c = p[0] + p[1] * np.sin(2.0 * np.pi * p[2] * t)
        return np.maximum(1.0 - np.abs(x - c) / p[3], 0.0)
    raise ValueError(f"unknown spatial factor kind {f.kind}")


def eval_time(term: "_in.Term", t: float) -> float:
    a, b = term.tp
    if term.tkind == _in.T_EXP:
        return float(np.exp(a * t))
    if term.tkind == _in.T_SIN:
        return float(np.sin(a * t + b))
    raise ValueError(f"unknown time factor kind {term.tkind}")


def eval_terms(terms, t, coords) -> np.ndarray:
    """sum_r amp_r time_r(t) prod_a factor_{r,a}(coords[a]) on a tensor grid of points.

    t = None drops the time factors (initial data are spatial only).
    """
    out = 0.0
    for term in terms:
        vals = term.amp * (1.0 if t is None else eval_time(term, t))
        prod = None
        for a, fac in enumerate(term.factors):
            v = eval_factor(fac, coords[a], t)
            prod = v if prod is None else np.multiply.outer(prod, v)
        out = out + vals * prod
    return out


def load_1d(fun, lo: float, hi: float, n: int, qp: int) -> np.ndarray:
    """F_k = int fun(x) phi_k(x) dx for the n interior hats of one axis.

    Element e = 0..n spans [lo + e h, lo + (e+1) h]; on it, the hat of its
    left node is 1 - s and that of its right node is s (s in [0,1]).
    """
    h, _ = axis_grid(lo, hi, n)
    s, w = gauss_legendre(qp)
    F = np.zeros(n + 2)  # include the two boundary nodes, dropped at the end
    for e in range(n + 1):
        xq = lo + (e + s) * h
        gq = fun(xq)
        F[e] += h * np.sum(w * gq * (1.0 - s))
        F[e + 1] += h * np.sum(w * gq * s)
    return F[1:-1]


def load_1d_periodic(fun, lo: float, hi: float, n: int, qp: int) -> np.ndarray:
    """F_k = int fun(x) phi_k(x) dx for the n hats of a periodic axis (nodes x_k = lo + k h,
    h = (hi - lo)/n): element e = 0..n-1 spans [lo + e h, lo + (e+1) h], its left node is e
    and its right node (e+1) mod n."""
    h, _ = axis_grid(lo, hi, n, True)
    s, w = gauss_legendre(qp)
    F = np.zeros(n)
    for e in range(n):
        gq = fun(lo + (e + s) * h)
        F[e] += h * np.sum(w * gq * (1.0 - s))
        F[(e + 1) % n] += h * np.sum(w * gq * s)
    return F


def load_full(terms, t, n, box, qp: int, periodic=()) -> np.ndarray:
    """d-D consistent load by tensor Gauss quadrature on every Q1 element.

    t = None loads the spatial part only (initial data).

    Evaluates the (possibly non-separable) function on all quadrature points
    of every element; each element adds w * f * prod_a (1-s_a or s_a) to its
    2^d vertices.  Slow, used on small grids.
    """
    d = len(n)
    per = tuple(periodic) + (False,) * (d - len(periodic))
    s, w = gauss_legendre(qp)
    hs = [axis_grid(box[a][0], box[a][1], n[a], per[a])[0] for a in range(d)]
    ne = [n[a] if per[a] else n[a] + 1 for a in range(d)]  # elements per axis
    # quadrature points along each axis for all elements: shape (ne_a, qp)
    pts = [box[a][0] + (np.arange(ne[a])[:, None] + s[None, :]) * hs[a] for a in range(d)]
    F = np.zeros(tuple(v + 1 for v in ne))
    # f at all points: shape (ne0, qp, ne1, qp, ...)
    fvals = eval_terms(terms, t, [p.reshape(-1) for p in pts])
    fvals = fvals.reshape(sum(((ne[a], qp) for a in range(d)), ()))
    for corner in range(2 ** d):
        bits = [(corner >> (d - 1 - a)) & 1 for a in range(d)]
        weight = None
        for a in range(d):
            shp = (s if bits[a] else 1.0 - s) * w * hs[a]
            weight = shp if weight is None else np.multiply.outer(weight, shp)
        # contract quadrature axes: fvals indices (e0,q0,e1,q1,...) with weight (q0,q1,...)
        contracted = _contract(fvals, weight, d, qp, ne)
        sl = tuple(slice(bits[a], bits[a] + ne[a]) for a in range(d))
        F[sl] += contracted
    # Dirichlet axes drop their two boundary nodes; periodic axes fold node n onto node 0
    for a in range(d):
        if per[a]:
            F = np.moveaxis(F, a, 0)
            F[0] += F[-1]
            F = np.moveaxis(F[:-1], 0, a)
        else:
            F = np.moveaxis(np.moveaxis(F, a, 0)[1:-1], 0, a)
    return F


def _contract(fvals, weight, d, qp, n):
    """sum over quadrature indices q_a of fvals[e0,q0,e1,q1,...] * weight[q0,q1,...]."""
    # reorder fvals to (e0,...,e_{d-1}, q0,...,q_{d-1})
    perm = [2 * a for a in range(d)] + [2 * a + 1 for a in range(d)]
    fv = np.transpose(fvals, perm)
    return np.tensordot(fv, weight, axes=(list(range(d, 2 * d)), list(range(d))))


def separable_load_factors(term, n, box, qp: int, periodic=()):
    """Per-axis 1D consistent loads of one separable term (spatial part only)."""
    per = tuple(periodic) + (False,) * (len(n) - len(periodic))
    out = []
    for a, fac in enumerate(term.factors):
        load = load_1d_periodic if per[a] else load_1d
        out.append(load(lambda x, fac=fac: eval_factor(fac, x), box[a][0], box[a][1], n[a], qp))
    return out


def l2_error_full(nodal: np.ndarray, exact_terms, t: float, n, box, qp: int = 5) -> float:
    """||u_h - u(t)||_0 with u_h the multilinear interpolant of the nodal values.

    Per-element tensor Gauss rule with qp points per axis.
    """
    d = len(n)
    s, w = gauss_legendre(qp)
    hs = [axis_grid(box[a][0], box[a][1], n[a])[0] for a in range(d)]
    U = np.zeros(tuple(v + 2 for v in n))
    U[tuple(slice(1, -1) for _ in range(d))] = nodal
    pts = [box[a][0] + (np.arange(n[a] + 1)[:, None] + s[None, :]) * hs[a] for a in range(d)]
    uex = eval_terms(exact_terms, t, [p.reshape(-1) for p in pts])
    uex = uex.reshape(sum(((n[a] + 1, qp) for a in range(d)), ()))
    # interpolant at the same points: sum over corners of U[e + bit] * prod shape
    uh = np.zeros_like(uex)
    for corner in range(2 ** d):
        bits = [(corner >> (d - 1 - a)) & 1 for a in range(d)]
        sl = tuple(slice(bits[a], bits[a] + n[a] + 1) for a in range(d))
        Uc = U[sl]  # (n0+1, n1+1, ...)
        shp = None
        for a in range(d):
            v = s if bits[a] else 1.0 - s
            shp = v if shp is None else np.multiply.outer(shp, v)
        # uh[e0,q0,e1,q1,..] += Uc[e0,e1,..] * shp[q0,q1,..]
        full = np.multiply.outer(Uc, shp)  # (e0..,q0..)
        inv = np.argsort([2 * a for a in range(d)] + [2 * a + 1 for a in range(d)])
        uh += np.transpose(full, inv)
    wt = None
    for a in range(d):
        wa = np.multiply.outer(np.full(n[a] + 1, hs[a]), w)  # (e_a, q_a)
        wt = wa if wt is None else np.multiply.outer(wt, wa)
    # wt has index order (e0,q0,e1,q1,...) already
    return float(np.sqrt(np.sum(wt * (uh - uex) ** 2)))


def l2_inner_1d(fun, nodal: np.ndarray, lo: float, hi: float, qp: int = 5):
    """Per-element Gauss sums int fun^2, int fun*v_h, int v_h^2 for one axis.

    v_h is the piecewise linear function with the given interior nodal values
    and zero boundary values.  Used for the L2 error of rank-one (separable)
    u and u_h, where ||u - u_h||^2 = prod int w_a^2 - 2 prod int w_a v_a + prod int v_a^2.
    """
    n = len(nodal)
    h, _ = axis_grid(lo, hi, n)
    s, w = gauss_legendre(qp)
    V = np.concatenate([[0.0], nodal, [0.0]])
    e = np.arange(n + 1)[:, None]
    xq = lo + (e + s[None, :]) * h
    fq = fun(xq)
    vq = V[:-1, None] * (1.0 - s[None, :]) + V[1:, None] * s[None, :]
    ww = h * w[None, :]
    return float(np.sum(ww * fq * fq)), float(np.sum(ww * fq * vq)), float(np.sum(ww * vq * vq))
