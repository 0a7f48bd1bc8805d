"""Exact time of impact for one vertex-face or edge-edge query.

TEST INFRASTRUCTURE ONLY (test suite, smoke check, CPU baseline).  Pure Python
on integers and ``fractions``; it shares nothing with the CUDA library.

Problem (Section "Preliminaries"): with linear trajectories
x(t) = x0 + t (x1 - x0), return the earliest t in [0, 1] at which the point
touches the triangle (vertex-face) or the two segments touch (edge-edge), or
None when they never do.  With min_sep = 0 this is the value that a
conservative method must never exceed (Section "Guarantees";
Section "Time of Impact Validation and Accuracy").

Method.  Vertex-face: F(t,u,v) = w - u e1 - v e2 with w = P - T0,
e1 = T1 - T0, e2 = T2 - T0, (u, v) in the simplex.  Edge-edge:
F = w + u ea - v eb with w = A0 - B0, ea = A1 - A0, eb = B1 - B0,
(u, v) in [0,1]^2.  Every coordinate of w, e1, e2 (ea, eb) is a polynomial of
degree <= 1 in t.  The set T of colliding times is closed and semi-algebraic;
its minimum is t = 0 or a point where a contact starts, which is a root of one
of these "event" polynomials:
  * the coplanarity cubic det[e1, e2, w] (det[ea, eb, w]) -- contact through
    the interior;
  * a coordinate of a point-segment cross product -- contact at a boundary
    edge of the parameter domain;
  * a coordinate of a point-point difference -- contact at a corner.
All real roots in (0, 1] of the non-zero event polynomials are isolated with
Sturm sequences, ordered exactly, and tested in increasing order by an exact
feasibility decision (polynomial sign conditions evaluated at the algebraic
root).  The first feasible one is the time of impact.
"""
from __future__ import annotations

import functools
from fractions import Fraction as Q
from typing import List, Optional, Sequence, Union

# ----------------------------------------------------------------------------
# Univariate polynomials: lists of Fractions, ascending powers, no trailing 0.
# ----------------------------------------------------------------------------


def ptrim(p):
    p = list(p)
    while p and p[-1] == 0:
        p.pop()
    return p


def padd(p, q):
    n = max(len(p), len(q))
    return ptrim([(p[i] if i < len(p) else 0) + (q[i] if i < len(q) else 0) for i in range(n)])


def pneg(p):
    return [-c for c in p]


def psub(p, q):
    return padd(p, pneg(q))


def pmul(p, q):
    if not p or not q:
        return []
    r = [Q(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        if a == 0:
            continue
        for j, b in enumerate(q):
            r[i + j] += a * b
    return ptrim(r)


def pderiv(p):
    return ptrim([i * p[i] for i in range(1, len(p))])


def peval(p, x):
    acc = Q(0)
    for c in reversed(p):
        acc = acc * x + c
    return acc


def pdivmod(p, q):
    p = ptrim(p)
    q = ptrim(q)
    if not q:
        raise ZeroDivisionError("polynomial division by zero")
    quo = [Q(0)] * max(len(p) - len(q) + 1, 1)
    r = list(p)
    lead = q[-1]
    while len(r) >= len(q) and r:
        c = r[-1] / lead
        k = len(r) - len(q)
        quo[k] = c
        for i, b in enumerate(q):
            r[i + k] -= c * b
        r = ptrim(r)
    return ptrim(quo), r


def pmonic(p):
    p = ptrim(p)
    return [c / p[-1] for c in p] if p else []


def pgcd(p, q):
    p, q = ptrim(p), ptrim(q)
    while q:
        p, q = q, pdivmod(p, q)[1]
    return pmonic(p)


def psquarefree(p):
    g = pgcd(p, pderiv(p))
    return pmonic(pdivmod(p, g)[0]) if len(g) > 1 else pmonic(p)


def sign(x) -> int:
    return (x > 0) - (x < 0)


def sturm_chain(p):
    chain = [ptrim(p), pderiv(p)]
    while chain[-1]:
        r = pdivmod(chain[-2], chain[-1])[1]
        chain.append(pneg(r))
    return [c for c in chain if c]


def variations(chain, x) -> int:
    signs = [sign(peval(c, x)) for c in chain]
    signs = [s for s in signs if s != 0]
    return sum(1 for a, b in zip(signs, signs[1:]) if a != b)


def count_roots(chain, a, b) -> int:
    """Distinct real roots of the (square-free) chain head in the half-open
    interval (a, b] (Sturm's theorem; the variation count is right-continuous
    at a root, so a and b may themselves be roots)."""
    return variations(chain, a) - variations(chain, b)


# ----------------------------------------------------------------------------
# Real algebraic numbers: a root of a square-free polynomial isolated in an
# open interval with rational ends that are not roots.
# ----------------------------------------------------------------------------


class Alg:
    __slots__ = ("p", "lo", "hi", "slo", "exact")

    def __init__(self, p, lo, hi):
        self.p = p
        self.lo = Q(lo)
        self.hi = Q(hi)
        self.slo = sign(peval(p, self.lo))
        self.exact: Optional[Q] = None
        assert self.slo != 0 and sign(peval(p, self.hi)) == -self.slo

    def refine(self):
        if self.exact is not None:
            return
        mid = (self.lo + self.hi) / 2
        s = sign(peval(self.p, mid))
        if s == 0:
            self.exact = mid
            self.lo = self.hi = mid
        elif s == self.slo:
            self.lo = mid
        else:
            self.hi = mid

    def bracket(self, bits: int = 60):
        while self.exact is None and self.hi - self.lo >= Q(1, 2 ** bits):
            self.refine()
        return self.lo, self.hi

    def __float__(self):
        lo, hi = self.bracket(70)
        return float((lo + hi) / 2)

    def __repr__(self):
        if self.exact is not None:
            return f"Alg(exact={self.exact})"
        return f"Alg({float(self.lo):.17g}..{float(self.hi):.17g})"


Exact = Union[Q, Alg]


def _as_rational(x: Exact) -> Optional[Q]:
    if isinstance(x, Q):
        return x
    return x.exact


def sign_at(q, x: Exact) -> int:
    """Sign of polynomial q at the exact number x."""
    q = ptrim(q)
    if not q:
        return 0
    r = _as_rational(x)
    if r is not None:
        return sign(peval(q, r))
    g = pgcd(x.p, q)
    if len(g) > 1 and sign(peval(g, x.lo)) * sign(peval(g, x.hi)) < 0:
        return 0
    qs = psquarefree(q)
    chain = sturm_chain(qs)
    while True:
        r = _as_rational(x)
        if r is not None:
            return sign(peval(q, r))
        if (peval(qs, x.lo) != 0 and peval(qs, x.hi) != 0
                and count_roots(chain, x.lo, x.hi) == 0):
            return sign(peval(q, x.lo))
        x.refine()


def compare(a: Exact, b: Exact) -> int:
    ra, rb = _as_rational(a), _as_rational(b)
    if ra is not None and rb is not None:
        return sign(ra - rb)
    if ra is not None:
        return -compare(b, a)
    # a is irrational (so far)
    if rb is not None:
        while True:
            if a.exact is not None:
                return sign(a.exact - rb)
            if rb <= a.lo:
                return 1
            if rb >= a.hi:
                return -1
            if peval(a.p, rb) == 0:
                return 0
            a.refine()
    g = pgcd(a.p, b.p)
    if len(g) > 1:
        lo, hi = max(a.lo, b.lo), min(a.hi, b.hi)
        if lo < hi and sign(peval(g, lo)) * sign(peval(g, hi)) < 0:
            return 0
    while True:
        ra, rb = _as_rational(a), _as_rational(b)
        if ra is not None or rb is not None:
            return compare(a, b)
        if a.hi <= b.lo:
            return -1
        if b.hi <= a.lo:
            return 1
        a.refine()
        b.refine()


def le_float(t: float, x: Exact) -> bool:
    """Exact test t <= x for a double t."""
    return compare(Q(t), x) <= 0


def isolate(p, a: Q, b: Q) -> List[Exact]:
    """All distinct real roots of p (not identically zero) in [a, b]."""
    p = psquarefree(p)
    if len(p) <= 1:
        return []
    chain = sturm_chain(p)
    out: List[Exact] = []
    if peval(p, a) == 0:
        out.append(Q(a))
    tail = [Q(b)] if (peval(p, b) == 0 and b != a) else []

    def step_off(x, direction):
        """A non-root y beside the root x with no other root between them."""
        h = Q(1, 2 ** 20)
        while True:
            y = x + direction * h
            if peval(p, y) != 0:
                if direction > 0:
                    ok = count_roots(chain, x, y) == 0      # (x, y] holds no root
                else:
                    ok = count_roots(chain, y, x) == 1      # (y, x] holds x only
                if ok:
                    return y
            h /= 2

    lo = step_off(a, 1) if peval(p, a) == 0 else a
    hi = step_off(b, -1) if peval(p, b) == 0 else b

    def rec(lo, hi):
        if lo >= hi:
            return
        n = count_roots(chain, lo, hi)
        if n == 0:
            return
        if n == 1:
            out.append(Alg(p, lo, hi))
            return
        mid = (lo + hi) / 2
        if peval(p, mid) == 0:
            m1 = step_off(mid, -1)
            m2 = step_off(mid, 1)
            rec(lo, m1)
            out.append(Q(mid))
            rec(m2, hi)
        else:
            rec(lo, mid)
            rec(mid, hi)

    rec(lo, hi)
    out.extend(tail)
    return out


def real_roots(p) -> List[Exact]:
    """All distinct real roots of p, increasing (Cauchy bound)."""
    p = ptrim(p)
    bound = 1 + max(abs(c / p[-1]) for c in p[:-1]) if len(p) > 1 else Q(1)
    roots = isolate(p, -Q(bound), Q(bound))
    return sorted(roots, key=functools.cmp_to_key(compare))


# ----------------------------------------------------------------------------
# Vectors of polynomials in t.
# ----------------------------------------------------------------------------


def vsub(a, b):
    return [psub(x, y) for x, y in zip(a, b)]


def vadd(a, b):
    return [padd(x, y) for x, y in zip(a, b)]


def vdot(a, b):
    r = []
    for x, y in zip(a, b):
        r = padd(r, pmul(x, y))
    return r


def vcross(a, b):
    return [psub(pmul(a[1], b[2]), pmul(a[2], b[1])),
            psub(pmul(a[2], b[0]), pmul(a[0], b[2])),
            psub(pmul(a[0], b[1]), pmul(a[1], b[0]))]


ZERO3 = [[], [], []]


def _trajectory(x0: Sequence[float], x1: Sequence[float]):
    return [ptrim([Q(a), Q(b) - Q(a)]) for a, b in zip(x0, x1)]


def _is_zero(vec, t) -> bool:
    return all(sign_at(c, t) == 0 for c in vec)


def _on_segment(p, a, b, t) -> bool:
    """Point p on the closed segment [a, b] at time t."""
    r = vsub(p, a)
    s = vsub(b, a)
    if _is_zero(s, t):
        return _is_zero(r, t)
    if not _is_zero(vcross(r, s), t):
        return False
    rs = vdot(r, s)
    return sign_at(rs, t) >= 0 and sign_at(psub(vdot(s, s), rs), t) >= 0


def _vf_feasible(w, e1, e2, t) -> bool:
    n = vcross(e1, e2)
    if not _is_zero(n, t):
        if sign_at(vdot(w, n), t) != 0:
            return False
        nn = vdot(n, n)
        su = vdot(vcross(w, e2), n)   # u |n|^2
        sv = vdot(vcross(e1, w), n)   # v |n|^2
        return (sign_at(su, t) >= 0 and sign_at(sv, t) >= 0
                and sign_at(psub(psub(nn, su), sv), t) >= 0)
    # degenerate triangle: it is the union of its three edges
    return (_on_segment(w, ZERO3, e1, t) or _on_segment(w, ZERO3, e2, t)
            or _on_segment(w, e1, e2, t))


def _ee_feasible(w, ea, eb, t) -> bool:
    n = vcross(ea, eb)
    if not _is_zero(n, t):
        if sign_at(vdot(w, n), t) != 0:
            return False
        nn = vdot(n, n)
        su = vdot(vcross(eb, w), n)   # u |n|^2
        sv = vdot(vcross(ea, w), n)   # v |n|^2
        return (sign_at(su, t) >= 0 and sign_at(psub(nn, su), t) >= 0
                and sign_at(sv, t) >= 0 and sign_at(psub(nn, sv), t) >= 0)
    # parallel or degenerate: some endpoint lies on the other segment
    a0, a1, b0, b1 = w, vadd(w, ea), ZERO3, eb
    return (_on_segment(a0, b0, b1, t) or _on_segment(a1, b0, b1, t)
            or _on_segment(b0, a0, a1, t) or _on_segment(b1, a0, a1, t))


def _setup(vf: bool, x0, x1):
    X = [_trajectory(x0[k], x1[k]) for k in range(4)]
    if vf:
        P, T0, T1, T2 = X
        return vsub(P, T0), vsub(T1, T0), vsub(T2, T0)
    A0, A1, B0, B1 = X
    return vsub(A0, B0), vsub(A1, A0), vsub(B1, B0)


def _events(vf: bool, w, a, b):
    polys = [vdot(w, vcross(a, b))]
    if vf:   # w = P - T0, a = e1, b = e2
        vecs = [vcross(w, a), vcross(w, b), vcross(vsub(w, a), vsub(b, a)),
                w, vsub(w, a), vsub(w, b)]
    else:    # w = A0 - B0, a = ea, b = eb
        wa = vadd(w, a)
        vecs = [vcross(w, b), vcross(wa, b), vcross(w, a), vcross(vsub(w, b), a),
                w, wa, vsub(w, b), vsub(wa, b)]
    for v in vecs:
        polys.extend(v)
    return [p for p in (ptrim(x) for x in polys) if len(p) > 1]


def feasible(vf: bool, x0, x1, t: Exact) -> bool:
    """Exact decision: do the primitives touch at time t?"""
    w, a, b = _setup(vf, x0, x1)
    return _vf_feasible(w, a, b, t) if vf else _ee_feasible(w, a, b, t)


def toi(vf: bool, x0, x1) -> Optional[Exact]:
    """Earliest time of impact in [0, 1], or None.  x0, x1: 4 points each
    (vertex-face: P, T0, T1, T2; edge-edge: A0, A1, B0, B1) at t = 0 and 1,
    given as exact numbers (floats are converted exactly)."""
    w, a, b = _setup(vf, x0, x1)
    feas = _vf_feasible if vf else _ee_feasible
    if feas(w, a, b, Q(0)):
        return Q(0)
    cands: List[Exact] = []
    for p in _events(vf, w, a, b):
        for r in isolate(p, Q(0), Q(1)):
            rr = _as_rational(r)
            if rr is not None and rr == 0:
                continue
            cands.append(r)
    cands.sort(key=functools.cmp_to_key(compare))
    last = None
    for r in cands:
        if last is not None and compare(last, r) == 0:
            continue
        last = r
        if feas(w, a, b, r):
            return r
    return None
