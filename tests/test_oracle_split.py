"""Pins of the oracle's split rule, worked out by hand.

The paper's Algorithm 3 only says "split"; this repository reads it as:
split the axis k in {t, u, v} with the largest L_k * 2^-l_k (l_k the
interval's level on k), ties in the order t, u, v, where
  L_t = max over axes x of |dw_x| + |de1_x| + |de2_x|   (d: value at t = 1
        minus value at t = 0; edge-edge: w, ea, eb),
  L_u = max over axes x and t in {0, 1} of |e1_x(t)|   (edge-edge: ea),
  L_v = the same with e2 (edge-edge: eb).
Nothing below calls a formula of the oracle to get an expected value: every
number is derived in the docstrings from the reading above, on inputs built
so that the derivation is short and every floating-point step is exact.

Two kinds of pin:
  * the weights of two queries whose maxima sit on different axes and at
    different time ends (catches a weight built from the wrong vector, the
    wrong time end, positions instead of displacements, a sum instead of a
    max);
  * the exact number of intervals the depth-first bisection evaluates, and
    the time it returns, on queries whose zero set is a single point: the
    count depends on the order in which the axes are split, so a wrong
    comparison, a dropped 2^-l factor or another tie order changes it.
"""
import numpy as np

from oracle import oracle as O


def _count(vf, x0, x1, delta):
    toi, flags, iters, _ = O.narrow_queries(np.array([1 if vf else 0], np.uint8),
                                            np.arange(4, dtype=np.int64).reshape(1, 4),
                                            np.asarray(x0, float), np.asarray(x1, float),
                                            delta=delta, min_sep=0.0, max_iter=10 ** 6, mode=0)
    return float(toi[0]), int(flags[0]), int(iters[0])


# ---------------------------------------------------------------------------
# Weights
# ---------------------------------------------------------------------------

# Vertex-face: points P, T0, T1, T2 at t = 0 and t = 1.
W_VF = (
    [[1, 2, 0], [0, 0, 0], [0.5, 0, 0], [0, 0.75, 0]],
    [[1.5, 2, -0.25], [0.25, 0, 0], [-1.25, 0, 0.5], [0.25, 1, 0]],
)
# Edge-edge: A0, A1, B0, B1.
W_EE = (
    [[0, 0, 0], [1, 0, 0], [0, 0, -1], [0, 2, -1]],
    [[0, 0, 1], [0.5, 0, 1], [0, 0.5, -1], [0, 0.5, -1]],
)


def pin_split_weights():
    """Vertex-face W_VF, with w = P - T0, e1 = T1 - T0, e2 = T2 - T0:
        w:  (1, 2, 0)     -> (1.25, 2, -0.25)  dw  = (0.25, 0, -0.25)
        e1: (0.5, 0, 0)   -> (-1.5, 0, 0.5)    de1 = (-2, 0, 0.5)
        e2: (0, 0.75, 0)  -> (0, 1, 0)         de2 = (0, 0.25, 0)
      L_t = max(0.25 + 2 + 0, 0 + 0 + 0.25, 0.25 + 0.5 + 0) = 2.25 (axis x)
      L_u = max(|0.5|, |-1.5|, |0.5|, ...) = 1.5 (x at t = 1; 0.5 at t = 0)
      L_v = max(0.75, 1) = 1 (y at t = 1)
    Edge-edge W_EE, with w = A0 - B0, ea = A1 - A0, eb = B1 - B0:
        w:  (0, 0, 1)  -> (0, -0.5, 2)   dw  = (0, -0.5, 1)
        ea: (1, 0, 0)  -> (0.5, 0, 0)    dea = (-0.5, 0, 0)
        eb: (0, 2, 0)  -> (0, 0, 0)      deb = (0, -2, 0)
      L_t = max(0 + 0.5 + 0, 0.5 + 0 + 2, 1 + 0 + 0) = 2.5 (axis y)
      L_u = 1 (x at t = 0), L_v = 2 (y at t = 0)."""
    a = O.split_weights(True, *W_VF)
    b = O.split_weights(False, *W_EE)
    return list(a) == [2.25, 1.5, 1.0] and list(b) == [2.5, 1.0, 2.0]


def test_split_weights_by_hand():
    assert pin_split_weights()


# ---------------------------------------------------------------------------
# Split order, through the number of evaluated intervals
# ---------------------------------------------------------------------------
#
# Both queries have e1 (ea) = (1/2, 0, 0) and e2 (eb) = (0, 1/4, 0), constant
# in time, and w moving along z only with dw_z = -1, so L = (1, 1/2, 1/4).
# F then separates by axis: F_x depends on u only, F_y on v only, F_z on t
# only, and its exact zero set is one point (t*, u*, v*).  Over an interval
# with levels (l_t, l_u, l_v) the hull's widths are exactly 2^-l_t (z),
# 2^-1 2^-l_u (x) and 2^-2 2^-l_v (y) -- the three values L_k 2^-l_k -- and
# all coordinates are dyadic with few bits, so every operation of the
# evaluation is exact.
#
# With delta = 2^-6 the largest of the three values is split until all are
# below 2^-6.  Values (t, u, v) before each split and the axis chosen:
#    1 (1, 1/2, 1/4) t      7 (1/8, 1/8, 1/8) t     13 (1/32 x3) t
#    2 (1/2, 1/2, 1/4) t    8 (1/16, 1/8, 1/8) u    14 (1/64, 1/32, 1/32) u
#    3 (1/4, 1/2, 1/4) u    9 (1/16, 1/16, 1/8) v   15 (1/64, 1/64, 1/32) v
#    4 (1/4 x3) t          10 (1/16 x3) t           16 (1/64 x3) t  (= delta: not below)
#    5 (1/8, 1/4, 1/4) u   11 (1/32, 1/16, 1/16) u  17 (1/128, 1/64, 1/64) u
#    6 (1/8, 1/8, 1/4) v   12 (1/32, 1/32, 1/16) v  18 (1/128, 1/128, 1/64) v
# after which all three are 1/128 < delta and the interval is accepted:
# levels (7, 6, 5), 18 splits, t split at steps 1, 2, 4, 7, 10, 13, 16.
#
# Counting evaluations (depth first, left child first; pruning at t >= t*):
# the root, then at each split the left child; when the point lies in the
# right child the left one misses and the right one is evaluated as well
# (+1).  After the accept, t* = T (the left end of the accepted interval);
# a pending right sibling of a left-going split is evaluated (and misses)
# only if it starts before T: for a t split never (it starts after T), for a
# u or v split exactly when a later t split went right.  So
#   count = 1 + 18 + (right-going splits)
#           + (left-going u/v splits before the last right-going t split).


def _query_vf(t_digits, u_star, v_star):
    """Vertex-face: T0 = 0, T1 = (1/2, 0, 0), T2 = (0, 1/4, 0) static;
    P(t) = (u*/2, v*/4, t* - t), so F = P - T0 - u e1 - v e2 =
    ((u* - u)/2, (v* - v)/4, t* - t).  t* has the given first 7 binary
    digits plus 2^-9 (never on a split point of levels <= 7)."""
    ts = sum(d * 2.0 ** -(i + 1) for i, d in enumerate(t_digits)) + 2.0 ** -9
    x0 = [[u_star / 2, v_star / 4, ts], [0, 0, 0], [0.5, 0, 0], [0, 0.25, 0]]
    x1 = [[u_star / 2, v_star / 4, ts - 1], [0, 0, 0], [0.5, 0, 0], [0, 0.25, 0]]
    return x0, x1


def _query_ee(t_digits, u_star, v_star):
    """Edge-edge: B0 = 0, B1 = (0, 1/4, 0) static; A0(t) = (-u*/2, v*/4,
    t* - t), A1 = A0 + (1/2, 0, 0), so F = w + u ea - v eb =
    ((u - u*)/2, (v* - v)/4, t* - t)."""
    ts = sum(d * 2.0 ** -(i + 1) for i, d in enumerate(t_digits)) + 2.0 ** -9
    a0 = [-u_star / 2, v_star / 4, ts]
    a0e = [-u_star / 2, v_star / 4, ts - 1]
    x0 = [a0, [a0[0] + 0.5, a0[1], a0[2]], [0, 0, 0], [0, 0.25, 0]]
    x1 = [a0e, [a0e[0] + 0.5, a0e[1], a0e[2]], [0, 0, 0], [0, 0.25, 0]]
    return x0, x1


DELTA = 2.0 ** -6


def pin_split_order():
    """Case A, vertex-face: t digits 0100100 (t* = 0.283203125), u* = v* =
    2^-8 (u and v always go left).  Right-going splits: the t splits of
    digits 2 and 5 (steps 2 and 10): 2.  Left-going u/v splits before step
    10: steps 3, 5, 6, 8, 9: 5.  count = 1 + 18 + 2 + 5 = 26;
    T = 0.0100100b = 0.28125.

    Case B, edge-edge: t digits 1001000 (t* = 0.564453125), u* = 2^-8,
    v* = 0.10101b + 2^-8 (v splits go right, left, right, left, right).
    Right-going: t splits of digits 1 and 4 (steps 1, 7) and v splits 1, 3, 5
    (steps 6, 12, 18): 5.  Left-going u/v splits before step 7: steps 3, 5:
    2.  count = 1 + 18 + 5 + 2 = 26; T = 0.1001b = 0.5625.

    Case C, vertex-face: t digits 1111111 (t* = 0.994140625), u* = v* = 2^-8.
    Every t split goes right (7), the last at step 16; left-going u/v splits
    before it: steps 3, 5, 6, 8, 9, 11, 12, 14, 15: 9.
    count = 1 + 18 + 7 + 9 = 35; T = 127/128 = 0.9921875.

    Case D, edge-edge: t digits 0000000 (t* = 2^-9), u* = 0.111111b + 2^-8
    (every u split goes right), v* = 2^-8.  Right-going: the 6 u splits.
    No t split goes right, so no pending sibling is evaluated.
    count = 1 + 18 + 6 = 25; T = 0."""
    want = {
        "A": (0.28125, 0, 26),
        "B": (0.5625, 0, 26),
        "C": (0.9921875, 0, 35),
        "D": (0.0, 0, 25),
    }
    got = {
        "A": _count(True, *_query_vf([0, 1, 0, 0, 1, 0, 0], 2.0 ** -8, 2.0 ** -8), DELTA),
        "B": _count(False, *_query_ee([1, 0, 0, 1, 0, 0, 0], 2.0 ** -8, 0.65625 + 2.0 ** -8), DELTA),
        "C": _count(True, *_query_vf([1] * 7, 2.0 ** -8, 2.0 ** -8), DELTA),
        "D": _count(False, *_query_ee([0] * 7, 1 - 2.0 ** -6 + 2.0 ** -8, 2.0 ** -8), DELTA),
    }
    return got == want


def test_split_order_by_hand():
    got = {
        "A": _count(True, *_query_vf([0, 1, 0, 0, 1, 0, 0], 2.0 ** -8, 2.0 ** -8), DELTA),
        "B": _count(False, *_query_ee([1, 0, 0, 1, 0, 0, 0], 2.0 ** -8, 0.65625 + 2.0 ** -8), DELTA),
        "C": _count(True, *_query_vf([1] * 7, 2.0 ** -8, 2.0 ** -8), DELTA),
        "D": _count(False, *_query_ee([0] * 7, 1 - 2.0 ** -6 + 2.0 ** -8, 2.0 ** -8), DELTA),
    }
    assert got == {"A": (0.28125, 0, 26), "B": (0.5625, 0, 26), "C": (0.9921875, 0, 35),
                   "D": (0.0, 0, 25)}
    assert pin_split_order()
