"""The oracle's pins must catch plausible mistakes.  Each test plants one
mistake in a copy of the oracle source (a dropped term, a flipped sign, a
transposed operand, a wrong index, a missing error box, a wrong comparison,
a missing rounding step, a missing filter, a wrong split rule or split
weight), builds it on the CPU, and checks that a pin fails on it while the
same pin passes on the real oracle.

Also here: the error-box pin itself (the C_eps derivation), checked against
exact rational corner values."""
import os
import subprocess
import tempfile
from fractions import Fraction as Q

import numpy as np
import pytest

from oracle import exact as X
from oracle import oracle as O
from paper_2112_06300_gb300 import scenes
from tests.test_oracle_split import pin_split_order, pin_split_weights

SRC = os.path.join(os.path.dirname(O.__file__), "ccd_oracle.c")


def build_variant(old: str, new: str):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    open(c, "w").write(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                    "-o", so, c, "-lm"], check=True, capture_output=True)
    return O.load_variant(so)


# ---- pins, each returning True when it holds ------------------------------

def pin_conservative(n=300, seed=21):
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(n, seed=seed)
    sc, vf, ee, order = scenes.pack_queries(X0, X1, is_vf)
    tv, te, *_ = O.narrow(vf, ee, sc.V0, sc.V1, sc.E, sc.F)
    toi = np.empty(n)
    toi[order] = np.concatenate([tv, te])
    for q in np.nonzero(kind == scenes.KINDS.index("collide"))[0]:
        r = X.toi(bool(is_vf[q]), X0[q].tolist(), X1[q].tolist())
        if r is not None and not (np.isfinite(toi[q]) and X.le_float(toi[q], r)):
            return False
    return True


def exact_corner(vf, x0, x1, t, u, v):
    P = [[Q(x0[k][i]) + t * (Q(x1[k][i]) - Q(x0[k][i])) for i in range(3)] for k in range(4)]
    if vf:
        return [P[0][i] - P[1][i] - u * (P[2][i] - P[1][i]) - v * (P[3][i] - P[1][i]) for i in range(3)]
    return [P[0][i] + u * (P[1][i] - P[0][i]) - P[2][i] - v * (P[3][i] - P[2][i]) for i in range(3)]


def pin_error_box(trials=300, seed=22):
    """Exact hull of F over the interval (hull of the exact corners, since F
    is affine in each variable) lies within the computed box widened by the
    error box, on every axis."""
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        vf = bool(rng.integers(2))
        scale = 2.0 ** rng.integers(-20, 20)
        x0 = rng.uniform(-1, 1, (4, 3)) * scale
        x1 = x0 + rng.uniform(-1, 1, (4, 3)) * scale * rng.choice([1e-8, 1e-3, 1.0])
        lv = rng.integers(0, 30, 3)
        nv = np.array([rng.integers(0, 2 ** int(l)) for l in lv], np.uint64)
        bmin, bmax, ebox = O.inclusion(vf, x0, x1, nv, lv)
        ends = [[Q(int(nv[k]), 2 ** int(lv[k])), Q(int(nv[k]) + 1, 2 ** int(lv[k]))] for k in range(3)]
        vals = [exact_corner(vf, x0, x1, t, u, v) for t in ends[0] for u in ends[1] for v in ends[2]]
        for a in range(3):
            lo = min(c[a] for c in vals)
            hi = max(c[a] for c in vals)
            if lo < Q(bmin[a]) - Q(ebox[a]) or hi > Q(bmax[a]) + Q(ebox[a]):
                return False
    return True


def pin_brute_equals_sweep():
    s = scenes.icosphere_on_plane(0, level=2, plane_n=9)
    b = O.broad(s.V0, s.V1, s.E, s.F, "brute")
    w = O.broad(s.V0, s.V1, s.E, s.F, "sweep")
    return np.array_equal(b[0], w[0]) and np.array_equal(b[1], w[1])


def pin_tight_rounding():
    rng = np.random.default_rng(23)
    vals = rng.normal(0, 1, 400)
    V = np.stack([vals, -vals, vals], 1)
    lo64, hi64, lo32, hi32 = O.boxes(V, V, np.zeros((0, 2), np.int32), np.zeros((0, 3), np.int32))
    up = np.nextafter(lo32, np.float32(np.inf)).astype(np.float64)
    return bool(np.all(lo32.astype(np.float64) <= lo64) and np.all(up > lo64))


def pin_definition_pairs():
    from tests.test_oracle_broad import numpy_pairs, random_scene
    rng = np.random.default_rng(24)
    V0, V1, E, F = random_scene(rng, 40, 40, motion=0.6)
    ref = numpy_pairs(V0, V1, E, F)
    vf, ee = O.broad(V0, V1, E, F, "brute")
    return np.array_equal(vf, ref[0]) and np.array_equal(ee, ref[1])


MUTATIONS = [
    ("drop the v term (vertex-face)",
     "double g = fma(-vs[iv], c[2][x], c[0][x]);", "double g = c[0][x];", pin_conservative),
    ("flip the sign of the u term (edge-edge)",
     "double g = fma(us[iu], c[1][x], c[0][x]);", "double g = fma(-us[iu], c[1][x], c[0][x]);",
     pin_conservative),
    ("transpose the trajectory operands",
     "c[j][x] = fma(ts[it], q->dc[j][x], q->c0[j][x]);",
     "c[j][x] = fma(ts[it], q->c0[j][x], q->dc[j][x]);", pin_conservative),
    ("wrong vertex index for e2",
     "x_of[2] = ids[3]; y_of[2] = ids[1];", "x_of[2] = ids[2]; y_of[2] = ids[1];", pin_conservative),
    ("no error box",
     "q->ebox[x] = nextafter(eps + min_sep, INFINITY);", "q->ebox[x] = min_sep; (void)eps;",
     pin_error_box),
    ("error box one ulp short of the derivation",
     "double eps = m * 0x1.8p-48; /* 48 * 2^-53 */", "double eps = m * 0x1p-53;", pin_error_box),
    ("sweep stops at touching boxes",
     "if (use32 ? (lo32[3 * j + ax] > hi32[3 * i + ax]) : (lo64[3 * j + ax] > hi64[3 * i + ax]))",
     "if (use32 ? (lo32[3 * j + ax] >= hi32[3 * i + ax]) : (lo64[3 * j + ax] >= hi64[3 * i + ax]))",
     pin_brute_equals_sweep),
    ("no nextafterf step when rounding down",
     "if ((double)f > x) f = nextafterf(f, -INFINITY);", "(void)0;", pin_tight_rounding),
    ("shared-vertex filter missing",
     "if (shares_vertex(a, na, b, nb)) return 0;", "(void)shares_vertex;", pin_definition_pairs),
    ("split the axis of the smallest weight",
     "if (val > bestval) { best = k; bestval = val; }",
     "if (best < 0 || val < bestval) { best = k; bestval = val; }", pin_split_order),
    ("split weight without the 2^-l factor",
     "double val = ldexp(q->L[k], -I->l[k]);", "double val = q->L[k];", pin_split_order),
    ("ties go to the later axis",
     "if (val > bestval) { best = k; bestval = val; }",
     "if (val >= bestval) { best = k; bestval = val; }", pin_split_order),
    ("L_u built from e2",
     "double su = fmax(fabs(q->c0[1][x]), fabs(c1u));",
     "double su = fmax(fabs(q->c0[2][x]), fabs(c1v));", pin_split_weights),
    ("L_u at t = 0 only",
     "double su = fmax(fabs(q->c0[1][x]), fabs(c1u));",
     "double su = fabs(q->c0[1][x]); (void)c1u;", pin_split_weights),
    ("L_t from the positions instead of the displacements",
     "double st = fabs(q->dc[0][x]) + fabs(q->dc[1][x]);",
     "double st = fabs(q->c0[0][x]) + fabs(q->c0[1][x]);", pin_split_weights),
]


def test_error_box_bound_holds_on_real_oracle():
    assert pin_error_box(trials=600)


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(name, old, new, pin):
    assert pin(), f"pin fails on the real oracle: {name}"
    handle = build_variant(old, new)
    with O.using(handle):
        caught = not pin()
    assert caught, f"planted mistake not caught: {name}"
