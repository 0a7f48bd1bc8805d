"""Seeded synthetic CCD inputs shaped like the paper's workloads.

This module only builds geometry and trajectories; it holds none of the
method's arithmetic and is shared by the tests, the benchmark and the oracle
checks.  Every array is float64 (positions) or int32 (topology):

    V0, V1  (nV, 3) vertex positions at t = 0 and t = 1
    E       (nE, 2) edges, F (nF, 3) triangles

The paper's six scenes (Section "Dataset Generation") are not available; these
stand in for them: a rigid body falling on a plane, a folded cloth pressed
into itself (like Cloth-Ball / Cloth-Funnel self contact), and standalone
narrow-phase queries with a controlled mix of generic, colliding, degenerate,
touching and near-miss cases.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field
from typing import Dict

import numpy as np


@dataclass
class Scene:
    V0: np.ndarray
    V1: np.ndarray
    E: np.ndarray
    F: np.ndarray
    info: Dict = field(default_factory=dict)

    @property
    def n_boxes(self) -> int:
        return len(self.V0) + len(self.E) + len(self.F)


def edges_of(F: np.ndarray) -> np.ndarray:
    """Unique undirected edges of a triangle list, sorted, as int32 (nE, 2)."""
    F = np.asarray(F, np.int64)
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
    e.sort(axis=1)
    e = np.unique(e, axis=0)
    return e.astype(np.int32)


def icosphere(level: int):
    """Unit icosphere by repeated 4-way subdivision of the icosahedron:
    10 * 4^level + 2 vertices, 20 * 4^level faces."""
    g = (1.0 + 5 ** 0.5) / 2.0
    V = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0),
         (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    Fl = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
          (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
          (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
          (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        for a, b, c in Fl:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        Fl = nf
    return np.array(V), np.array(Fl, np.int32)


def grid(n: int, x0: float, x1: float, y0: float, y1: float):
    """n x n vertex grid, two triangles per cell (same diagonal everywhere)."""
    xs = np.linspace(x0, x1, n)
    ys = np.linspace(y0, y1, n)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), np.zeros(n * n)], axis=1)
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    a = (i * n + j).ravel()
    b = a + n
    c = a + n + 1
    d = a + 1
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0).astype(np.int32)
    return V, F


def icosphere_on_plane(seed: int = 0, level: int = 4, plane_n: int = 33,
                       jitter: float = 1e-3) -> Scene:
    """Sphere falling onto a plane: icosphere (radius 0.5, centre z = 0.52,
    level 4: 2,562 V / 7,680 E / 5,120 F) translated by -0.1 in z, each sphere
    vertex offset by the same N(0, jitter^2) at t = 0 and t = 1; a static
    plane_n x plane_n grid on [-1, 1]^2 at z = 0.  21,635 boxes."""
    rng = np.random.default_rng(seed)
    Vs, Fs = icosphere(level)
    Vs = 0.5 * Vs + np.array([0.0, 0.0, 0.52])
    Vs = Vs + rng.normal(0.0, jitter, Vs.shape) if jitter > 0 else Vs
    Vp, Fp = grid(plane_n, -1.0, 1.0, -1.0, 1.0)
    V0 = np.concatenate([Vs, Vp], 0)
    V1 = np.concatenate([Vs + np.array([0.0, 0.0, -0.1]), Vp], 0)
    F = np.concatenate([Fs, Fp + len(Vs)], 0).astype(np.int32)
    E = edges_of(F)
    return Scene(V0, V1, E, F, {"name": "icosphere-on-plane", "level": level,
                                "plane_n": plane_n, "seed": seed})


def folded_cloth(n: int = 512, seed: int = 1, gap: float = 1e-3, n_waves: int = 8,
                 amplitude: float = 0.01, wavelength=(0.05, 0.5)) -> Scene:
    """Cloth self contact: an n x n grid on [0,1]^2 folded once along x = 0.5
    (x > 0.5 maps to (1 - x, y, gap)); the lower half moves by +s(x, y) in z and
    the upper half by -s(x, y), s a sum of n_waves seeded sinusoids (given
    amplitude, wavelength uniform in the range, random direction and phase),
    evaluated at the folded position.  n = 512: 262,144 V, 784,385 E,
    522,242 F."""
    rng = np.random.default_rng(seed)
    V, F = grid(n, 0.0, 1.0, 0.0, 1.0)
    upper = V[:, 0] > 0.5
    V0 = V.copy()
    V0[upper, 0] = 1.0 - V[upper, 0]
    V0[upper, 2] = gap
    lam = rng.uniform(wavelength[0], wavelength[1], n_waves)
    th = rng.uniform(0.0, 2 * np.pi, n_waves)
    ph = rng.uniform(0.0, 2 * np.pi, n_waves)
    x, y = V0[:, 0], V0[:, 1]
    s = np.zeros(len(V0))
    for k in range(n_waves):
        s += amplitude * np.sin(2 * np.pi * (x * np.cos(th[k]) + y * np.sin(th[k])) / lam[k] + ph[k])
    V1 = V0.copy()
    V1[:, 2] += np.where(upper, -s, s)
    E = edges_of(F)
    return Scene(V0, V1, E, F, {"name": "folded-cloth", "n": n, "seed": seed, "gap": gap})


# ---------------------------------------------------------------------------
# Standalone narrow-phase queries on a dyadic grid.
# ---------------------------------------------------------------------------

KINDS = ("generic", "collide", "degenerate", "touch", "near_miss")
MIX = (0.4, 0.2, 0.1, 0.1, 0.2)


def _grid_pts(rng, shape, bits=20, lim=1.0):
    k = 2 ** bits
    return rng.integers(-int(lim * k), int(lim * k) + 1, size=shape) / k


def _construct(rng, is_vf, tstar, m):
    """m queries that touch exactly at time tstar (a dyadic k / 2^10, or 0 or
    1): pick the contact configuration X* on the 2^-20 grid, displacements D on
    the 2^-10 grid, X0 = X* - tstar D, X1 = X0 + D (all exact)."""
    C = _grid_pts(rng, (m, 1, 3), 20, 0.5)
    if is_vf:
        R0 = 2 * _grid_pts(rng, (m, 1, 3), 20, 0.1)
        R1 = 2 * _grid_pts(rng, (m, 1, 3), 20, 0.1)
        R2 = -(R0 + R1) / 2            # barycentric (1/4, 1/4, 1/2) of the triangle is C
        star = np.concatenate([C, C + R0, C + R1, C + R2], axis=1)
    else:
        RA = _grid_pts(rng, (m, 1, 3), 20, 0.1)
        RB = _grid_pts(rng, (m, 1, 3), 20, 0.1)
        star = np.concatenate([C - RA, C + RA, C - RB, C + RB], axis=1)   # midpoints meet
    D = _grid_pts(rng, (m, 4, 3), 10, 0.25)
    ts = np.asarray(tstar, float).reshape(m, 1, 1)
    X0 = star - ts * D
    X1 = X0 + D
    return X0, X1


def _degenerate(rng, is_vf, m):
    """Coplanar for all t (vertex-face: all four points keep z = c) or parallel
    for all t (edge-edge: both edges along one fixed direction)."""
    if is_vf:
        X0 = _grid_pts(rng, (m, 4, 3), 20, 0.5)
        D = _grid_pts(rng, (m, 4, 3), 20, 0.5)
        c = _grid_pts(rng, (m, 1), 20, 0.5)
        X0[:, :, 2] = c
        D[:, :, 2] = 0.0
        return X0, X0 + D
    d = _grid_pts(rng, (m, 1, 3), 20, 0.25)
    A0 = _grid_pts(rng, (m, 1, 3), 20, 0.5)
    B0 = _grid_pts(rng, (m, 1, 3), 20, 0.5)
    a = rng.integers(1, 3, (m, 1, 1)) / 2.0
    b = rng.integers(1, 3, (m, 1, 1)) / 2.0
    X0 = np.concatenate([A0, A0 + a * d, B0, B0 + b * d], axis=1)
    shift = _grid_pts(rng, (m, 4, 3), 20, 0.25)
    shift[:, 1] = shift[:, 0]
    shift[:, 3] = shift[:, 2]
    return X0, X0 + shift


def _near_miss(rng, is_vf, m):
    """Separated by s = 2^-j, j in [30, 40], for all t: the primitives lie in
    parallel planes z = c and z = c + s (off the 2^-20 grid by s)."""
    s = 2.0 ** -rng.integers(30, 41, (m, 1)).astype(float)
    c = _grid_pts(rng, (m, 1), 20, 0.5)
    X0 = _grid_pts(rng, (m, 4, 3), 20, 0.5)
    D = _grid_pts(rng, (m, 4, 3), 20, 0.5)
    D[:, :, 2] = 0.0
    if is_vf:     # point above the triangle's plane
        X0[:, 0, 2] = (c + s)[:, 0]
        X0[:, 1:, 2] = c
    else:         # first edge above the second
        X0[:, :2, 2] = c + s
        X0[:, 2:, 2] = c
    return X0, X0 + D


def narrow_stress_queries(n: int, seed: int = 2):
    """n standalone queries, half vertex-face and half edge-edge, mixed
    40/20/10/10/20 % generic / collide at a seeded dyadic t* / coplanar or
    parallel / touching at t = 0 or 1 / near miss at 2^-30..2^-40; counts are
    floor(p n) per kind, the remainder generic.  Returns (X0, X1, is_vf, kind)
    with X0, X1 of shape (n, 4, 3) (vertex-face: P, T0, T1, T2; edge-edge: A0,
    A1, B0, B1) and kind an index into KINDS."""
    rng = np.random.default_rng(seed)
    counts = [int(np.floor(p * n)) for p in MIX]
    counts[0] += n - sum(counts)
    kind = np.concatenate([np.full(c, k, np.int8) for k, c in enumerate(counts)])
    rng.shuffle(kind)
    is_vf = np.zeros(n, bool)
    is_vf[rng.permutation(n)[: n // 2]] = True
    X0 = np.empty((n, 4, 3))
    X1 = np.empty((n, 4, 3))
    for k in range(len(KINDS)):
        for vf in (True, False):
            idx = np.nonzero((kind == k) & (is_vf == vf))[0]
            m = len(idx)
            if m == 0:
                continue
            if KINDS[k] == "generic":
                a, b = _grid_pts(rng, (m, 4, 3)), _grid_pts(rng, (m, 4, 3))
            elif KINDS[k] == "collide":
                a, b = _construct(rng, vf, rng.integers(1, 1024, m) / 1024.0, m)
            elif KINDS[k] == "touch":
                a, b = _construct(rng, vf, rng.integers(0, 2, m).astype(float), m)
            elif KINDS[k] == "degenerate":
                a, b = _degenerate(rng, vf, m)
            else:
                a, b = _near_miss(rng, vf, m)
            X0[idx], X1[idx] = a, b
    return X0, X1, is_vf, kind


def pack_queries(X0, X1, is_vf):
    """Lay standalone queries out as one mesh: query q owns vertices 4q..4q+3;
    a vertex-face query becomes face (4q+1, 4q+2, 4q+3) and pair (4q, face),
    an edge-edge query edges (4q, 4q+1), (4q+2, 4q+3) and their pair.
    Returns (Scene, vf_pairs, ee_pairs, order) where order maps the stacked
    [vf..., ee...] query list back to input positions."""
    n = len(is_vf)
    V0 = X0.reshape(-1, 3).copy()
    V1 = X1.reshape(-1, 3).copy()
    base = 4 * np.arange(n, dtype=np.int64)
    ivf = np.nonzero(is_vf)[0]
    iee = np.nonzero(~is_vf)[0]
    F = np.stack([base[ivf] + 1, base[ivf] + 2, base[ivf] + 3], 1).astype(np.int32)
    vf = np.stack([base[ivf], np.arange(len(ivf))], 1).astype(np.int32)
    E = np.empty((2 * len(iee), 2), np.int32)
    E[0::2] = np.stack([base[iee], base[iee] + 1], 1)
    E[1::2] = np.stack([base[iee] + 2, base[iee] + 3], 1)
    ee = np.stack([2 * np.arange(len(iee)), 2 * np.arange(len(iee)) + 1], 1).astype(np.int32)
    order = np.concatenate([ivf, iee])
    return Scene(V0, V1, E, F, {"name": "standalone-queries", "n": n}), vf, ee, order


# ---------------------------------------------------------------------------
# Batched rigid-body environments.
# ---------------------------------------------------------------------------

def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.35):
    """Torus with nu x nv quads (2 * nu * nv triangles)."""
    u = np.arange(nu) * 2 * np.pi / nu
    v = np.arange(nv) * 2 * np.pi / nv
    U, W = np.meshgrid(u, v, indexing="ij")
    V = np.stack([(R + r * np.cos(W)) * np.cos(U), (R + r * np.cos(W)) * np.sin(U), r * np.sin(W)], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a = (i * nv + j).ravel()
    b = (((i + 1) % nu) * nv + j).ravel()
    c = (((i + 1) % nu) * nv + (j + 1) % nv).ravel()
    d = (i * nv + (j + 1) % nv).ravel()
    F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)], 0).astype(np.int32)
    return V, F


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


@functools.lru_cache(maxsize=None)
def _body(kind: str, k: int):
    """Template body (vertices, faces, edges), built once: kind 'ico' with
    subdivision level k, or 'torus' with k x max(4, k // 2) quads (scaled by
    1 / 1.35 to about unit radius)."""
    if kind == "ico":
        V, F = icosphere(k)
    else:
        V, F = torus(k, max(4, k // 2))
        V = V / 1.35
    V.setflags(write=False)
    F.setflags(write=False)
    E = edges_of(F)
    E.setflags(write=False)
    return V, F, E


def rigid_environment(seed: int, tri_lo: float = 500, tri_hi: float = 50000, vmax: float = 0.05) -> Scene:
    """One environment: rigid icospheres (levels 1-3) and tori added until a
    total triangle count drawn log-uniformly from [tri_lo, tri_hi] is reached,
    randomly placed, rotated and scaled (0.2-0.5) in a cube sized for about one
    body diameter between neighbours, each translated by a random velocity of
    norm <= vmax over the step."""
    rng = np.random.default_rng(seed)
    target = float(np.exp(rng.uniform(np.log(tri_lo), np.log(tri_hi))))
    bodies = []
    total = 0
    while total < target or not bodies:
        if rng.random() < 0.5:
            b = _body("ico", int(rng.integers(1, 4)))
        else:
            b = _body("torus", int(rng.integers(6, 25)))
        bodies.append(b)
        total += len(b[1])
    nb = len(bodies)
    side = max(1.0, 1.1 * nb ** (1.0 / 3.0))
    Vs0, Vs1, Fs, Es = [], [], [], []
    off = 0
    for Vb, Fb, Eb in bodies:
        Rm = _random_rotation(rng)
        sc = rng.uniform(0.2, 0.5)
        pos = rng.uniform(0, side, 3)
        vel = rng.normal(size=3)
        vel *= rng.uniform(0, vmax) / max(np.linalg.norm(vel), 1e-12)
        P = (Vb @ Rm.T) * sc + pos
        Vs0.append(P)
        Vs1.append(P + vel)
        Fs.append(Fb + off)
        Es.append(Eb + off)
        off += len(Vb)
    V0 = np.concatenate(Vs0, 0)
    V1 = np.concatenate(Vs1, 0)
    F = np.concatenate(Fs, 0).astype(np.int32)
    # bodies own disjoint, increasing vertex ranges: the per-body sorted edge
    # lists concatenate to the sorted edge list of the whole environment
    E = np.concatenate(Es, 0).astype(np.int32)
    return Scene(V0, V1, E, F, {"name": "rigid-environment", "seed": seed, "bodies": nb,
                                "triangles": len(F)})


def concat_scenes(scs):
    """Concatenate scenes for a batched step: vertex ids of edges and faces are
    shifted to global ids; returns (V0, V1, E, F, vert_off, edge_off,
    face_off) with the offsets as int64 arrays of len(scs) + 1."""
    voff = np.zeros(len(scs) + 1, np.int64)
    eoff = np.zeros(len(scs) + 1, np.int64)
    foff = np.zeros(len(scs) + 1, np.int64)
    for k, s in enumerate(scs):
        voff[k + 1] = voff[k] + len(s.V0)
        eoff[k + 1] = eoff[k] + len(s.E)
        foff[k + 1] = foff[k] + len(s.F)
    V0 = np.concatenate([s.V0 for s in scs], 0) if scs else np.zeros((0, 3))
    V1 = np.concatenate([s.V1 for s in scs], 0) if scs else np.zeros((0, 3))
    E = np.concatenate([s.E.astype(np.int64) + voff[k] for k, s in enumerate(scs)], 0).astype(np.int32)
    F = np.concatenate([s.F.astype(np.int64) + voff[k] for k, s in enumerate(scs)], 0).astype(np.int32)
    return V0, V1, E.reshape(-1, 2), F.reshape(-1, 3), voff, eoff, foff


def cloth_and_bodies(n: int = 512, n_ico: int = 500, n_torus: int = 500, seed: int = 1, body_seed: int = 0,
                     min_gap: float = 0.01) -> Scene:
    """The folded cloth plus rigid bodies: n_ico icospheres (level 4, 5,120
    triangles) and n_torus tori (48 x 32 quads, 3,072 triangles) placed
    uniformly in [0, 10]^3 with random rotation and scale 0.2-0.5, each
    translated by U(-0.02, 0.02)^3 over the step (500 + 500 bodies: 4,096,000
    body triangles).  Placement is by rejection: a body's bounding sphere
    (radius = its scale) keeps min_gap from every earlier body's sphere and
    from the cloth's slab [0, 1]^2 x [-0.03, 0.03], so nothing interpenetrates
    at t = 0 and the narrow phase has real work (bodies that come within the
    step's relative motion can still collide)."""
    cl = folded_cloth(n, seed=seed)
    rng = np.random.default_rng(body_seed)
    ico = _body("ico", 4)
    Vt, Ft = torus(48, 32)
    Vt = Vt / 1.35
    tor = (Vt, Ft, edges_of(Ft))
    Vs0, Vs1, Fs, Es = [cl.V0], [cl.V1], [cl.F], [cl.E]
    off = len(cl.V0)
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    for Vb, Fb, Eb in [ico] * n_ico + [tor] * n_torus:
        Rm = _random_rotation(rng)
        sc = rng.uniform(0.2, 0.5)
        while True:
            pos = rng.uniform(0.0, 10.0, 3)
            # distance from the sphere's centre to the cloth slab
            q = np.clip(pos, [0.0, 0.0, -0.03], [1.0, 1.0, 0.03])
            if np.linalg.norm(pos - q) < sc + min_gap:
                continue
            if len(radii) and np.any(np.linalg.norm(centres - pos, axis=1) < radii + sc + min_gap):
                continue
            break
        centres = np.vstack([centres, pos])
        radii = np.append(radii, sc)
        d = rng.uniform(-0.02, 0.02, 3)
        P = (Vb @ Rm.T) * sc + pos
        Vs0.append(P)
        Vs1.append(P + d)
        Fs.append(Fb + off)
        Es.append(Eb + off)
        off += len(Vb)
    return Scene(np.concatenate(Vs0, 0), np.concatenate(Vs1, 0), np.concatenate(Es, 0).astype(np.int32),
                 np.concatenate(Fs, 0).astype(np.int32),
                 {"name": "cloth-and-bodies", "n": n, "icospheres": n_ico, "tori": n_torus})
