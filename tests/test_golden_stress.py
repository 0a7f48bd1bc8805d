"""The stored exact times of the narrow-phase stress subset
(tests/golden/stress_exact_1e5.txt.gz, written by make_stress_exact.py with
the exact rational oracle only) against a fresh run of the same oracle.

Checks that the generator still produces the queries the file was made from
(SHA-256 of the subset's inputs), recomputes 300 seeded entries exactly and
compares them with the file, and checks the FP64 oracle on those queries:
never later than the exact time, and a collision wherever one exists."""
import numpy as np

from oracle import exact as X
from oracle import oracle as O
from paper_2112_06300_gb300 import scenes
from tests.golden import make_stress_exact as G


def test_stress_exact_file_matches_exact_oracle():
    head, idx, rd = G.read()
    assert len(idx) == G.SUBSET and np.all(np.diff(idx) > 0)
    assert np.array_equal(idx, G.subset_indices())
    X0, X1, is_vf, kind = scenes.narrow_stress_queries(G.N_QUERIES, G.GEN_SEED)
    assert head["sha256"] == G.fingerprint(X0, X1, is_vf, idx), "generator changed: regenerate the file"
    pick = np.random.default_rng(7).choice(len(idx), size=300, replace=False)
    q = idx[pick]
    for k, qq in zip(pick, q):
        r = X.toi(bool(is_vf[qq]), X0[qq].tolist(), X1[qq].tolist())
        if r is None:
            assert np.isnan(rd[k]), qq
        else:
            assert rd[k] == G._round_down(r), qq
    sc, vf, ee, order = scenes.pack_queries(X0[q], X1[q], is_vf[q])
    o = O.narrow(vf, ee, sc.V0, sc.V1, sc.E, sc.F, 1e-6, 0.0, 10 ** 6, 0)
    toi = np.empty(len(q))
    toi[order] = np.concatenate([o[0], o[1]])
    hit = ~np.isnan(rd[pick])
    assert np.all(np.isfinite(toi[hit])), "false negative of the FP64 oracle"
    assert np.all(toi[hit] <= rd[pick][hit]), "FP64 oracle later than the exact time"
