"""CPU tests of the autotuner's learned performance model (regression trees).

Pinned against brute force (the squared-error split chosen by the tree is the
best of all candidate splits, enumerated here), exact interpolation of
training data by an unrestricted tree, a step function whose threshold is
known, and the selection quality on a synthetic performance surface whose
best variant per shape is known in closed form.
"""
import itertools

import numpy as np
import pytest

from paper_1910_04796_gb300 import perfmodel as P


def test_q_and_lane_fill():
    assert [P.q_of(x) for x in (1, 32, 33, 64, 65, 128, 129, 256, 257, 512, 513, 1024)] == \
        [1, 1, 2, 2, 4, 4, 8, 8, 16, 16, 16, 16]
    f = dict(zip(P.FEATURES, P.features(13, 23, 5, 2)))
    # 299 elements: 10 per lane (lanes 12..31 hold 9), issued in 5 groups of 2
    assert f["mn"] == 299 and f["q"] == 16 and f["passes"] == 1
    assert f["lane_fill"] == pytest.approx(299 / 320)
    # 32 x 32: two passes of 16 per lane, every slot used; 5 x 5: one group of one
    assert P.issued_slots(1024, 16) == 1024 and P.issued_slots(25, 1) == 32
    assert P.issued_slots(17 * 32 + 1, 16) == 32 * 16 + 32 * 2   # second pass: 33 elements, one group of two
    assert f["team_warps"] == 2 and f["cta_threads"] == 256 and f["teams_per_cta"] == 4
    assert f["bytes_per_product"] == 8 * (13 * 5 + 5 * 23)


def test_full_tree_interpolates_training_data():
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 1, (60, 3))
    y = rng.normal(size=60)
    t = P.RegressionTree(max_depth=64, min_leaf=1).fit(X, y)
    assert np.array_equal(t.predict(X), y)


def test_step_threshold():
    X = np.arange(8, dtype=float)[:, None]
    y = (X[:, 0] > 3).astype(float) * 5.0
    t = P.RegressionTree(max_depth=1).fit(X, y)
    assert t.root.feature == 0 and t.root.threshold == pytest.approx(3.5)
    assert np.array_equal(t.predict(np.array([[0.0], [3.2], [3.8], [9.0]])), [0, 0, 5, 5])


def test_root_split_is_brute_force_optimum():
    rng = np.random.default_rng(1)
    X = rng.integers(0, 6, (40, 3)).astype(float)
    y = X[:, 1] * 2.0 + rng.normal(0, 0.3, 40)
    t = P.RegressionTree(max_depth=1, min_leaf=2).fit(X, y)
    best = np.inf
    for f in range(3):
        for thr in np.unique(X[:, f])[:-1] + 0.5:
            L, R = y[X[:, f] <= thr], y[X[:, f] > thr]
            if len(L) < 2 or len(R) < 2:
                continue
            best = min(best, ((L - L.mean()) ** 2).sum() + ((R - R.mean()) ** 2).sum())
    m = X[:, t.root.feature] <= t.root.threshold
    got = ((y[m] - y[m].mean()) ** 2).sum() + ((y[~m] - y[~m].mean()) ** 2).sum()
    assert got == pytest.approx(best, rel=1e-12)


def _synthetic_perf(m, n, k, v):
    # a made-up GPU: wider teams pay off for long inner products of small C
    # blocks; TFLOP/s grows with the lane fill
    f = dict(zip(P.FEATURES, P.features(m, n, k, v)))
    base = 0.2 + 0.8 * f["lane_fill"] * min(1.0, f["mnk"] / 4000.0)
    if v in (2, 3):
        base *= (1.0 + 0.02 * f["k_per_warp"]) if f["mn"] <= 128 else 0.8
    return base


def test_forest_picks_best_variant_on_unseen_shapes():
    sizes = (2, 4, 5, 8, 9, 13, 16, 22, 23, 26, 29, 32)
    shapes = list(itertools.product(sizes, sizes, sizes))
    rng = np.random.default_rng(2)
    rng.shuffle(shapes)
    train, test = shapes[: len(shapes) // 5], shapes[len(shapes) // 5:]
    recs = [(m, n, k, v, _synthetic_perf(m, n, k, v)) for (m, n, k) in train for v in range(4)]
    model = P.PerfModel(P.RandomForest(n_trees=20, seed=3)).fit(recs)
    measured = {s: {v: _synthetic_perf(*s, v) for v in range(4)} for s in test}
    chosen = {s: model.best_variant(*s) for s in test}
    q = P.choice_quality(measured, chosen)
    assert q["mean_of_best"] > 0.97
    assert q["within_5pct"] > 0.9
    # the fixed default (variant 0) is clearly worse on this surface
    q0 = P.choice_quality(measured, {s: 0 for s in test})
    assert q0["mean_of_best"] < q["mean_of_best"]


def test_table_format():
    recs = [(m, n, 8, v, float(v == (m % 4))) for m in (4, 8) for n in (4, 8) for v in range(4)]
    model = P.PerfModel(P.RandomForest(n_trees=5, seed=0)).fit(recs)
    tab = model.table((4, 8), (4, 8), (8,))
    assert len(tab) == 4 and all(len(e) == 4 and 0 <= e[2] < 4 for e in tab)


def test_choice_quality_arithmetic():
    measured = {(1, 1, 1): {0: 1.0, 1: 2.0}, (2, 2, 2): {0: 3.0, 1: 1.5}}
    q = P.choice_quality(measured, {(1, 1, 1): 0, (2, 2, 2): 0})
    assert q["mean_of_best"] == pytest.approx(0.75) and q["min_of_best"] == pytest.approx(0.5)
    assert q["optimal"] == 0.5 and q["within_5pct"] == 0.5


def test_table_mnk_matches_best_variant():
    # per-(m, n, k) entries are the model's argmax on every shape; the (m, n)
    # table averages over k and can differ from them
    sizes = (4, 8, 16, 32)
    recs = [(m, n, k, v, _synthetic_perf(m, n, k, v)) for m in sizes for n in sizes for k in sizes
            for v in range(4)]
    model = P.PerfModel(P.RandomForest(n_trees=5, seed=1)).fit(recs)
    tab = model.table_mnk((4, 13), (8,), (2, 32))
    assert [e[:3] for e in tab] == [(4, 8, 2), (4, 8, 32), (13, 8, 2), (13, 8, 32)]
    for (m, n, k, v, t) in tab:
        assert v == model.best_variant(m, n, k)
        assert t == pytest.approx(model.predict(m, n, k).max())


def test_mnk_table_string_roundtrip():
    from paper_1910_04796_gb300 import autotune
    E = 5
    rng = np.random.default_rng(4)
    entries = [(m, n, k, int(rng.integers(0, 4))) for m in range(1, E + 1) for n in range(1, E + 1)
               for k in range(1, E + 1)]
    code = autotune.encode_mnk(entries, E)
    assert len(code) == E ** 3 and set(code) <= set("0123")
    # the stated index: ((m-1)*E + (n-1))*E + (k-1)
    m, n, k, v = entries[37]
    assert code[((m - 1) * E + (n - 1)) * E + (k - 1)] == str(v)
    assert autotune.decode_mnk(code, E) == entries


def test_shipped_tables_follow_from_their_records():
    # the GB300 model file keeps the timed training records; refitting the
    # performance model on them (no GPU) gives the very tables the file ships
    import json
    from paper_1910_04796_gb300 import autotune
    with open(autotune.MODEL_TABLE) as f:
        d = json.load(f)
    recs = [tuple(r) for r in d["records"]]
    assert len(recs) == 4 * d["report"]["timed_for_training"]
    E = int(d["variants_mnk"]["max_edge"])
    entries, entries_mnk, _, _ = autotune.model_tune(d["report"]["sizes"], d["report"]["train_frac"], 3, E, False,
                                                     recs=recs)
    assert [e[:3] for e in entries] == [e[:3] for e in d["entries"]]
    assert autotune.encode_mnk(entries_mnk, E) == d["variants_mnk"]["variants"]
