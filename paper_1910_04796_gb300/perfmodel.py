"""Learned performance model of the FP64 stack kernels: regression trees.

The paper's LIBCUSMM cannot time every parameter combination of every
requestable (m, n, k) kernel, so it times a subset and predicts the rest with
a performance model built from regression trees over hand-engineered
features of the matrix dimensions, the kernel parameters and the GPU's
constraints (Sec. II). This module does the same for this library's FP64
stack kernels: a record is (m, n, k, variant, measured TFLOP/s); a random
forest of CART regression trees (bootstrap samples, random feature subsets,
squared-error splits) learns TFLOP/s from the features below, and the
variant with the highest prediction is chosen for shapes never timed.

Everything here is host-side numpy; the measurements come from
``autotune.measure`` (the library's own CUDA-event kernel timer).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# (warps per C block, threads per CTA) of the FP64 stack-kernel variants
# (dbcsr_opts.kernel = variant + 1); variant 1 runs as variant 0 (the single
# persistent launch has 256-thread CTAs)
VARIANTS = ((1, 256), (1, 256), (2, 256), (4, 256))
FEATURES = ("m", "n", "k", "mn", "mnk", "q", "lane_fill", "passes", "team_warps", "cta_threads",
            "teams_per_cta", "k_per_warp", "bytes_per_product", "flops_per_byte", "regs_class",
            "acc_per_lane")
Q_MAX = 16          # elements per lane of the largest kernel instance
GROUP = 2           # elements per inner-loop group (FMAs issue for whole groups)


def q_of(mn: int) -> int:
    """Elements per lane the kernel instantiates for an m*n C block: 1, 2, 4, 8, 16."""
    q = (mn + 31) // 32
    for c in (1, 2, 4, 8):
        if q <= c:
            return c
    return Q_MAX


def issued_slots(mn: int, q: int) -> int:
    """Lane slots of the FMAs issued per inner step over the whole C block:
    each pass covers up to 32 q elements, in groups of GROUP per lane."""
    slots, e0 = 0, 0
    while e0 < mn:
        nq = min(q, -(-(mn - e0) // 32))
        g = min(GROUP, q)
        slots += 32 * g * -(-nq // g)
        e0 += 32 * q
    return slots


def features(m: int, n: int, k: int, variant: int) -> np.ndarray:
    """Hand-engineered features of one (shape, variant) pair."""
    w, t = VARIANTS[variant]
    mn = m * n
    q = q_of(mn)
    passes = math.ceil(mn / (32 * q))          # sweeps of the lane grid over the C block
    lane_fill = mn / issued_slots(mn, q)       # useful fraction of the issued lane slots
    bytes_pp = 8.0 * (m * k + k * n)           # A and B block per product
    return np.array([
        m, n, k, mn, mn * k, q, lane_fill, passes, w, t, t // (32 * w), k / w, bytes_pp,
        2.0 * mn * k / bytes_pp, math.log2(q), q * passes,
    ], dtype=np.float64)


def feature_matrix(records) -> tuple[np.ndarray, np.ndarray]:
    """records: iterable of (m, n, k, variant, tflops) -> X, y."""
    rec = list(records)
    X = np.array([features(int(r[0]), int(r[1]), int(r[2]), int(r[3])) for r in rec], dtype=np.float64)
    y = np.array([float(r[4]) for r in rec], dtype=np.float64)
    return X, y


# ------------------------------------------------------------------ CART tree
@dataclass
class _Node:
    value: float
    feature: int = -1
    threshold: float = 0.0
    left: "._Node | None" = None
    right: "._Node | None" = None


def _best_split(X, y, feats, min_leaf):
    """Split (feature, threshold) minimising the summed squared error of the two children."""
    n = len(y)
    best = (None, None, np.inf)
    for f in feats:
        order = np.argsort(X[:, f], kind="stable")
        xs, ys = X[order, f], y[order]
        csum = np.cumsum(ys)
        csq = np.cumsum(ys * ys)
        tot, totsq = csum[-1], csq[-1]
        # candidate cut after position i (left = 0..i): between distinct values only
        i = np.arange(min_leaf - 1, n - min_leaf)
        if len(i) == 0:
            continue
        ok = xs[i] < xs[i + 1]
        i = i[ok]
        if len(i) == 0:
            continue
        nl = i + 1.0
        nr = n - nl
        sl, sr = csum[i], tot - csum[i]
        sse = (csq[i] - sl * sl / nl) + ((totsq - csq[i]) - sr * sr / nr)
        j = int(np.argmin(sse))
        if sse[j] < best[2] - 1e-12:
            best = (f, 0.5 * (xs[i[j]] + xs[i[j] + 1]), sse[j])
    return best


class RegressionTree:
    """CART regression tree: greedy binary splits on squared error, leaf = mean."""

    def __init__(self, max_depth: int = 12, min_leaf: int = 1, max_features: int | None = None, seed: int = 0):
        self.max_depth = max_depth
        self.min_leaf = max(1, min_leaf)
        self.max_features = max_features
        self.rng = np.random.default_rng(seed)
        self.root: _Node | None = None

    def fit(self, X: np.ndarray, y: np.ndarray) -> "RegressionTree":
        X = np.asarray(X, np.float64)
        y = np.asarray(y, np.float64)
        self.root = self._grow(X, y, 0)
        self._flatten()
        return self

    def _flatten(self):
        """Node arrays for vectorised prediction (feature -1 marks a leaf)."""
        feat, thr, left, right, val = [], [], [], [], []
        stack = [(self.root, -1, False)]
        while stack:
            nd, parent, is_right = stack.pop()
            k = len(feat)
            feat.append(nd.feature)
            thr.append(nd.threshold)
            left.append(k)
            right.append(k)
            val.append(nd.value)
            if parent >= 0:
                (right if is_right else left)[parent] = k
            if nd.feature >= 0:
                stack.append((nd.right, k, True))
                stack.append((nd.left, k, False))
        self._feat = np.array(feat, np.int64)
        self._thr = np.array(thr, np.float64)
        self._left = np.array(left, np.int64)
        self._right = np.array(right, np.int64)
        self._val = np.array(val, np.float64)

    def _grow(self, X, y, depth):
        node = _Node(float(np.mean(y)))
        if depth >= self.max_depth or len(y) < 2 * self.min_leaf or np.all(y == y[0]):
            return node
        nf = X.shape[1]
        if self.max_features and self.max_features < nf:
            feats = self.rng.choice(nf, self.max_features, replace=False)
        else:
            feats = range(nf)
        f, thr, sse = _best_split(X, y, feats, self.min_leaf)
        if f is None:
            return node
        mask = X[:, f] <= thr
        node.feature, node.threshold = int(f), float(thr)
        node.left = self._grow(X[mask], y[mask], depth + 1)
        node.right = self._grow(X[~mask], y[~mask], depth + 1)
        return node

    def predict(self, X: np.ndarray) -> np.ndarray:
        X = np.atleast_2d(np.asarray(X, np.float64))
        idx = np.zeros(len(X), np.int64)
        rows = np.arange(len(X))
        while True:
            f = self._feat[idx]
            inner = f >= 0
            if not inner.any():
                return self._val[idx]
            go_left = X[rows, np.where(inner, f, 0)] <= self._thr[idx]
            idx = np.where(inner, np.where(go_left, self._left[idx], self._right[idx]), idx)


class RandomForest:
    """Average of regression trees grown on bootstrap samples with random feature subsets."""

    def __init__(self, n_trees: int = 40, max_depth: int = 12, min_leaf: int = 2, max_features: int | None = 6,
                 seed: int = 0):
        self.n_trees, self.max_depth, self.min_leaf, self.max_features = n_trees, max_depth, min_leaf, max_features
        self.seed = seed
        self.trees: list[RegressionTree] = []

    def fit(self, X, y) -> "RandomForest":
        X = np.asarray(X, np.float64)
        y = np.asarray(y, np.float64)
        rng = np.random.default_rng(self.seed)
        self.trees = []
        for t in range(self.n_trees):
            idx = rng.integers(0, len(y), len(y))
            tree = RegressionTree(self.max_depth, self.min_leaf, self.max_features, seed=self.seed * 1000 + t)
            self.trees.append(tree.fit(X[idx], y[idx]))
        return self

    def predict(self, X) -> np.ndarray:
        return np.mean([t.predict(X) for t in self.trees], axis=0)


# ------------------------------------------------------------ the tuner's model
@dataclass
class PerfModel:
    """TFLOP/s of (m, n, k, variant) learned from measured records."""
    forest: RandomForest = field(default_factory=RandomForest)

    def fit(self, records) -> "PerfModel":
        X, y = feature_matrix(records)
        self.forest.fit(X, y)
        return self

    def predict(self, m: int, n: int, k: int) -> np.ndarray:
        """Predicted TFLOP/s of every variant for one shape."""
        X = np.stack([features(m, n, k, v) for v in range(len(VARIANTS))])
        return self.forest.predict(X)

    def best_variant(self, m: int, n: int, k: int) -> int:
        return int(np.argmax(self.predict(m, n, k)))

    def table(self, msizes, nsizes, ksizes) -> list[tuple[int, int, int, float]]:
        """(m, n, variant, predicted TFLOP/s) entries for dbcsr_set_tuning; the kernel is
        chosen per C-block shape (m, n), so the prediction is averaged over the inner sizes k."""
        out = []
        nv = len(VARIANTS)
        for m in msizes:
            for n in nsizes:
                X = np.stack([features(int(m), int(n), int(k), v) for k in ksizes for v in range(nv)])
                p = self.forest.predict(X).reshape(len(ksizes), nv).mean(axis=0)
                out.append((int(m), int(n), int(np.argmax(p)), float(p.max())))
        return out

    def table_mnk(self, msizes, nsizes, ksizes) -> list[tuple[int, int, int, int, float]]:
        """(m, n, k, variant, predicted TFLOP/s) entries for dbcsr_set_tuning_mnk: the
        predicted best variant of every (m, n, k) shape."""
        nv = len(VARIANTS)
        shapes = [(int(m), int(n), int(k)) for m in msizes for n in nsizes for k in ksizes]
        X = np.stack([features(m, n, k, v) for (m, n, k) in shapes for v in range(nv)])
        p = self.forest.predict(X).reshape(len(shapes), nv)
        return [(m, n, k, int(np.argmax(p[i])), float(p[i].max())) for i, (m, n, k) in enumerate(shapes)]


def choice_quality(measured: dict, chosen: dict) -> dict:
    """How good a per-shape choice is against the measured optimum.

    measured: {(m, n, k): {variant: tflops}}; chosen: {(m, n, k): variant}.
    Returns the mean and minimum of (TFLOP/s of the choice) / (best TFLOP/s),
    and the fraction of shapes where the choice is optimal, or within 5 %.
    """
    ratios, exact, near = [], 0, 0
    for shape, perf in measured.items():
        best = max(perf.values())
        got = perf[chosen[shape]]
        r = got / best if best > 0 else 1.0
        ratios.append(r)
        exact += int(got >= best)
        near += int(r >= 0.95)
    n = max(1, len(ratios))
    return {"shapes": len(ratios), "mean_of_best": float(np.mean(ratios)) if ratios else 1.0,
            "min_of_best": float(np.min(ratios)) if ratios else 1.0, "optimal": exact / n, "within_5pct": near / n}
