"""Learned per-mode solver-and-tile selector (Sec. IV, with an MLP in place of
the paper's decision tree).

Every step here is a call into the CUDA library: features come from
``atucker_mode_features``, the network is trained on the GPU by
``atucker_mlp_train`` (the project's own forward/backward/Adam kernels), and
plans created with solver ``AUTO`` run the library's host-side inference
(``atucker_selector_predict``).  This module only marshals data.

Labels are measured with the library's own kernels: for each shape, every mode is timed under
every class (CUDA events around each mode inside the plan), and the network
learns, per class, y = log2(t_class / t_fastest) (capped at 4, i.e. 16x).  The
selector takes the class with the smallest prediction.

``python -m paper_2010_10131_b300.selector collect`` measures the timing set on
the current GPU; ``... train`` fits the network and writes the weights that
``install()`` loads.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import time

import numpy as np

from . import (AUTO, NUM_CLASSES, CLASS_NAMES, SELECTOR_FEATURES, SELECTOR_HIDDEN, Plan, _check, _i32arr, _i64arr,
               lib)

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "selector_weights.json")
TIMINGS = os.path.join(HERE, "selector_timings.json")
TARGET_CAP = 4.0  # log2 of the largest slowdown the network is asked to resolve


# ---------------------------------------------------------------- features
def mode_features(dims, ranks, mode_order=None) -> np.ndarray:
    """Model inputs (log2, not standardised) of every mode: (N, 12), row n = mode n."""
    n = len(dims)
    out = np.zeros(n * SELECTOR_FEATURES)
    mo = _i32arr(mode_order) if mode_order is not None else None
    _check(lib().atucker_mode_features(n, _i64arr(dims), _i64arr(ranks), mo,
                                       out.ctypes.data_as(ctypes.c_void_p)), "atucker_mode_features")
    return out.reshape(n, SELECTOR_FEATURES)


def targets(times: np.ndarray):
    """Per-row log2 slowdown vs the fastest measured class, and its mask."""
    t = np.asarray(times, dtype=np.float64)
    mask = np.isfinite(t) & (t > 0)
    best = np.where(mask, t, np.inf).min(axis=1, keepdims=True)
    y = np.where(mask, np.log2(np.where(mask, t, 1.0) / best), 0.0)
    return np.minimum(y, TARGET_CAP), mask.astype(np.float64)


# ------------------------------------------------------------------ network
def param_count(n_in=SELECTOR_FEATURES, hidden=SELECTOR_HIDDEN, n_out=NUM_CLASSES) -> int:
    return int(lib().atucker_mlp_param_count(n_in, hidden, n_out))


def init_params(seed: int = 0, n_in=SELECTOR_FEATURES, hidden=SELECTOR_HIDDEN, n_out=NUM_CLASSES) -> np.ndarray:
    """He-normal weights, zero biases (float32, the layout of atucker_mlp_param_count)."""
    g = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((n_in, hidden), (hidden, hidden), (hidden, n_out)):
        parts.append(g.standard_normal(fan_out * fan_in) * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


class GpuMLP:
    """Device-resident network trained by the library's kernels."""

    def __init__(self, params: np.ndarray, n_in=SELECTOR_FEATURES, hidden=SELECTOR_HIDDEN, n_out=NUM_CLASSES):
        import torch
        self.torch = torch
        self.shape = (n_in, hidden, n_out)
        self.params = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).cuda()
        self.state = torch.zeros(2 * self.params.numel(), device="cuda")
        self.steps = 0

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _dev(self, a):
        t = self.torch
        return a if isinstance(a, t.Tensor) else t.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()

    def forward(self, X) -> np.ndarray:
        X = self._dev(X)
        B = X.shape[0]
        out = self.torch.empty(B, self.shape[2], device="cuda")
        _check(lib().atucker_mlp_forward(ctypes.c_void_p(X.data_ptr()), B, *self.shape,
                                         ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         self._stream()), "atucker_mlp_forward")
        return out.cpu().numpy()

    def loss_grad(self, X, Y, M):
        X, Y, M = self._dev(X), self._dev(Y), self._dev(M)
        loss = self.torch.empty(1, device="cuda")
        grad = self.torch.empty_like(self.params)
        _check(lib().atucker_mlp_loss_grad(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                           ctypes.c_void_p(M.data_ptr()), X.shape[0], *self.shape,
                                           ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                           ctypes.c_void_p(grad.data_ptr()), self._stream()), "atucker_mlp_loss_grad")
        return float(loss.item()), grad.cpu().numpy()

    def train(self, X, Y, M, steps: int, lr: float) -> np.ndarray:
        X, Y, M = self._dev(X), self._dev(Y), self._dev(M)
        losses = self.torch.empty(max(steps, 1), device="cuda")
        _check(lib().atucker_mlp_train(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                       ctypes.c_void_p(M.data_ptr()), X.shape[0], *self.shape,
                                       ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(self.state.data_ptr()),
                                       int(steps), int(self.steps), ctypes.c_float(lr),
                                       ctypes.c_void_p(losses.data_ptr()), self._stream()), "atucker_mlp_train")
        self.steps += steps
        return losses[:steps].cpu().numpy()

    def host_params(self) -> np.ndarray:
        return self.params.cpu().numpy()


# ---------------------------------------------------------- selector state
def pack(fmean, fscale, params) -> np.ndarray:
    return np.concatenate([np.asarray(fmean, np.float32), np.asarray(fscale, np.float32),
                           np.asarray(params, np.float32)])


def install(packed=None, path: str = WEIGHTS) -> bool:
    """Load a selector into the library (atucker_selector_set); from `path` when
    no packed vector is given.  Returns False when there is nothing to load."""
    if packed is None:
        if not os.path.exists(path):
            return False
        with open(path) as f:
            packed = np.asarray(json.load(f)["packed"], dtype=np.float32)
    packed = np.ascontiguousarray(packed, dtype=np.float32)
    _check(lib().atucker_selector_set(packed.ctypes.data_as(ctypes.c_void_p), packed.size), "atucker_selector_set")
    return True


def predict(features: np.ndarray):
    """(classes, scores) from the loaded selector (host inference in the library)."""
    f = np.ascontiguousarray(features, dtype=np.float64)
    rows = f.shape[0]
    cls = (ctypes.c_int * rows)()
    scores = np.zeros(rows * NUM_CLASSES, dtype=np.float32)
    _check(lib().atucker_selector_predict(f.ctypes.data_as(ctypes.c_void_p), rows, cls,
                                          scores.ctypes.data_as(ctypes.c_void_p)), "atucker_selector_predict")
    return np.array(list(cls)), scores.reshape(rows, NUM_CLASSES)


# ------------------------------------------------------------ timing labels
def random_tucker_gpu(dims, ranks, seed: int, noise: float = 1e-3):
    """Random Tucker tensor + noise built on the GPU with torch (timing inputs
    only; the content sets the spectra the solvers see).  Column-major flat."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(int(seed))
    x = torch.randn(*[int(r) for r in reversed(ranks)], device="cuda", generator=g)  # C order = reversed dims
    for n in range(len(dims)):
        u, _ = torch.linalg.qr(torch.randn(int(dims[n]), int(ranks[n]), device="cuda", generator=g))
        ax = len(dims) - 1 - n
        x = torch.movedim(torch.tensordot(u, x, dims=([1], [ax])), 0, ax)
    x = x + noise * torch.randn(x.shape, device="cuda", generator=g)
    return x.contiguous().view(-1)


def time_shape(dims, ranks, x, reps: int = 2, slow_ms: float = 1500.0):
    """Per-mode ms of every class: array (N, NUM_CLASSES), NaN where a class
    failed.  One warm-up run per shape, then the median of `reps` timed runs
    per class (one, when a mode already took over `slow_ms`)."""
    import torch
    N = len(dims)
    out = np.full((N, NUM_CLASSES), np.nan)
    for c in range(NUM_CLASSES):
        try:
            p = Plan(dims, ranks, classes=[c] * N)
        except Exception:
            continue
        try:
            core = torch.empty(p.core_numel, device="cuda")
            fac = torch.empty(p.factors_numel, device="cuda")
            if c == 0:  # one warm-up per shape
                p.run(x, core, fac)
                p.sync()
            p.set_timing(True)
            runs = []
            for _ in range(max(reps, 1)):
                p.run(x, core, fac)
                p.sync()
                runs.append(p.mode_timings())
                p.timings()  # drop the phase records
                if max(runs[-1]) > slow_ms:
                    break
            out[:, c] = np.median(np.array(runs), axis=0)
        except Exception:
            pass
        finally:
            p.close()
    return out


def collect(shapes, seed: int = 0, reps: int = 2, log=None):
    """Timing set for `shapes` [(dims, ranks)]: list of per-shape (N, K) arrays."""
    import torch
    res = []
    for i, (dims, ranks) in enumerate(shapes):
        t0 = time.time()
        x = random_tucker_gpu(dims, ranks, seed * 100003 + i)
        res.append(time_shape(dims, ranks, x, reps=reps))
        del x
        torch.cuda.empty_cache()
        if log:
            log(f"{i + 1}/{len(shapes)} {dims} {ranks} {time.time() - t0:.1f}s")
    return res


# ------------------------------------------------------------- train / eval
def dataset(shapes, times):
    """Stack (features, times) of every (shape, mode)."""
    F = np.concatenate([mode_features(d, r) for d, r in shapes])
    T = np.concatenate([np.asarray(t, dtype=np.float64) for t in times])
    return F, T


def fit(F, T, steps: int = 4000, lr: float = 3e-3, seed: int = 0):
    """Standardise the features, train on the GPU; returns (packed vector, losses)."""
    fmean = F.mean(axis=0)
    fscale = F.std(axis=0)
    fscale[fscale < 1e-6] = 1.0
    X = ((F - fmean) / fscale).astype(np.float32)
    Y, M = targets(T)
    net = GpuMLP(init_params(seed))
    losses = net.train(X, Y.astype(np.float32), M.astype(np.float32), steps, lr)
    return pack(fmean, fscale, net.host_params()), losses


def regret(T, chosen):
    """Sum of chosen times / sum of best times - 1, over rows with a measured choice."""
    T = np.asarray(T, dtype=np.float64)
    rows = np.arange(len(T))
    tc = T[rows, chosen]
    best = np.nanmin(T, axis=1)
    ok = np.isfinite(tc) & np.isfinite(best)
    return float(tc[ok].sum() / best[ok].sum() - 1.0), ok


# The product path's policy (atucker_plan_create): the network's best class
# and up to SEARCH_MAX - 1 more predicted within SEARCH_MARGIN log2 units of
# it are timed at the plan's first run, which keeps the fastest.
SEARCH_MARGIN = 2.0
SEARCH_MAX = 3


def class_fits(k: int, lg: float) -> bool:
    """Whether class k can run a mode with log2 I_n = lg (the full Jacobi needs I_n <= 1024)."""
    if k == NUM_CLASSES - 1:
        return True
    return lg <= (10.0 if k in (2, 3) else 15.0) + 1e-9


def with_search(F, T, cls, scores, margin: float = SEARCH_MARGIN, top: int = SEARCH_MAX):
    """Classes the product path ends with: the prediction, or, where other
    fitting classes are predicted within `margin` of it (at most `top`
    candidates in all), whichever candidate measured fastest (the timed
    search).  Returns (classes, number of modes searched)."""
    out = np.array(cls, copy=True)
    searched = 0
    for i in range(len(F)):
        if not np.all(np.isfinite(scores[i])):
            continue
        pick = int(cls[i])
        rest = sorted((k for k in range(NUM_CLASSES) if k != pick and class_fits(k, float(F[i, 0]))),
                      key=lambda k: scores[i, k])
        cands = [pick] + [k for k in rest[:top - 1] if scores[i, k] - scores[i, pick] < margin]
        if len(cands) < 2:
            continue
        searched += 1
        tt = [T[i, k] if np.isfinite(T[i, k]) else np.inf for k in cands]
        out[i] = cands[int(np.argmin(tt))]
    return out, searched


def evaluate(F, T, shapes_rows=None):
    """Regret of the loaded selector on (F, T), and its gain over fixed classes."""
    cls, scores = predict(F)
    r, ok = regret(T, cls)
    best = np.nanmin(T, axis=1)
    out = {"rows": int(ok.sum()), "regret": r,
           "chosen_ms": float(T[np.arange(len(T)), cls][ok].sum()), "best_ms": float(best[ok].sum()),
           "class_counts": {CLASS_NAMES[k]: int((cls == k).sum()) for k in range(NUM_CLASSES)}}
    for k, name in enumerate(CLASS_NAMES):
        tk = T[:, k]
        m = ok & np.isfinite(tk)
        out[f"fixed_{name}_ms"] = float(tk[m].sum())
        out[f"gain_vs_fixed_{name}"] = float(tk[m].sum() / T[np.arange(len(T)), cls][m].sum())
    if shapes_rows is not None:
        per_shape = []
        for a, b in shapes_rows:
            rr, _ = regret(T[a:b], cls[a:b])
            per_shape.append(rr)
        out["max_shape_regret"] = float(np.max(per_shape))
    if np.any(scores != 0):
        # the product path: the network, with the timed search on close calls;
        # and, for scale, the search over the network's top three always
        for key, margin in (("with_timed_search", SEARCH_MARGIN), ("top3_always_searched", np.inf)):
            cs, searched = with_search(F, T, cls, scores, margin=margin)
            rs, _ = regret(T, cs)
            out[key] = {"regret": rs, "modes_searched": searched,
                        "gain_vs_fixed_EIG": float(T[:, 0][ok].sum() / T[np.arange(len(T)), cs][ok].sum())}
    return out


def shape_rows(shapes):
    rows, o = [], 0
    for d, _ in shapes:
        rows.append((o, o + len(d)))
        o += len(d)
    return rows


RMAX = 128  # the library's rank limit (atucker_plan_create)


def selector_shapes(count: int = 256, seed: int = 0):
    """The selector workload: synth.selector_shapes with every rank clamped to
    the library's limit of 128 (then made Tucker-feasible again)."""
    import synth
    return [(list(d), synth.feasible_ranks(d, [min(r, RMAX) for r in rr]))
            for d, rr in synth.selector_shapes(count=count, seed=seed)]


TIMINGS_EXTRA = os.path.join(HERE, "selector_timings_extra.json")


def load_timings(path):
    with open(path) as f:
        data = json.load(f)
    shapes = [(list(d), list(r)) for d, r in data["shapes"]]
    times = [np.where(np.asarray(t) < 0, np.nan, np.asarray(t, dtype=np.float64)) for t in data["times_ms"]]
    return shapes, times


def train_and_evaluate(timings=TIMINGS, extra=TIMINGS_EXTRA, n_train: int = 192, steps: int = 4000,
                       lr: float = 3e-3, seed: int = 0):
    """Fit on the first n_train shapes of `timings` (the protocol of the
    selector workload), and again with the `extra` timing set added to the
    training data; evaluate both on the remaining shapes of `timings`.
    Returns (report, packed vector of the better-data model)."""
    shapes, times = load_timings(timings)
    F, T = dataset(shapes[:n_train], times[:n_train])
    Fh, Th = dataset(shapes[n_train:], times[n_train:])
    rows = shape_rows(shapes[n_train:])
    report = {"held_out_shapes": len(shapes) - n_train, "held_out_modes": int(len(Fh)),
              "best_possible_gain_vs_fixed_EIG": float(Th[:, 0].sum() / np.nanmin(Th, axis=1).sum())}
    packed, losses = fit(F, T, steps=steps, lr=lr, seed=seed)
    install(packed)
    report["train_192"] = dict(evaluate(Fh, Th, rows), train_modes=int(len(F)), final_loss=float(losses[-1]))
    if extra and os.path.exists(extra):
        es, et = load_timings(extra)
        Fe, Te = dataset(es, et)
        packed, losses = fit(np.concatenate([F, Fe]), np.concatenate([T, Te]), steps=steps, lr=lr, seed=seed)
        install(packed)
        report["train_192_plus_extra"] = dict(evaluate(Fh, Th, rows), train_modes=int(len(F) + len(Fe)),
                                              extra_shapes=len(es), final_loss=float(losses[-1]))
    return report, packed


# ------------------------------------------- decision tree (the paper's selector)
# Sec. IV-B trains a decision tree classifier on Table I's features to pick
# the solver.  Here, as a baseline for the MLP: a CART tree (Gini impurity,
# binary splits at midpoints between consecutive distinct values, depth <= 10)
# on the ten Table I features, labelled with the fastest measured class of
# each (shape, mode).  Features enter as the library computes them (log2):
# a tree's splits are invariant under monotone maps of a feature.  Training is
# an offline host step; inference runs in the library
# (atucker_selector_set_tree / atucker_selector_predict).
TABLE_I = tuple(range(10))


def best_labels(T):
    """Fastest measured class of every row, -1 where none was measured."""
    T = np.asarray(T, dtype=np.float64)
    ok = np.isfinite(T).any(axis=1)
    lab = np.full(len(T), -1, dtype=np.int64)
    lab[ok] = np.nanargmin(np.where(np.isfinite(T[ok]), T[ok], np.nan), axis=1)
    return lab


def _gini(counts):
    n = counts.sum(axis=-1)
    with np.errstate(invalid="ignore", divide="ignore"):
        p = counts / np.maximum(n, 1)[..., None]
    return 1.0 - (p * p).sum(axis=-1)


def fit_tree(F, labels, max_depth: int = 10, min_leaf: int = 2, features=TABLE_I, n_classes: int = NUM_CLASSES):
    """CART classification tree.  Returns a dict of node arrays (feature,
    threshold, left, right, cls) in creation order (children after their
    parent), as atucker_selector_set_tree takes them."""
    F = np.asarray(F, dtype=np.float64)
    y = np.asarray(labels, dtype=np.int64)
    keep = y >= 0
    F, y = F[keep], y[keep]
    nodes = {"feature": [], "threshold": [], "left": [], "right": [], "cls": [], "depth": []}

    def new_node(depth):
        for k in nodes:
            nodes[k].append(-1 if k != "threshold" else 0.0)
        nodes["depth"][-1] = depth
        return len(nodes["feature"]) - 1

    root = new_node(0)
    stack = [(root, np.arange(len(y)), 0)]
    while stack:
        node, idx, depth = stack.pop()
        counts = np.bincount(y[idx], minlength=n_classes).astype(np.float64)
        nodes["cls"][node] = int(np.argmax(counts))  # majority, ties to the lower class
        if depth >= max_depth or len(idx) < 2 * min_leaf or counts.max() == len(idx):
            continue
        parent = _gini(counts) * len(idx)
        best = (parent - 1e-12, None, None)
        for f in features:
            order = idx[np.argsort(F[idx, f], kind="stable")]
            v = F[order, f]
            onehot = np.zeros((len(order), n_classes))
            onehot[np.arange(len(order)), y[order]] = 1.0
            left = np.cumsum(onehot, axis=0)[:-1]
            right = counts[None, :] - left
            nl = np.arange(1, len(order))
            nr = len(order) - nl
            cost = _gini(left) * nl + _gini(right) * nr
            valid = (v[1:] > v[:-1]) & (nl >= min_leaf) & (nr >= min_leaf)
            if not valid.any():
                continue
            j = int(np.argmin(np.where(valid, cost, np.inf)))
            if cost[j] < best[0]:
                best = (cost[j], f, 0.5 * (v[j] + v[j + 1]))
        if best[1] is None:
            continue
        f, thr = best[1], best[2]
        go_left = F[idx, f] <= thr
        li, ri = new_node(depth + 1), new_node(depth + 1)
        nodes["feature"][node], nodes["threshold"][node] = int(f), float(thr)
        nodes["left"][node], nodes["right"][node] = li, ri
        stack.append((ri, idx[~go_left], depth + 1))
        stack.append((li, idx[go_left], depth + 1))
    return {k: np.asarray(v) for k, v in nodes.items()}


def tree_predict_host(tree, F) -> np.ndarray:
    """The tree's class for every row (numpy walk; the library's
    atucker_selector_predict does the same in C)."""
    F = np.asarray(F, dtype=np.float64)
    out = np.empty(len(F), dtype=np.int64)
    for r, f in enumerate(F):
        node = 0
        while tree["feature"][node] >= 0:
            node = tree["left"][node] if f[tree["feature"][node]] <= tree["threshold"][node] else tree["right"][node]
        out[r] = tree["cls"][node]
    return out


def install_tree(tree) -> None:
    """Make the tree the library's active selector (atucker_selector_set_tree)."""
    n = len(tree["feature"])
    feat = np.ascontiguousarray(tree["feature"], dtype=np.int32)
    thr = np.ascontiguousarray(tree["threshold"], dtype=np.float64)
    left = np.ascontiguousarray(tree["left"], dtype=np.int32)
    right = np.ascontiguousarray(tree["right"], dtype=np.int32)
    cls = np.ascontiguousarray(tree["cls"], dtype=np.int32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib().atucker_selector_set_tree(n, vp(feat), vp(thr), vp(left), vp(right), vp(cls)),
           "atucker_selector_set_tree")


def inference_us(F, reps: int = 20) -> float:
    """Host inference time of the active selector, microseconds per mode."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    predict(F)
    t0 = time.perf_counter()
    for _ in range(reps):
        predict(F)
    return (time.perf_counter() - t0) / reps / len(F) * 1e6


def compare_tree_mlp(timings=TIMINGS, extra=TIMINGS_EXTRA, n_train: int = 192, max_depth: int = 10):
    """The paper's decision tree against the installed MLP on the held-out
    shapes: regret, gain over always-EIG and host inference time per mode.
    The tree is trained on the same timing sets as the installed network
    (the first n_train shapes plus the extra set).  Leaves the installed
    network active afterwards."""
    shapes, times = load_timings(timings)
    F, T = dataset(shapes[:n_train], times[:n_train])
    if extra and os.path.exists(extra):
        es, et = load_timings(extra)
        Fe, Te = dataset(es, et)
        F, T = np.concatenate([F, Fe]), np.concatenate([T, Te])
    Fh, Th = dataset(shapes[n_train:], times[n_train:])
    rows = shape_rows(shapes[n_train:])
    out = {}
    if install():
        out["mlp"] = dict(evaluate(Fh, Th, rows), inference_us_per_mode=inference_us(Fh))
    tree = fit_tree(F, best_labels(T), max_depth=max_depth)
    install_tree(tree)
    out["tree"] = dict(evaluate(Fh, Th, rows), inference_us_per_mode=inference_us(Fh),
                       nodes=int(len(tree["feature"])), depth=int(tree["depth"].max()),
                       train_modes=int(len(F)))
    lib().atucker_selector_clear()
    install()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2010_10131_b300.selector")
    ap.add_argument("cmd", choices=["collect", "train", "tree"])
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--train", type=int, default=192)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--seed", type=int, default=0, help="shape-set seed (collect)")
    ap.add_argument("--timings", default=TIMINGS, help="timing set (written by collect, read by train)")
    ap.add_argument("--weights", default=WEIGHTS, help="weights written by train")
    ap.add_argument("--extra", default=TIMINGS_EXTRA, help="additional training timings (train)")
    args = ap.parse_args(argv)
    shapes = selector_shapes(args.count, seed=args.seed)
    if args.cmd == "collect":
        times = collect(shapes, seed=args.seed, reps=args.reps, log=lambda s: print(s, flush=True))
        with open(args.timings, "w") as f:
            json.dump({"shapes": shapes, "classes": list(CLASS_NAMES),
                       "times_ms": [np.where(np.isfinite(t), t, -1.0).tolist() for t in times]}, f)
        return 0
    if args.cmd == "tree":
        print(json.dumps(compare_tree_mlp(args.timings, args.extra, n_train=args.train)))
        return 0
    report, packed = train_and_evaluate(args.timings, args.extra, n_train=args.train, steps=args.steps)
    with open(args.weights, "w") as f:
        json.dump({"packed": packed.tolist(), "steps": args.steps, "report": report}, f)
    print(json.dumps(report))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
