"""The paper's selector as a baseline: a depth-limited CART decision tree on
Table I's features (Sec. IV-B), trained offline on the timing sets, with its
inference in the C library (atucker_selector_set_tree).  Host only."""
import ctypes

import numpy as np
import pytest

import paper_2010_10131_b300 as atk
from paper_2010_10131_b300 import selector as sel


def test_tree_finds_the_single_threshold():
    """Labels that one threshold separates give a one-split tree at the
    midpoint between the two groups."""
    F = np.zeros((10, atk.SELECTOR_FEATURES))
    F[:, 3] = np.arange(1, 11)
    y = (F[:, 3] > 3).astype(int) * atk.CLASS_ALS
    tree = sel.fit_tree(F, y)
    assert tree["feature"][0] == 3 and tree["threshold"][0] == pytest.approx(3.5)
    assert sorted(tree["cls"][[tree["left"][0], tree["right"][0]]]) == [0, atk.CLASS_ALS]
    assert len(tree["feature"]) == 3
    np.testing.assert_array_equal(sel.tree_predict_host(tree, F), y)


def test_tree_respects_depth_and_library_inference_matches():
    g = np.random.default_rng(1)
    F = g.uniform(0, 10, size=(400, atk.SELECTOR_FEATURES))
    F[:, 0] = g.uniform(4, 10, size=400)  # log2 I_n within the EIG limit
    y = g.integers(0, atk.NUM_CLASSES, size=400)  # no structure: the tree grows to its depth limit
    tree = sel.fit_tree(F, y, max_depth=6)
    assert tree["depth"].max() <= 6
    assert np.all(tree["left"][tree["feature"] >= 0] > np.flatnonzero(tree["feature"] >= 0))
    try:
        sel.install_tree(tree)
        cls, _ = sel.predict(F)
        np.testing.assert_array_equal(cls, sel.tree_predict_host(tree, F))
    finally:
        atk.lib().atucker_selector_clear()


def test_set_tree_rejects_malformed_trees():
    lib = atk.lib()
    i32 = lambda *v: (ctypes.c_int * len(v))(*v)  # noqa: E731
    thr = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    # a child numbered before its parent (a possible cycle)
    assert lib.atucker_selector_set_tree(3, i32(0, -1, -1), thr, i32(0, 2, 0), i32(2, 0, 0), i32(0, 0, 4)) == atk.EINVAL
    # a leaf class out of range
    assert lib.atucker_selector_set_tree(1, i32(-1), thr, i32(0), i32(0), i32(9)) == atk.EINVAL
    # a split on a feature that does not exist
    assert lib.atucker_selector_set_tree(3, i32(12, -1, -1), thr, i32(1, 0, 0), i32(2, 0, 0), i32(0, 0, 4)) == atk.EINVAL


def test_tree_baseline_against_the_mlp_on_held_out_shapes():
    """Trained on the same measured timings as the installed network
    (192 shapes plus the extra set), evaluated on the 64 held-out shapes: the
    tree must beat always-EIG, and the comparison is reported (regret and host
    inference per mode for both)."""
    out = sel.compare_tree_mlp()
    tree, mlp = out["tree"], out["mlp"]
    assert tree["depth"] <= 10
    assert tree["rows"] == mlp["rows"] == 258
    assert tree["gain_vs_fixed_EIG"] > 1.0
    assert tree["regret"] < 0.10 and mlp["regret"] < 0.10
    assert tree["inference_us_per_mode"] < mlp["inference_us_per_mode"]
