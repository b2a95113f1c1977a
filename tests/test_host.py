"""CPU tests of the host logic and the library boundary (no GPU calls)."""
import os
import re

import numpy as np
import pytest

import paper_1908_07392_gb300 as V
from paper_1908_07392_gb300 import build as B
from paper_1908_07392_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return V.load_library()


def header_functions():
    names = set()
    for h in ("vp.h", "bie.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b((?:vp|bie|ws)_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    assert "vp_eval" in names and "vp_tables_build" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(V.exported_symbols()) >= set(names)


def test_error_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert V.vp_strerror(code)
    assert V.vp_strerror(-99) == "unknown error"


@pytest.mark.parametrize("seed", range(5))
def test_lists_cover_every_pair_once(lib, seed):
    t = I.random_balanced_tree(np.random.default_rng(seed), 30, 7, min_depth=1)
    a, b, m = V.vp_plan_pairs(t.level, t.ix, t.iy)
    L = t.n_leaves
    cnt = np.zeros((L, L), int)
    np.add.at(cnt, (a, b), 1)
    assert (cnt == 1).all()
    # near interactions are exactly the adjacent pairs
    x0, y0, h = t.leaf_boxes()
    near = m == 0
    gap_x = np.maximum(x0[a] - (x0[b] + h[b]), x0[b] - (x0[a] + h[a]))
    gap_y = np.maximum(y0[a] - (y0[b] + h[b]), y0[b] - (y0[a] + h[a]))
    adjacent = (gap_x <= 1e-12) & (gap_y <= 1e-12)
    assert np.array_equal(near, adjacent)


def test_uniform_tree_has_no_mixed_level_lists(lib):
    t = I.uniform_tree(4)
    a, b, m = V.vp_plan_pairs(t.level, t.ix, t.iy)
    assert set(np.unique(m)) == {0, 1}


def test_root_leaf(lib):
    a, b, m = V.vp_plan_pairs([0], [0], [0])
    assert list(a) == [0] and list(b) == [0] and list(m) == [0]


def test_rejects_bad_trees(lib):
    # unbalanced: level-1 leaf next to level-3 leaves
    leaves = {(1, 0, 0), (1, 1, 0), (1, 0, 1)}
    sub = {(2, 3, 2), (2, 2, 3), (2, 3, 3)}
    sub |= {(3, 4, 4), (3, 5, 4), (3, 4, 5), (3, 5, 5)}  # level-3 leaves touching level-1 leaves
    t = I.tree_from_set(leaves | sub, 0, 0, 2)
    with pytest.raises(V.VPError) as e:
        V.vp_plan_pairs(t.level, t.ix, t.iy)
    assert e.value.code == -2
    # gap
    with pytest.raises(V.VPError) as e:
        V.vp_plan_pairs([1, 1, 1], [0, 1, 0], [0, 0, 1])
    assert e.value.code == -6
    # overlap
    with pytest.raises(V.VPError) as e:
        V.vp_plan_pairs([0, 1], [0, 0], [0, 0])
    assert e.value.code == -6
    # outside the root
    with pytest.raises(V.VPError) as e:
        V.vp_plan_pairs([1, 1, 1, 1], [0, 1, 0, 2], [0, 0, 1, 1])
    assert e.value.code == -6
    # negative level
    with pytest.raises(V.VPError):
        V.vp_plan_pairs([-1], [0], [0])


def test_balance_generator_produces_valid_trees(lib):
    rng = np.random.default_rng(9)
    for _ in range(3):
        t = I.random_balanced_tree(rng, 40, 8)
        V.vp_plan_pairs(t.level, t.ix, t.iy)  # raises if unbalanced or not a tiling
        x0, y0, h = t.leaf_boxes()
        assert abs((h * h).sum() - t.side ** 2) < 1e-12


def test_node_coordinates_follow_the_layout():
    t = I.uniform_tree(1, cx=0.5, cy=-0.25, side=2.0)
    X, Y = I.node_coords(t, 3)
    xi, _ = np.polynomial.legendre.leggauss(3)
    # leaf 0 is (1, 0, 0): [-0.5, 0.5] x [-1.25, -0.25]; node (i, j) at j*p + i
    assert np.allclose(X[:3], -0.5 + (xi + 1) / 2)
    assert np.allclose(Y[0:9:3], -1.25 + (xi + 1) / 2)
