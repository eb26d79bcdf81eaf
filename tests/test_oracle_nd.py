"""Pins for the nested-dissection hierarchy (Sec. 2.2.1, Sec. 3.3)."""
import json
import os

import numpy as np
import pytest

from oracle.nd import NDTree, build_hierarchy, nd_permutation, symbolic_blocks

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_enumerated_12x6():
    g = json.load(open(os.path.join(GOLD, "nd_12x6_D2.json")))
    t, levels = build_hierarchy(g["n_theta"], g["n_r"], g["D"])
    owner = np.array(g["owner_rows_i0_to_i5"]).ravel()
    assert np.array_equal(t.owner, owner)
    assert t.level == g["node_level"]
    for l, want in enumerate(g["levels"]):
        got = levels[l]
        assert len(got) == len(want)
        for c, w in zip(got, want):
            assert c["node"] == w["node"] and list(c["key"]) == w["key"]
            assert c["interior"] == w["interior"]
            if "elems" in w:
                assert c["elems"] == w["elems"]
            else:
                assert c["children"] == w["children"]


def test_hand_enumerated_8x4_single_split():
    # D=1: root separator j in {0, 4}; two 4x3 leaves
    t, levels = build_hierarchy(8, 4, 1)
    own = t.owner.reshape(4, 8)
    assert np.all(own[:, 0] == 0) and np.all(own[:, 4] == 0)
    assert np.all(own[:, 1:4] == 1) and np.all(own[:, 5:8] == 2)
    assert [c["interior"] for c in levels[0]] == [False, True, True]
    assert len(levels[1]) == 1 and levels[1][0]["interior"]


@pytest.mark.parametrize("nt,nr,D", [(16, 8, 2), (12, 6, 2), (64, 32, 6), (24, 20, 4), (10, 3, 3)])
def test_permutation_is_bijection(nt, nr, D):
    _, levels = build_hierarchy(nt, nr, D)
    perm = nd_permutation(levels)
    assert np.array_equal(np.sort(perm), np.arange(nt * nr))
    # every element is in exactly one level-0 cluster; every cluster at a level
    # is the union of its children
    for l in range(1, len(levels)):
        surv = [c for c in levels[l - 1] if not c["interior"]]
        kids = sorted(k for c in levels[l] for k in c["children"])
        assert kids == list(range(len(surv)))
        for c in levels[l]:
            assert c["elems"] == sorted(e for k in c["children"] for e in surv[k]["elems"])


@pytest.mark.parametrize("nt,nr,D", [(16, 8, 2), (12, 6, 2), (32, 16, 4), (24, 20, 4)])
def test_separator_property_brute_force(nt, nr, D):
    """Graph elimination on the element graph: before level l, no edge joins two
    different level-l interiors (so their elimination creates no fill between them)."""
    t, levels = build_hierarchy(nt, nr, D)
    K = nt * nr
    adj = [set(t.neighbours(e)) for e in range(K)]
    alive = np.ones(K, bool)
    for l, cl in enumerate(levels):
        inter = [c["elems"] for c in cl if c["interior"]]
        tag = np.full(K, -1)
        for i, el in enumerate(inter):
            tag[el] = i
        for el in inter:
            for e in el:
                for n in adj[e]:
                    assert tag[n] == -1 or tag[n] == tag[e]
        for el in inter:                                   # eliminate with fill
            for e in el:
                nb = [n for n in adj[e] if alive[n] and n != e]
                for a in nb:
                    adj[a].discard(e)
                    adj[a].update(x for x in nb if x != a)
                alive[e] = False
    assert not alive.any()


def test_symbolic_blocks_no_interior_interior():
    t, levels = build_hierarchy(32, 16, 4)
    pats = symbolic_blocks(t, levels)
    for l, pat in enumerate(pats):
        inter = {i for i, c in enumerate(levels[l]) if c["interior"]}
        for a, b in pat:
            if a != b:
                assert not (a in inter and b in inter)
            assert (b, a) in set(pat)                      # symmetric pattern


def test_levels_match_depth():
    t = NDTree(64, 32, 6)
    for v in range(len(t.depth)):
        if t.is_leaf[v]:
            assert t.level[v] == 0
        else:
            assert t.level[v] == 6 - t.depth[v] and t.depth[v] < 6
