"""Nested dissection of the (i, j) element grid and the spaND cluster hierarchy.

Sec. 2.2.1: an ND ordering defines interiors, separators and interfaces at each
level 0 <= l < l_max (0 = leaves); interfaces are the parts of a separator
that touch the same interiors.  Sec. 3.3: elements are mapped to integer
(i, j) (i radial, j angular) and partitioned by recursive bisection.

Readings (the paper does not fix these details):
  * The ring is periodic in j.  The root separator is the two radial lines
    j = 0 and j = floor(n_theta/2); its two children are the j-ranges between
    them.  Below the root a box is split across its longer extent (ties split
    j) at index lo + floor((n-1)/2).  A box becomes a leaf at depth D or when
    its longer extent is < 3.
  * Leaves are eliminated at level 0; the separator of a box at depth d is
    eliminated at level D - d.
  * box_k(e), the depth-k box holding element e: the depth-k ancestor of the
    node owning e when that node is at depth >= k; the owning leaf itself when
    it is a shallower leaf; none when e lies on a separator shallower than k.
  * Level-0 clusters: one per leaf, and separator elements grouped by
    (separator, sorted set of box_D of their face neighbours).  The clusters
    remaining after level l are grouped into level-(l+1) clusters by
    (separator, union over the cluster's elements of box_{D-l-1} of their
    face neighbours); a coarse cluster concatenates its children in order.
  * Clusters at a level are ordered by (separator/leaf preorder id, key);
    elements inside a level-0 cluster ascend by e.
"""
import numpy as np


class NDTree:
    def __init__(self, n_theta, n_r, D):
        if n_theta < 4 or n_r < 1:
            raise ValueError("need n_theta >= 4 and n_r >= 1")
        self.n_theta, self.n_r, self.D = n_theta, n_r, D
        self.K = n_theta * n_r
        self.depth, self.parent, self.is_leaf, self.elems = [], [], [], []
        self.owner = np.full(self.K, -1, dtype=np.int64)
        J2 = n_theta // 2
        root = self._new(0, -1, False)
        sep = sorted([i * n_theta + 0 for i in range(n_r)] + [i * n_theta + J2 for i in range(n_r)])
        self._own(root, sep)
        self._rec(0, n_r, 1, J2, 1, root)
        self._rec(0, n_r, J2 + 1, n_theta, 1, root)
        assert np.all(self.owner >= 0)
        self.level = [0 if self.is_leaf[v] else D - self.depth[v] for v in range(len(self.depth))]

    def _new(self, depth, parent, leaf):
        self.depth.append(depth)
        self.parent.append(parent)
        self.is_leaf.append(leaf)
        self.elems.append([])
        return len(self.depth) - 1

    def _own(self, v, elems):
        self.elems[v] = sorted(elems)
        self.owner[self.elems[v]] = v

    def _rec(self, i0, i1, j0, j1, depth, parent):
        ni, nj = i1 - i0, j1 - j0
        nt = self.n_theta
        if depth == self.D or max(ni, nj) < 3:
            v = self._new(depth, parent, True)
            self._own(v, [i * nt + j for i in range(i0, i1) for j in range(j0, j1)])
            return
        v = self._new(depth, parent, False)
        if nj >= ni:
            js = j0 + (nj - 1) // 2
            self._own(v, [i * nt + js for i in range(i0, i1)])
            self._rec(i0, i1, j0, js, depth + 1, v)
            self._rec(i0, i1, js + 1, j1, depth + 1, v)
        else:
            is_ = i0 + (ni - 1) // 2
            self._own(v, [is_ * nt + j for j in range(j0, j1)])
            self._rec(i0, is_, j0, j1, depth + 1, v)
            self._rec(is_ + 1, i1, j0, j1, depth + 1, v)

    # ------------------------------------------------------------------
    def neighbours(self, e):
        nt, nr = self.n_theta, self.n_r
        i, j = divmod(e, nt)
        out = [i * nt + (j + 1) % nt, i * nt + (j - 1) % nt]
        if i > 0:
            out.append(e - nt)
        if i < nr - 1:
            out.append(e + nt)
        return out

    def box(self, e, k):
        v = int(self.owner[e])
        if self.depth[v] >= k:
            while self.depth[v] > k:
                v = self.parent[v]
            return v
        return v if self.is_leaf[v] else None

    def adj_boxes(self, elems, k):
        s = set()
        for e in elems:
            for n in self.neighbours(e):
                b = self.box(n, k)
                if b is not None:
                    s.add(b)
        return tuple(sorted(s))


def build_hierarchy(n_theta, n_r, D):
    """Return (tree, levels).

    levels[l] is the ordered list of clusters present at the start of level l;
    each cluster is a dict with node, key, elems (sorted union of its
    elements), children (indices into the surviving clusters of level l-1,
    None at level 0) and interior (eliminated at level l).
    """
    t = NDTree(n_theta, n_r, D)
    groups = {}
    for v in range(len(t.depth)):
        if t.is_leaf[v]:
            groups[(v, ())] = list(t.elems[v])
    for e in range(t.K):
        v = int(t.owner[e])
        if not t.is_leaf[v]:
            groups.setdefault((v, t.adj_boxes([e], D)), []).append(e)
    lv0 = [dict(node=k[0], key=k[1], elems=sorted(g), children=None,
                interior=(t.level[k[0]] == 0)) for k, g in sorted(groups.items())]
    levels = [lv0]
    for l in range(D):
        surv = [c for c in levels[l] if not c["interior"]]
        groups = {}
        for ci, c in enumerate(surv):
            key = (c["node"], t.adj_boxes(c["elems"], D - l - 1))
            groups.setdefault(key, []).append(ci)
        nxt = []
        for key in sorted(groups):
            ch = groups[key]
            el = sorted(e for ci in ch for e in surv[ci]["elems"])
            nxt.append(dict(node=key[0], key=key[1], elems=el, children=ch,
                            interior=(t.level[key[0]] == l + 1)))
        levels.append(nxt)
    assert all(c["interior"] for c in levels[D])
    return t, levels


def nd_permutation(levels):
    """Elements in level-0 cluster order (the ND ordering of the level-0 DOFs)."""
    return np.array([e for c in levels[0] for e in c["elems"]], dtype=np.int64)


def symbolic_blocks(tree, levels):
    """Cluster-pair block pattern per level (before elimination), with fill-in.

    Returns a list over levels of sorted lists of (a, b) index pairs into
    levels[l]; pairs follow the pattern rule of Eq. 10 (elimination of an
    interior couples every pair of its neighbours).
    """
    out = []
    # level 0 from element adjacency
    cl_of = np.empty(tree.K, dtype=np.int64)
    for ci, c in enumerate(levels[0]):
        cl_of[c["elems"]] = ci
    pat = set()
    for e in range(tree.K):
        a = int(cl_of[e])
        pat.add((a, a))
        for n in tree.neighbours(e):
            pat.add((a, int(cl_of[n])))
    for l in range(len(levels)):
        cl = levels[l]
        out.append(sorted(pat))
        inter = {i for i, c in enumerate(cl) if c["interior"]}
        nb = {}
        for a, b in pat:
            nb.setdefault(a, set()).add(b)
        newpat = {(a, b) for a, b in pat if a not in inter and b not in inter}
        for s in inter:
            ns = sorted(n for n in nb.get(s, ()) if n != s)
            for n1 in ns:
                for n2 in ns:
                    newpat.add((n1, n2))
        if l + 1 == len(levels):
            break
        surv = [i for i, c in enumerate(cl) if not c["interior"]]
        pos = {old: k for k, old in enumerate(surv)}
        parent_of = {}
        for pi, pc in enumerate(levels[l + 1]):
            for ch in pc["children"]:
                parent_of[surv[ch]] = pi
        pat = {(parent_of[a], parent_of[b]) for a, b in newpat}
        del pos
    return out
