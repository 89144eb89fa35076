"""Nested-dissection solve of a quasi-2D slab subproblem (Section 4).

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the product
path imports this module.

Section 4 solves every 3D slab subproblem H_q^M, H_p^R, H_p^L (a quasi-2D
problem: n x n points in x1, x2 and w planes in x3) by first grouping the
unknowns along dimension 3 -- each (x1, x2) column holds its w unknowns -- and
then ordering the grouped problem by nested dissection (George 1973), with the
elimination organised around dense frontal matrices (Duff and Reid 1983).  This
module writes that out plainly, in complex128:

* ``separator_tree``: the column grid is cut recursively.  A region of more
  than ``leaf_cols`` columns is split by the middle line across its longer side;
  the line is the node's separator and the two halves are its children.  A
  region of at most ``leaf_cols`` columns is a leaf that owns all its columns.
* ``factor``: the nodes are eliminated children before parents.  Node t owns
  the unknowns I(t) (its columns, every plane) and its front also holds the
  unknowns B(t) outside its region that are coupled to the region.  The front
  is assembled from the entries of H that couple I(t) to I(t) and B(t) (and
  B(t) to I(t)) plus the children's update matrices; F_II is factored by LU
  with partial pivoting (scipy), and U = F_BB - F_BI F_II^-1 F_IB is the
  node's update matrix for its parent.
* ``solve``: forward (children first) and backward (parents first)
  substitution through the fronts.

The result is H^-1 g up to rounding, so it is pinned against a sparse direct
solve of the same matrix and against brute-force checks of the tree.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


@dataclass
class Node:
    region: tuple            # (x0, x1, y0, y1): columns x in [x0, x1), y in [y0, y1)
    own: list                # column ids y*n + x owned by the node
    children: list = field(default_factory=list)
    parent: int = -1
    depth: int = 0


def separator_tree(n: int, leaf_cols: int = 8) -> list[Node]:
    """Nodes of the nested dissection of the n x n column grid (root first)."""
    nodes: list[Node] = []

    def cut(x0, x1, y0, y1, parent, depth):
        t = len(nodes)
        nodes.append(Node((x0, x1, y0, y1), [], [], parent, depth))
        W, Hh = x1 - x0, y1 - y0
        if W * Hh <= leaf_cols:
            nodes[t].own = [y * n + x for y in range(y0, y1) for x in range(x0, x1)]
            return t
        if W >= Hh:
            xs = (x0 + x1) // 2
            nodes[t].own = [y * n + xs for y in range(y0, y1)]
            halves = [(x0, xs, y0, y1), (xs + 1, x1, y0, y1)]
        else:
            ys = (y0 + y1) // 2
            nodes[t].own = [ys * n + x for x in range(x0, x1)]
            halves = [(x0, x1, y0, ys), (x0, x1, ys + 1, y1)]
        for r in halves:
            nodes[t].children.append(cut(*r, t, depth + 1))
        return t

    cut(0, n, 0, n, -1, 0)
    return nodes


def _unknowns(cols, n: int, w: int) -> np.ndarray:
    """Indices, in the slab's natural order (x1 fastest, x3 slowest), of every
    plane of the given columns: column by column, planes inside a column."""
    out = [pl * n * n + col for col in cols for pl in range(w)]
    return np.asarray(out, dtype=np.int64)


def _region_cols(region, n):
    x0, x1, y0, y1 = region
    return {y * n + x for y in range(y0, y1) for x in range(x0, x1)}


@dataclass
class NDFactor:
    n: int
    w: int
    nodes: list
    I: list                  # per node: owned unknowns
    B: list                  # per node: boundary unknowns
    lu: list                 # per node: LU factors of F_II
    FIB: list
    FBI: list


def factor(H: sp.spmatrix, n: int, w: int, leaf_cols: int = 8) -> NDFactor:
    """Multifrontal nested-dissection factorization of the slab matrix H
    (natural order: index = i3*n*n + i2*n + i1, 0-based)."""
    H = sp.csr_matrix(H, dtype=np.complex128)
    nodes = separator_tree(n, leaf_cols)
    N = n * n * w
    assert H.shape == (N, N)
    # the region of a node's subtree, and its boundary: the unknowns outside the
    # region that H couples to an unknown inside it
    I, B = [None] * len(nodes), [None] * len(nodes)
    for t, nd in enumerate(nodes):
        I[t] = _unknowns(nd.own, n, w)
        inside = _unknowns(sorted(_region_cols(nd.region, n)), n, w)
        inside_set = set(inside.tolist())
        coupled = set(H[inside].indices.tolist()) - inside_set
        B[t] = np.asarray(sorted(coupled), dtype=np.int64)
    lu, FIB, FBI = [None] * len(nodes), [None] * len(nodes), [None] * len(nodes)
    update = [None] * len(nodes)
    eliminated = np.zeros(N, dtype=bool)
    for t in sorted(range(len(nodes)), key=lambda k: -nodes[k].depth):  # children before parents
        idx = np.concatenate([I[t], B[t]])
        pos = {int(g): k for k, g in enumerate(idx)}
        s = len(I[t])
        F = np.zeros((len(idx), len(idx)), dtype=np.complex128)
        # entries of H coupling I(t) to the front, and B(t) to I(t)
        sub = H[idx][:, idx].toarray()
        F[:s, :] = sub[:s, :]
        F[s:, :s] = sub[s:, :s]
        for c in nodes[t].children:
            Bc, Uc = B[c], update[c]
            at = np.array([pos[int(g)] for g in Bc], dtype=np.int64)
            F[np.ix_(at, at)] += Uc
        lu[t] = sla.lu_factor(F[:s, :s])
        FIB[t] = F[:s, s:]
        FBI[t] = F[s:, :s]
        update[t] = F[s:, s:] - FBI[t] @ sla.lu_solve(lu[t], FIB[t])
        eliminated[I[t]] = True
    assert eliminated.all()
    return NDFactor(n, w, nodes, I, B, lu, FIB, FBI)


def solve(fac: NDFactor, g: np.ndarray) -> np.ndarray:
    """x = H^-1 g for g of shape (N,) or (N, nrhs), natural order."""
    g = np.asarray(g, dtype=np.complex128)
    vec = g.ndim == 1
    rhs = g.reshape(g.shape[0], -1).copy()
    nodes = fac.nodes
    order = sorted(range(len(nodes)), key=lambda k: -nodes[k].depth)
    z = [None] * len(nodes)
    for t in order:  # forward: eliminate I(t) from the right-hand side
        z[t] = sla.lu_solve(fac.lu[t], rhs[fac.I[t]])
        if len(fac.B[t]):
            rhs[fac.B[t]] -= fac.FBI[t] @ z[t]
    x = np.zeros_like(rhs)
    for t in reversed(order):  # backward: parents first
        xi = z[t]
        if len(fac.B[t]):
            xi = xi - sla.lu_solve(fac.lu[t], fac.FIB[t] @ x[fac.B[t]])
        x[fac.I[t]] = xi
    return x[:, 0] if vec else x
