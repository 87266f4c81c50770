"""Brute-force block-tree helpers for tests: random 2:1-balanced trees and a
touching test written from the definition (closed-box overlap with periodic
images), independent of both the oracle and the CUDA library's tree code."""
import numpy as np


def block_box(level, c, ndim, max_level):
    s = 1 << (max_level - level)
    return [(c[d] * s, (c[d] + 1) * s) for d in range(ndim)]


def touching(a, b, ndim, base, max_level, periodic):
    (la, ca), (lb, cb) = a, b
    A = block_box(la, ca, ndim, max_level)
    B = block_box(lb, cb, ndim, max_level)
    for d in range(ndim):
        N = base[d] << (max_level - 1)
        shifts = (-N, 0, N) if periodic[d] else (0,)
        if not any(A[d][0] <= B[d][1] + s and B[d][0] + s <= A[d][1] for s in shifts):
            return False
    return True


def is_balanced(leaves, ndim, base, max_level, periodic):
    L = list(leaves)
    for i in range(len(L)):
        for j in range(i + 1, len(L)):
            if abs(L[i][0] - L[j][0]) > 1 and touching(L[i], L[j], ndim, base, max_level, periodic):
                return False
    return True


def covers_domain(leaves, ndim, base, max_level):
    vol = 0
    for lev, c in leaves:
        vol += (1 << (max_level - lev)) ** ndim
    total = 1
    for d in range(ndim):
        total *= base[d] << (max_level - 1)
    return vol == total


def random_balanced_tree(ndim, base, max_level, rng, n_refine, periodic=(True, True, True)):
    """Refine random leaves, then refine coarser touching leaves until 2:1 balanced."""
    leaves = set()
    for z in range(base[2] if ndim > 2 else 1):
        for y in range(base[1] if ndim > 1 else 1):
            for x in range(base[0]):
                leaves.add((1, (x, y, z)))

    def children(leaf):
        lev, c = leaf
        out = []
        for o in range(1 << ndim):
            cc = [2 * c[d] + ((o >> d) & 1) if d < ndim else 0 for d in range(3)]
            out.append((lev + 1, tuple(cc)))
        return out

    for _ in range(n_refine):
        cand = sorted(l for l in leaves if l[0] < max_level)
        if not cand:
            break
        pick = cand[rng.integers(len(cand))]
        todo = [pick]
        while todo:
            leaf = todo.pop()
            if leaf not in leaves:
                continue
            # coarser touching leaves must be refined first
            coarser = [m for m in leaves if m[0] < leaf[0] and
                       touching(leaf, m, ndim, base, max_level, periodic)]
            if coarser:
                todo.append(leaf)
                todo.extend(coarser)
                continue
            leaves.remove(leaf)
            leaves.update(children(leaf))
    out = sorted(leaves)
    lev = np.array([l[0] for l in out], dtype=np.int32)
    crd = np.array([l[1] for l in out], dtype=np.int32)
    return lev, crd
