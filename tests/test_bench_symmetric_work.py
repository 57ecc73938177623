"""The work accounting of the symmetric Hessian in bench.py, on CPU.

bench.symmetric_lt_entries counts the L^T-sweep entries the symmetric tiles of
the library sweep.  This test counts them a second way, by brute force on the
filled pattern: for each tile, the rows whose Psi the assembly reads (the
right-hand-side rows of the controls from the tile's first column position
on), their elimination-tree ancestors (walked through the parents of L), and
the rows of every bus block that holds one of them; then the strictly upper
entries of those rows.  It also checks the two ends that hold for any tiling:
the last columns sweep at most what the first sweep, and no tile sweeps more
than the whole L^T.
"""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
import paper_2110_02590_b300 as P  # noqa: E402
from paper_2110_02590_b300 import synth  # noqa: E402


def brute_force(net, sym, nu, k, sm_count):
    rp, ci, perm = sym["rowptr"], sym["colidx"], sym["perm"]
    nx = len(perm)
    pos = np.empty(nx, np.int64)
    pos[perm] = np.arange(nx)
    # strictly lower pattern of L by rows, parents, and the upper entries of each row
    parent = [-1] * nx
    upper = np.zeros(nx, np.int64)
    for i in range(nx):
        for j in ci[rp[i]:rp[i + 1]]:
            if j < i and (parent[j] < 0 or i < parent[j]):
                parent[j] = i
            if j > i:
                upper[i] += 1
    nb, ref = net.n_bus, int(net.ref_bus)
    typ = np.zeros(nb, int)
    typ[np.asarray(net.gen_bus, int)] = 1
    typ[ref] = 2
    pv = [b for b in range(nb) if typ[b] == 1]
    pq = [b for b in range(nb) if typ[b] == 0]
    pth = {b: int(pos[q]) for q, b in enumerate(pv + pq)}
    pvv = {b: int(pos[len(pv) + len(pq) + q]) for q, b in enumerate(pq)}
    block = {}
    for b in range(nb):
        rows = [r for r in (pth.get(b), pvv.get(b)) if r is not None]
        for r in rows:
            block[r] = rows
    adj = [set() for _ in range(nb)]
    for f, t in zip(net.br_from, net.br_to):
        adj[int(f)].add(int(t))
        adj[int(t)].add(int(f))
    # the column order of the library's full-Hessian tiling
    children = [[] for _ in range(nx)]
    for j in range(nx):
        if parent[j] >= 0:
            children[parent[j]].append(j)
    post, order = {}, []

    def visit(v):
        stack = [(v, iter(children[v]))]
        while stack:
            node, it = stack[-1]
            nxt = next(it, None)
            if nxt is None:
                post[node] = len(order)
                order.append(node)
                stack.pop()
            else:
                stack.append((nxt, iter(children[nxt])))
    for r in range(nx - 1, -1, -1):
        if parent[r] < 0:
            visit(r)
    cols = [("v", ref)] + [c for b in sorted(pv, key=lambda b: post[pth[b]]) for c in (("v", b), ("p", b))]

    def rhs_rows(c):
        kind, b = c
        if kind == "p":
            return {pth[b]}
        out = {pth[o] for o in adj[b] if typ[o] != 2} | {pvv[o] for o in adj[b] if typ[o] == 0}
        if typ[b] == 1:
            out.add(pth[b])
        return out

    waves = nu // (k * sm_count)
    n1 = waves * sm_count
    rem = nu - n1 * k
    n2 = -(-rem // (k // 2))
    if waves >= 1 and rem > 0 and n2 <= sm_count:
        tiles = [(t * k, k) for t in range(n1)] + \
            [(n1 * k + t * (k // 2), min(k // 2, nu - n1 * k - t * (k // 2))) for t in range(n2)]
    else:
        tiles = [(t * k, min(k, nu - t * k)) for t in range(-(-nu // k))]
    ent = 0
    for p, w in tiles:
        need = set()
        for q in range(p, nu):
            for r in rhs_rows(cols[q]):
                x = r
                while x >= 0 and x not in need:
                    need.add(x)
                    x = parent[x]
        rows = set()
        for r in need:
            rows.update(block[r])
        ent += w * int(sum(upper[r] for r in rows))
    return ent, tiles


@pytest.mark.parametrize("name,k,sm", [("tiny30", 4, 148), ("tiny30", 2, 2), ("batchA500", 8, 148),
                                       ("batchA500", 8, 8)])
def test_symmetric_lt_entries_match_brute_force(name, k, sm):
    net = synth.workload(name)
    sym = P.symbolic_analyze(net)
    nu = 1 + 2 * (net.n_gen - 1)
    ent, ent_tiles, rows = bench.symmetric_lt_entries(net, sym, nu, k, sm)
    ref, tiles = brute_force(net, sym, nu, k, sm)
    assert ent == ref
    nx = len(sym["perm"])
    nnz_strict = (len(sym["colidx"]) - nx) // 2
    assert 0 < ent <= nu * nnz_strict
    assert ent_tiles <= len(tiles) * nnz_strict and rows <= nu * nx
