"""Pins for the oracle's edge numbering, orientation signs and boundary detection.

Checked against brute force on small meshes, closed-form Kuhn counts, the Euler
characteristic of a ball, and the local edge table of Appendix B (eqs. B.1-B.6, stored in
tests/golden/local_edge_table.txt) with the sign rule of eq. B.16.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1808_00186_gb300 import synth
from tests.golden.tables import local_edge_table


def relabelled(mesh, seed):
    """Same mesh with node ids shuffled, so sorting by id is not trivially the lattice order."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(mesh.n_nodes)
    nodes = np.empty_like(mesh.nodes)
    nodes[perm] = mesh.nodes
    return nodes, perm[mesh.tets].astype(np.int32)


def brute_edges(tets):
    table = local_edge_table()
    pairs = set()
    for t in tets:
        for a, b in table:
            pairs.add((min(t[a], t[b]), max(t[a], t[b])))
    return sorted(pairs)


def brute_boundary_faces(tets):
    count = {}
    for t in tets:
        for f in itertools.combinations(sorted(t.tolist()), 3):
            count[f] = count.get(f, 0) + 1
    return count


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_counts_match_closed_form(n):
    m = synth.kuhn_mesh(n, (0, 0, 0), (1, 1, 1))
    s = oracle.System(m.nodes, m.tets, topology_only=True)
    edges, te, sg, bd = s.topology()
    c = synth.kuhn_counts(n)
    assert s.n_edges == c["edges"]
    assert int(bd.sum()) == c["boundary_edges"]
    # Euler characteristic of a closed ball: V - E + F - T = 1.
    faces = brute_boundary_faces(m.tets)
    assert c["nodes"] - s.n_edges + len(faces) - m.n_tets == 1


def test_single_cube_by_hand():
    m = synth.kuhn_mesh(1, (0, 0, 0), (1, 1, 1))
    s = oracle.System(m.nodes, m.tets, topology_only=True)
    edges, te, sg, bd = s.topology()
    assert s.n_edges == 19
    # The only interior edge of one Kuhn-split cube is its main diagonal, node 0 -> node 7.
    interior = [tuple(e) for e, b in zip(edges, bd) if not b]
    assert interior == [(0, 7)]


@pytest.mark.parametrize("seed", [0, 1])
def test_edges_signs_brute_force(seed):
    m = synth.kuhn_mesh(3, (0, 0, 0), (3, 3, 3))
    nodes, tets = relabelled(m, seed)
    s = oracle.System(nodes, tets, topology_only=True)
    edges, te, sg, bd = s.topology()
    ref = brute_edges(tets)
    assert [tuple(e) for e in edges] == ref               # lexicographic rank = edge id
    table = local_edge_table()
    for t in range(tets.shape[0]):
        for i, (a, b) in enumerate(table):
            n1, n2 = tets[t, a], tets[t, b]
            assert tuple(edges[te[t, i]]) == (min(n1, n2), max(n1, n2))
            assert sg[t, i] == (1 if n2 > n1 else -1)       # eq. B.16


def test_boundary_brute_force():
    m = synth.kuhn_mesh(3, (0, 0, 0), (3, 3, 3))
    nodes, tets = relabelled(m, 7)
    s = oracle.System(nodes, tets, topology_only=True)
    edges, te, sg, bd = s.topology()
    faces = brute_boundary_faces(tets)
    ref = set()
    for f, c in faces.items():
        if c == 1:
            for a, b in itertools.combinations(f, 2):
                ref.add((a, b))
    got = {tuple(e) for e, b in zip(edges, bd) if b}
    assert got == ref
    # Every boundary edge lies on the surface of the box.
    mid = 0.5 * (nodes[edges[:, 0]] + nodes[edges[:, 1]])
    on_surface = np.any((np.abs(mid) < 1e-12) | (np.abs(mid - 3.0) < 1e-12), axis=1)
    # an interior edge can touch the surface only at one end, never have its midpoint on it
    assert np.array_equal(on_surface.astype(np.uint8), bd)


def test_rejects_nonmanifold_and_repeated_nodes():
    tets = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], np.int32)
    nodes = np.random.default_rng(0).normal(size=(6, 3))
    with pytest.raises(ValueError):
        oracle.System(nodes, tets, topology_only=True)
    with pytest.raises(ValueError):
        oracle.System(nodes, np.array([[0, 1, 1, 3]], np.int32), topology_only=True)
