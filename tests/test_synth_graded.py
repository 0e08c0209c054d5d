"""The frequency-adapted graded Kuhn generator (synth.graded_axis, synth.graded_marine_model)
against the spacing rules of the paper's Section 5.3, written out here from their definitions:
skin depth sqrt(2 / (mu0 w sigma)) (about 503 / sqrt(f sigma) m, 275 / sqrt(f) in 3.3 S/m
seawater), d_delta = delta_min / r_delta, d_s = min(L_s / r_s, d_delta), core steps
min(s_c^i d_s, d_delta), boundary steps growing by s_b, and the domain extents."""
import math

import numpy as np
import pytest

from paper_1808_00186_gb300 import synth


def test_skin_depth_matches_the_papers_rules_of_thumb():
    for f in (0.25, 1.0, 2.0):
        assert synth.skin_depth(f, 1.0) == pytest.approx(503.0 / math.sqrt(f), rel=2e-3)
        assert synth.skin_depth(f, 3.3) == pytest.approx(275.0 / math.sqrt(f), rel=1e-2)
        assert synth.skin_depth(f, 0.5) == pytest.approx(503.0 * math.sqrt(1.0 / (f * 0.5)), rel=2e-3)


def test_graded_axis_steps_follow_the_power_laws():
    d_s, d_delta, s_c, s_b = 10.0, 40.0, 1.04, 1.1
    a = synth.graded_axis(0.0, -1000.0, 2000.0, d_s, d_delta, 500.0, 300.0, s_c, s_b)
    assert np.all(np.diff(a) > 0)
    assert a[0] == pytest.approx(-1500.0) and a[-1] == pytest.approx(2300.0)
    c = int(np.argmin(np.abs(a)))
    assert a[c] == 0.0
    up = np.diff(a[c:])
    # core: step i = min(s_c^i d_s, d_delta), i = 1, 2, ... (the last core step may absorb a remainder)
    core_hi = int(np.argmin(np.abs(a - 2000.0)))
    n_core = core_hi - c
    for i in range(1, n_core):
        assert up[i - 1] == pytest.approx(min(s_c ** i * d_s, d_delta), rel=1e-12)
    # boundary layer above: each step s_b times the previous one (the last may absorb a remainder)
    layer = np.diff(a[core_hi:])
    prev = a[core_hi] - a[core_hi - 1]
    for k in range(len(layer) - 1):
        assert layer[k] == pytest.approx(s_b * prev, rel=1e-12)
        prev = layer[k]
    # the same rules walking down from the centre
    down = np.diff(a[:c + 1])[::-1]
    for i in range(1, 20):
        assert down[i - 1] == pytest.approx(min(s_c ** i * d_s, d_delta), rel=1e-12)


def test_graded_marine_model_extent_spacing_and_mesh():
    f = 1.0
    m = synth.graded_marine_model(f)
    d_ave, d_min = synth.skin_depth(f, 1.0), synth.skin_depth(f, 3.3)
    assert m.extra["d_delta"] == pytest.approx(d_min / 3.0)
    assert m.extra["d_s"] == pytest.approx(min(250.0 / 13.0, d_min / 3.0))
    nx, ny, nz = m.mesh.n
    assert m.mesh.n_tets == 6 * nx * ny * nz
    # core +- 8 delta_ave plus boundary layers of 4 delta_ave; vertically 4 delta_ave below the
    # source plus a boundary layer, up to the sea surface
    assert m.mesh.hi[0] == pytest.approx(0.0 + 8 * d_ave + 4 * d_ave)
    assert m.mesh.lo[0] == pytest.approx(0.0 - 8 * d_ave - 4 * d_ave)
    assert m.mesh.hi[2] == pytest.approx(1000.0)
    assert m.mesh.lo[2] == pytest.approx(50.0 - 4 * d_ave - 4 * d_ave)
    z = np.unique(m.mesh.nodes[:, 2])
    x = np.unique(m.mesh.nodes[:, 0])
    for v in (0.0, -1000.0, -1100.0):
        assert v in z  # seafloor and reservoir faces are node planes
    for v in (-1000.0, 1000.0):
        assert v in x
    core = (x >= -8 * d_ave) & (x <= 8 * d_ave)
    assert np.diff(x[core]).max() <= m.extra["d_delta"] * (1 + 1e-9) * 1.5  # a merged remainder at most
    assert np.diff(x).min() >= 0.5 * m.extra["d_s"]
    vol = synth.signed_volumes6(m.mesh)
    assert np.all(np.abs(vol) > 0)


def test_graded_small_model_is_conforming():
    m = synth.graded_marine_model(8.0, L_s=400.0, r_xy=1.5, r_z=1.0, r_b=0.5)
    assert m.mesh.n_tets < 120000
    # every tet lies entirely on one side of the seafloor plane z = 0
    zt = m.mesh.nodes[m.mesh.tets][:, :, 2]
    assert np.all((zt.min(axis=1) >= 0.0) | (zt.max(axis=1) <= 0.0))


def test_relabel_keeps_the_geometry_and_each_tets_conductivity():
    m = synth.marine_model(4, n_src=2)
    r = synth.relabel(m, seed=3)
    assert r.mesh.nodes.shape == m.mesh.nodes.shape and r.mesh.tets.shape == m.mesh.tets.shape
    assert r.mesh.tets.dtype == np.int32 and r.mesh.tets.min() >= 0 and r.mesh.tets.max() < r.mesh.n_nodes

    def keyed(mesh, sig):  # each tet as its sorted vertex coordinates, with its conductivity
        P = mesh.nodes[mesh.tets]                                  # [T, 4, 3]
        order = np.lexsort(P.transpose(2, 0, 1)[::-1])            # sort the 4 vertices of each tet
        Ps = np.take_along_axis(P, order[..., None], axis=1).reshape(len(P), 12)
        k = np.lexsort(Ps.T[::-1])
        return Ps[k], sig[k]

    a, sa = keyed(m.mesh, m.sigma)
    b, sb = keyed(r.mesh, r.sigma)
    assert np.array_equal(a, b) and np.array_equal(sa, sb)
    assert not np.array_equal(r.mesh.tets, m.mesh.tets)           # the numbering did change
    assert r.sources == m.sources and r.freq == m.freq and r.sigma_p == m.sigma_p
