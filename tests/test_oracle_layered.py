"""Pins for the layered-Earth primary field oracle (oracle/layered.py; Section 2, layered background).

Nothing here retypes the oracle's formulas.  The pins are what the physics fixes:
  * the Hankel integrals of the whole-space spectra reproduce App. A's closed form (checks the
    TE/TM decomposition of the dipole, the angular integrals and the quadrature rule);
  * a model whose layers all have one conductivity is the whole space (the 1-D solves then carry
    no reflection, also through interfaces between equal layers);
  * tangential E and the normal current sigma E_z are continuous across interfaces;
  * the field satisfies the source-free curl-curl equation of each layer (finite differences);
  * a y-directed dipole is the x-directed one rotated by 90 degrees.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import layered as LY

MU0 = 4e-7 * math.pi


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("sigma,freq", [(1.0, 1.0), (3.3, 0.25), (0.3, 3.0)])
def test_hankel_integrals_of_whole_space_spectra_are_appendix_a(axis, sigma, freq):
    src = (5.0, -3.0, -400.0, axis, 1.0)
    for dz, rho, th in [(30.0, 0.0, 0.0), (30.0, 150.0, 0.7), (-200.0, 900.0, 2.1), (120.0, 2500.0, -1.0)]:
        p = np.array([src[0] + rho * math.cos(th), src[1] + rho * math.sin(th), src[2] + dz])
        e_h = LY.spectral_field(p, src, sigma, freq, abs(dz))
        e_a = LY.whole_space_field(p, src, sigma, freq)
        assert rel(e_h, e_a) <= 2e-8, (dz, rho, th, e_h, e_a)


def test_equal_layers_are_the_whole_space():
    z_if = np.array([0.0, -700.0, -1100.0])
    sig = np.array([1.7, 1.7, 1.7, 1.7])
    src = (0.0, 0.0, -350.0, 0, 1.0)
    pts = np.array([[300.0, 40.0, -350.0], [800.0, -500.0, 120.0], [50.0, 20.0, -1500.0], [1200.0, 0.0, -700.0],
                    [-250.0, 60.0, -20.0]])
    e = LY.primary_field(pts, src, z_if, sig, 0.75)
    ref = oracle.primary_field(pts, src, 1.7, 0.75)
    for a, b in zip(e, ref):
        assert rel(a, b) <= 1e-11


@pytest.mark.parametrize("axis", [0, 1])
def test_tangential_field_and_normal_current_are_continuous(axis):
    z_if = np.array([0.0, -900.0, -1000.0])        # seawater, sediment, thin resistor, sediment
    sig = np.array([3.3, 1.0, 0.02, 1.0])
    src = (0.0, 0.0, 50.0, axis, 1.0)
    freq = 0.5
    eps = 1e-6
    for zi, (sa, sb) in zip(z_if, [(3.3, 1.0), (1.0, 0.02), (0.02, 1.0)]):
        for x, y in [(400.0, 0.0), (1500.0, 700.0), (0.0, 2600.0)]:
            up = LY.primary_field(np.array([[x, y, zi + eps]]), src, z_if, sig, freq)[0]
            dn = LY.primary_field(np.array([[x, y, zi - eps]]), src, z_if, sig, freq)[0]
            scale = np.linalg.norm(up[:2])
            assert np.abs(up[:2] - dn[:2]).max() <= 1e-6 * scale, (zi, x, y, up, dn)
            assert abs(sa * up[2] - sb * dn[2]) <= 1e-6 * abs(sa * up[2]) + 1e-6 * scale * sa
    # and the layering matters: the field differs from the source layer's whole space
    p = np.array([[1500.0, 0.0, -500.0]])
    assert rel(LY.primary_field(p, src, z_if, sig, freq)[0], oracle.primary_field(p, src, 3.3, freq)[0]) > 0.1


def test_field_satisfies_each_layers_curl_curl_equation():
    """curl curl E + i w mu0 sigma_j E = 0 inside every layer off the source (fourth-order central
    differences of the oracle's own field)."""
    z_if = np.array([0.0, -800.0])
    sig = np.array([3.3, 1.0, 0.05])
    src = (0.0, 0.0, 60.0, 0, 1.0)
    freq = 1.0
    F = lambda xs: LY.primary_field(np.asarray(xs).reshape(-1, 3), src, z_if, sig, freq)

    def jac(x, h):
        pts = []
        for j in range(3):
            for s in (-2, -1, 1, 2):
                p = np.array(x, dtype=float)
                p[j] += s * h
                pts.append(p)
        v = F(np.array(pts)).reshape(3, 4, 3)
        return ((v[:, 0] - 8 * v[:, 1] + 8 * v[:, 2] - v[:, 3]) / (12 * h)).T   # [i][j] = dE_i/dx_j

    def curl_at(x, h):
        J = jac(x, h)
        return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])

    def curl_curl(x, h):
        pts, vals = [], []
        for j in range(3):
            for s in (-2, -1, 1, 2):
                p = np.array(x, dtype=float)
                p[j] += s * h
                vals.append(curl_at(p, h))
        v = np.array(vals).reshape(3, 4, 3)
        J = ((v[:, 0] - 8 * v[:, 1] + 8 * v[:, 2] - v[:, 3]) / (12 * h)).T
        return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])

    w = 2 * math.pi * freq
    for x, sj in [([700.0, 300.0, 250.0], 3.3), ([900.0, -200.0, -400.0], 1.0), ([600.0, 500.0, -1300.0], 0.05)]:
        h = 8.0
        cc = curl_curl(x, h)
        E = F(np.array([x]))[0]
        res = cc + 1j * w * MU0 * sj * E
        assert np.linalg.norm(res) <= 2e-3 * np.linalg.norm(1j * w * MU0 * sj * E), (x, res, E)


def test_y_dipole_is_the_rotated_x_dipole():
    z_if = np.array([0.0, -600.0])
    sig = np.array([3.3, 1.0, 0.1])
    sx = (10.0, 20.0, 40.0, 0, 2.0)
    sy = (10.0, 20.0, 40.0, 1, 2.0)
    p = np.array([[410.0, -130.0, -80.0]])
    # rotating the configuration by +90 degrees about the source's vertical line
    d = p[0, :2] - np.array(sx[:2])
    pr = np.array([[sx[0] - d[1], sx[1] + d[0], p[0, 2]]])
    ex = LY.primary_field(p, sx, z_if, sig, 0.8)[0]
    ey = LY.primary_field(pr, sy, z_if, sig, 0.8)[0]
    assert rel(ey, np.array([-ex[1], ex[0], ex[2]])) <= 1e-12


def test_quadrature_rule_and_layer_lookup():
    e = LY.panel_edges(0.0, 10.0, 1e-3)
    assert e[0] == 0.0 and np.isclose(e[1], 1e-3 / 16) and e[-1] == LY.DECAY / 10.0
    assert np.all(np.diff(e) > 0) and np.allclose(np.diff(e)[1:6], e[1:6])   # doubling at first
    lam, w = LY.quadrature_nodes(2000.0, 50.0, 1e-3)
    assert np.isclose(np.sum(w * np.exp(-lam * 50.0)), (1 - math.exp(-LY.DECAY)) / 50.0, rtol=1e-13)
    assert np.diff(LY.panel_edges(2000.0, 50.0, 1e-3)).max() <= math.pi / 2000.0 * (1 + 1e-12)
    z_if = np.array([0.0, -100.0])
    assert [LY.layer_of(z, z_if) for z in (5.0, 0.0, -50.0, -100.0, -101.0)] == [0, 0, 1, 1, 2]


def test_layered_rhs_with_equal_layers_is_the_assembled_whole_space_rhs():
    """The layered right-hand side restated in Python equals the C++ oracle's assembled b (its own
    whole-space field and quadrature, pinned elsewhere) when every layer has the background
    conductivity."""
    from paper_1808_00186_gb300 import synth
    m = synth.kuhn_mesh(3, (-600.0, -600.0, -600.0), (600.0, 600.0, 600.0), jitter=0.1)
    cen = m.centroids()
    sigma = np.where(np.all(np.abs(cen - 150.0) < 250.0, axis=1), 0.05, 1.3)
    srcs = [(20.0, -10.0, 400.0, 0, 1.0), (-30.0, 15.0, 420.0, 1, 2.0)]
    ref = oracle.System(m.nodes, m.tets, sigma, 1.3, 1.5, np.array(srcs))
    edges, te, sg, bd = ref.topology()
    b_ref = ref.system()[3]
    b = LY.rhs(m.nodes, m.tets, sigma, [100.0, -200.0], [1.3, 1.3, 1.3], 1.5, srcs, te, sg, bd, ref.n_edges)
    assert np.abs(b_ref).max() > 0
    assert rel(b, b_ref) <= 1e-10
