"""FP64 CPU oracle of the primary field of a horizontal electric dipole in a horizontally layered
Earth (Section 2: for a layered background the primary field is computed semi-analytically by
Hankel transforms).

TEST INFRASTRUCTURE (like the rest of oracle/): used only by tests/ and the benchmark's CPU legs;
it shares no code with the CUDA library.

The paper names Hankel transform filters without giving any; this oracle evaluates the same
Hankel integrals by a fixed Gauss-Legendre panel rule (quadrature_nodes below), written out so
that the CUDA kernel uses the same nodes.  Convention as for the whole-space field (App. A):
operator curl curl E + i w mu0 sigma E, e^{-ikr} decay, d = x - x_s.

Derivation (quasi-static Maxwell equations, horizontal Fourier transform with e^{+i kappa . rho},
the frame rotated so that kappa = lambda x'): the field of a unit horizontal current sheet splits
into two scalar problems in z, with u_j^2 = lambda^2 + i w mu0 sigma_j (Re u_j > 0):
  TE (current along z x kappa):  e'' - u^2 e = i w mu0 delta(z - z_s); e, e' continuous at
      interfaces; e -> 0 at +-infinity.  E_TE = e (the field along z x kappa).
  TM (current along kappa):      h'' - u^2 h = 0 off the source, [h]_{z_s} = -1, [h']_{z_s} = 0;
      h and h' / sigma continuous at interfaces.  E_TM = -h' / sigma (along kappa),
      E_z = i lambda h / sigma.
The angular integrals (int cos^2 phi e^{i a cos(phi - theta)} = pi (J0 - J2 cos 2 theta) etc.) give,
for an x-directed dipole of moment p and (rho, theta) the polar offset of the point,
  E_x = p / (4 pi) int lambda [(E_TM + E_TE) J0 - (E_TM - E_TE) J2 cos 2 theta] dlambda
  E_y = -p / (4 pi) int lambda (E_TM - E_TE) J2 sin 2 theta dlambda
  E_z = i p / (2 pi) int lambda E_z,TM J1 cos theta dlambda.
In a whole space E_TE = -i w mu0 e^{-u|z-z_s|} / (2u), E_TM = -u e^{-u|z-z_s|} / (2 sigma): the
integrals then equal App. A's closed form.  Here the field is written as App. A's whole-space
field of the source layer's conductivity plus the Hankel integrals of (layered - whole-space)
spectra, which decay exponentially in lambda away from the source depth.
"""
from __future__ import annotations

import numpy as np
import scipy.special as ss

MU0 = 4e-7 * np.pi
GL_ORDER = 8
DECAY = 36.0          # integrate up to lambda_max = DECAY / D (e^-36 ~ 2e-16 of the spectrum left)
MAX_PANELS = 16384


# ---------------------------------------------------------------- layered model
def layer_of(z: float, z_if: np.ndarray) -> int:
    """Index of the layer holding height z: interfaces z_if strictly decreasing (z up), layer 0
    above z_if[0], layer j between z_if[j] and z_if[j-1]; a point on an interface belongs to the
    layer above it."""
    j = 0
    for zi in z_if:
        if z < zi:
            j += 1
        else:
            break
    return j


def mode_spectra(lam: np.ndarray, z: float, zs: float, z_if: np.ndarray, sig: np.ndarray, omega: float):
    """(E_TE, E_TM, Ez_TM) at height z for unit currents at zs, for every lambda: the two 1-D
    boundary-value problems solved as one linear system per lambda.  Unknowns: in every layer
    (the source layer split at zs into two) the amplitudes of two exponentials normalised to 1 at
    the layer's own top and bottom, e^{-u (z_top - z)} and e^{-u (z - z_bot)}; half-spaces keep
    only the decaying one.  Rows: continuity (or the source jump) of f and of f' / eps across every
    interface, eps = 1 (TE) or sigma (TM)."""
    lam = np.asarray(lam, dtype=np.float64)
    # sub-layers: boundaries from the top, the source depth inserted
    bounds = list(z_if)
    s = layer_of(zs, z_if)
    bounds.insert(s, zs)                       # zs lies between z_if[s-1] and z_if[s]
    sub_sig = list(sig[:s + 1]) + list(sig[s:])  # the source layer appears twice
    nsub = len(sub_sig)
    # unknown index: sub-layer k has (top-anchored, bottom-anchored) amplitudes; the top half-space
    # keeps only its bottom-anchored term (decays upward), the bottom half-space only its top-anchored
    idx = {}
    n = 0
    for k in range(nsub):
        if k > 0:
            idx[(k, "t")] = n
            n += 1
        if k < nsub - 1:
            idx[(k, "b")] = n
            n += 1
    u = np.sqrt(lam[:, None] ** 2 + 1j * omega * MU0 * np.asarray(sub_sig)[None, :])   # [M, nsub]

    def basis(k, zz):
        """values and z-derivatives of sub-layer k's two exponentials at height zz: [M] each."""
        out = {}
        if k > 0:   # e^{-u (z_top - z)}, z_top = bounds[k-1]
            ztop = bounds[k - 1]
            v = np.exp(-u[:, k] * (ztop - zz))
            out["t"] = (v, u[:, k] * v)
        if k < nsub - 1:  # e^{-u (z - z_bot)}, z_bot = bounds[k]
            zbot = bounds[k]
            v = np.exp(-u[:, k] * (zz - zbot))
            out["b"] = (v, -u[:, k] * v)
        return out

    results = {}
    for mode in ("TE", "TM"):
        eps = np.ones(nsub) if mode == "TE" else np.asarray(sub_sig, dtype=np.float64)
        A = np.zeros((lam.size, n, n), dtype=np.complex128)
        rhs = np.zeros((lam.size, n), dtype=np.complex128)
        row = 0
        for i in range(nsub - 1):                 # boundary between sub-layers i (above) and i + 1
            zb = bounds[i]
            up, dn = basis(i, zb), basis(i + 1, zb)
            src = i == s                          # the boundary at zs
            # f(above) - f(below) = jump_f ; f'/eps(above) - f'/eps(below) = jump_g
            for key, (v, dv) in up.items():
                A[:, row, idx[(i, key)]] += v
                A[:, row + 1, idx[(i, key)]] += dv / eps[i]
            for key, (v, dv) in dn.items():
                A[:, row, idx[(i + 1, key)]] -= v
                A[:, row + 1, idx[(i + 1, key)]] -= dv / eps[i + 1]
            if src:
                if mode == "TE":   # g'' - u^2 g = delta: [g] = 0, [g'] = 1 (above minus below)
                    rhs[:, row + 1] = 1.0
                else:              # [h] = -1, [h'] = 0
                    rhs[:, row] = -1.0
            row += 2
        coef = np.linalg.solve(A, rhs[..., None])[..., 0]
        # evaluate at z: its sub-layer (ties go to the layer above, and z = zs to the part above)
        k = layer_of(z, np.asarray(bounds))
        f = np.zeros(lam.size, dtype=np.complex128)
        df = np.zeros(lam.size, dtype=np.complex128)
        for key, (v, dv) in basis(k, z).items():
            f += coef[:, idx[(k, key)]] * v
            df += coef[:, idx[(k, key)]] * dv
        results[mode] = (f, df, sub_sig[k])
    e, _, _ = results["TE"]
    h, dh, sk = results["TM"]
    return 1j * omega * MU0 * e, -dh / sk, 1j * lam * h / sk


def whole_space_spectra(lam, z, zs, sigma, omega):
    """The same three spectra in a whole space of conductivity sigma (closed form)."""
    u = np.sqrt(lam ** 2 + 1j * omega * MU0 * sigma)
    dz = z - zs
    ex = np.exp(-u * abs(dz))
    sgn = 1.0 if dz >= 0 else -1.0
    return -1j * omega * MU0 * ex / (2 * u), -u * ex / (2 * sigma), -1j * lam * sgn * ex / (2 * sigma)


# ---------------------------------------------------------------- the quadrature rule
def decay_length(z: float, zs: float, z_if: np.ndarray) -> float:
    """Distance D over which the (layered - whole-space) spectrum decays like e^{-lambda D}: the
    shortest reflected path (source to an interface of the source layer and back to z) when z is in
    the source layer, else |z - zs| (the transmitted field); at least 1e-3 m."""
    s, j = layer_of(zs, z_if), layer_of(z, z_if)
    if j != s:
        return max(abs(z - zs), 1e-3)
    d = np.inf
    if s > 0:
        d = min(d, (z_if[s - 1] - zs) + (z_if[s - 1] - z))
    if s < len(z_if):
        d = min(d, (zs - z_if[s]) + (z - z_if[s]))
    return max(d, 1e-3)


def panel_edges(rho: float, D: float, kmin: float) -> np.ndarray:
    """Panel edges of the lambda rule: lambda_max = DECAY / D; the first panel [0, kmin / 16]
    (kmin = the smallest |k_j| = sqrt(w mu0 sigma_j) of the model, the scale of the spectra's branch
    points near lambda = 0), then panels that double in width until they reach the cap
    w = min(pi / rho, lambda_max / 16) (half a period of the Bessel kernels), then panels of width w;
    the last edge is lambda_max; at most MAX_PANELS panels."""
    lmax = DECAY / D
    w = lmax / 16.0
    if rho > 0.0:
        w = min(w, np.pi / rho)
    edges = [0.0, min(kmin / 16.0, lmax)]
    while edges[-1] < lmax and len(edges) <= MAX_PANELS:
        edges.append(min(edges[-1] + min(edges[-1], w), lmax))
    return np.array(edges)


def quadrature_nodes(rho: float, D: float, kmin: float):
    """Gauss-Legendre nodes and weights (GL_ORDER points per panel) on the panels of panel_edges."""
    e = panel_edges(rho, D, kmin)
    x, wt = np.polynomial.legendre.leggauss(GL_ORDER)
    a, h = e[:-1, None], (e[1:] - e[:-1])[:, None]
    return (a + 0.5 * h * (x[None, :] + 1.0)).reshape(-1), (0.5 * h * wt[None, :]).reshape(-1)


def kmin_of(sig, freq: float) -> float:
    return float(np.sqrt(2.0 * np.pi * freq * MU0 * np.min(np.atleast_1d(sig))))


# ---------------------------------------------------------------- the field
def whole_space_field(p, src, sigma, freq):
    """App. A closed form (the oracle's own whole-space routine)."""
    import oracle
    return oracle.primary_field(np.asarray(p, dtype=np.float64).reshape(1, 3), src, sigma, freq)[0]


def primary_field(pts: np.ndarray, src, z_if, sig, freq: float) -> np.ndarray:
    """Primary field [n, 3] (complex) of a horizontal dipole src = (x, y, z, axis, moment), axis 0
    (x) or 1 (y), in the layered model (interfaces z_if decreasing, conductivities sig, one more
    than interfaces), at the points pts [n, 3]."""
    z_if = np.asarray(z_if, dtype=np.float64)
    sig = np.asarray(sig, dtype=np.float64)
    xs, ys, zs, axis, mom = src
    axis = int(axis)
    if axis not in (0, 1):
        raise ValueError("layered primary field: horizontal dipoles only")
    omega = 2.0 * np.pi * freq
    s = layer_of(zs, z_if)
    out = np.zeros((len(pts), 3), dtype=np.complex128)
    for i, p in enumerate(np.asarray(pts, dtype=np.float64)):
        dx, dy, z = p[0] - xs, p[1] - ys, p[2]
        if axis == 1:                        # rotate the offset by -90 degrees: x-dipole frame
            dx, dy = dy, -dx
        rho = np.hypot(dx, dy)
        th = np.arctan2(dy, dx) if rho > 0 else 0.0
        lam, w = quadrature_nodes(rho, decay_length(z, zs, z_if), kmin_of(sig, freq))
        te, tm, tz = mode_spectra(lam, z, zs, z_if, sig, omega)
        te0, tm0, tz0 = whole_space_spectra(lam, z, zs, sig[s], omega)
        dte, dtm, dtz = te - te0, tm - tm0, tz - tz0
        x = lam * rho
        J0, J1, J2 = ss.jv(0, x), ss.jv(1, x), ss.jv(2, x)
        ex = np.sum(w * lam * ((dtm + dte) * J0 - (dtm - dte) * J2 * np.cos(2 * th))) / (4 * np.pi)
        ey = -np.sum(w * lam * (dtm - dte) * J2) * np.sin(2 * th) / (4 * np.pi)
        ez = 1j * np.sum(w * lam * dtz * J1) * np.cos(th) / (2 * np.pi)
        e = mom * np.array([ex, ey, ez])
        if axis == 1:                        # rotate the field back by +90 degrees
            e = np.array([-e[1], e[0], e[2]])
        out[i] = e + whole_space_field(p, src, sig[s], freq)
    return out


def spectral_field(p, src, sigma, freq, D):
    """The whole-space field of an x- or y-dipole from the Hankel integrals of the whole-space
    spectra with the same quadrature rule (decay length D = |z - z_s|), for the pin against App. A."""
    xs, ys, zs, axis, mom = src
    omega = 2.0 * np.pi * freq
    dx, dy, z = p[0] - xs, p[1] - ys, p[2]
    if int(axis) == 1:
        dx, dy = dy, -dx
    rho = np.hypot(dx, dy)
    th = np.arctan2(dy, dx) if rho > 0 else 0.0
    lam, w = quadrature_nodes(rho, D, kmin_of(sigma, freq))
    te, tm, tz = whole_space_spectra(lam, z, zs, sigma, omega)
    x = lam * rho
    J0, J1, J2 = ss.jv(0, x), ss.jv(1, x), ss.jv(2, x)
    ex = np.sum(w * lam * ((tm + te) * J0 - (tm - te) * J2 * np.cos(2 * th))) / (4 * np.pi)
    ey = -np.sum(w * lam * (tm - te) * J2) * np.sin(2 * th) / (4 * np.pi)
    ez = 1j * np.sum(w * lam * tz * J1) * np.cos(th) / (2 * np.pi)
    e = mom * np.array([ex, ey, ez])
    if int(axis) == 1:
        e = np.array([-e[1], e[0], e[2]])
    return e


# ---------------------------------------------------------------- right-hand sides (eq. 6)
LOCAL_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (3, 1), (2, 3)]   # eqs. B.1-B.6 (N5 = W42)


def layer_sigma(z: float, z_if, sig) -> float:
    return float(np.asarray(sig)[layer_of(z, np.asarray(z_if, dtype=np.float64))])


def rhs(nodes, tets, sigma, z_if, sig, freq, sources, tet_edges, signs, boundary, n_edges):
    """b[s][e] of eq. 6 with the layered background: for every tet whose conductivity differs from
    that of the layer holding its centroid, b^e_k = -i w mu0 (sigma_e - sigma_layer) sum_q (V/4)
    N_k(x_q) . E_p(x_q) on the oracle's 4-point rule (oracle.quadrature), N_k = S_k l_k (lambda_a
    grad lambda_b - lambda_b grad lambda_a); gathered over the edges, zero on boundary edges."""
    import oracle
    z_if = np.asarray(z_if, dtype=np.float64)
    omega = 2.0 * np.pi * freq
    Q = oracle.quadrature()                 # rows: barycentric coordinates of the 4 points
    b = np.zeros((len(sources), n_edges), dtype=np.complex128)
    for t in range(len(tets)):
        P = nodes[tets[t]]
        ds = sigma[t] - layer_sigma(P[:, 2].mean(), z_if, sig)
        if ds == 0.0:
            continue
        c0, grad, ln, vol = oracle.geometry(P)
        xq = Q[:, :4] @ P                    # [4 points][3]
        for si, src in enumerate(sources):
            Ep = primary_field(xq, src, z_if, sig, freq)
            for k, (a, bb) in enumerate(LOCAL_EDGES):
                acc = 0.0
                for q in range(4):
                    lam = Q[q, :4]
                    N = signs[t, k] * ln[k] * (lam[a] * grad[bb] - lam[bb] * grad[a])
                    acc = acc + N @ Ep[q]
                b[si, tet_edges[t, k]] += -1j * omega * MU0 * ds * (vol / 4.0) * acc
    b[:, boundary == 1] = 0.0
    return b
