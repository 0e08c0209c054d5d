"""Seeded synthetic CSEM models: Kuhn-split tetrahedral meshes, conductivity models,
dipole sources and receiver lines.

This module builds INPUTS only.  It holds none of the method's arithmetic (no basis
functions, no element integrals, no primary field): both the CUDA path and the CPU
oracle receive what it returns as plain arrays.

The paper meshes its models with Gmsh (Section 4) and reads the mesh from files; those
meshes are not available, so structured cubes split into six tetrahedra each (the Kuhn
split) stand in for them.  The marine geometry follows the canonical reservoir model of
Section 5.1 (seawater over sediment with a thin resistive slab) and the bathymetry
model of Section 5.2 (a non-flat seafloor); the numeric choices of each model are
stated in the functions below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1

# The six axis orders of the Kuhn split, in lexicographic order.  Tet 6*c + p of cell c
# walks from the cell's lowest corner along axes PERMS[p][0], PERMS[p][1], PERMS[p][2].
PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood 2014) on a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def counter_uniform(seed: int, counter: np.ndarray) -> np.ndarray:
    """Counter-based uniform numbers in [0, 1): u = top 53 bits of
    SplitMix64(seed * 2^32 + counter) / 2^53.  Reproducible from the definition alone."""
    key = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) + np.asarray(counter, dtype=np.uint64)
    return (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Mesh:
    n: tuple                     # cells per axis (nx, ny, nz)
    lo: tuple                    # box corner (m)
    hi: tuple                    # box corner (m)
    nodes: np.ndarray            # float64 [n_nodes, 3]
    tets: np.ndarray             # int32 [n_tets, 4]

    @property
    def n_nodes(self) -> int:
        return self.nodes.shape[0]

    @property
    def n_tets(self) -> int:
        return self.tets.shape[0]

    @property
    def h(self) -> tuple:
        return tuple((self.hi[a] - self.lo[a]) / self.n[a] for a in range(3))

    def centroids(self) -> np.ndarray:
        return self.nodes[self.tets].mean(axis=1)


def kuhn_mesh(n, lo, hi, jitter: float = 0.0, seed: int = 12345, warp=None) -> Mesh:
    """Structured box split into n^3 cubes, each cut into 6 tetrahedra.

    Node (i, j, k) has id i + (nx+1) * (j + (ny+1) * k).  Cell (i, j, k) has id
    c = i + nx * (j + ny * k); its tet 6c + p starts at the cell's lowest corner and steps
    +1 along PERMS[p][0], then PERMS[p][1], then PERMS[p][2].  Odd permutations give
    negatively oriented tets; both orientations are left in on purpose.

    jitter: interior nodes move by (2u - 1) * jitter * h_axis per axis, with u from
      counter_uniform(seed, 3 * node + axis).
    warp: optional callable (x, y, z) -> new z applied after the jitter.
    """
    if isinstance(n, int):
        n = (n, n, n)
    xs = [np.linspace(lo[a], hi[a], n[a] + 1) for a in range(3)]
    return kuhn_mesh_axes(xs, jitter=jitter, seed=seed, warp=warp)


def kuhn_mesh_axes(xs, jitter: float = 0.0, seed: int = 12345, warp=None) -> Mesh:
    """The Kuhn split of the tensor-product grid with node coordinates xs[0], xs[1], xs[2]
    (strictly increasing; spacings may vary), numbered as in kuhn_mesh.  jitter is relative to
    the mean spacing of each axis."""
    n = tuple(len(x) - 1 for x in xs)
    nx, ny, nz = n
    lo = tuple(float(x[0]) for x in xs)
    hi = tuple(float(x[-1]) for x in xs)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    nodes = np.stack([xs[0][ii], xs[1][jj], xs[2][kk]], axis=1).astype(np.float64)
    if jitter > 0.0:
        interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny) & (kk > 0) & (kk < nz)
        ids = np.arange(nodes.shape[0], dtype=np.uint64)
        for a in range(3):
            h = (hi[a] - lo[a]) / n[a]
            u = counter_uniform(seed, ids * np.uint64(3) + np.uint64(a))
            nodes[:, a] += np.where(interior, (2.0 * u - 1.0) * jitter * h, 0.0)
    if warp is not None:
        nodes[:, 2] = warp(nodes[:, 0], nodes[:, 1], nodes[:, 2])

    ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    sx, sy = nx + 1, (nx + 1) * (ny + 1)
    step = (1, sx, sy)
    base = ci + sx * cj + sy * ck
    tets = np.empty((base.size, 6, 4), dtype=np.int64)
    for p, perm in enumerate(PERMS):
        v = base.copy()
        tets[:, p, 0] = v
        for m in range(3):
            v = v + step[perm[m]]
            tets[:, p, m + 1] = v
    tets = tets.reshape(-1, 4).astype(np.int32)
    mesh = Mesh(n=tuple(n), lo=tuple(lo), hi=tuple(hi), nodes=nodes, tets=tets)
    if jitter > 0.0 or warp is not None:
        _check_shape(mesh)
    return mesh


def signed_volumes6(mesh: Mesh) -> np.ndarray:
    """6 x signed volume of every tet (a generator-side quality check only)."""
    p = mesh.nodes[mesh.tets]
    return np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]))


def _check_shape(mesh: Mesh) -> None:
    hx, hy, hz = mesh.h
    ref = hx * hy * hz                     # |6V| of an undistorted Kuhn tet
    d = np.abs(signed_volumes6(mesh))
    sign_ok = np.sign(signed_volumes6(mesh))
    parity = np.tile(np.array([1, -1, -1, 1, 1, -1]), mesh.n_tets // 6)
    if d.min() <= 0.05 * ref or not np.all(sign_ok == parity):
        raise ValueError("distorted mesh rejected: min |6V| / h^3 = %.3g" % (d.min() / ref))


# ---------------------------------------------------------------- sources, receivers

@dataclass
class Dipole:
    x: float
    y: float
    z: float
    axis: int = 0          # 0 = x, 1 = y, 2 = z directed (Appendix A, eqs. A.1-A.3)
    moment: float = 1.0    # I * dS in A m


@dataclass
class Model:
    name: str
    mesh: Mesh
    sigma: np.ndarray      # float64 [n_tets], S/m, constant per element
    sigma_p: float         # background conductivity of the primary field
    freq: float            # Hz
    sources: list
    receivers: np.ndarray  # float64 [R, 3]
    extra: dict = field(default_factory=dict)


def _boxes(cen: np.ndarray, sigma: np.ndarray, boxes) -> None:
    for (x0, x1, y0, y1, z0, z1), s in boxes:
        inside = ((cen[:, 0] >= x0) & (cen[:, 0] <= x1) & (cen[:, 1] >= y0) & (cen[:, 1] <= y1)
                  & (cen[:, 2] >= z0) & (cen[:, 2] <= z1))
        sigma[inside] = s


def cube_block_model(n: int = 16) -> Model:
    """Smallest case: cube [-1000, 1000]^3 m, 1 S/m with a 400 x 400 x 100 m block of
    0.01 S/m centred 300 m deep; x-directed unit dipole at (1, 1, 1) m, f = 2 Hz,
    sigma_p = 1 S/m; 21 receivers x = -500..500 m every 50 m, y = 0, z = -100 m."""
    mesh = kuhn_mesh(n, (-1000.0, -1000.0, -1000.0), (1000.0, 1000.0, 1000.0))
    sigma = np.ones(mesh.n_tets)
    _boxes(mesh.centroids(), sigma, [((-200, 200, -200, 200, -350, -250), 0.01)])
    rx = np.stack([np.linspace(-500.0, 500.0, 21), np.zeros(21), np.full(21, -100.0)], axis=1)
    return Model("cube_block_n%d" % n, mesh, sigma, 1.0, 2.0, [Dipole(1.0, 1.0, 1.0, 0, 1.0)], rx)


def whole_space_model(n: int, half: float = 500.0, sigma: float = 0.5, sigma_p: float = 1.0,
                      freq: float = 2.0, src=(0.0, 0.0, 800.0)) -> Model:
    """Uniform whole space sigma != sigma_p, seen through the window [-half, half]^3.
    The dipole sits outside the window, so the primary field is smooth inside it."""
    mesh = kuhn_mesh(n, (-half,) * 3, (half,) * 3)
    rx = np.stack([np.linspace(-0.6 * half, 0.6 * half, 13), np.full(13, 0.11 * half),
                   np.full(13, 0.23 * half)], axis=1)
    return Model("whole_space_n%d" % n, mesh, np.full(mesh.n_tets, sigma), sigma_p, freq,
                 [Dipole(*src, 0, 1.0)], rx)


def relabel(model: Model, seed: int = 20260) -> Model:
    """The same model with its node ids and its tet order randomly permuted (seeded): the geometry,
    the conductivity of every tet and the sources are unchanged, only the numbering loses the
    lattice's locality, as a general unstructured mesher's output may."""
    rng = np.random.default_rng(seed)
    nn, nt = model.mesh.n_nodes, len(model.mesh.tets)
    pn = rng.permutation(nn)           # new node k is old node pn[k]
    inv = np.empty(nn, dtype=np.int64)
    inv[pn] = np.arange(nn)
    pt = rng.permutation(nt)           # new tet k is old tet pt[k]
    mesh = Mesh(model.mesh.n, model.mesh.lo, model.mesh.hi, np.ascontiguousarray(model.mesh.nodes[pn]),
                np.ascontiguousarray(inv[model.mesh.tets[pt]].astype(np.int32)))
    return Model(model.name + "_relabelled", mesh, np.ascontiguousarray(model.sigma[pt]), model.sigma_p, model.freq,
                 list(model.sources), model.receivers, dict(model.extra))


def marine_model(n: int = 64, n_src: int = 1, freq: float = 1.0, jitter: float = 0.18) -> Model:
    """Marine layered model on [-5, 5] x [-5, 5] x [-4, 1] km: seawater 3.3 S/m above
    z = 0, sediment 1 S/m below, a 2 x 2 km x 100 m reservoir slab of 0.01 S/m 1 km below
    the seafloor.  Interior nodes jittered by up to 0.18 h (0.2 h leaves slivers below
    5 % of the undistorted volume at n = 64, which the shape check rejects).  Dipoles 50 m above the
    seafloor (one at x = 0, or n_src spread over x in [-4, 4] km), sigma_p = 3.3 S/m;
    101 receivers on the seafloor, x = -4..4 km every 80 m."""
    mesh = kuhn_mesh(n, (-5000.0, -5000.0, -4000.0), (5000.0, 5000.0, 1000.0), jitter=jitter)
    cen = mesh.centroids()
    sigma = np.where(cen[:, 2] > 0.0, 3.3, 1.0)
    _boxes(cen, sigma, [((-1000, 1000, -1000, 1000, -1100, -1000), 0.01)])
    xs = [0.0] if n_src == 1 else list(np.linspace(-4000.0, 4000.0, n_src))
    rx = np.stack([np.linspace(-4000.0, 4000.0, 101), np.zeros(101), np.zeros(101)], axis=1)
    return Model("marine_n%d" % n, mesh, sigma, 3.3, freq, [Dipole(x, 0.0, 50.0, 0, 1.0) for x in xs], rx)


def seafloor(x: np.ndarray) -> np.ndarray:
    """Sinusoidal bathymetry: amplitude 200 m, wavelength 3 km."""
    return 200.0 * np.sin(2.0 * math.pi * x / 3000.0)


def bathymetry_model(n: int = 96, n_src: int = 32, freq: float = 0.5) -> Model:
    """Largest case: the marine box with the seafloor warped to seafloor(x); nodes move
    vertically by seafloor(x) * w(z), w falling linearly to 0 at the top and bottom faces.
    Two resistive bodies (0.01 and 0.02 S/m) in 1 S/m sediment under 3.3 S/m seawater.
    n_src x-directed dipoles 50 m above the mean seafloor, x in [-4, 4] km."""
    z0, z1 = -4000.0, 1000.0

    def warp(x, y, z):
        w = np.where(z <= 0.0, (z - z0) / (0.0 - z0), (z1 - z) / z1)
        return z + seafloor(x) * w

    mesh = kuhn_mesh(n, (-5000.0, -5000.0, z0), (5000.0, 5000.0, z1), warp=warp)
    cen = mesh.centroids()
    sigma = np.where(cen[:, 2] > seafloor(cen[:, 0]), 3.3, 1.0)
    _boxes(cen, sigma, [((-2000, 0, -1000, 1000, -1200, -1100), 0.01),
                        ((500, 2500, -1000, 1000, -1600, -1500), 0.02)])
    xs = list(np.linspace(-4000.0, 4000.0, n_src)) if n_src > 1 else [0.0]
    srcs = [Dipole(x, 0.0, float(seafloor(np.array([x]))[0]) + 50.0, 0, 1.0) for x in xs]
    rxx = np.linspace(-4000.0, 4000.0, 101)
    rx = np.stack([rxx, np.zeros(101), seafloor(rxx) + 1.0], axis=1)
    return Model("bathymetry_n%d" % n, mesh, sigma, 3.3, freq, srcs, rx)


MU0 = 4.0e-7 * math.pi


def skin_depth(freq: float, sigma: float) -> float:
    """Skin depth sqrt(2 / (mu0 w sigma)) in m (Section 5.3): the depth at which a plane wave in a
    whole space of conductivity sigma has decayed to 1/e."""
    return math.sqrt(2.0 / (MU0 * 2.0 * math.pi * freq * sigma))


def graded_axis(center: float, core_lo: float, core_hi: float, d_s: float, d_delta: float,
                t_lo: float, t_hi: float, s_c: float = 1.04, s_b: float = 1.1) -> np.ndarray:
    """Node coordinates of one axis by the spacing rules of Section 5.3.

    Core [core_lo, core_hi], walked from `center` outward on both sides: the i-th step (i = 1,
    2, ...) is min(s_c^i d_s, d_delta), the power-law stretching of the core.  Boundary layers of
    thickness t_lo below core_lo and t_hi above core_hi: each step is s_b times the one before (the
    boundary stretching), starting from the last core step.  A walk ends exactly on its bound: a
    final step shorter than half the step before it is merged into that step.
    """
    def walk(start, end, first_steps):
        sign = 1.0 if end > start else -1.0
        length = abs(end - start)
        pos, out, i = 0.0, [], 0
        while pos < length:
            step = first_steps(i)
            i += 1
            if pos + step >= length or length - (pos + step) < 0.5 * step:
                out.append(length)
                break
            pos += step
            out.append(pos)
        return [start + sign * v for v in out]

    def layer(start, last_step, thickness, sign):
        if thickness <= 0.0:
            return []
        pos, step, out = 0.0, last_step, []
        while pos < thickness:
            step *= s_b
            if pos + step >= thickness or thickness - (pos + step) < 0.5 * step:
                out.append(thickness)
                break
            pos += step
            out.append(pos)
        return [start + sign * v for v in out]

    core_step = lambda i: min(s_c ** (i + 1) * d_s, d_delta)
    hi_side = walk(center, core_hi, core_step) if core_hi > center else []
    lo_side = walk(center, core_lo, core_step) if core_lo < center else []
    pts = lo_side[::-1] + [center] + hi_side
    last_lo = pts[1] - pts[0] if len(pts) > 1 else d_s
    last_hi = pts[-1] - pts[-2] if len(pts) > 1 else d_s
    pts = layer(core_lo, last_lo, t_lo, -1.0)[::-1] + pts + layer(core_hi, last_hi, t_hi, 1.0)
    return np.array(pts, dtype=np.float64)


def snap_interfaces(axis: np.ndarray, interfaces) -> np.ndarray:
    """Move the interior node nearest to each interface coordinate onto it, so that material
    interfaces are node planes (conforming), as long as both neighbouring spacings stay above
    half their original size."""
    a = axis.copy()
    for v in interfaces:
        if not (a[0] < v < a[-1]):
            continue
        i = int(np.argmin(np.abs(a - v)))
        if i == 0 or i == len(a) - 1:
            continue
        left, right = a[i] - a[i - 1], a[i + 1] - a[i]
        if v - a[i - 1] >= 0.5 * left and a[i + 1] - v >= 0.5 * right:
            a[i] = v
    return a


def graded_marine_model(freq: float = 1.0, L_s: float = 250.0, r_delta: float = 3.0, r_s: float = 13.0,
                        r_xy: float = 8.0, r_z: float = 4.0, r_b: float = 4.0, sigma_min_depth: float = 3.3,
                        sigma_ave: float = 1.0, n_src: int = 1, reservoir: bool = True,
                        z_surface: float = 1000.0) -> Model:
    """The marine model of marine_model on a frequency-adapted graded Kuhn mesh (Section 5.3).

    Spacings: d_delta = delta_min / r_delta with delta_min the skin depth in seawater; near the
    source d_s = min(L_s / r_s, d_delta) (L_s the dipole length).  Extent: the core spans
    x_s +- r_xy delta_ave, y_s +- r_xy delta_ave and, vertically, from r_z delta_ave below the
    source up to the sea surface (the air-water interface closes the domain at the top); boundary
    layers of r_b delta_ave on every other side.  delta_ave is the skin depth at sigma_ave (the
    sediment).  The core is centred on the (first) source.  Conductivities, sources and receivers
    as in marine_model (seawater 3.3 S/m above z = 0 up to the surface at z = 1000 m, sediment
    1 S/m, the 0.01 S/m reservoir slab 1 km down; reservoir=False leaves the two half-spaces alone,
    z_surface moves the top of the domain)."""
    d_min = skin_depth(freq, sigma_min_depth)
    d_ave = skin_depth(freq, sigma_ave)
    d_delta = d_min / r_delta
    d_s = min(L_s / r_s, d_delta)
    xs_src = [0.0] if n_src == 1 else list(np.linspace(-4000.0, 4000.0, n_src))
    src = (xs_src[0], 0.0, 50.0)
    tb = r_b * d_ave
    ax = graded_axis(src[0], src[0] - r_xy * d_ave, src[0] + r_xy * d_ave, d_s, d_delta, tb, tb)
    ay = graded_axis(src[1], src[1] - r_xy * d_ave, src[1] + r_xy * d_ave, d_s, d_delta, tb, tb)
    az = graded_axis(src[2], src[2] - r_z * d_ave, z_surface, d_s, d_delta, tb, 0.0)
    # the seafloor and the reservoir's faces as node planes
    ax = snap_interfaces(ax, (-1000.0, 1000.0))
    ay = snap_interfaces(ay, (-1000.0, 1000.0))
    az = snap_interfaces(az, (0.0, -1000.0, -1100.0))
    mesh = kuhn_mesh_axes([ax, ay, az])
    cen = mesh.centroids()
    sigma = np.where(cen[:, 2] > 0.0, 3.3, 1.0)
    if reservoir:
        _boxes(cen, sigma, [((-1000, 1000, -1000, 1000, -1100, -1000), 0.01)])
    rx = np.stack([np.linspace(-4000.0, 4000.0, 101), np.zeros(101), np.zeros(101)], axis=1)
    return Model("graded_marine_%gHz" % freq, mesh, sigma, 3.3, freq,
                 [Dipole(x, 0.0, 50.0, 0, 1.0) for x in xs_src], rx,
                 extra={"d_delta": d_delta, "d_s": d_s, "delta_ave": d_ave, "delta_min": d_min})


def kuhn_counts(n: int) -> dict:
    """Closed-form counts of a Kuhn-split n^3 cube mesh (a generator property)."""
    e = 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    return {"nodes": (n + 1) ** 3, "tets": 6 * n ** 3, "edges": e, "boundary_edges": 18 * n * n,
            "faces": 12 * n ** 3 + 6 * n * n}


def sources_array(sources) -> np.ndarray:
    """Pack dipoles as float64 [S, 5] = (x, y, z, axis, moment) for the C interfaces."""
    return np.array([[s.x, s.y, s.z, float(s.axis), s.moment] for s in sources], dtype=np.float64)
