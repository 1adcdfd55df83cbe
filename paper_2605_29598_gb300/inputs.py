"""Seeded synthetic inputs: hex/quad meshes with 2:1 refinement and the
initial atmospheres of the rotating IMEX-DG test cases.

This module holds no DG arithmetic.  It produces the host lists that
``dg_mesh_create`` takes (cell vertices, interior / hanging / boundary face
lists) and evaluates analytic initial states at given physical points.  Both
the CUDA path and the CPU oracle consume what it returns.

Conventions (shared by every consumer of these lists):

* Reference cell [0,1]^d.  Vertex ``v`` of a cell sits at reference corner
  ``(v & 1, (v >> 1) & 1[, (v >> 2) & 1])`` (lexicographic, x fastest).
* Face ``f = 2*a + s`` lies at reference coordinate ``xi_a = s``;
  2D: 0/1 = -x/+x, 2/3 = -z/+z; 3D: 0..5 = -x,+x,-y,+y,-z,+z.
* Interior face row ``[eL, fL, eR, fR]`` with ``fL = 2a+1`` and ``fR = 2a``:
  ``eL`` lies on the low side in direction ``a``.  Periodic pairs are listed
  the same way.
* Hanging face row ``[e_coarse, f_coarse, e_fine, f_fine, subface]``: the
  fine cell's face covers one half (2D) or quarter (3D) of the coarse face;
  bit ``t`` of ``subface`` says which half along the ``t``-th tangential
  direction (tangential directions in increasing order).
* Boundary face row ``[e, f, bc]`` with ``bc = BC_WALL`` (or ``BC_FARFIELD``,
  see ``with_boundary``; the oracle and the CUDA library support it).
* Physical coordinates are (x, z) in 2D (vertical x-z slice) and (x, y, z)
  in 3D; the vertical is always the last coordinate.

The vertical-slice, hill, background and perturbation formulas follow the
paper's test cases: the slice model (Section 2, eq. vertical_slice), the bell
mountain (eq. bell_mountain), the Exner-pressure background (eq. init_cond)
and the Gal-Chen terrain-following map named in Section 4.3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_WALL = 1
BC_FARFIELD = 2

# physical constants of the paper's experiments (Section 4: gamma, g, R)
GAMMA = 1.4
GRAV = 9.81
R_GAS = 287.0
CP = GAMMA * R_GAS / (GAMMA - 1.0)
P_REF = 1.0e5


@dataclass
class Mesh:
    """Host description of a mesh, in the layout ``dg_mesh_create`` takes."""

    dim: int
    vertices: np.ndarray          # (n_elem, 2**dim, dim) float64
    int_faces: np.ndarray         # (n_int, 4) int64
    hang_faces: np.ndarray        # (n_hang, 5) int64
    bdry_faces: np.ndarray        # (n_bdry, 3) int64
    level: np.ndarray = field(default=None)  # (n_elem,) refinement level
    name: str = ""

    @property
    def n_elem(self) -> int:
        return int(self.vertices.shape[0])


def bell_height(x, y, h0, a_c, xc, yc):
    """Bell-shaped mountain h(x, y) of eq. bell_mountain."""
    return h0 / (1.0 + ((x - xc) ** 2 + (y - yc) ** 2) / a_c ** 2)


def _corner_bits(dim):
    return np.array([[(v >> a) & 1 for a in range(dim)] for v in range(1 << dim)],
                    dtype=np.float64)


def _multilinear(verts, ref_pts):
    """Multilinear interpolation of cell vertices at reference points.

    verts: (..., 2**d, d); ref_pts: (m, d) -> (..., m, d)."""
    d = ref_pts.shape[1]
    bits = _corner_bits(d)                                   # (2^d, d)
    w = np.prod(np.where(bits[None, :, :] > 0.5, ref_pts[:, None, :],
                         1.0 - ref_pts[:, None, :]), axis=2)  # (m, 2^d)
    return np.einsum("mv,...vd->...md", w, verts)


def _uniform_mesh(cells, periodic, verts, name):
    """Face lists of an unrefined structured mesh (cell index x fastest),
    built with array arithmetic."""
    d = len(cells)
    n = int(np.prod(cells))
    e = np.arange(n, dtype=np.int64)
    coords = [(e // int(np.prod(cells[:a]))) % cells[a] for a in range(d)]
    int_faces, bdry_faces = [], []
    for a in range(d):
        stride = int(np.prod(cells[:a]))
        ca = coords[a]
        inner = ca < cells[a] - 1
        eL = e[inner]
        int_faces.append(np.stack([eL, np.full_like(eL, 2 * a + 1), eL + stride,
                                   np.full_like(eL, 2 * a)], axis=1))
        last = e[ca == cells[a] - 1]
        first = e[ca == 0]
        if periodic[a]:
            if cells[a] > 1:
                int_faces.append(np.stack([last, np.full_like(last, 2 * a + 1),
                                           last - (cells[a] - 1) * stride,
                                           np.full_like(last, 2 * a)], axis=1))
        else:
            bdry_faces.append(np.stack([first, np.full_like(first, 2 * a),
                                        np.full_like(first, BC_WALL)], axis=1))
            bdry_faces.append(np.stack([last, np.full_like(last, 2 * a + 1),
                                        np.full_like(last, BC_WALL)], axis=1))
    i64 = lambda lst, w: (np.concatenate(lst).astype(np.int64) if lst
                          else np.zeros((0, w), dtype=np.int64))
    return Mesh(dim=d, vertices=verts, int_faces=i64(int_faces, 4),
                hang_faces=np.zeros((0, 5), dtype=np.int64), bdry_faces=i64(bdry_faces, 3),
                level=np.zeros(n, dtype=np.int64), name=name)


def box_mesh(cells, extent, periodic=None, hill=None, z_top=None,
             refine_level=None, name=""):
    """Structured box mesh, optionally terrain-following and locally refined.

    cells:    (nx, nz) or (nx, ny, nz) base cells.
    extent:   (Lx, Lz) or (Lx, Ly, Lz) in metres; the box starts at 0.
    periodic: per direction; default periodic horizontally, walls in z.
    hill:     dict(h0, a_c, xc, yc) for the Gal-Chen map
              z = zeta + h(x, y) (1 - zeta / z_top) applied to base vertices.
    refine_level: callable(center (d,)) -> int level in {0, 1, 2} for a base
              cell with flat-box centre ``center``; levels are then raised
              until face neighbours differ by at most one (2:1 balance).
              Refined children are placed by multilinear interpolation of
              their parent, which keeps hanging faces watertight; a
              horizontal coordinate that depends on its own reference
              direction only (every Gal-Chen cell) keeps that property
              exactly, so refined meshes stay terrain-following.
    """
    d = len(cells)
    cells = tuple(int(c) for c in cells)
    extent = tuple(float(e) for e in extent)
    if periodic is None:
        periodic = tuple([True] * (d - 1) + [False])
    z_top = extent[-1] if z_top is None else z_top
    nb = int(np.prod(cells))
    strides = [int(np.prod(cells[:a])) for a in range(d)]

    def bidx(c):
        return sum(int(c[a]) * strides[a] for a in range(d))

    bcoords = np.stack(np.meshgrid(*[np.arange(n) for n in cells], indexing="ij"),
                       axis=-1).reshape(-1, d)
    # lexicographic with x fastest
    order = np.lexsort([bcoords[:, a] for a in range(d)])
    bcoords = bcoords[order]
    h = [extent[a] / cells[a] for a in range(d)]
    bits = _corner_bits(d).astype(np.int64)
    base_verts = np.zeros((nb, 1 << d, d))
    for v in range(1 << d):
        base_verts[:, v, :] = (bcoords + bits[v]) * np.array(h)
    if hill is not None:
        xs = base_verts[..., 0]
        ys = base_verts[..., 1] if d == 3 else np.full_like(xs, hill.get("yc", 0.0))
        hh = bell_height(xs, ys, hill["h0"], hill["a_c"], hill["xc"],
                         hill.get("yc", 0.0))
        zeta = base_verts[..., d - 1]
        base_verts[..., d - 1] = zeta + hh * (1.0 - zeta / z_top)

    if refine_level is None:
        return _uniform_mesh(cells, periodic, base_verts, name)

    # refinement levels per base cell, then 2:1 balance across faces
    lev = np.zeros(nb, dtype=np.int64)
    if refine_level is not None:
        centers = (bcoords + 0.5) * np.array(h)
        lev = np.array([int(refine_level(c)) for c in centers], dtype=np.int64)

    def nbr_base(c, a, s):
        c2 = np.array(c)
        c2[a] += 1 if s else -1
        if c2[a] < 0 or c2[a] >= cells[a]:
            if not periodic[a]:
                return -1
            c2[a] %= cells[a]
        return bidx(c2)

    changed = True
    while changed:
        changed = False
        for b in range(nb):
            for a in range(d):
                for s in (0, 1):
                    nbb = nbr_base(bcoords[b], a, s)
                    if nbb >= 0 and lev[nbb] < lev[b] - 1:
                        lev[nbb] = lev[b] - 1
                        changed = True

    # enumerate cells: each base cell replaced by its 2^(d*L) children
    start = np.zeros(nb + 1, dtype=np.int64)
    start[1:] = np.cumsum((1 << (d * lev)).astype(np.int64))
    n_elem = int(start[-1])
    verts = np.zeros((n_elem, 1 << d, d))
    level = np.zeros(n_elem, dtype=np.int64)
    local = []          # per cell: (base, local coords)
    for b in range(nb):
        L = int(lev[b])
        m = 1 << L
        lc = np.stack(np.meshgrid(*[np.arange(m)] * d, indexing="ij"), axis=-1).reshape(-1, d)
        lc = lc[np.lexsort([lc[:, a] for a in range(d)])]
        corners = ((lc[:, None, :] + bits[None, :, :]) / m).reshape(-1, d)
        cv = _multilinear(base_verts[b], corners)
        # a horizontal coordinate that depends only on its own reference
        # direction in the base cell keeps that property exactly in the
        # children: (1 - t) x0 + t x1 is the same number for every corner
        # with the same t (the sum over all corners is not)
        for c in range(d - 1):
            bit = 1 << c
            x0, x1 = base_verts[b, 0, c], base_verts[b, bit, c]
            if all(base_verts[b, k, c] == base_verts[b, k & bit, c] for k in range(1 << d)):
                tt = corners[:, c]
                cv[:, c] = (1.0 - tt) * x0 + tt * x1
        cv = cv.reshape(len(lc), 1 << d, d)
        verts[start[b]:start[b + 1]] = cv
        level[start[b]:start[b + 1]] = L
        for row in lc:
            local.append((b, row.copy()))

    def child_id(b, lc):
        L = int(lev[b])
        m = 1 << L
        return int(start[b] + sum(int(lc[a]) * m ** a for a in range(d)))

    int_faces, hang_faces, bdry_faces = [], [], []
    for e in range(n_elem):
        b, lc = local[e]
        L = int(lev[b])
        m = 1 << L
        for a in range(d):
            for s in (0, 1):
                f = 2 * a + s
                inside = (lc[a] + (1 if s else -1))
                if 0 <= inside < m:
                    if s == 1:
                        lc2 = lc.copy()
                        lc2[a] = inside
                        int_faces.append((e, f, child_id(b, lc2), 2 * a))
                    continue
                nbb = nbr_base(bcoords[b], a, s)
                if nbb < 0:
                    bdry_faces.append((e, f, BC_WALL))
                    continue
                L2 = int(lev[nbb])
                if L2 == L:
                    if s == 1:
                        lc2 = lc.copy()
                        lc2[a] = 0
                        int_faces.append((e, f, child_id(nbb, lc2), 2 * a))
                elif L2 == L - 1:
                    # this cell is the fine side; the coarse neighbour is the
                    # level-(L-1) child of nbb touching this face
                    lc2 = lc // 2
                    lc2[a] = 0 if s == 1 else (1 << L2) - 1
                    ec = child_id(nbb, lc2)
                    tang = [t for t in range(d) if t != a]
                    sub = sum(int(lc[t] & 1) << k for k, t in enumerate(tang))
                    hang_faces.append((ec, 2 * a + (1 - s), e, f, sub))
                elif L2 == L + 1:
                    pass  # listed from the fine side
                else:
                    raise ValueError("2:1 balance violated")
    i64 = lambda x, w: np.array(x, dtype=np.int64).reshape(-1, w)
    return Mesh(dim=d, vertices=verts, int_faces=i64(int_faces, 4),
                hang_faces=i64(hang_faces, 5), bdry_faces=i64(bdry_faces, 3),
                level=level, name=name)


# ----------------------------------------------------------------------------
# Analytic atmospheres (evaluated at physical points supplied by the caller)
# ----------------------------------------------------------------------------

def exner_background(z, theta_ref, n_bv, g=GRAV, p_ref=P_REF, cp=CP, R=R_GAS):
    """Hydrostatic stratified background of eq. init_cond.

    theta = theta_ref exp(N^2 z / g); Exner pi per eq. init_cond with
    T_ref = theta_ref; returns (rho, p, theta, pi)."""
    kappa_inv = GAMMA / (GAMMA - 1.0)
    pi = 1.0 + g * g / (cp * theta_ref * n_bv * n_bv) * (np.exp(-n_bv * n_bv * z / g) - 1.0)
    theta = theta_ref * np.exp(n_bv * n_bv * z / g)
    p = p_ref * pi ** kappa_inv
    rho = p / (R * pi * theta)
    return rho, p, theta, pi


def stratified_state(points, theta_ref=300.0, n_bv=0.01, wind=(0.0, 0.0, 0.0),
                     bubble=None, gamma=GAMMA):
    """Conserved state (rho, rho u, rho v, rho w, rho E) at physical points.

    points: (..., d) physical coordinates; vertical = last coordinate.
    wind:   uniform (u, v, w).
    bubble: dict(A, xc, a, H): potential-temperature perturbation
            A exp(-(x - xc)^2 / a^2) sin(pi z / H) added at constant pressure
            (the Gaussian-in-x, sine-in-z shape of the inertia-gravity-wave
            test of Section 4.1).
    Returns an array of shape (5, ...)."""
    pts = np.asarray(points, dtype=np.float64)
    z = pts[..., -1]
    x = pts[..., 0]
    rho, p, theta, pi = exner_background(z, theta_ref, n_bv)
    if bubble is not None:
        dth = bubble["A"] * np.exp(-((x - bubble["xc"]) / bubble["a"]) ** 2) * \
            np.sin(math.pi * z / bubble["H"])
        rho = p / (R_GAS * pi * (theta + dth))
    u = np.broadcast_to(np.asarray(wind, dtype=np.float64), pts.shape[:-1] + (3,))
    m = rho[..., None] * u
    E = p / (gamma - 1.0) + 0.5 * rho * np.sum(u * u, axis=-1)
    return np.stack([rho, m[..., 0], m[..., 1], m[..., 2], E], axis=0)


def isothermal_state(points, T0=250.0, ps=P_REF, bubble=None, g=GRAV, R=R_GAS, gamma=GAMMA):
    """Isothermal hydrostatic atmosphere at rest (Section 4, inertia-gravity
    wave): p0 = ps exp(-delta z), rho0 = rho_s exp(-delta z), delta = g/(R T0),
    rho_s = ps/(R T0), u = 0.

    bubble: dict(dT, xc, a, H): the Bretherton-transformed perturbation
            T' = exp(delta z / 2) T_b, rho' = exp(-delta z / 2) rho_b, p' = 0,
            T_b = dT exp(-(x - xc)^2 / a^2) sin(pi z / H),
            rho_b = rho_s (-T_b / T0).
    Returns (5, ...) conserved variables."""
    pts = np.asarray(points, dtype=np.float64)
    z = pts[..., -1]
    x = pts[..., 0]
    delta = g / (R * T0)
    rho_s = ps / (R * T0)
    p = ps * np.exp(-delta * z)
    rho = rho_s * np.exp(-delta * z)
    if bubble is not None:
        tb = bubble["dT"] * np.exp(-((x - bubble["xc"]) / bubble["a"]) ** 2) * \
            np.sin(math.pi * z / bubble["H"])
        rho = rho + np.exp(-0.5 * delta * z) * rho_s * (-tb / T0)
    zeros = np.zeros_like(rho)
    return np.stack([rho, zeros, zeros, zeros, p / (gamma - 1.0)], axis=0)


def with_boundary(mesh, faces, bc):
    """Copy of ``mesh`` whose boundary faces with local face index in
    ``faces`` (e.g. 2d - 1 for the top) carry boundary id ``bc``."""
    b = np.array(mesh.bdry_faces, dtype=np.int64, copy=True).reshape(-1, 3)
    sel = np.isin(b[:, 1], list(faces))
    b[sel, 2] = bc
    return Mesh(dim=mesh.dim, vertices=mesh.vertices, int_faces=mesh.int_faces,
                hang_faces=mesh.hang_faces, bdry_faces=b, level=mesh.level,
                name=mesh.name + "_bc")


def perturb(state, rng, rel=1e-3):
    """Seeded multiplicative noise on every field (parity-test inputs).

    Momentum gets additive noise scaled by rho * 10 m/s so that zero wind
    still yields a non-trivial velocity field."""
    q = np.array(state, dtype=np.float64, copy=True)
    q[0] *= 1.0 + rel * rng.uniform(-1, 1, q[0].shape)
    q[1:4] += rel * 10.0 * q[0] * rng.uniform(-1, 1, q[1:4].shape)
    q[4] *= 1.0 + rel * rng.uniform(-1, 1, q[4].shape)
    return q


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def planetary_igw_case(nx=300, nz=20, r=4):
    """Planetary-scale inertia-gravity wave (Section 4): 60 000 km x 10 km
    x-z channel, periodic in x, walls in z, 300 x 20 cells, degree 4;
    isothermal background at rest (T0 = 250 K, ps = 1e5 Pa), Bretherton
    perturbation dT = 0.01 K, half-width a = 1000 km at x_c = 30 000 km,
    H = 10 km; f = 1.03126e-4 1/s (45 degrees); dt = 10 s, 96 h."""
    mesh = box_mesh((nx, nz), (60000e3, 10e3), name="planetary_igw")
    params = dict(T0=250.0, ps=P_REF, bubble=dict(dT=0.01, xc=30000e3, a=1000e3, H=10e3))
    return dict(mesh=mesh, degree=r, f=1.03126e-4, dt=10.0, hours=96.0, state_params=params)


def igw2d_case(seed=0, nx=100, nz=5, r=2):
    """2D x-z rotating inertia-gravity wave: 300 km x 10 km periodic channel,
    100 x 5 quads, degree 2, N = 0.01 1/s, theta0 = 300 K, mean wind 20 m/s,
    f = 1e-4 1/s, dt = 12 s; theta' amplitude 0.01 K (seed jitters it by
    +-1%), Gaussian half-width 5 km at x = 100 km, sin(pi z / 10 km)."""
    rng = np.random.default_rng(seed)
    amp = 0.01 * (1.0 + 0.01 * rng.uniform(-1.0, 1.0))
    mesh = box_mesh((nx, nz), (300e3, 10e3), name="igw2d")
    params = dict(theta_ref=300.0, n_bv=0.01, wind=(20.0, 0.0, 0.0),
                  bubble=dict(A=amp, xc=100e3, a=5e3, H=10e3))
    return dict(mesh=mesh, degree=r, f=1e-4, dt=12.0, state_params=params)


def hill3d_case(nx=60, ny=60, nz=20, r=3, refine=False, refine_box=None):
    """3D stratified flow over a bell hill (h0 = 400 m, a_c = 10 km) in a
    200 x 200 x 20 km box, Gal-Chen terrain-following, N = 0.01 1/s,
    theta_ref = 293.15 K, inflow 10 m/s along x, f = 1e-4 1/s, dt = 4 s.

    refine=True adds two levels of 2:1 refinement for base cells whose
    centre lies in |x-100 km|, |y-100 km| <= 20 km and z <= 6 km, with a
    one-cell level-1 ring from the 2:1 balance."""
    L = (200e3, 200e3, 20e3)
    hill = dict(h0=400.0, a_c=10e3, xc=100e3, yc=100e3)
    rl = None
    if refine:
        bx = refine_box or dict(x=(80e3, 120e3), y=(80e3, 120e3), z=(0.0, 6e3))

        def rl(c):
            ok = (bx["x"][0] <= c[0] <= bx["x"][1] and bx["y"][0] <= c[1] <= bx["y"][1]
                  and bx["z"][0] <= c[2] <= bx["z"][1])
            return 2 if ok else 0
    mesh = box_mesh((nx, ny, nz), L, hill=hill, refine_level=rl,
                    name="hill3d_nc" if refine else "hill3d")
    params = dict(theta_ref=293.15, n_bv=0.01, wind=(10.0, 0.0, 0.0), bubble=None)
    return dict(mesh=mesh, degree=r, f=1e-4, dt=4.0, state_params=params)


def paper_igw_case(nx=300, nz=20, r=4):
    """Inertia-gravity wave, reference run of Section 4.1: 6000 km x 10 km
    x-z channel, periodic in x, walls in z, 300 x 20 cells, degree 4;
    isothermal background at rest (T0 = 250 K), Bretherton perturbation at
    x_c = 3000 km with half-width a = 100 km, f = 1.03126e-4 1/s, dt = 0.5 s,
    8 h."""
    mesh = box_mesh((nx, nz), (6000e3, 10e3), name="paper_igw")
    params = dict(T0=250.0, ps=P_REF, bubble=dict(dT=0.01, xc=3000e3, a=100e3, H=10e3))
    return dict(mesh=mesh, degree=r, f=1.03126e-4, dt=0.5, hours=8.0, state_params=params)


def paper_hill_benchmark_case(f=1e-4):
    """Medium-steep bell hill, benchmark test of Section 4.3: 60 x 40 x 16 km,
    hill at (30, 20) km with h0 = 400 m and a_c = 1 km, 30 x 20 x 8 cells of
    degree 4, dt = 8 s, 8 h; N = 0.01 1/s, theta_ref = 293.15 K, inflow
    10 m/s along x; f = 0 or 1e-4 1/s.  Damping layers (for
    ``Mesh.set_sponge``): 20 km at both ends of x, 10 km at both ends of y,
    the top 6 km, lambda_bar dt = 1.2.  The geostrophic pressure correction
    of a rotating run is left out (it is not periodic)."""
    dt = 8.0
    mesh = box_mesh((30, 20, 8), (60e3, 40e3, 16e3), hill=dict(h0=400.0, a_c=1e3, xc=30e3, yc=20e3),
                    name="paper_hill")
    sponge = dict(lambda_bar=1.2 / dt, z_b=10e3, z_t=16e3, x_layers=(0.0, 60e3, 20e3),
                  y_layers=(0.0, 40e3, 10e3))
    params = dict(theta_ref=293.15, n_bv=0.01, wind=(10.0, 0.0, 0.0), bubble=None)
    return dict(mesh=mesh, degree=4, f=f, dt=dt, hours=8.0, state_params=params, sponge=sponge)


def paper_hill_large_case(f=1e-4):
    """Larger-scale hill test of Section 4.3: 240 x 240 x 30 km, hill at
    (120, 120) km with h0 = 100 m and a_c = 10 km, 50 x 50 x 50 cells of
    degree 4, dt = 4 s, 8 h; isothermal background at 250 K (its buoyancy
    frequency g / sqrt(c_p T) = 0.0196 1/s, printed as 0.02), inflow 10 m/s
    along x.  Damping layers: 60 km at both ends of x and y, the top 14 km,
    lambda_bar dt = 1.2."""
    dt = 4.0
    T = 250.0
    mesh = box_mesh((50, 50, 50), (240e3, 240e3, 30e3), hill=dict(h0=100.0, a_c=10e3, xc=120e3, yc=120e3),
                    name="paper_hill_large")
    sponge = dict(lambda_bar=1.2 / dt, z_b=16e3, z_t=30e3, x_layers=(0.0, 240e3, 60e3),
                  y_layers=(0.0, 240e3, 60e3))
    params = dict(theta_ref=T, n_bv=GRAV / math.sqrt(CP * T), wind=(10.0, 0.0, 0.0), bubble=None)
    return dict(mesh=mesh, degree=4, f=f, dt=dt, hours=8.0, state_params=params, sponge=sponge)


def ensemble_cases(n=32, seed0=1000):
    """Ensemble of independent instances of uneven sizes and degrees.

    Instance i draws from PCG64(seed0 + i): dim 2 when i % 4 == 0 else 3;
    degree 2 + i % 3; cell count log-uniform in [2 000, 60 000]; f uniform in
    [0, 1.4e-4] 1/s; theta' amplitude uniform in [0.005, 0.02] K.  2D: the
    inertia-gravity-wave channel with 10 layers (3 km x 1 km cells, dt 12 s);
    3D: the hill box with 10 layers and the hill workload's cell size
    (3.33 km x 3.33 km x 2 km, dt 4 s), hill at the centre."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        dim = 2 if i % 4 == 0 else 3
        r = 2 + i % 3
        ne = float(np.exp(rng.uniform(np.log(2000.0), np.log(60000.0))))
        f = float(rng.uniform(0.0, 1.4e-4))
        amp = float(rng.uniform(0.005, 0.02))
        if dim == 2:
            nz = 10
            nx = max(4, int(round(ne / nz)))
            mesh = box_mesh((nx, nz), (nx * 3e3, 10e3), name=f"ens{i}")
            params = dict(theta_ref=300.0, n_bv=0.01, wind=(20.0, 0.0, 0.0),
                          bubble=dict(A=amp, xc=nx * 3e3 / 3, a=5e3, H=10e3))
            dt = 12.0
        else:
            nz = 10
            nxy = max(3, int(round(np.sqrt(ne / nz))))
            dx = 200e3 / 60
            L = nxy * dx
            mesh = box_mesh((nxy, nxy, nz), (L, L, 20e3),
                            hill=dict(h0=400.0, a_c=10e3, xc=L / 2, yc=L / 2), name=f"ens{i}")
            params = dict(theta_ref=293.15, n_bv=0.01, wind=(10.0, 0.0, 0.0),
                          bubble=dict(A=amp, xc=L / 3, a=5e3, H=20e3))
            dt = 4.0
        out.append(dict(mesh=mesh, degree=r, f=f, dt=dt, state_params=params))
    return out
