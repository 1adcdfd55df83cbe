"""FP64 CPU oracle for the rotating IMEX-DG hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this module.  The product path (``paper_2605_29598_gb300``) never does.

It restates the paper's discretisation in the plainest form available:

* nodal DG, Lagrange basis on (r+1)^d Gauss-Legendre nodes per cell, Q_r
  space (Section 3, spatial discretisation); Gauss-Lobatto nodes are
  supported too, always with (r+1)-point Gauss-Legendre quadrature;
* every cell integral is a full quadrature sum over all quadrature points
  against all basis functions, with dense interpolation matrices (no sum
  factorisation, no collocation shortcut); every inverse mass or (A+R)
  block is a dense LU solve per cell;
* hanging faces evaluate the coarse cell's polynomial directly at the fine
  face's quadrature points (no 1D prolongation matrices);
* face normals come from cross products of the tangent vectors of the
  multilinear cell map (not from the inverse Jacobian);
* the weak operators are the paper's matrices: A (eq. A), B, R, f_g, f
  (momentum), C, D, k, M_g, g (energy), the Schur systems of R1 and R2, the
  Picard (fixed-point) loop, restarted GMRES with modified Gram-Schmidt and
  Givens rotations, and the three-stage ARK2 step (Butcher tableau);
* the Rayleigh damping layers of the orography tests (Section 4, eq.
  damping) as an extra non-stiff rate -lambda (q - q_bar), in weak form;
* far-field boundary faces (the upper boundary of the orography tests,
  Section 4.3), whose outer state is a given background state.

Readings where the paper is silent or garbled (each also used by the CUDA
path) are marked ``READING`` below.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` and ``tests/test_golden.py`` (closed forms, invariants, brute force, values the
paper prints).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CHI = 2.0 - math.sqrt(2.0)

# boundary ids of the mesh's boundary face rows [e, f, bc]
BC_WALL = 1        # slip wall, mirror state (READING c12)
BC_FARFIELD = 2    # outer state = a given background state (READING R-farfield)


# ----------------------------------------------------------------------------
# Butcher tableaux (Section 3, Table "Butcher tableau")
# ----------------------------------------------------------------------------

def ark2_tableau(a32=0.5):
    """Explicit (a) and implicit (at) tableaux, weights b, nodes c."""
    chi = CHI
    a = np.array([[0.0, 0.0, 0.0],
                  [chi, 0.0, 0.0],
                  [1.0 - a32, a32, 0.0]])
    bw = np.array([0.5 - chi / 4.0, 0.5 - chi / 4.0, chi / 2.0])
    at = np.array([[0.0, 0.0, 0.0],
                   [chi / 2.0, chi / 2.0, 0.0],
                   [bw[0], bw[1], bw[2]]])
    c = np.array([0.0, chi, 1.0])
    return a, at, bw, c


# ----------------------------------------------------------------------------
# 1D bases and quadrature
# ----------------------------------------------------------------------------

def gauss_legendre01(n):
    """n-point Gauss-Legendre rule mapped to [0, 1]."""
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def gauss_lobatto01(n):
    """n-point Gauss-Lobatto points on [0, 1] (endpoints + roots of P'_{n-1})."""
    if n == 1:
        return np.array([0.5])
    c = np.zeros(n)
    c[-1] = 1.0
    inner = np.polynomial.legendre.Legendre(c).deriv().roots()
    t = np.concatenate([[-1.0], np.sort(inner.real), [1.0]])
    return 0.5 * (t + 1.0)


def lagrange(nodes, t):
    """Values l_j(t_p) of the Lagrange polynomials on ``nodes``: (len(t), n)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(t), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                out[:, j] *= (t - nodes[k]) / (nodes[j] - nodes[k])
    return out


def dlagrange(nodes, t):
    """Derivatives l_j'(t_p) by the product rule: (len(t), n)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    out = np.zeros((len(t), n))
    for j in range(n):
        for m in range(n):
            if m == j:
                continue
            term = np.full(len(t), 1.0 / (nodes[j] - nodes[m]))
            for k in range(n):
                if k != j and k != m:
                    term *= (t - nodes[k]) / (nodes[j] - nodes[k])
            out[:, j] += term
    return out


def _tensor_index(n, d):
    """Multi-indices (i0, i1[, i2]) of the n^d nodes, x fastest: (n^d, d)."""
    k = np.arange(n ** d)
    return np.stack([(k // n ** a) % n for a in range(d)], axis=-1).astype(np.int64)


def _tensor_points(pts1d, d):
    """Tensor grid of 1D values (points or weights), x fastest: (n^d, d)."""
    pts1d = np.asarray(pts1d, dtype=np.float64)
    return pts1d[_tensor_index(len(pts1d), d)]


# ----------------------------------------------------------------------------
# Reference cell and geometry
# ----------------------------------------------------------------------------

def _corner_bits(d):
    return np.array([[(v >> a) & 1 for a in range(d)] for v in range(1 << d)])


def map_points(verts, ref):
    """Multilinear cell map x(xi) at reference points: (E, m, d)."""
    bits = _corner_bits(ref.shape[1])
    N = np.ones((ref.shape[0], len(bits)))
    for v, bv in enumerate(bits):
        for a, b in enumerate(bv):
            N[:, v] *= ref[:, a] if b else (1.0 - ref[:, a])
    return np.einsum("mv,evd->emd", N, verts)


def map_jacobian(verts, ref):
    """J[e, p, b, c] = d x_b / d xi_c of the multilinear map."""
    d = ref.shape[1]
    bits = _corner_bits(d)
    dN = np.ones((d, ref.shape[0], len(bits)))
    for c in range(d):
        for v, bv in enumerate(bits):
            for a, b in enumerate(bv):
                if a == c:
                    dN[c, :, v] *= 1.0 if b else -1.0
                else:
                    dN[c, :, v] *= ref[:, a] if b else (1.0 - ref[:, a])
    return np.einsum("cmv,evb->embc", dN, verts)


def spatial_components(d):
    """Velocity component carried by each spatial direction.

    3D: x, y, z -> u, v, w.  2D vertical slice (eq. vertical_slice): the two
    spatial directions are x and z, carrying u and w; v has no derivative."""
    return [0, 1, 2] if d == 3 else [0, 2]


class Discretisation:
    """Reference matrices, geometry and face lists of one mesh.

    q arrays are (fields, E, Np) with nodes in tensor order, x fastest."""

    def __init__(self, mesh, degree, node_set="gl"):
        self.mesh = mesh
        self.d = d = mesh.dim
        self.r = degree
        self.n = n = degree + 1
        self.Np = n ** d
        self.E = mesh.vertices.shape[0]
        self.comp = spatial_components(d)
        if node_set == "gl":
            self.nodes1d = gauss_legendre01(n)[0]
        elif node_set == "gll":
            self.nodes1d = gauss_lobatto01(n)
        else:
            raise ValueError(node_set)
        # quadrature: (r+1)-point Gauss-Legendre per direction
        self.qx1d, self.qw1d = gauss_legendre01(n)
        L = lagrange(self.nodes1d, self.qx1d)
        dL = dlagrange(self.nodes1d, self.qx1d)
        idx = _tensor_index(n, d)
        self.qpts = _tensor_points(self.qx1d, d)
        self.qw = np.prod(_tensor_points(self.qw1d, d), axis=1)
        Nq = len(self.qw)
        # dense interpolation / gradient matrices (reference cell)
        self.V = np.ones((Nq, self.Np))
        self.Dxi = np.ones((d, Nq, self.Np))
        for qi in range(Nq):
            for i in range(self.Np):
                for a in range(d):
                    self.V[qi, i] *= L[idx[qi, a], idx[i, a]]
                    for c in range(d):
                        self.Dxi[c, qi, i] *= (dL if c == a else L)[idx[qi, a], idx[i, a]]
        # geometry at volume quadrature points
        J = map_jacobian(mesh.vertices, self.qpts)
        self.detJ = np.linalg.det(J)
        if np.any(self.detJ <= 0):
            raise ValueError("inverted cell")
        Jinv = np.linalg.inv(J)                                 # [e,q,c,b] = dxi_c/dx_b
        # physical gradients of basis functions: G[e,q,b,i]
        self.G = np.einsum("eqcb,cqi->eqbi", Jinv, self.Dxi)
        self.wJ = self.qw[None, :] * self.detJ                 # (E, Nq)
        self.M = np.einsum("qi,eq,qj->eij", self.V, self.wJ, self.V)
        self._build_faces()

    # -- faces ---------------------------------------------------------------
    def _face_ref(self, f, sub=None):
        """Reference points of face f's quadrature; with ``sub``, the points
        of that subface expressed in the coarse cell's reference frame."""
        d, n = self.d, self.n
        a, s = f // 2, f % 2
        tang = [t for t in range(d) if t != a]
        tp = _tensor_points(self.qx1d, d - 1) if d > 1 else np.zeros((1, 0))
        P = np.zeros((len(tp), d))
        P[:, a] = float(s)
        for k, t in enumerate(tang):
            x = tp[:, k]
            if sub is not None:
                x = 0.5 * (x + ((sub >> k) & 1))
            P[:, t] = x
        w = np.prod(_tensor_points(self.qw1d, d - 1), axis=1)
        return P, w

    def _basis_at(self, P):
        """Dense values of all Np basis functions at reference points P."""
        idx = _tensor_index(self.n, self.d)
        out = np.ones((len(P), self.Np))
        for a in range(self.d):
            La = lagrange(self.nodes1d, P[:, a])              # (m, n)
            out *= La[:, idx[:, a]]
        return out

    def _normals(self, elems, faces):
        """Outward (area * weight) normals at face quadrature points.

        Built from tangent vectors of the cell map: 3D cross product, 2D
        rotated tangent; sign fixed by the orientation of the face."""
        d = self.d
        out = np.zeros((len(elems), self.n ** (d - 1), d))
        for f in range(2 * d):
            sel = np.nonzero(faces == f)[0]
            if len(sel) == 0:
                continue
            P, w = self._face_ref(f)
            J = map_jacobian(self.mesh.vertices[elems[sel]], P)   # (m, p, b, c)
            a, s = f // 2, f % 2
            tang = [t for t in range(d) if t != a]
            sgn = 1.0 if s == 1 else -1.0
            if d == 3:
                t1, t2 = J[..., tang[0]], J[..., tang[1]]
                nv = np.cross(t1, t2)
                # (a, t1, t2) is an even permutation of (0,1,2) for a = 0, 2
                if a == 1:
                    nv = -nv
            else:
                t = J[..., tang[0]]
                nv = np.stack([t[..., 1], -t[..., 0]], axis=-1)
                if a == 1:
                    nv = -nv
            out[sel] = sgn * nv * w[None, :, None]
        return out

    def _build_faces(self):
        """One uniform list of face quadrature groups.

        Each group has a minus cell (whose geometry defines the normal), its
        trace matrix, and a plus cell (-1 for a wall) with its trace matrix.
        Interior: minus = eL.  Hanging: minus = fine, plus = coarse evaluated
        at the fine points.  Boundary: plus = -1."""
        m = self.mesh
        d = self.d
        Vf = [self._basis_at(self._face_ref(f)[0]) for f in range(2 * d)]
        Vh = [[self._basis_at(self._face_ref(f, sub)[0]) for sub in range(1 << (d - 1))]
              for f in range(2 * d)]
        em, fm, ep, Vm_list, Vp_list, bcs = [], [], [], [], [], []
        for eL, fL, eR, fR in m.int_faces:
            em.append(eL); fm.append(fL); ep.append(eR); bcs.append(0)
            Vm_list.append(Vf[fL]); Vp_list.append(Vf[fR])
        for ec, fc, ef, ff, sub in m.hang_faces:
            em.append(ef); fm.append(ff); ep.append(ec); bcs.append(0)
            Vm_list.append(Vf[ff]); Vp_list.append(Vh[fc][sub])
        for e, f, bc in m.bdry_faces:
            if bc not in (BC_WALL, BC_FARFIELD):
                raise ValueError(f"unknown boundary condition {bc}")
            em.append(e); fm.append(f); ep.append(-1); bcs.append(bc)
            Vm_list.append(Vf[f]); Vp_list.append(Vf[f])
        self.f_em = np.array(em, dtype=np.int64)
        self.f_fm = np.array(fm, dtype=np.int64)
        self.f_ep = np.array(ep, dtype=np.int64)
        nfp = self.n ** (d - 1)
        self.f_Vm = np.array(Vm_list).reshape(-1, nfp, self.Np)
        self.f_Vp = np.array(Vp_list).reshape(-1, nfp, self.Np)
        self.f_nS = self._normals(self.f_em, self.f_fm)              # (F, p, d)
        self.f_dS = np.linalg.norm(self.f_nS, axis=-1)              # (F, p)
        self.f_nhat = self.f_nS / self.f_dS[..., None]
        self.f_wall = self.f_ep < 0                 # boundary faces: no plus cell
        self.f_far = np.array(bcs) == BC_FARFIELD   # ... of them, the far-field ones
        self.f_mirror = self.f_wall & ~self.f_far   # ... and the slip walls
        self.f_epc = np.where(self.f_wall, self.f_em, self.f_ep)
        self.far_tr = None

    def set_far_state(self, q_far):
        """Outer state of the far-field faces: traces, at their face points,
        of the nodal background state q_far (5, E, Np) from the inner cell."""
        self.far_tr = self.traces(np.asarray(q_far, dtype=np.float64))[0]

    def far_primitives(self, gamma):
        """(u, p) of the outer state at every face point, (3, F, p) and
        (F, p), from its conserved traces (meaningful on far-field faces)."""
        if self.f_far.any() and self.far_tr is None:
            raise ValueError("far-field faces need set_far_state()")
        t = self.far_tr
        u = t[1:4] / t[0]
        p = (gamma - 1.0) * (t[4] - 0.5 * np.sum(t[1:4] * u, axis=0))
        return u, p

    # -- small helpers --------------------------------------------------------
    def at_quad(self, v):
        """Interpolate nodal fields (..., E, Np) to volume quadrature points."""
        return np.einsum("qi,...ei->...eq", self.V, v)

    def traces(self, v):
        """Minus / plus traces of nodal fields (..., E, Np) at face points."""
        tm = np.einsum("fpi,...fi->...fp", self.f_Vm, v[..., self.f_em, :])
        tp = np.einsum("fpi,...fi->...fp", self.f_Vp, v[..., self.f_epc, :])
        return tm, tp

    def lift(self, res, flux):
        """Add the face term  -int_F flux * test  to both sides.

        ``flux`` (..., F, p) already carries weight * area * (. n_minus); the
        minus cell receives -flux, the plus cell +flux (its normal is -n)."""
        lead = flux.shape[:-2]
        cm = np.einsum("...fp,fpi->...fi", flux, self.f_Vm)
        cp = np.einsum("...fp,fpi->...fi", flux, self.f_Vp)
        inner = ~self.f_wall
        for k in np.ndindex(*lead) if lead else [()]:
            np.add.at(res[k], self.f_em, -cm[k])
            np.add.at(res[k], self.f_ep[inner], cp[k][inner])

    def vol_weak(self, vals):
        """int_K vals * phi_i  for values at quadrature points (..., E, Nq)."""
        return np.einsum("...eq,eq,qi->...ei", vals, self.wJ, self.V)

    def vol_grad(self, flux):
        """sum_b int_K flux_b * d phi_i / dx_b;  flux (..., d, E, Nq)."""
        return np.einsum("...beq,eq,eqbi->...ei", flux, self.wJ, self.G)

    def mass_solve(self, res):
        """Apply the inverse (unweighted) mass matrix cell by cell (dense
        LU, factorised once per mesh)."""
        if not hasattr(self, "_Minv"):
            self._Minv = np.linalg.inv(self.M)
        lead = res.shape[:-2]
        r = res.reshape((-1,) + res.shape[-2:])
        out = np.einsum("eij,kej->kei", self._Minv, r)
        return out.reshape(lead + res.shape[-2:])

    def node_points(self):
        """Physical coordinates of the nodes: (E, Np, d)."""
        return map_points(self.mesh.vertices, _tensor_points(self.nodes1d, self.d))


@dataclass
class Phys:
    gamma: float = 1.4
    g: float = 9.81
    f: float = 1.0e-4
    variant: str = "R2"          # "R1" | "R2"
    penalty: bool = True         # implicit Rusanov term on rho e (READING c5)
    sponge: "Sponge" = None      # Rayleigh damping layers (Section 4), or none
    lambda_min: float = 0.0      # floor (m/s) of the non-stiff Rusanov coefficient; 0: the paper's
                                 # lambda = |u.n| (a floor is not in the paper: see rusanov_floor)


@dataclass
class Sponge:
    """Rayleigh damping (sponge) layers of the orography tests (Section 4,
    eq. damping).

    lam_bar (1/s): the damping coefficient at the boundary.  Top layer:
    lambda = 0 below z_b, lam_bar sin^2(pi/2 (z - z_b)/(z_t - z_b)) above.
    Lateral layers, (lo, hi, width) for x and/or y: the same sin^2 ramp over
    ``width`` from the layer's inner edge (lo + width, hi - width) out to the
    boundary lo or hi.  q_bar (5, E, Np): the nodal state the layers relax.
    READINGS (the paper gives the top profile and says the lateral layers are
    analogous): the damping term -lambda (q - q_bar) acts on all five
    conserved fields and belongs to the non-stiff (explicit) part; where
    layers overlap the largest coefficient applies; the ramp argument is
    clipped to [0, 1]."""
    lam_bar: float
    z_b: float
    z_t: float
    x_layers: tuple = None
    y_layers: tuple = None
    q_bar: np.ndarray = None


def sponge_coefficient(points, s):
    """lambda at physical points (..., d) for the layers ``s``."""
    pts = np.asarray(points, dtype=np.float64)

    def ramp(t):
        t = np.clip(t, 0.0, 1.0)
        return s.lam_bar * np.sin(0.5 * math.pi * t) ** 2

    z = pts[..., -1]
    lam = np.where(z >= s.z_b, ramp((z - s.z_b) / (s.z_t - s.z_b)), 0.0)
    for axis, lay in ((0, s.x_layers), (1, s.y_layers)):
        if lay is None or (axis == 1 and pts.shape[-1] < 3):
            continue
        lo, hi, w = lay
        c = pts[..., axis]
        lam = np.maximum(lam, np.where(c <= lo + w, ramp((lo + w - c) / w), 0.0))
        lam = np.maximum(lam, np.where(c >= hi - w, ramp((c - (hi - w)) / w), 0.0))
    return lam


# ----------------------------------------------------------------------------
# Explicit operator: weak residuals of f_NS and f_S, then rates M^{-1} r
# ----------------------------------------------------------------------------

def explicit_residuals(disc, q, phys):
    """Weak residuals (r_NS, r_S) of the non-stiff and stiff parts at state q.

    Non-stiff (advective) part, weights a_lm in the RHS vectors f and g:
      mass  rho u,  momentum rho u (x) u,  energy kappa rho u, with Rusanov
      stabilisation lambda/2 [.] on rho, rho u and rho kappa.
    Stiff part, weights at_lm: pressure p I with centred flux {p}, enthalpy
      flux h rho u with centred flux and Rusanov lambda/2 [rho e]
      (READING c4: the second energy Rusanov term of the g vector, on
      [rho E], duplicates this one and is dropped), gravity -rho g k and
      Coriolis -f rho k x u in momentum, -g rho k.u in energy.
    lambda = max(|u- . n|, |u+ . n|) pointwise at face points (READING c3).
    Walls use the mirror state (READING c12); far-field faces use the given
    outer state (READING R-farfield) in the same fluxes as interior faces.

    Option not in the paper: phys.lambda_min > 0 floors lambda in the three
    non-stiff Rusanov terms (the stiff rho e term keeps |u.n|, as does its
    implicit counterpart).  With the flow at rest lambda = |u.n| vanishes,
    and a cell-to-cell checkerboard of vertical momentum, which the centred
    pressure flux does not see, oscillates at the buoyancy frequency and
    grows through the explicit density (about 9 % per step on the planetary
    wave's columns at dt = 10 s); a floor of 1 m/s damps it."""
    gm = phys.gamma
    d, comp = disc.d, disc.comp
    Q = disc.at_quad(q)                                   # (5, E, Nq)
    rho, m, E = Q[0], Q[1:4], Q[4]
    u = m / rho
    kin = 0.5 * np.sum(u * u, axis=0)
    p = (gm - 1.0) * (E - rho * kin)
    hrho = gm / (gm - 1.0) * p
    uS = np.stack([u[c] for c in comp])                  # spatial velocity (d, E, Nq)
    r_ns = np.zeros((5,) + q.shape[1:])
    r_s = np.zeros((5,) + q.shape[1:])
    r_ns[0] += disc.vol_grad(rho * uS)
    for c in range(3):
        r_ns[1 + c] += disc.vol_grad(m[c] * uS)
    r_ns[4] += disc.vol_grad(rho * kin * uS)
    if phys.sponge is not None:
        # -lambda (q - q_bar) in weak form, lambda at the quadrature points
        lam = sponge_coefficient(map_points(disc.mesh.vertices, disc.qpts), phys.sponge)
        r_ns += disc.vol_weak(-lam[None] * (Q - disc.at_quad(phys.sponge.q_bar)))
    for b, c in enumerate(comp):
        pf = np.zeros((d,) + p.shape)
        pf[b] = p
        r_s[1 + c] += disc.vol_grad(pf)
    r_s[4] += disc.vol_grad(hrho * uS)
    # sources: -rho g k - f rho k x u  (k x u = (-v, u, 0)),  -g rho k.u
    r_s[1] += disc.vol_weak(phys.f * m[1])
    r_s[2] += disc.vol_weak(-phys.f * m[0])
    r_s[3] += disc.vol_weak(-phys.g * rho)
    r_s[4] += disc.vol_weak(-phys.g * m[2])

    # faces
    tm, tp = disc.traces(q)                               # (5, F, p)
    nS, dS, nh = disc.f_nS, disc.f_dS, disc.f_nhat
    wall = disc.f_mirror
    # mirror state on walls: m+ = m- - 2 (m-.n) n
    mS_m = np.stack([tm[1 + c] for c in comp], axis=-1)  # (F, p, d)
    mn = np.sum(mS_m * nh, axis=-1)
    mirror = tm.copy()
    for b, c in enumerate(comp):
        mirror[1 + c] = tm[1 + c] - 2.0 * mn * nh[..., b]
    tp = np.where(wall[None, :, None], mirror, tp)
    if disc.f_far.any():
        disc.far_primitives(gm)                           # checks that the state is set
        tp = np.where(disc.f_far[None, :, None], disc.far_tr, tp)

    def prim(t):
        r_, m_, E_ = t[0], t[1:4], t[4]
        u_ = m_ / r_
        k_ = 0.5 * np.sum(u_ * u_, axis=0)
        p_ = (gm - 1.0) * (E_ - r_ * k_)
        un_ = sum(u_[c] * nS[..., b] for b, c in enumerate(comp))   # u . nS
        unh_ = sum(u_[c] * nh[..., b] for b, c in enumerate(comp))  # u . n
        return r_, m_, E_, u_, k_, p_, un_, unh_

    rm, mm, Em, um, km, pm, unm, unhm = prim(tm)
    rp, mp, Ep, up, kp, pp, unp, unhp = prim(tp)
    lam = np.maximum(np.abs(unhm), np.abs(unhp))
    pen = 0.5 * lam * dS
    # non-stiff fluxes: lambda floored at phys.lambda_min (0: the paper's)
    pen_ns = 0.5 * np.maximum(lam, phys.lambda_min) * dS
    fl_ns = np.zeros((5,) + lam.shape)
    fl_s = np.zeros((5,) + lam.shape)
    fl_ns[0] = 0.5 * (rm * unm + rp * unp) + pen_ns * (rm - rp)
    for c in range(3):
        fl_ns[1 + c] = 0.5 * (mm[c] * unm + mp[c] * unp) + pen_ns * (mm[c] - mp[c])
    fl_ns[4] = 0.5 * (rm * km * unm + rp * kp * unp) + pen_ns * (rm * km - rp * kp)
    for b, c in enumerate(comp):
        fl_s[1 + c] = 0.5 * (pm + pp) * nS[..., b]
    fl_s[4] = 0.5 * gm / (gm - 1.0) * (pm * unm + pp * unp) \
        + pen * (pm - pp) / (gm - 1.0)
    disc.lift(r_ns, fl_ns)
    disc.lift(r_s, fl_s)
    return r_ns, r_s


def explicit_rates(disc, q, phys):
    """Rates F = M^{-1} r of the non-stiff and stiff parts (5 fields each)."""
    r_ns, r_s = explicit_residuals(disc, q, phys)
    return disc.mass_solve(r_ns), disc.mass_solve(r_s)


def geostrophic_error(disc, q, phys):
    """Geostrophic imbalance E_geo of Section 4 (planetary-scale wave, eq.
    egeo): the domain mean of |(1/rho) dp/dx - f v|.

    The pressure gradient and the Coriolis term are the scheme's own: the
    stiff x-momentum rate F_S = -dp/dx + f rho v of the explicit operator
    (weak DG gradient with centred face pressures, M^{-1} applied), so the
    integrand is |F_S / rho|.  The integral is the volume quadrature
    sum_q wJ_q |.| of the values interpolated to the quadrature points.
    READING: the domain measure sum_q wJ_q replaces x_max z_max (equal on a
    flat box); in 3D the same x-momentum balance is averaged over the volume."""
    _, Fs = explicit_rates(disc, q, phys)
    ratio = disc.at_quad(Fs[1]) / disc.at_quad(q[0])
    return float(np.sum(disc.wJ * np.abs(ratio)) / np.sum(disc.wJ))


# ----------------------------------------------------------------------------
# Implicit (acoustic) operators of one stage: the paper's matrices
# ----------------------------------------------------------------------------

@dataclass
class StageCoeffs:
    """Coefficients frozen during one Picard iteration of stage l.

    rho: rho^(n,l) nodal (E, Np);  p_lag: p^(n,l,k) nodal;  u_lag:
    u^(n,l,k) nodal (3, E, Np);  adt: at_ll * dt."""
    rho: np.ndarray
    p_lag: np.ndarray
    u_lag: np.ndarray
    adt: float
    cache: dict = None


def op_B(disc, cf, x):
    """B x:  -adt int div(phi_i) x  +  adt int_Gamma {x} [phi_i]  (3, E, Np).

    Walls: {x} = x-.  Far-field faces: {x} = (x- + p_far)/2, of which this
    linear operator holds x-/2 (the p_far/2 part is in far_affine)."""
    X = disc.at_quad(x)
    out = np.zeros((3,) + x.shape)
    for b, c in enumerate(disc.comp):
        fl = np.zeros((disc.d,) + X.shape)
        fl[b] = X
        out[c] = -cf.adt * disc.vol_grad(fl)
    tm, tp = disc.traces(x)
    avg = np.where(disc.f_mirror[:, None], tm, 0.5 * (tm + tp))
    avg = np.where(disc.f_far[:, None], 0.5 * tm, avg)
    flux = np.zeros((3,) + avg.shape)
    for b, c in enumerate(disc.comp):
        # +adt {x} phi.n  enters with the opposite sign of the generic lift
        flux[c] = -cf.adt * avg * disc.f_nS[..., b]
    disc.lift(out, flux)
    return out


def op_A(disc, cf, u):
    """A u = int rho phi_j . phi_i  (eq. A), per component."""
    R = disc.at_quad(cf.rho)
    return disc.vol_weak(R[None] * disc.at_quad(u))


def op_R(disc, cf, u, f):
    """R u = adt f int rho (k x u) . phi_i,  k x u = (-v, u, 0)."""
    R = disc.at_quad(cf.rho)
    U = disc.at_quad(u)
    kxu = np.stack([-U[1], U[0], np.zeros_like(U[0])])
    return cf.adt * f * disc.vol_weak(R[None] * kxu)


def _cell_block_AR(disc, cf, f, with_R):
    """Dense per-cell matrix of (A + R) on the 3 Np velocity unknowns."""
    R = disc.at_quad(cf.rho)                                       # (E, Nq)
    Mr = np.einsum("qi,eq,qj->eij", disc.V, disc.wJ * R, disc.V)  # (E, Np, Np)
    Np = disc.Np
    blk = np.zeros((disc.E, 3 * Np, 3 * Np))
    for c in range(3):
        blk[:, c * Np:(c + 1) * Np, c * Np:(c + 1) * Np] = Mr
    if with_R:
        beta = cf.adt * f
        # row u gets -beta * v-column, row v gets +beta * u-column
        blk[:, 0:Np, Np:2 * Np] = -beta * Mr
        blk[:, Np:2 * Np, 0:Np] = beta * Mr
    return blk


def solve_AR(disc, cf, f, rhs, with_R=True):
    """(A + R)^{-1} rhs (or A^{-1} rhs) by a dense inverse per cell (the
    cell blocks are factorised once per set of frozen coefficients)."""
    if cf.cache is None:
        cf.cache = {}
    key = ("AR", f, with_R)
    if key not in cf.cache:
        cf.cache[key] = np.linalg.inv(_cell_block_AR(disc, cf, f, with_R))
    inv = cf.cache[key]
    r = np.concatenate([rhs[0], rhs[1], rhs[2]], axis=-1)          # (E, 3Np)
    s = np.einsum("eij,ej->ei", inv, r)
    Np = disc.Np
    return np.stack([s[:, :Np], s[:, Np:2 * Np], s[:, 2 * Np:]])


def op_C(disc, cf, u, gamma):
    """C u:  -adt int h rho phi . grad psi_i + adt int_Gamma {h rho phi}.[psi_i].

    h rho = gamma p_lag / (gamma - 1) (h = e + p / rho for the ideal gas).
    Walls: the mirror velocity makes {h rho u}.n vanish.  Far-field faces:
    the linear part (h rho u)-.n / 2 (the outer state's half is in
    far_affine)."""
    H = gamma / (gamma - 1.0) * disc.at_quad(cf.p_lag)
    U = disc.at_quad(u)
    fl = np.stack([H * U[c] for c in disc.comp])
    out = -cf.adt * disc.vol_grad(fl)
    Hm, Hp = disc.traces(gamma / (gamma - 1.0) * cf.p_lag)
    um, up = disc.traces(u)
    fm = sum(Hm * um[c] * disc.f_nS[..., b] for b, c in enumerate(disc.comp))
    fp = sum(Hp * up[c] * disc.f_nS[..., b] for b, c in enumerate(disc.comp))
    avg = np.where(disc.f_mirror[:, None], 0.0, 0.5 * (fm + fp))
    avg = np.where(disc.f_far[:, None], 0.5 * fm, avg)
    out = out[None]
    disc.lift(out, (-cf.adt * avg)[None])
    return out[0]


def op_D(disc, p, gamma):
    """D p = int p psi_i / (gamma - 1)."""
    return disc.vol_weak(disc.at_quad(p)) / (gamma - 1.0)


def face_lambda(disc, u_lag, gamma=1.4):
    """lambda = max(|u- . n|, |u+ . n|) at face points from nodal u (the
    outer state's velocity on far-field faces)."""
    um, up = disc.traces(u_lag)
    unm = sum(um[c] * disc.f_nhat[..., b] for b, c in enumerate(disc.comp))
    unp = sum(up[c] * disc.f_nhat[..., b] for b, c in enumerate(disc.comp))
    unp = np.where(disc.f_mirror[:, None], -unm, unp)
    if disc.f_far.any():
        uf, _ = disc.far_primitives(gamma)
        unf = sum(uf[c] * disc.f_nhat[..., b] for b, c in enumerate(disc.comp))
        unp = np.where(disc.f_far[:, None], unf, unp)
    return np.maximum(np.abs(unm), np.abs(unp))


def op_P(disc, cf, p, gamma):
    """Implicit Rusanov term on rho e = p/(gamma-1) at stage l (READING c5):
    adt/(2(gamma-1)) int_Gamma lambda^(k) [p].[psi_i]; zero on walls; on
    far-field faces the linear part lambda p- (-lambda p_far in far_affine)."""
    lam = face_lambda(disc, cf.u_lag, gamma)
    pm, pp = disc.traces(p)
    jump = np.where(disc.f_mirror[:, None], 0.0, pm - pp)
    jump = np.where(disc.f_far[:, None], pm, jump)
    flux = cf.adt / (2.0 * (gamma - 1.0)) * lam * disc.f_dS * jump
    out = np.zeros((1,) + p.shape)
    # [p].[psi_i]: minus cell gets +flux psi-, plus cell -flux psi+
    disc.lift(out, -flux[None])
    return out[0]


def op_Mg(disc, cf, u, g):
    """M_g u = adt g int rho (k . u) psi_i  (READING c6: row index on psi)."""
    R = disc.at_quad(cf.rho)
    U = disc.at_quad(u)
    return cf.adt * g * disc.vol_weak(R * U[2])


def vec_k(disc, cf, u):
    """k_i = int rho kappa psi_i,  kappa = |u|^2 / 2."""
    R = disc.at_quad(cf.rho)
    U = disc.at_quad(u)
    return disc.vol_weak(R * 0.5 * np.sum(U * U, axis=0))


def vec_fg(disc, cf, g):
    """f_g = adt g int rho k . phi_i  (z component only)."""
    out = np.zeros((3,) + cf.rho.shape)
    out[2] = cf.adt * g * disc.vol_weak(disc.at_quad(cf.rho))
    return out


def far_affine(disc, cf, phys):
    """Parts of B p, C u and the implicit Rusanov term P p that the outer
    state of far-field faces contributes (READING R-farfield): known data,
    moved to the right-hand sides of the coupled stage system.

    Returns (b_far (3, E, Np), g_far (E, Np)): B p = B_lin p + b_far and
    C u + P p = C_lin u + P_lin p + g_far, with
      b_far:  adt int_far (p_far / 2) n . phi_i,
      g_far:  adt int_far (h rho u)_far . n / 2 psi_i
              - adt / (2 (gamma - 1)) int_far lambda p_far psi_i."""
    gm = phys.gamma
    fb = np.zeros((3,) + cf.rho.shape)
    gb = np.zeros((1,) + cf.rho.shape)
    if not disc.f_far.any():
        return fb, gb[0]
    far = disc.f_far[:, None]
    uf, pf = disc.far_primitives(gm)
    flux = np.zeros((3,) + pf.shape)
    for b, c in enumerate(disc.comp):
        flux[c] = np.where(far, -cf.adt * 0.5 * pf * disc.f_nS[..., b], 0.0)
    disc.lift(fb, flux)
    unS = sum(uf[c] * disc.f_nS[..., b] for b, c in enumerate(disc.comp))
    cfl = np.where(far, 0.5 * gm / (gm - 1.0) * pf * unS, 0.0)
    disc.lift(gb, (-cf.adt * cfl)[None])
    if phys.penalty:
        lam = face_lambda(disc, cf.u_lag, gm)
        pfl = np.where(far, cf.adt / (2.0 * (gm - 1.0)) * lam * disc.f_dS * (-pf), 0.0)
        disc.lift(gb, -pfl[None])
    return fb, gb[0]


def D_solve(disc, r, gamma):
    """D^{-1} r, D = mass / (gamma - 1)  (left scaling of the Schur system,
    READING c10b: GMRES runs on D^{-1} S)."""
    return (gamma - 1.0) * disc.mass_solve(r[None])[0]


def schur_apply(disc, cf, phys, x):
    """Scaled Schur operator D^{-1} S x.

    R2: S = D + P - (C + M_g)(A + R)^{-1} B
    R1: S = D + P - C A^{-1} B"""
    gm = phys.gamma
    Bx = op_B(disc, cf, x)
    if phys.variant == "R2":
        w = solve_AR(disc, cf, phys.f, Bx, with_R=True)
        cw = op_C(disc, cf, w, gm) + op_Mg(disc, cf, w, phys.g)
    else:
        w = solve_AR(disc, cf, phys.f, Bx, with_R=False)
        cw = op_C(disc, cf, w, gm)
    Sx = op_D(disc, x, gm) - cw
    if phys.penalty:
        Sx = Sx + op_P(disc, cf, x, gm)
    return D_solve(disc, Sx, gm)


def schur_rhs(disc, cf, phys, f_w, g_w):
    """Scaled right-hand side D^{-1} RHS of the pressure system.

    R2: RHS = g - k - (C + M_g)(A + R)^{-1}(f - f_g)
    R1: RHS = g - M_g u^k - k - C A^{-1}(f - R u^k - f_g)
    f_w, g_w are the weak momentum (3, E, Np) and energy (E, Np) vectors."""
    gm = phys.gamma
    fg = vec_fg(disc, cf, phys.g)
    kv = vec_k(disc, cf, cf.u_lag)
    if phys.variant == "R2":
        w = solve_AR(disc, cf, phys.f, f_w - fg, with_R=True)
        rhs = g_w - kv - op_C(disc, cf, w, gm) - op_Mg(disc, cf, w, phys.g)
    else:
        rr = f_w - op_R(disc, cf, cf.u_lag, phys.f) - fg
        w = solve_AR(disc, cf, phys.f, rr, with_R=False)
        rhs = g_w - op_Mg(disc, cf, cf.u_lag, phys.g) - kv - op_C(disc, cf, w, gm)
    return D_solve(disc, rhs, gm)


def recover_velocity(disc, cf, phys, f_w, p):
    """u^(k+1) from the momentum equation once p^(k+1) is known.

    R2: u = (A + R)^{-1}(f - f_g - B p);  R1: u = A^{-1}(f - f_g - R u^k - B p)."""
    fg = vec_fg(disc, cf, phys.g)
    rr = f_w - fg - op_B(disc, cf, p)
    if phys.variant == "R2":
        return solve_AR(disc, cf, phys.f, rr, with_R=True)
    rr = rr - op_R(disc, cf, cf.u_lag, phys.f)
    return solve_AR(disc, cf, phys.f, rr, with_R=False)


# ----------------------------------------------------------------------------
# GMRES (restarted, modified Gram-Schmidt, Givens rotations)
# ----------------------------------------------------------------------------

def gmres(apply, b, x0, rtol=1e-12, restart=30, maxit=1000):
    """Solve apply(x) = b; stop when ||b - apply(x)|| <= rtol ||b||.

    Returns (x, iterations, final relative residual, converged)."""
    shape = b.shape
    bv = b.reshape(-1)
    x = x0.reshape(-1).copy()
    bnorm = np.linalg.norm(bv)
    if bnorm == 0.0:
        return np.zeros(shape), 0, 0.0, True
    it = 0
    while True:
        r = bv - apply(x.reshape(shape)).reshape(-1)
        beta = np.linalg.norm(r)
        if beta <= rtol * bnorm:
            return x.reshape(shape), it, beta / bnorm, True
        if it >= maxit:
            return x.reshape(shape), it, beta / bnorm, False
        m = restart
        Vb = np.zeros((m + 1, len(bv)))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        Vb[0] = r / beta
        j_used = 0
        for j in range(m):
            w = apply(Vb[j].reshape(shape)).reshape(-1)
            for i in range(j + 1):
                H[i, j] = np.dot(w, Vb[i])
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                Vb[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            it += 1
            j_used = j + 1
            if abs(gvec[j + 1]) <= rtol * bnorm or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_used, :j_used]), gvec[:j_used])
        x = x + Vb[:j_used].T @ y


# ----------------------------------------------------------------------------
# Picard iteration and the ARK2 step (Section 3)
# ----------------------------------------------------------------------------

@dataclass
class StepOpts:
    picard_rtol: float = 1e-10
    picard_maxit: int = 10
    picard_fixed: int = 0        # > 0: exactly this many Picard iterations
    gmres_rtol: float = 1e-12
    gmres_restart: int = 30
    gmres_maxit: int = 1000


def nodal_primitives(q, gamma):
    """Nodal u = m / rho and p = (gamma - 1)(E - |m|^2 / (2 rho))."""
    u = q[1:4] / q[0][None]
    p = (gamma - 1.0) * (q[4] - 0.5 * np.sum(q[1:4] * u, axis=0))
    return u, p


def picard_solve(disc, phys, rho, f_w, g_w, u0, p0, adt, opts, info=None):
    """Fixed-point iteration of one implicit stage (R1 or R2).

    Initial guess: the previous stage (u0, p0).  Stops when
    max(||dp||/||p||, ||du||/||u||) < picard_rtol (READING c9), or after
    exactly ``picard_fixed`` iterations when that is set."""
    u, p = u0.copy(), p0.copy()
    kmax = opts.picard_fixed if opts.picard_fixed > 0 else opts.picard_maxit
    for k in range(kmax):
        cf = StageCoeffs(rho=rho, p_lag=p, u_lag=u, adt=adt)
        # far-field faces: their known outer data on the right-hand sides
        fb, gb = far_affine(disc, cf, phys)
        fk, gk = f_w - fb, g_w - gb
        rhs = schur_rhs(disc, cf, phys, fk, gk)
        p_new, its, rr, ok = gmres(lambda x: schur_apply(disc, cf, phys, x), rhs, p,
                                   rtol=opts.gmres_rtol, restart=opts.gmres_restart,
                                   maxit=opts.gmres_maxit)
        u_new = recover_velocity(disc, cf, phys, fk, p_new)
        dp = np.linalg.norm(p_new - p) / max(np.linalg.norm(p_new), 1e-300)
        nu = np.linalg.norm(u_new)
        du = np.linalg.norm(u_new - u) / nu if nu > 0 else 0.0
        if info is not None:
            info.setdefault("gmres_iters", []).append(its)
            info.setdefault("gmres_relres", []).append(rr)
            info.setdefault("picard_change", []).append(max(dp, du))
        u, p = u_new, p_new
        if opts.picard_fixed <= 0 and max(dp, du) < opts.picard_rtol:
            break
    return u, p, k + 1


def stage_state(disc, phys, rho, u, p, adt):
    """Conserved stage state from (rho, u, p): rho u = M^{-1} A u and
    rho E = M^{-1}(D p + k(u))."""
    cf = StageCoeffs(rho=rho, p_lag=p, u_lag=u, adt=adt)
    m = disc.mass_solve(op_A(disc, cf, u))
    E = disc.mass_solve((op_D(disc, p, phys.gamma) + vec_k(disc, cf, u))[None])[0]
    return np.concatenate([rho[None], m, E[None]], axis=0)


def imex_ark2_step(disc, phys, q, dt, opts=None, info=None):
    """One step of the three-stage IMEX ARK2 scheme (TR-BDF2 implicit part).

    Stage l = 2, 3: rho explicit, then the coupled (u, p) system solved by
    Picard + Schur + GMRES; final update with weights b (literal form,
    READING c8)."""
    opts = opts or StepOpts()
    a, at, bw, _ = ark2_tableau()
    Mq = disc.vol_weak(disc.at_quad(q))          # weak form of q^n: int q phi_i
    r_ns, r_s = [], []
    rn, rs = explicit_residuals(disc, q, phys)
    r_ns.append(rn); r_s.append(rs)
    y = q
    for l in (1, 2):
        adt = at[l, l] * dt
        rho_w = Mq[0] + dt * sum(a[l, m] * r_ns[m][0] for m in range(l))
        rho = disc.mass_solve(rho_w[None])[0]
        f_w = Mq[1:4] + dt * sum(a[l, m] * r_ns[m][1:4] + at[l, m] * r_s[m][1:4]
                                 for m in range(l))
        g_w = Mq[4] + dt * sum(a[l, m] * r_ns[m][4] + at[l, m] * r_s[m][4]
                               for m in range(l))
        u0, p0 = nodal_primitives(y, phys.gamma)
        u, p, k = picard_solve(disc, phys, rho, f_w, g_w, u0, p0, adt, opts, info)
        if info is not None:
            info.setdefault("picard_iters", []).append(k)
        y = stage_state(disc, phys, rho, u, p, adt)
        rn, rs = explicit_residuals(disc, y, phys)
        r_ns.append(rn); r_s.append(rs)
    upd = sum(bw[l] * (r_ns[l] + r_s[l]) for l in range(3))
    return q + dt * disc.mass_solve(upd)


# ----------------------------------------------------------------------------
# Sub-meshes for sampled checks at full size
# ----------------------------------------------------------------------------

def submesh(mesh, targets, layers):
    """Cells ``targets`` plus ``layers`` rings of face neighbours.

    Faces with a side outside the set are dropped, so results are exact only
    on cells at least ``layers`` rings inside; returns (sub-mesh, old ids,
    positions of the targets in the sub-mesh)."""
    from types import SimpleNamespace
    keep = set(int(t) for t in targets)
    adj = {}
    for eL, _, eR, _ in mesh.int_faces:
        adj.setdefault(int(eL), set()).add(int(eR))
        adj.setdefault(int(eR), set()).add(int(eL))
    for ec, _, ef, _, _ in mesh.hang_faces:
        adj.setdefault(int(ec), set()).add(int(ef))
        adj.setdefault(int(ef), set()).add(int(ec))
    for _ in range(layers):
        new = set(keep)
        for e in keep:
            new |= adj.get(e, set())
        keep = new
    old = np.array(sorted(keep), dtype=np.int64)
    new_of = -np.ones(mesh.vertices.shape[0], dtype=np.int64)
    new_of[old] = np.arange(len(old))
    inf = mesh.int_faces
    ok = (new_of[inf[:, 0]] >= 0) & (new_of[inf[:, 2]] >= 0)
    int_f = inf[ok].copy()
    int_f[:, 0] = new_of[int_f[:, 0]]
    int_f[:, 2] = new_of[int_f[:, 2]]
    hf = mesh.hang_faces
    ok = (new_of[hf[:, 0]] >= 0) & (new_of[hf[:, 2]] >= 0)
    hang_f = hf[ok].copy()
    hang_f[:, 0] = new_of[hang_f[:, 0]]
    hang_f[:, 2] = new_of[hang_f[:, 2]]
    bf = mesh.bdry_faces
    ok = new_of[bf[:, 0]] >= 0
    bd_f = bf[ok].copy()
    bd_f[:, 0] = new_of[bd_f[:, 0]]
    sub = SimpleNamespace(dim=mesh.dim, vertices=mesh.vertices[old], int_faces=int_f,
                          hang_faces=hang_f, bdry_faces=bd_f)
    pos = new_of[np.asarray(targets, dtype=np.int64)]
    return sub, old, pos
