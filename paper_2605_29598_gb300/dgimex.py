"""ctypes binding of ``libdgimex.so`` (declared in ``include/dgimex.h``).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (FP64, contiguous,
field-major ``[field][cell][node]``); streams are taken from torch.

The library is loaded on first use and must have been built
(``paper_2605_29598_gb300.build.build()``); a missing library raises
:class:`RuntimeError` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DG_OK = 0
DG_NODES_GL, DG_NODES_GLL = 0, 1
DG_R1, DG_R2 = 1, 2
DG_FP64, DG_MIXED, DG_MIXED_EXPLICIT, DG_PAIRS = 0, 1, 2, 3
PRECISIONS = {"fp64": DG_FP64, "mixed": DG_MIXED, "mixed_explicit": DG_MIXED_EXPLICIT, "pairs": DG_PAIRS}
STATUS = {0: "DG_OK", -1: "DG_ERR_ARG", -2: "DG_ERR_UNSUPPORTED", -3: "DG_ERR_CUDA",
          -4: "DG_ERR_NOT_CONVERGED", -5: "DG_ERR_TIMEOUT", -6: "DG_ERR_NONFINITE",
          -7: "DG_ERR_OOM"}

_I64P = C.POINTER(C.c_int64)
_DP = C.POINTER(C.c_double)


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("degree", C.c_int), ("node_set", C.c_int),
                ("n_elem", C.c_int64), ("vertices", _DP),
                ("n_int", C.c_int64), ("int_faces", _I64P),
                ("n_hang", C.c_int64), ("hang_faces", _I64P),
                ("n_bdry", C.c_int64), ("bdry_faces", _I64P)]


class MeshStats(C.Structure):
    _fields_ = [("dim", C.c_int), ("degree", C.c_int), ("n1d", C.c_int),
                ("nodes_per_elem", C.c_int), ("n_elem", C.c_int64), ("n_nodes", C.c_int64),
                ("n_face_points", C.c_int64), ("n_hang_points", C.c_int64),
                ("workspace_bytes", C.c_int64), ("tile_fp64", C.c_int * 3),
                ("tile_fp32", C.c_int * 3), ("terrain_following", C.c_int),
                ("fused_stage", C.c_int * 3)]


class Sponge(C.Structure):
    _fields_ = [("lambda_bar", C.c_double), ("z_b", C.c_double), ("z_t", C.c_double),
                ("x_layers", C.c_int), ("x_lo", C.c_double), ("x_hi", C.c_double),
                ("x_width", C.c_double), ("y_layers", C.c_int), ("y_lo", C.c_double),
                ("y_hi", C.c_double), ("y_width", C.c_double)]


class Phys(C.Structure):
    _fields_ = [("gamma", C.c_double), ("g", C.c_double), ("f", C.c_double),
                ("variant", C.c_int), ("penalty", C.c_int), ("precision", C.c_int),
                ("f_cell", C.c_void_p), ("lambda_min", C.c_double)]


class ImplicitCoeffs(C.Structure):
    _fields_ = [("rho", C.c_void_p), ("p_lag", C.c_void_p), ("u_lag", C.c_void_p),
                ("a_dt", C.c_double)]


# GMRES preconditioner choice (dg_gmres_opts.precond)
DG_PRECOND_NONE = 0
DG_PRECOND_VLINE = 1
DG_PRECOND_CELL = 2


def _precond_kind(p):
    """False/None: none; True or "vline": vertical lines; "cell": cell blocks."""
    if not p:
        return DG_PRECOND_NONE
    if p is True or p == "vline":
        return DG_PRECOND_VLINE
    if p == "cell":
        return DG_PRECOND_CELL
    raise ValueError(f"unknown preconditioner {p!r}")


class GmresOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int),
                ("inner_rtol", C.c_double), ("precond", C.c_int)]


class GmresInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("relres", C.c_double), ("refinements", C.c_int)]


class StepOpts(C.Structure):
    _fields_ = [("picard_rtol", C.c_double), ("picard_maxit", C.c_int),
                ("picard_fixed", C.c_int), ("gmres", GmresOpts), ("graph", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("picard_iters", C.c_int * 3), ("gmres_iters_total", C.c_int),
                ("max_relres", C.c_double), ("refinements_total", C.c_int)]


EXPORTS = {
    "dg_status_string": (C.c_char_p, [C.c_int]),
    "dg_last_error": (C.c_char_p, []),
    "dg_ctx_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "dg_ctx_destroy": (None, [C.c_void_p]),
    "dg_mesh_create": (C.c_int, [C.c_void_p, C.POINTER(MeshDesc), C.POINTER(C.c_void_p)]),
    "dg_mesh_destroy": (None, [C.c_void_p]),
    "dg_mesh_validate": (C.c_int, [C.POINTER(MeshDesc)]),
    "dg_mesh_info": (C.c_int, [C.c_void_p, C.POINTER(MeshStats)]),
    "dg_mesh_node_coords": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_apply_explicit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys), C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_apply_implicit": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys),
                                    C.POINTER(ImplicitCoeffs), C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "dg_precond_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys),
                                   C.POINTER(ImplicitCoeffs), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_schur_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys), C.POINTER(ImplicitCoeffs),
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dg_recover_velocity": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys),
                                      C.POINTER(ImplicitCoeffs), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    "dg_gmres_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys),
                                 C.POINTER(ImplicitCoeffs), C.c_void_p, C.c_void_p,
                                 C.POINTER(GmresOpts), C.POINTER(GmresInfo), C.c_void_p]),
    "imex_ark2_step": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys), C.c_void_p, C.c_double,
                                 C.POINTER(StepOpts), C.POINTER(StepInfo), C.c_void_p]),
}


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("timed_launches", C.c_int64),
                ("total_ms", C.c_double)]


EXPORTS["dg_apply_explicit_noalloc"] = (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys),
                                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p])
EXPORTS["dg_ensemble_create"] = (C.c_int, [C.c_void_p, C.POINTER(MeshDesc), C.POINTER(C.c_double),
                                           C.c_int, C.POINTER(C.c_void_p)])
EXPORTS["dg_ensemble_destroy"] = (None, [C.c_void_p])
EXPORTS["dg_ensemble_info"] = (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64)])
EXPORTS["dg_ensemble_instance_nodes"] = (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64)])
EXPORTS["dg_ensemble_set_state"] = (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p])
EXPORTS["dg_ensemble_get_state"] = (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p])
EXPORTS["dg_ensemble_step"] = (C.c_int, [C.c_void_p, C.POINTER(Phys), C.POINTER(C.c_double),
                                         C.POINTER(StepOpts), C.POINTER(StepInfo), C.c_void_p])
EXPORTS["dg_mesh_autotune"] = (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p])
EXPORTS["dg_mesh_set_fused_stage"] = (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int])
EXPORTS["dg_mesh_set_vmult_tile"] = (C.c_int, [C.c_void_p, C.c_int, C.c_int])
EXPORTS["dg_mesh_set_far_state"] = (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p])
EXPORTS["dg_geostrophic_error"] = (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys), C.c_void_p,
                                              C.POINTER(C.c_double), C.c_void_p])
EXPORTS["dg_mesh_set_background"] = (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Phys), C.c_void_p,
                                                C.c_void_p])
EXPORTS["dg_mesh_set_sponge"] = (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Sponge), C.c_void_p,
                                            C.c_void_p])
EXPORTS["dg_probe_fma"] = (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.c_void_p])
EXPORTS["dg_profile_begin"] = (C.c_int, [C.c_void_p, C.c_uint32])
EXPORTS["dg_profile_end"] = (C.c_int, [C.c_void_p, C.POINTER(KernelStat), C.c_int,
                                       C.POINTER(C.c_int)])

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Open libdgimex.so (once) and declare every exported signature."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"libdgimex.so not found at {path}: build it with "
            "paper_2605_29598_gb300.build.build() (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DGError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.dg_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status, where, allow=()):
    if status != DG_OK and status not in allow:
        raise DGError(status, where)
    return status


def _validate(numel, device_index, n=None, device=None):
    """The C ABI takes raw pointers and cannot see a buffer's length or
    device, so the binding checks both: a short buffer would be read or
    written out of bounds on the GPU."""
    if n is not None and numel != n:
        raise ValueError(f"expected {n} elements, got {numel}")
    if device is not None and device_index != device:
        raise ValueError(f"tensor on cuda:{device_index}, context on cuda:{device}")


def _ptr(t, n=None, device=None):
    """Device pointer of a contiguous FP64 CUDA tensor (of n elements on
    cuda:device when given)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    _validate(t.numel(), t.device.index, n, device)
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def make_phys(gamma=1.4, g=9.81, f=1e-4, variant="R2", penalty=True, precision="fp64", lambda_min=0.0):
    """lambda_min > 0: floor of the non-stiff Rusanov coefficient (not in the paper)."""
    return Phys(gamma=gamma, g=g, f=f, variant=DG_R2 if variant == "R2" else DG_R1,
                penalty=1 if penalty else 0,
                precision=PRECISIONS[precision], lambda_min=lambda_min)


def validate_mesh(mesh, degree, node_set=DG_NODES_GL):
    """Run dg_mesh_create's host-side checks on a host mesh (see
    ``inputs.Mesh``) without a context or GPU; raises DGError on failure."""
    lib = load()
    v = np.ascontiguousarray(mesh.vertices, dtype=np.float64)
    a = np.ascontiguousarray(mesh.int_faces, dtype=np.int64).reshape(-1, 4)
    h = np.ascontiguousarray(mesh.hang_faces, dtype=np.int64).reshape(-1, 5)
    b = np.ascontiguousarray(mesh.bdry_faces, dtype=np.int64).reshape(-1, 3)
    d = MeshDesc(dim=int(mesh.dim), degree=int(degree), node_set=int(node_set), n_elem=v.shape[0],
                 vertices=v.ctypes.data_as(_DP),
                 n_int=a.shape[0], int_faces=a.ctypes.data_as(_I64P),
                 n_hang=h.shape[0], hang_faces=h.ctypes.data_as(_I64P),
                 n_bdry=b.shape[0], bdry_faces=b.ctypes.data_as(_I64P))
    return _check(lib.dg_mesh_validate(C.byref(d)), "dg_mesh_validate")


class Context:
    def __init__(self, device=0):
        self.lib = load()
        h = C.c_void_p()
        _check(self.lib.dg_ctx_create(device, C.byref(h)), "dg_ctx_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.dg_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """Device mesh built from host lists (see ``inputs.Mesh``)."""

    def __init__(self, ctx: Context, mesh, degree: int, node_set: int = DG_NODES_GL):
        self.ctx = ctx
        self.lib = ctx.lib
        self.dim = int(mesh.dim)
        self.degree = int(degree)
        self._verts = np.ascontiguousarray(mesh.vertices, dtype=np.float64)
        self._int = np.ascontiguousarray(mesh.int_faces, dtype=np.int64).reshape(-1, 4)
        self._hang = np.ascontiguousarray(mesh.hang_faces, dtype=np.int64).reshape(-1, 5)
        self._bdry = np.ascontiguousarray(mesh.bdry_faces, dtype=np.int64).reshape(-1, 3)
        d = MeshDesc(dim=self.dim, degree=self.degree, node_set=node_set,
                     n_elem=self._verts.shape[0],
                     vertices=self._verts.ctypes.data_as(_DP),
                     n_int=self._int.shape[0], int_faces=self._int.ctypes.data_as(_I64P),
                     n_hang=self._hang.shape[0], hang_faces=self._hang.ctypes.data_as(_I64P),
                     n_bdry=self._bdry.shape[0], bdry_faces=self._bdry.ctypes.data_as(_I64P))
        h = C.c_void_p()
        _check(self.lib.dg_mesh_create(ctx.h, C.byref(d), C.byref(h)), "dg_mesh_create")
        self.h = h
        st = self.stats()
        self.n_elem = st.n_elem
        self.N = st.n_nodes
        self.Np = st.nodes_per_elem

    def _p(self, t, fields=1):
        """Pointer of a field-major device array of `fields` x N values."""
        return _ptr(t, fields * self.N, self.ctx.device)

    def _cf(self, cf):
        """Coefficients built by `coeffs` for another mesh size or device are
        rejected before they reach the library."""
        _validate(getattr(cf, "_n", self.N), getattr(cf, "_dev", self.ctx.device), self.N, self.ctx.device)
        return C.byref(cf)

    def geostrophic_error(self, phys, q, stream=None):
        """E_geo: domain mean of |(1/rho) dp/dx - f v| (scheme's own operators)."""
        out = C.c_double()
        _check(self.lib.dg_geostrophic_error(self.ctx.h, self.h, C.byref(phys), self._p(q, 5), C.byref(out),
                                             _stream(stream)), "dg_geostrophic_error")
        return out.value

    def set_background(self, phys, q_bg, stream=None):
        """Background state for the perturbation-form (mixed) explicit operator."""
        _check(self.lib.dg_mesh_set_background(self.ctx.h, self.h, C.byref(phys), self._p(q_bg, 5),
                                               _stream(stream)), "dg_mesh_set_background")

    def set_sponge(self, q_bar=None, lambda_bar=0.0, z_b=0.0, z_t=1.0, x_layers=None, y_layers=None,
                   stream=None):
        """Rayleigh damping layers (see dg_mesh_set_sponge); x_layers / y_layers
        are (lo, hi, width) or None; q_bar=None switches the layers off."""
        if q_bar is None:
            _check(self.lib.dg_mesh_set_sponge(self.ctx.h, self.h, None, None, _stream(stream)),
                   "dg_mesh_set_sponge")
            return
        s = Sponge(lambda_bar=lambda_bar, z_b=z_b, z_t=z_t)
        if x_layers is not None:
            s.x_layers, (s.x_lo, s.x_hi, s.x_width) = 1, x_layers
        if y_layers is not None:
            s.y_layers, (s.y_lo, s.y_hi, s.y_width) = 1, y_layers
        _check(self.lib.dg_mesh_set_sponge(self.ctx.h, self.h, C.byref(s), self._p(q_bar, 5), _stream(stream)),
               "dg_mesh_set_sponge")

    def autotune(self, precision="mixed", stream=None):
        """Pick the cells-per-block multiplier of each cell kernel by timing."""
        prec = PRECISIONS[precision]
        _check(self.lib.dg_mesh_autotune(self.ctx.h, self.h, prec, _stream(stream)),
               "dg_mesh_autotune")
        s = self.stats()
        return list(s.tile_fp64), list(s.tile_fp32), list(s.fused_stage)

    def set_far_state(self, q_far, stream=None):
        """Outer state (5 x N) of the far-field faces (dg_mesh_set_far_state)."""
        _check(self.lib.dg_mesh_set_far_state(self.ctx.h, self.h, self._p(q_far, 5), _stream(stream)),
               "dg_mesh_set_far_state")

    def set_fused_stage(self, fp64, fp32, pairs=0):
        """Schedule of the fused vmult kernels per precision (1: neighbour
        node lines, 0: trace array, 2: one thread per x-line); see
        dg_mesh_set_fused_stage."""
        _check(self.lib.dg_mesh_set_fused_stage(self.h, int(fp64), int(fp32), int(pairs)),
               "dg_mesh_set_fused_stage")

    def set_vmult_tile(self, precision, tile):
        """Cells-per-block multiplier (1, 2, 4) of the schedule-2 vmult
        passes of one precision; see dg_mesh_set_vmult_tile."""
        _check(self.lib.dg_mesh_set_vmult_tile(self.h, PRECISIONS[precision], int(tile)),
               "dg_mesh_set_vmult_tile")

    def stats(self) -> MeshStats:
        s = MeshStats()
        _check(self.lib.dg_mesh_info(self.h, C.byref(s)), "dg_mesh_info")
        return s

    def close(self):
        if self.h:
            self.lib.dg_mesh_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- operators -----------------------------------------------------------
    def node_coords(self, stream=None):
        import torch
        xyz = torch.empty((self.dim, self.N), dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        _check(self.lib.dg_mesh_node_coords(self.ctx.h, self.h, self._p(xyz, self.dim), _stream(stream)),
               "dg_mesh_node_coords")
        return xyz

    def apply_explicit(self, phys, q, f_ns=None, f_s=None, stream=None):
        import torch
        f_ns = torch.empty((5, self.N), dtype=torch.float64, device=q.device) if f_ns is None else f_ns
        f_s = torch.empty((4, self.N), dtype=torch.float64, device=q.device) if f_s is None else f_s
        _check(self.lib.dg_apply_explicit(self.ctx.h, self.h, C.byref(phys), self._p(q, 5), self._p(f_ns, 5),
                                          self._p(f_s, 4), _stream(stream)), "dg_apply_explicit")
        return f_ns, f_s

    @staticmethod
    def coeffs(rho, p_lag, u_lag, a_dt):
        """Frozen stage coefficients: rho and p_lag (N values), u_lag (3 x N),
        all on one device.  The returned struct holds the three tensors, so
        they live at least as long as it does."""
        n = rho.numel()
        dev = rho.device.index
        cf = ImplicitCoeffs(rho=_ptr(rho), p_lag=_ptr(p_lag, n, dev), u_lag=_ptr(u_lag, 3 * n, dev),
                            a_dt=float(a_dt))
        cf._n, cf._dev, cf._keep = n, dev, (rho, p_lag, u_lag)
        return cf

    def apply_implicit(self, phys, cf, x, y=None, stream=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(self.lib.dg_apply_implicit(self.ctx.h, self.h, C.byref(phys), self._cf(cf), self._p(x),
                                          self._p(y), _stream(stream)), "dg_apply_implicit")
        return y

    def precond_apply(self, phys, cf, r, z=None, stream=None, kind="vline"):
        """z = P^{-1} r, P the Schur GMRES preconditioner of `kind` ("vline" or "cell")."""
        import torch
        z = torch.empty_like(r) if z is None else z
        _check(self.lib.dg_precond_apply(self.ctx.h, self.h, C.byref(phys), self._cf(cf), _precond_kind(kind),
                                         self._p(r), self._p(z), _stream(stream)), "dg_precond_apply")
        return z

    def schur_rhs(self, phys, cf, m_hat, e_hat, rhs=None, stream=None):
        import torch
        rhs = torch.empty_like(e_hat) if rhs is None else rhs
        _check(self.lib.dg_schur_rhs(self.ctx.h, self.h, C.byref(phys), self._cf(cf), self._p(m_hat, 3),
                                     self._p(e_hat), self._p(rhs), _stream(stream)), "dg_schur_rhs")
        return rhs

    def recover_velocity(self, phys, cf, m_hat, p, u=None, stream=None):
        import torch
        u = torch.empty_like(m_hat) if u is None else u
        _check(self.lib.dg_recover_velocity(self.ctx.h, self.h, C.byref(phys), self._cf(cf),
                                            self._p(m_hat, 3), self._p(p), self._p(u, 3), _stream(stream)),
               "dg_recover_velocity")
        return u

    def gmres_solve(self, phys, cf, b, x, rtol=1e-12, restart=30, maxit=1000, stream=None,
                    allow_not_converged=False, inner_rtol=0.0, precond=False):
        """precond=True: right preconditioning by the vertical-line solve."""
        opts = GmresOpts(rtol=rtol, restart=restart, maxit=maxit, inner_rtol=inner_rtol,
                         precond=_precond_kind(precond))
        info = GmresInfo()
        st = self.lib.dg_gmres_solve(self.ctx.h, self.h, C.byref(phys), self._cf(cf), self._p(b),
                                     self._p(x), C.byref(opts), C.byref(info), _stream(stream))
        _check(st, "dg_gmres_solve", allow=(-4,) if allow_not_converged else ())
        return info

    def step(self, phys, q, dt, picard_rtol=1e-10, picard_maxit=10, picard_fixed=0,
             gmres_rtol=1e-10, gmres_restart=30, gmres_maxit=1000, stream=None,
             gmres_inner_rtol=0.0, graph=False, gmres_precond=False):
        opts = StepOpts(picard_rtol=picard_rtol, picard_maxit=picard_maxit,
                        picard_fixed=picard_fixed,
                        gmres=GmresOpts(rtol=gmres_rtol, restart=gmres_restart, maxit=gmres_maxit,
                                        inner_rtol=gmres_inner_rtol,
                                        precond=_precond_kind(gmres_precond)),
                        graph=1 if graph else 0)
        info = StepInfo()
        _check(self.lib.imex_ark2_step(self.ctx.h, self.h, C.byref(phys), self._p(q, 5), float(dt),
                                       C.byref(opts), C.byref(info), _stream(stream)),
               "imex_ark2_step")
        return info


def probe_fma(ctx: "Context", bits: int, iters: int | None = None, stream=None):
    """FMA throughput of the device (dg_probe_fma): (TFLOP/s, ms)."""
    iters = iters or (8192 if bits == 64 else 524288)
    tf, ms = C.c_double(), C.c_double()
    _check(ctx.lib.dg_probe_fma(ctx.h, int(bits), int(iters), C.byref(tf), C.byref(ms), _stream(stream)),
           "dg_probe_fma")
    return tf.value, ms.value


# ----------------------------------------------------------------------------
# launch accounting
# ----------------------------------------------------------------------------

KERNEL_CLASSES = ["trace", "face_explicit", "hang_gather", "volume_explicit", "face_lambda",
                  "face_grad", "volume_grad", "face_div", "volume_div", "ustar", "multidot",
                  "reduce", "multiaxpy", "vector", "stage", "picard_norms", "precond", "precond_setup"]


def profile_begin(mesh: "Mesh", timed=()):
    """Count every launch on ``mesh``; bracket the classes in ``timed`` with
    CUDA events."""
    mask = 0
    for name in timed:
        mask |= 1 << KERNEL_CLASSES.index(name)
    _check(mesh.lib.dg_profile_begin(mesh.h, mask), "dg_profile_begin")


def profile_end(mesh: "Mesh"):
    """Return {class: (launches, timed_launches, total_ms)}."""
    out = (KernelStat * len(KERNEL_CLASSES))()
    n = C.c_int()
    _check(mesh.lib.dg_profile_end(mesh.h, out, len(KERNEL_CLASSES), C.byref(n)),
           "dg_profile_end")
    return {out[k].name.decode(): (out[k].launches, out[k].timed_launches, out[k].total_ms)
            for k in range(n.value)}


class Ensemble:
    """Independent instances advanced together (see dg_ensemble_create).

    meshes: list of host meshes (``inputs.Mesh``); degrees: list of ints;
    f: list of Coriolis parameters (one per instance)."""

    def __init__(self, ctx: Context, meshes, degrees, f):
        self.ctx = ctx
        self.lib = ctx.lib
        n = len(meshes)
        keep = []
        descs = (MeshDesc * n)()
        for i, (m, r) in enumerate(zip(meshes, degrees)):
            v = np.ascontiguousarray(m.vertices, dtype=np.float64)
            a = np.ascontiguousarray(m.int_faces, dtype=np.int64).reshape(-1, 4)
            h = np.ascontiguousarray(m.hang_faces, dtype=np.int64).reshape(-1, 5)
            b = np.ascontiguousarray(m.bdry_faces, dtype=np.int64).reshape(-1, 3)
            keep += [v, a, h, b]
            descs[i] = MeshDesc(dim=int(m.dim), degree=int(r), node_set=DG_NODES_GL,
                                n_elem=v.shape[0], vertices=v.ctypes.data_as(_DP),
                                n_int=a.shape[0], int_faces=a.ctypes.data_as(_I64P),
                                n_hang=h.shape[0], hang_faces=h.ctypes.data_as(_I64P),
                                n_bdry=b.shape[0], bdry_faces=b.ctypes.data_as(_I64P))
        fa = (C.c_double * n)(*[float(x) for x in f])
        hnd = C.c_void_p()
        _check(self.lib.dg_ensemble_create(ctx.h, descs, fa, n, C.byref(hnd)), "dg_ensemble_create")
        self.h = hnd
        self.n = n
        self.nodes = []
        for i in range(n):
            k = C.c_int64()
            _check(self.lib.dg_ensemble_instance_nodes(self.h, i, C.byref(k)), "instance_nodes")
            self.nodes.append(k.value)
        g = C.c_int()
        t = C.c_int64()
        _check(self.lib.dg_ensemble_info(self.h, C.byref(g), C.byref(t)), "dg_ensemble_info")
        self.n_groups = g.value
        self.total_nodes = t.value

    def _q(self, i, q):
        if not 0 <= i < self.n:
            raise IndexError(f"instance {i} of {self.n}")
        return _ptr(q, 5 * self.nodes[i], self.ctx.device)

    def set_state(self, i, q, stream=None):
        _check(self.lib.dg_ensemble_set_state(self.h, i, self._q(i, q), _stream(stream)), "set_state")

    def get_state(self, i, q, stream=None):
        _check(self.lib.dg_ensemble_get_state(self.h, i, self._q(i, q), _stream(stream)), "get_state")
        return q

    def step(self, phys, dt, picard_rtol=1e-10, picard_maxit=10, picard_fixed=0, gmres_rtol=1e-10,
             gmres_restart=30, gmres_maxit=1000, gmres_inner_rtol=0.0, stream=None, graph=False,
             gmres_precond=False):
        opts = StepOpts(picard_rtol=picard_rtol, picard_maxit=picard_maxit,
                        picard_fixed=picard_fixed,
                        gmres=GmresOpts(rtol=gmres_rtol, restart=gmres_restart, maxit=gmres_maxit,
                                        inner_rtol=gmres_inner_rtol,
                                        precond=_precond_kind(gmres_precond)),
                        graph=1 if graph else 0)
        if len(dt) != self.n:
            raise ValueError(f"{len(dt)} time steps for {self.n} instances")
        dts = (C.c_double * self.n)(*[float(x) for x in dt])
        info = StepInfo()
        _check(self.lib.dg_ensemble_step(self.h, C.byref(phys), dts, C.byref(opts), C.byref(info),
                                         _stream(stream)), "dg_ensemble_step")
        return info

    def close(self):
        if self.h:
            self.lib.dg_ensemble_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
