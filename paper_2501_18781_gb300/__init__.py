"""Matrix-free Q_k hexahedral operators for one GB300 (sm_103a).

A thin binding over libmfgb.so (C ABI in include/mfgb.h).  Every numerical step runs in
the library's CUDA kernels; this module only marshals arguments.  PyTorch tensors
provide device memory: pass CUDA tensors, their data pointers go to the library.
"""
import ctypes as C

from . import _lib
from ._lib import (MF_F64, MF_F32, MF_F16, MF_BF16, MF_OP_HELMHOLTZ, MF_OP_HEAT, MF_OP_OSEEN, MF_OP_REINIT,
                   MF_HEAVISIDE_TANH, MF_HEAVISIDE_SINE, MF_COEF_INKERNEL, MF_COEF_QPOINT,
                   MF_FIELD_PHI, MF_FIELD_T_PREV, MF_FIELD_BETA, MF_FIELD_K_QPOINT,
                   MF_SOLVER_CG, MF_SOLVER_GMRES, MF_SOLVER_DEFECT_CORRECTION,
                   MF_PREC_NONE, MF_PREC_JACOBI, MF_PREC_CHEBYSHEV, MF_PREC_BLOCK_JACOBI, MF_PREC_BLOCK_TRIANGULAR,
                   MFError, check)

__all__ = ["Context", "Mesh", "DofMap", "Operator", "MFError", "build_library", "load_library"]


def build_library(force=False):
    from .build import build
    return build(force=force)


def load_library():
    return _lib.load()


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return MF_F64
    if t.dtype == torch.float32:
        return MF_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


class Context:
    """Library context on one CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device=0, stream=None):
        import torch
        lib = _lib.load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        # torch's default stream has handle 0; hand the library cudaStreamLegacy (0x1) so that
        # its work stays ordered with torch's copies and kernels
        handle = stream.cuda_stream or 0x1
        h = C.c_void_p()
        check(lib.mf_context_create(device, C.c_void_p(handle), C.byref(h)))
        self.h = h
        self.device = device

    def dot(self, x, y, nvec=1):
        """Deterministic fp64-accumulated inner products of nvec vector pairs (device tensor out)."""
        import torch
        out = torch.empty(nvec, dtype=torch.float64, device="cuda")
        n = x.numel() // nvec
        check(_lib.load().mf_dot(self.h, _ptr(x), _ptr(y), n, n, nvec, _dtype_code(x), _ptr(out)))
        return out

    def launch_count(self):
        return int(_lib.load().mf_context_launch_count(self.h))

    def close(self):
        if self.h:
            _lib.load().mf_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx, h, keep=None):
        self.ctx, self.h, self._keep = ctx, h, keep

    @classmethod
    def uniform(cls, ctx, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        nn = (C.c_int * 3)(*([n] * 3 if isinstance(n, int) else n))
        h = C.c_void_p()
        check(_lib.load().mf_mesh_uniform(ctx.h if ctx else None, nn, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi), C.byref(h)))
        return cls(ctx, h)

    @classmethod
    def octree(cls, ctx, base, levels, leaves, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        import numpy as np
        lv = np.ascontiguousarray(leaves, dtype=np.int32)
        h = C.c_void_p()
        check(_lib.load().mf_mesh_octree(ctx.h if ctx else None, base, levels, (C.c_double * 3)(*lo), (C.c_double * 3)(*hi),
                                         lv.ctypes.data_as(C.POINTER(C.c_int32)), lv.shape[0], C.byref(h)))
        return cls(ctx, h)

    def __del__(self):
        try:
            if self.h:
                _lib.load().mf_mesh_destroy(self.h)
        except Exception:
            pass


class DofMap:
    def __init__(self, mesh, degree=2, dirichlet_faces=0):
        h = C.c_void_p()
        check(_lib.load().mf_dofmap_create(mesh.h, degree, dirichlet_faces, C.byref(h)))
        self.mesh, self.h, self.degree = mesh, h, degree
        nd, nc, ncon, nent = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        check(_lib.load().mf_dofmap_query(h, C.byref(nd), C.byref(nc), C.byref(ncon), C.byref(nent)))
        self.n_dofs, self.n_cells = nd.value, nc.value
        self.n_constraints, self.n_constraint_entries = ncon.value, nent.value

    def export(self, cell_map=True, constraints=True, coords=True, dirichlet=True):
        """Host numpy copies: cell_map (n_cells, (k+1)^3), constraint CSR, coordinates, Dirichlet flags."""
        import numpy as np
        nb = (self.degree + 1) ** 3
        cm = np.empty((self.n_cells, nb), np.int32) if cell_map else None
        rp = np.empty(self.n_constraints + 1, np.int64) if constraints else None
        cols = np.empty(max(self.n_constraint_entries, 1), np.int32) if constraints else None
        w = np.empty(max(self.n_constraint_entries, 1), np.float64) if constraints else None
        xyz = np.empty((self.n_dofs, 3), np.float64) if coords else None
        dr = np.empty(self.n_dofs, np.uint8) if dirichlet else None
        p = lambda a, t: a.ctypes.data_as(C.POINTER(t)) if a is not None else None
        check(_lib.load().mf_dofmap_export(self.h, p(cm, C.c_int32), p(rp, C.c_int64), p(cols, C.c_int32),
                                           p(w, C.c_double), p(xyz, C.c_double), p(dr, C.c_uint8)))
        out = {}
        if cell_map:
            out["cell_map"] = cm
        if constraints:
            out["con_rowptr"] = rp
            out["con_cols"] = cols[:self.n_constraint_entries]
            out["con_w"] = w[:self.n_constraint_entries]
        if coords:
            out["coords"] = xyz
        if dirichlet:
            out["dirichlet"] = dr.astype(bool)
        return out

    def coords(self):
        return self.export(cell_map=False, constraints=False, dirichlet=False)["coords"]

    def __del__(self):
        try:
            if self.h:
                _lib.load().mf_dofmap_destroy(self.h)
        except Exception:
            pass


def solver_params(solver="cg", precond="jacobi", tol=1e-10, maxit=5000, restart=50, cheby_degree=4,
                  inner_tol=1e-4, inner_maxit=100, use_graph=False, cheby_ratio=30.0, lanczos_steps=20,
                  fp64_arith="f64", schur_tol=0.1, schur_maxit=30, velocity_steps=10, inner_arith="f32"):
    s = _lib.SolverParams()
    s.fp64_arith = {"f64": 0, "df64": 1, "auto": 2}[fp64_arith]
    s.solver = {"cg": MF_SOLVER_CG, "gmres": MF_SOLVER_GMRES, "defect_correction": MF_SOLVER_DEFECT_CORRECTION}[solver]
    s.precond = {"none": MF_PREC_NONE, "jacobi": MF_PREC_JACOBI, "chebyshev": MF_PREC_CHEBYSHEV,
                 "block_jacobi": MF_PREC_BLOCK_JACOBI, "block_triangular": MF_PREC_BLOCK_TRIANGULAR}[precond]
    s.schur_tol, s.schur_maxit, s.velocity_steps = schur_tol, schur_maxit, velocity_steps
    s.inner_arith = {"f32": MF_F32, "f16": MF_F16, "bf16": MF_BF16, "tc": _lib.MF_INNER_TENSOR_CORES}[inner_arith]
    s.inner_dtype = MF_F32
    s.restart, s.cheby_degree, s.maxit, s.inner_maxit = restart, cheby_degree, maxit, inner_maxit
    s.use_graph = 1 if use_graph else 0
    s.tol, s.inner_tol, s.cheby_ratio, s.lanczos_steps = tol, inner_tol, cheby_ratio, lanczos_steps
    return s


class Operator:
    """A matrix-free operator; ``params`` are the fields of mf_op_params (kind given by name)."""

    KINDS = {"helmholtz": MF_OP_HELMHOLTZ, "heat": MF_OP_HEAT, "oseen": MF_OP_OSEEN, "reinit": MF_OP_REINIT}
    FIELDS = {"phi": MF_FIELD_PHI, "t_prev": MF_FIELD_T_PREV, "beta": MF_FIELD_BETA, "k_qpoint": MF_FIELD_K_QPOINT,
              "rhocp_qpoint": _lib.MF_FIELD_RHOCP_QPOINT, "beta_qpoint": _lib.MF_FIELD_BETA_QPOINT}

    def __init__(self, ctx, kind, maps, **params):
        p = _lib.OpParams()
        p.kind = self.KINDS[kind]
        for k, v in params.items():
            setattr(p, k, v)
        arr = (C.c_void_p * len(maps))(*[m.h for m in maps])
        h = C.c_void_p()
        check(_lib.load().mf_operator_create(ctx.h, C.byref(p), arr, len(maps), C.byref(h)))
        self.ctx, self.h, self.maps, self.kind = ctx, h, maps, kind
        n = C.c_int64()
        check(_lib.load().mf_operator_size(h, C.byref(n)))
        self.n = n.value
        self._fields = {}

    def set_field(self, name, tensor):
        """Borrow a CUDA fp64 tensor as a coefficient field (kept alive by the operator)."""
        t = tensor.contiguous()
        self._fields[name] = t
        check(_lib.load().mf_operator_set_field(self.h, self.FIELDS[name], _ptr(t), _dtype_code(t), t.numel()))

    def apply(self, src, dst=None, nrhs=1, transpose=False, arith=None):
        """dst = A src; fp64 tensors may ask for arith="df64" (double-float cell arithmetic), fp32
        tensors for arith="f16" or "bf16" (packed 16-bit arithmetic, pairs of right-hand sides) or,
        on Q3 Helmholtz operators, arith="tc" (the tensor-core kernel)."""
        import torch
        if dst is None:
            dst = torch.empty_like(src)
        code = _dtype_code(src)
        if arith == "tc":
            if code != MF_F32 or transpose:
                raise TypeError("tensor-core applies take fp32 tensors, forward (the operator is symmetric)")
            check(_lib.load().mf_apply_tc(self.h, _ptr(src), _ptr(dst), nrhs, src.numel() // nrhs))
            return dst
        if arith in ("f16", "bf16"):
            if code != MF_F32 or transpose:
                raise TypeError("16-bit arithmetic applies to fp32 tensors, forward only")
            check(_lib.load().mf_apply_packed16(self.h, _ptr(src), _ptr(dst), nrhs, src.numel() // nrhs,
                                                MF_F16 if arith == "f16" else MF_BF16))
            return dst
        if arith == "df64":
            if code != MF_F64:
                raise TypeError("df64 arithmetic applies to fp64 tensors")
            code = _lib.MF_DF64
        fn = _lib.load().mf_apply_transpose if transpose else _lib.load().mf_apply
        check(fn(self.h, _ptr(src), _ptr(dst), nrhs, src.numel() // nrhs, code))
        return dst

    def diagonal(self, dtype=None):
        import torch
        dst = torch.empty(self.n, dtype=dtype or torch.float64, device="cuda")
        check(_lib.load().mf_diagonal(self.h, _ptr(dst), _dtype_code(dst)))
        return dst

    def solve(self, b, x=None, nrhs=1, **kw):
        import torch
        if x is None:
            x = torch.empty_like(b)
        sp = solver_params(**kw)
        info = _lib.SolveInfo()
        st = _lib.load().mf_solve(self.h, C.byref(sp), _ptr(b), _ptr(x), nrhs, C.byref(info))
        if st not in (_lib.MF_OK, _lib.MF_ENOTCONV):
            check(st)
        return x, {"status": st, "iterations": info.iterations, "outer_iterations": info.outer_iterations,
                   "rel_residual": info.rel_residual, "lambda_max": info.lambda_max, "seconds": info.seconds,
                   "inner_steps": info.inner_steps}

    def coupling(self, which, src):
        """Oseen coupling blocks alone: which="grad" gives B^T p (velocity blocks) from a pressure
        vector, which="div" gives B u (pressure block) from the velocity blocks, which="schur"
        gives B D^-1 B^T p (D: the 3 x 3 nodal blocks of A_uu) from a pressure vector."""
        import torch
        nu, npr = self.maps[0].n_dofs, self.maps[1].n_dofs
        w = {"grad": 0, "div": 1, "schur": 2}[which]
        src = src.contiguous()
        dst = torch.empty(3 * nu if w == 0 else npr, dtype=src.dtype, device=src.device)
        check(_lib.load().mf_oseen_coupling(self.h, w, _ptr(src), _ptr(dst), _dtype_code(src)))
        return dst

    def interface_sources(self, T, p_ambient, latent_heat, molar_mass, t_boil, rhocp_liquid, rhocp_gas,
                          mass_flux="knight", sticking=1.0, tanasawa_coef=0.0, gas_constant=8.314,
                          outputs=("u", "p", "T")):
        """Interface source loads of an Oseen operator from the nodal temperature T (fp64 device,
        n_u values): dict with "u" (hybrid recoil force, 3 n_u), "p" (evaporative dilation, n_p),
        "T" (evaporative cooling, n_u) for the requested outputs."""
        import torch
        ev = _lib.Evaporation()
        ev.mass_flux = {"knight": 0, "tanasawa": 1}[mass_flux]
        ev.p_ambient, ev.latent_heat, ev.molar_mass, ev.t_boil = p_ambient, latent_heat, molar_mass, t_boil
        ev.sticking, ev.tanasawa_coef, ev.gas_constant = sticking, tanasawa_coef, gas_constant
        ev.rhocp_liquid, ev.rhocp_gas = rhocp_liquid, rhocp_gas
        nu = self.maps[0].n_dofs
        npr = self.maps[1].n_dofs if len(self.maps) > 1 else 0   # the library rejects non-Oseen operators
        T = T.contiguous()
        out = {}
        for key, size in (("u", 3 * nu), ("p", npr), ("T", nu)):
            if key in outputs:
                out[key] = torch.empty(size, dtype=torch.float64, device=T.device)
        ptr = lambda k: _ptr(out[k]) if k in out else None
        check(_lib.load().mf_interface_sources(self.h, C.byref(ev), _ptr(T), ptr("u"), ptr("p"), ptr("T")))
        return out

    def laser_load(self, power, radius, x0, y0, absorptivity, derivatives=False):
        import torch
        lz = _lib.Laser(power, radius, x0, y0, absorptivity)
        nd = self.maps[0].n_dofs
        f = torch.empty(nd, dtype=torch.float64, device="cuda")
        dF = torch.empty(4 * nd, dtype=torch.float64, device="cuda") if derivatives else None
        check(_lib.load().mf_laser_load(self.h, C.byref(lz), _ptr(f), _ptr(dF)))
        return (f, dF.view(4, nd)) if derivatives else f

    def heat_step_gradient(self, laser, theta_prev, theta_target, box_half, box_depth, with_kq=True, **kw):
        import torch
        lz = _lib.Laser(*laser)
        sp = solver_params(**kw)
        J = C.c_double()
        g = (C.c_double * 4)()
        nd = self.maps[0].n_dofs
        gk = torch.empty(self.maps[0].n_cells * 27, dtype=torch.float64, device="cuda") if with_kq else None
        th = torch.empty(nd, dtype=torch.float64, device="cuda")
        lam = torch.empty(nd, dtype=torch.float64, device="cuda")
        check(_lib.load().mf_heat_step_gradient(self.h, C.byref(lz), C.byref(sp), _ptr(theta_prev),
                                                _ptr(theta_target), box_half, box_depth, C.byref(J), g,
                                                _ptr(gk), _ptr(th), _ptr(lam)))
        return J.value, list(g), gk, th, lam

    def autotune(self, cache_path=None):
        check(_lib.load().mf_autotune(self.h, cache_path.encode() if cache_path else None))

    @property
    def variant(self):
        return _lib.load().mf_operator_variant(self.h).decode()

    def set_variant(self, name, value):
        """Select an apply variant by name in place of the autotuner's choice ("q2_line": 0 or 1)."""
        check(_lib.load().mf_operator_set_variant(self.h, name.encode(), int(value)))

    def __del__(self):
        try:
            if self.h:
                _lib.load().mf_operator_destroy(self.h)
        except Exception:
            pass


class MeltPoolStep:
    """One time step of the melt-pool algorithm (mf_meltpool_create / mf_meltpool_advance) on the
    maps (velocity Q2, pressure Q1, level set Q2 without Dirichlet faces, temperature Q2).
    ``params`` are the fields of mf_meltpool_params; ``evaporation`` a dict of mf_evaporation
    fields (mass_flux "knight" | "tanasawa"), ``laser`` a dict (power, radius, absorptivity, focus,
    direction) or None."""

    TRACE = ("u_star", "T_star", "phi_star", "u_gamma", "b_advection", "phi_advected", "r_heat", "b_flow",
             "T_update")

    def __init__(self, ctx, maps, evaporation, laser=None, gravity=(0.0, 0.0, 0.0), **params):
        p = _lib.MeltPoolParams()
        ev = dict(evaporation)
        ev["mass_flux"] = {"knight": 0, "tanasawa": 1}[ev.get("mass_flux", "knight")]
        for k, v in ev.items():
            setattr(p.evaporation, k, v)
        if p.evaporation.gas_constant == 0:
            p.evaporation.gas_constant = 8.314
        for k, v in params.items():
            setattr(p, k, v)
        p.gravity[:] = list(gravity)
        if laser is not None:
            p.laser_on = 1
            p.laser_power, p.laser_radius = laser["power"], laser["radius"]
            p.laser_absorptivity = laser["absorptivity"]
            p.laser_focus[:] = list(laser["focus"])
            p.laser_direction[:] = list(laser["direction"])
        h = C.c_void_p()
        check(_lib.load().mf_meltpool_create(ctx.h, C.byref(p), *[m.h for m in maps], C.byref(h)))
        self.ctx, self.h, self.maps, self.params = ctx, h, maps, p

    def advance(self, state, trace=False):
        """state: dict of fp64 CUDA tensors u, u_prev (3 n_u), T, T_prev, phi, phi_prev (n_u).
        Returns (dict u (3, n_u), p, T, phi [, trace tensors]), info dict."""
        import torch
        mu, mp = self.maps[0], self.maps[1]
        nu, npr, nc = mu.n_dofs, mp.n_dofs, mu.n_cells
        kw = dict(dtype=torch.float64, device="cuda")
        up = torch.empty(3 * nu + npr, **kw)
        T = torch.empty(nu, **kw)
        phi = torch.empty(nu, **kw)
        tr, trp = {}, None
        if trace:
            sizes = dict(u_star=3 * nu, T_star=nu, phi_star=nu, u_gamma=81 * nc, b_advection=nu,
                         phi_advected=nu, r_heat=nu, b_flow=3 * nu + npr, T_update=nu)
            tr = {k: torch.empty(sizes[k], **kw) for k in self.TRACE}
            trp = _lib.MeltPoolTrace(*[tr[k].data_ptr() for k in self.TRACE])
        inf = _lib.MeltPoolInfo()
        s = {k: state[k].contiguous() for k in ("u_prev", "u", "T_prev", "T", "phi_prev", "phi")}
        st = _lib.load().mf_meltpool_advance(self.h, *[_ptr(s[k]) for k in ("u_prev", "u", "T_prev", "T",
                                                                             "phi_prev", "phi")],
                                             _ptr(up), _ptr(T), _ptr(phi), C.byref(trp) if trp else None,
                                             C.byref(inf))
        if st not in (_lib.MF_OK, _lib.MF_ENOTCONV):
            check(st)
        out = dict(u=up[:3 * nu].view(3, nu), p=up[3 * nu:], T=T, phi=phi, **tr)
        info = {k: getattr(inf, k) for k, _ in _lib.MeltPoolInfo._fields_ if k != "seconds"}
        info["seconds"] = list(inf.seconds)
        info["status"] = st
        return out, info

    def __del__(self):
        try:
            if self.h:
                _lib.load().mf_meltpool_destroy(self.h)
        except Exception:
            pass
