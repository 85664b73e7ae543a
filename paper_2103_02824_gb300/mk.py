"""Python binding of the mk C ABI (include/mk.h): argument marshalling only.

Every function here forwards to the CUDA library libmk.so; device arrays are torch CUDA tensors (float64, C
contiguous), host arrays numpy.  If the library has not been built, importing this module raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmk.so")

MK_OK = 0
MK_ERR_INVALID_ARG = -1
MK_ERR_CUDA = -2
MK_ERR_OOM = -3
MK_ERR_NOT_CONVERGED = -4
MK_ERR_BREAKDOWN = -5
MK_ERR_TIMEOUT = -6
MK_ERR_SINGULAR_AUG = -7
MK_ERR_UNSUPPORTED = -8
MK_MAX_RHS = 64
MK_FAULT_PATCH_WAIT, MK_FAULT_PATCH_RECORD, MK_FAULT_TC_WAIT = 1, 2, 4

MK_XC = {"none": 0, "slater": 1, "xalpha": 2, "lda": 3}
MK_PREC_FP64, MK_PREC_MIXED, MK_PREC_PAIRS = 0, 1, 2
MK_PRECOND = {"jacobi": 0, "chebyshev": 1, "learned": 2}
MK_BC = {"zero": 0, "multipole": 1}


class MkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mk error {code}: {msg}")
        self.code = code


class mk_mesh_desc(C.Structure):
    _fields_ = [("order", C.c_int), ("n_vertices", C.c_int64), ("coords", C.POINTER(C.c_double)),
                ("n_elems", C.c_int64), ("tets", C.POINTER(C.c_int32))]


class mk_molecule(C.Structure):
    _fields_ = [("n_nuclei", C.c_int), ("Z", C.POINTER(C.c_double)), ("R", C.POINTER(C.c_double))]


class mk_xc(C.Structure):
    _fields_ = [("kind", C.c_int), ("alpha", C.c_double)]


class mk_solve_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("precond", C.c_int), ("rtol", C.c_double), ("maxit", C.c_int),
                ("inner_rtol", C.c_double), ("max_refine", C.c_int), ("check_every", C.c_int),
                ("mlp", C.c_void_p), ("mlp_precision", C.c_int), ("trace_every", C.c_int), ("trace_cap", C.c_int),
                ("trace_x", C.c_void_p), ("trace_r", C.c_void_p), ("coarse", C.c_int)]


class mk_solve_report(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("refinements", C.c_int), ("n_rhs", C.c_int),
                ("max_rel_residual", C.c_double), ("iters", C.c_int * MK_MAX_RHS),
                ("rel_residual", C.c_double * MK_MAX_RHS), ("n_traced", C.c_int)]

    def to_dict(self):
        n = self.n_rhs
        return dict(status=self.status, iterations=self.iterations, refinements=self.refinements, n_rhs=n,
                    max_rel_residual=self.max_rel_residual, iters=list(self.iters[:n]),
                    rel_residual=list(self.rel_residual[:n]), n_traced=self.n_traced)


class mk_adam(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double)]


class mk_mesh_info(C.Structure):
    _fields_ = [("order", C.c_int), ("nloc", C.c_int), ("n_nodes", C.c_int64), ("n_free", C.c_int64),
                ("n_elems", C.c_int64), ("n_colours", C.c_int64), ("n_nodes_coarse", C.c_int64),
                ("n_free_coarse", C.c_int64), ("n_elems_coarse", C.c_int64), ("n_quad", C.c_int)]


_vp = C.c_void_p
_SIGS = {
    "mk_ctx_create": [C.POINTER(_vp), C.c_int],
    "mk_ctx_destroy": [_vp],
    "mk_last_error": [C.c_char_p, C.c_size_t],
    "mk_ctx_fault": [_vp, C.POINTER(C.c_int)],
    "mk_version": [],
    "mk_launch_count": [],
    "mk_profile_enable": [_vp, C.c_int],
    "mk_profile_read": [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong)],
    "mk_mesh_upload": [_vp, C.POINTER(mk_mesh_desc), C.POINTER(mk_mesh_desc), C.POINTER(C.c_int32), C.POINTER(_vp)],
    "mk_mesh_destroy": [_vp],
    "mk_mesh_get_info": [_vp, C.POINTER(mk_mesh_info)],
    "mk_mesh_get_topology": [_vp, C.c_int, _vp, _vp, _vp, _vp],
    "mk_prolongate": [_vp, _vp, _vp, C.c_int, C.c_int, _vp, C.c_int, _vp],
    "mk_density": [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_double), C.c_int, _vp, _vp],
    "mk_hartree_poisson": [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_double), C.c_int, _vp, C.c_int, _vp,
                           C.POINTER(mk_solve_opts), C.POINTER(mk_solve_report), _vp],
    "mk_assemble_rhs": [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int, _vp,
                        C.c_double, mk_xc, _vp, _vp, _vp],
    "mk_correction_solve": [_vp, _vp, C.POINTER(mk_molecule), C.c_double, _vp, _vp, C.c_int, C.c_int,
                            C.POINTER(mk_solve_opts), C.POINTER(mk_solve_report), _vp],
    "mk_augmented_project": [_vp, _vp, C.POINTER(mk_molecule), _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp,
                             _vp, _vp, _vp, _vp],
    "mk_small_eigensolve": [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "mk_coarse_pencil": [_vp, _vp, C.POINTER(mk_molecule), _vp, _vp, _vp, _vp],
    "mk_operator_apply": [_vp, _vp, C.POINTER(mk_molecule), C.c_double, C.c_int, _vp, _vp, C.c_int, _vp],
    "mk_coarse_decompose": [_vp, _vp, _vp, _vp, _vp, _vp],
    "mk_decompose_info": [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)],
    "mk_coarse_decompose_warm": [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp],
    "mk_small_eigensolve_shared": [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "mk_small_eigensolve_static": [C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "mk_orbital_assemble": [_vp, _vp, _vp, _vp, _vp, C.c_int, C.c_int, _vp, _vp],
    "mk_lowest_ritz": [_vp, _vp, C.POINTER(mk_molecule), C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double), _vp],
    "mk_correction_shift": [_vp, _vp, C.POINTER(mk_molecule), C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double),
                            C.POINTER(C.c_double), _vp],
    "mk_ctx_set_option": [_vp, C.c_int, C.c_int],
    "mk_mesh_set_hierarchy": [_vp, C.c_int, C.POINTER(mk_mesh_desc), C.POINTER(C.POINTER(C.c_int32))],
    "mk_joint_ritz": [_vp, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(C.c_int),
                      _vp],
    "mk_joint_assemble": [_vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp, C.c_int, _vp, _vp],
    "mk_batch_correction_solve": [_vp, C.c_int, C.POINTER(_vp), C.POINTER(mk_molecule), C.POINTER(C.c_double),
                                  C.POINTER(_vp), C.POINTER(_vp), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(mk_solve_opts), C.POINTER(mk_solve_report), _vp],
    "mk_mesh_set_patch_elems": [_vp, C.c_int],
    "mk_autotune_patches": [_vp, _vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "mk_frozen_potential": [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_double), C.c_int, _vp, _vp, mk_xc, _vp, _vp],
    "mk_assemble_rhs_from_vq": [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_double), C.c_int, _vp, C.c_double, _vp, _vp],
    "mk_correction_solve_vq": [_vp, _vp, C.POINTER(mk_molecule), _vp, C.c_double, _vp, _vp, C.c_int, C.c_int,
                               C.POINTER(mk_solve_opts), C.POINTER(mk_solve_report), _vp],
    "mk_inner_create": [_vp, _vp, C.POINTER(mk_molecule), _vp, C.c_int, C.c_int, _vp, _vp, C.POINTER(_vp), _vp],
    "mk_inner_run": [_vp, _vp, C.POINTER(C.c_double), C.c_double, C.c_int, C.c_double, _vp, _vp, _vp, _vp,
                     C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_double), _vp],
    "mk_inner_potential": [_vp, _vp, _vp, _vp],
    "mk_inner_info": [_vp, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "mk_inner_destroy": [_vp],
    "mk_error_indicators": [_vp, _vp, C.POINTER(mk_molecule), _vp, C.c_int, C.c_int, C.POINTER(C.c_double), _vp,
                            _vp, _vp],
    "mk_dorfler_mark": [_vp, C.c_int64, _vp, C.c_double, _vp, C.POINTER(C.c_int64), C.POINTER(C.c_double), _vp],
    "mk_refine": [_vp, C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, _vp, C.c_int64, C.c_int64, C.POINTER(C.c_int64),
                  C.POINTER(C.c_int64), C.POINTER(C.c_int), _vp],
    "mk_mlp_param_count": [C.c_int],
    "mk_mlp_create": [_vp, C.c_int, C.POINTER(C.c_float), C.POINTER(_vp)],
    "mk_mlp_destroy": [_vp],
    "mk_mlp_save": [_vp, C.POINTER(C.c_float)],
    "mk_mlp_load": [_vp, C.POINTER(C.c_float)],
    "mk_mlp_forward": [_vp, _vp, _vp, C.c_int64, _vp, C.c_int, _vp],
    "mk_mlp_train_step": [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int64, C.POINTER(mk_adam), C.POINTER(C.c_double), _vp,
                          _vp],
    "mk_mlp_harvest": [_vp, _vp, _vp, _vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp],
    "mk_learned_precond": [_vp, _vp, _vp, C.POINTER(mk_molecule), C.c_double, _vp, _vp, C.c_int, C.c_int, C.c_int,
                           _vp],
}


def header_symbols():
    """Names of the entry points declared in include/mk.h (parsed from the header)."""
    import re
    hdr = open(os.path.join(os.path.dirname(_HERE), "include", "mk.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|long long|const char\*)\s+(mk_\w+)\s*\(", hdr, re.M)))


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libmk.so not built at {path}: run `python -m paper_2103_02824_gb300.build`")
    lib = C.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = {"mk_version": C.c_char_p, "mk_launch_count": C.c_longlong,
                     "mk_mlp_param_count": C.c_int64}.get(name, C.c_int)
    return lib


def launch_count() -> int:
    return int(lib().mk_launch_count())


def ctx_fault(ctx) -> int:
    """The context's device fault word (0 = none; MK_FAULT_* bits), read after waiting for the device, then
    cleared."""
    f = C.c_int()
    _check(lib().mk_ctx_fault(ctx.h, C.byref(f)))
    return int(f.value)


PROF_APPLY64, PROF_APPLY32, PROF_HALO, PROF_LEARNED, PROF_STIFF, PROF_PAIRS = 0, 1, 2, 3, 4, 5
MK_OPT_GRAPHS, MK_OPT_PATCH_PIPELINE, MK_OPT_WAIT_LIMIT, MK_OPT_DECOMPOSE_CTAS, MK_OPT_PAIR_RESIDUAL = 1, 2, 3, 4, 5


def ctx_set_option(ctx, option, value):
    _check(lib().mk_ctx_set_option(ctx.h, option, int(value)))


def profile_enable(ctx, on=True):
    _check(lib().mk_profile_enable(ctx.h, 1 if on else 0))


def profile_read(ctx, kind):
    """(total_ms, count) of the operator applications timed since profile_enable."""
    t, n = C.c_double(), C.c_longlong()
    _check(lib().mk_profile_read(ctx.h, kind, C.byref(t), C.byref(n)))
    return t.value, n.value


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _err():
    buf = C.create_string_buffer(2048)
    lib().mk_last_error(buf, 2048)
    return buf.value.decode(errors="replace")


def _check(code, allow=()):
    if code != MK_OK and code not in allow:
        raise MkError(code, _err())
    return code


def _ptr(t):
    """Device pointer of a torch tensor (must be contiguous float64/int32 on CUDA) or None."""
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream)


def _host_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


class Molecule:
    def __init__(self, Z, R):
        self.Z, zp = _host_f64(np.asarray(Z).ravel())
        self.R, rp = _host_f64(np.asarray(R).reshape(-1, 3))
        self.c = mk_molecule(len(self.Z), zp, rp)


MK_MLP_FP32, MK_MLP_BF16 = 0, 1


def opts(precision="fp64", precond="jacobi", rtol=1e-8, maxit=20000, inner_rtol=1e-4, max_refine=20, check_every=10,
         mlp=None, mlp_precision="bf16", trace=None, coarse=False):
    """Solver options.  mlp: an Mlp (precond='learned'); trace: (every, x_buf, r_buf) device float64 tensors of
    shape [cap, n_nodes, ld] receiving iterates and residuals of the FP64 PCG; coarse: add the two-level coarse
    correction (mixed precision)."""
    o = mk_solve_opts(MK_PREC_MIXED if precision == "mixed" else MK_PREC_FP64, MK_PRECOND[precond], rtol, maxit,
                      inner_rtol, max_refine, check_every)
    o.coarse = 2 if coarse in (2, "multigrid") else (1 if coarse else 0)
    if mlp is not None:
        o.mlp = mlp.h.value
        o.mlp_precision = MK_MLP_BF16 if mlp_precision == "bf16" else MK_MLP_FP32
    if trace is not None:
        every, xb, rb = trace
        o.trace_every, o.trace_cap = int(every), int(xb.shape[0])
        o.trace_x, o.trace_r = _ptr(xb).value, _ptr(rb).value
        o._keep = (xb, rb)
    return o


class Mlp:
    """The learned preconditioner's network (device-resident FP32 weights, Adam state, BF16 copy)."""

    def __init__(self, ctx, nloc, params):
        self.ctx, self.nloc = ctx, nloc
        self.count = int(lib().mk_mlp_param_count(nloc))
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        assert p.size == self.count, (p.size, self.count)
        self.h = _vp()
        _check(lib().mk_mlp_create(ctx.h, nloc, p.ctypes.data_as(C.POINTER(C.c_float)), C.byref(self.h)))

    def save(self):
        out = np.zeros(self.count, dtype=np.float32)
        _check(lib().mk_mlp_save(self.h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def load(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        assert p.size == self.count
        _check(lib().mk_mlp_load(self.h, p.ctypes.data_as(C.POINTER(C.c_float))))

    def close(self):
        if self.h:
            lib().mk_mlp_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mk_mlp_forward(ctx, mlp: Mlp, X, Y, precision="fp32", stream=None):
    _check(lib().mk_mlp_forward(ctx.h, mlp.h, _ptr(X), X.shape[0], _ptr(Y),
                                MK_MLP_BF16 if precision == "bf16" else MK_MLP_FP32, _stream(stream)))


def mk_mlp_train_step(ctx, mlp: Mlp, X, U, E, idx=None, S=None, lr=0.0, beta1=0.9, beta2=0.999, eps=1e-8, grad=None,
                      stream=None):
    """Loss (before the update) of one training step; Adam update when lr > 0."""
    S = int(S if S is not None else (idx.shape[0] if idx is not None else X.shape[0]))
    loss = C.c_double()
    a = mk_adam(lr, beta1, beta2, eps)
    _check(lib().mk_mlp_train_step(ctx.h, mlp.h, _ptr(X), _ptr(U), _ptr(E), _ptr(idx), S, C.byref(a),
                                   C.byref(loss), _ptr(grad), _stream(stream)))
    return loss.value


def mk_mlp_harvest(ctx, mesh, Rk, Xk, Xstar, N, X, U, E, stream=None):
    ld = Rk.shape[1] if Rk.dim() == 2 else 1
    _check(lib().mk_mlp_harvest(ctx.h, mesh.h, _ptr(Rk), _ptr(Xk), _ptr(Xstar), ld, N, _ptr(X), _ptr(U), _ptr(E),
                                _stream(stream)))


def mk_learned_precond(ctx, mesh, mlp: Mlp, mol: Molecule, sigma, r, z, N, precision="bf16", stream=None):
    ld = r.shape[1] if r.dim() == 2 else 1
    _check(lib().mk_learned_precond(ctx.h, mesh.h, mlp.h, C.byref(mol.c), float(sigma), _ptr(r), _ptr(z), ld, N,
                                    MK_MLP_BF16 if precision == "bf16" else MK_MLP_FP32, _stream(stream)))


class Context:
    def __init__(self, device: int = 0):
        self.h = C.c_void_p()
        _check(lib().mk_ctx_create(C.byref(self.h), device))

    def close(self):
        if self.h:
            lib().mk_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx: Context, fine_coords, fine_tets, coarse_coords, coarse_tets, parent, order: int):
        self.ctx = ctx
        keep = []

        def desc(coords, tets):
            c, cp = _host_f64(coords)
            t = np.ascontiguousarray(tets, dtype=np.int32)
            keep.extend([c, t])
            return mk_mesh_desc(order, c.shape[0], cp, t.shape[0], t.ctypes.data_as(C.POINTER(C.c_int32)))

        f = desc(fine_coords, fine_tets)
        cdesc = desc(coarse_coords, coarse_tets)
        par = np.ascontiguousarray(parent, dtype=np.int32)
        self.h = C.c_void_p()
        _check(lib().mk_mesh_upload(ctx.h, C.byref(f), C.byref(cdesc), par.ctypes.data_as(C.POINTER(C.c_int32)),
                                    C.byref(self.h)))
        info = mk_mesh_info()
        _check(lib().mk_mesh_get_info(self.h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in mk_mesh_info._fields_}

    def topology(self, level: int = 0):
        n = self.info["n_nodes"] if level == 0 else self.info["n_nodes_coarse"]
        E = self.info["n_elems"] if level == 0 else self.info["n_elems_coarse"]
        nodes = np.zeros((n, 3))
        bnd = np.zeros(n, dtype=np.uint8)
        elem = np.zeros((E, self.info["nloc"]), dtype=np.int32)
        col = np.zeros(E, dtype=np.int32)
        _check(lib().mk_mesh_get_topology(self.h, level, nodes.ctypes.data, bnd.ctypes.data, elem.ctypes.data,
                                          col.ctypes.data))
        return nodes, bnd.astype(bool), elem, col

    def set_hierarchy(self, meshes, parents):
        """Intermediate levels (coarsest first) of the multigrid hierarchy: meshes [(coords, tets)], parents as
        synth.cube_hierarchy returns them."""
        keep = []
        descs = (mk_mesh_desc * max(len(meshes), 1))()
        for k, (c, t) in enumerate(meshes):
            c, cp = _host_f64(c)
            t = np.ascontiguousarray(t, dtype=np.int32)
            keep.extend([c, t])
            descs[k] = mk_mesh_desc(self.info["order"], c.shape[0], cp, t.shape[0],
                                    t.ctypes.data_as(C.POINTER(C.c_int32)))
        pars = (C.POINTER(C.c_int32) * max(len(parents), 1))()
        for k, p in enumerate(parents):
            p = np.ascontiguousarray(p, dtype=np.int32)
            keep.append(p)
            pars[k] = p.ctypes.data_as(C.POINTER(C.c_int32))
        _check(lib().mk_mesh_set_hierarchy(self.h, len(meshes), descs, pars))

    def close(self):
        if self.h:
            lib().mk_mesh_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mk_prolongate(ctx, mesh, psiH, N, u, stream=None):
    ldc = psiH.shape[1] if psiH.dim() == 2 else 1
    ld = u.shape[1] if u.dim() == 2 else 1
    _check(lib().mk_prolongate(ctx.h, mesh.h, _ptr(psiH), ldc, N, _ptr(u), ld, _stream(stream)))


def mk_density(ctx, mesh, u, occ, N, rho_q, stream=None):
    """rho_H at the quadrature points [n_elems, n_quad] (float64 device tensor rho_q)."""
    ld = u.shape[1] if u.dim() == 2 else 1
    occ_h, occ_p = _host_f64(occ)
    _check(lib().mk_density(ctx.h, mesh.h, _ptr(u), ld, occ_p, N, _ptr(rho_q), _stream(stream)))


def mk_hartree_poisson(ctx, mesh, u, occ, N, w, bc="multipole", opt=None, stream=None, rho_q=None):
    ld = u.shape[1] if u.dim() == 2 else 1
    occ_h, occ_p = _host_f64(occ)
    rep = mk_solve_report()
    o = opt or opts(rtol=1e-12)
    code = lib().mk_hartree_poisson(ctx.h, mesh.h, _ptr(u), ld, occ_p, N, None if rho_q is None else _ptr(rho_q),
                                    MK_BC[bc], _ptr(w), C.byref(o), C.byref(rep), _stream(stream))
    _check(code)
    return rep.to_dict()


def mk_assemble_rhs(ctx, mesh, u, lamH, occ, N, w, sigma, xc, rhs, vq, alpha=0.77298, stream=None):
    ld = u.shape[1] if u.dim() == 2 else 1
    lam_h, lam_p = _host_f64(lamH)
    occ_h, occ_p = _host_f64(occ)
    _check(lib().mk_assemble_rhs(ctx.h, mesh.h, _ptr(u), ld, lam_p, occ_p, N, _ptr(w), float(sigma),
                                 mk_xc(MK_XC[xc], alpha), _ptr(rhs), _ptr(vq), _stream(stream)))


def mk_frozen_potential(ctx, mesh, u, occ, N, w, xc, vq, alpha=0.77298, stream=None, rho_q=None):
    ld = u.shape[1] if u.dim() == 2 else 1
    occ_h, occ_p = _host_f64(occ)
    _check(lib().mk_frozen_potential(ctx.h, mesh.h, _ptr(u), ld, occ_p, N, None if rho_q is None else _ptr(rho_q),
                                     _ptr(w), mk_xc(MK_XC[xc], alpha), _ptr(vq), _stream(stream)))


def mk_assemble_rhs_from_vq(ctx, mesh, u, lamH, N, vq, sigma, rhs, stream=None):
    ld = u.shape[1] if u.dim() == 2 else 1
    lam_h, lam_p = _host_f64(lamH)
    _check(lib().mk_assemble_rhs_from_vq(ctx.h, mesh.h, _ptr(u), ld, lam_p, N, _ptr(vq), float(sigma), _ptr(rhs),
                                         _stream(stream)))


def mk_correction_solve(ctx, mesh, mol: Molecule, sigma, rhs, x, N, opt=None, stream=None, allow=()):
    ld = x.shape[1] if x.dim() == 2 else 1
    rep = mk_solve_report()
    o = opt or opts()
    code = lib().mk_correction_solve(ctx.h, mesh.h, C.byref(mol.c), float(sigma), _ptr(rhs), _ptr(x), ld, N,
                                     C.byref(o), C.byref(rep), _stream(stream))
    _check(code, allow)
    d = rep.to_dict()
    d["code"] = code
    return d


def mk_correction_solve_vq(ctx, mesh, mol: Molecule, vq, sigma, rhs, x, N, opt=None, stream=None, allow=()):
    """The paper's form of the correction solve: (K/2 + M_Vext + M_vq + sigma M) x = rhs."""
    ld = x.shape[1] if x.dim() == 2 else 1
    rep = mk_solve_report()
    o = opt or opts()
    code = lib().mk_correction_solve_vq(ctx.h, mesh.h, C.byref(mol.c), _ptr(vq), float(sigma), _ptr(rhs), _ptr(x),
                                        ld, N, C.byref(o), C.byref(rep), _stream(stream))
    _check(code, allow)
    d = rep.to_dict()
    d["code"] = code
    return d


class Inner:
    """Handle of the inner SCF iteration (Algorithm 2 with Algorithm 3's precomputations; see include/mk.h):
    created from the corrections phit [n_nodes, ld], their Hartree potential wt [n_nodes] and V_xc at the
    quadrature points vxc_q [n_elems, n_quad] (all device float64)."""

    def __init__(self, ctx, mesh, mol: Molecule, phit, N, wt, vxc_q, stream=None):
        self.ctx, self.mesh, self.N = ctx, mesh, N
        self.NH = mesh.info["n_free_coarse"]
        ld = phit.shape[1] if phit.dim() == 2 else 1
        h = _vp()
        _check(lib().mk_inner_create(ctx.h, mesh.h, C.byref(mol.c), _ptr(phit), ld, N, _ptr(wt), _ptr(vxc_q),
                                     C.byref(h), _stream(stream)))
        self.h = h
        wv, sc = C.c_int(), C.c_double()
        _check(lib().mk_inner_info(self.h, C.byref(wv), C.byref(sc)))
        self.w_in_VH, self.schur = bool(wv.value), sc.value

    def run(self, occ, lam, coef, status=None, wH=None, tol=1e-10, max_inner=200, mix=0.5, stream=None):
        """Returns dict(theta1, iters, delta); lam [N], coef [(N_H+1), N], status [N] int32, wH [N_H] device."""
        occ_h, occ_p = _host_f64(occ)
        th, it, dl = C.c_double(), C.c_int(), C.c_double()
        _check(lib().mk_inner_run(self.ctx.h, self.h, occ_p, float(tol), int(max_inner), float(mix), _ptr(lam),
                                  _ptr(coef), _ptr(status), _ptr(wH), C.byref(th), C.byref(it), C.byref(dl),
                                  _stream(stream)))
        return dict(theta1=th.value, iters=it.value, delta=dl.value)

    def potential(self, w, stream=None):
        _check(lib().mk_inner_potential(self.ctx.h, self.h, _ptr(w), _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().mk_inner_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mk_error_indicators(ctx, mesh, mol: Molecule, psi, N, lam, vq, eta2, stream=None):
    """eta2 [n_elems] device: the residual a posteriori indicator of (lam, psi) with vq = w + V_xc at the points."""
    ld = psi.shape[1] if psi.dim() == 2 else 1
    lam_h, lam_p = _host_f64(lam)
    _check(lib().mk_error_indicators(ctx.h, mesh.h, C.byref(mol.c), _ptr(psi), ld, N, lam_p, _ptr(vq), _ptr(eta2),
                                     _stream(stream)))


def mk_dorfler_mark(ctx, eta2, theta, marked, stream=None):
    """marked [n] device uint8; returns (n_marked, threshold)."""
    nm, th = C.c_int64(), C.c_double()
    _check(lib().mk_dorfler_mark(ctx.h, int(eta2.numel()), _ptr(eta2), float(theta), _ptr(marked), C.byref(nm),
                                 C.byref(th), _stream(stream)))
    return nm.value, th.value


def mk_refine(ctx, coords, tets, tags, parent, marked, n_vertices, n_elems, stream=None):
    """Newest-vertex bisection of the marked elements with closure, in place in the device buffers coords
    [max_v, 3] float64, tets [max_e, 4] int32, tags [max_e] int8, parent [max_e] int32 (marked [n_elems] uint8);
    returns (n_vertices, n_elems, rounds)."""
    nv, ne, r = C.c_int64(), C.c_int64(), C.c_int()
    _check(lib().mk_refine(ctx.h, int(n_vertices), int(n_elems), _ptr(coords), _ptr(tets), _ptr(tags), _ptr(parent),
                           _ptr(marked), int(coords.shape[0]), int(tets.shape[0]), C.byref(nv), C.byref(ne),
                           C.byref(r), _stream(stream)))
    return nv.value, ne.value, r.value


def refine_mesh(ctx, X, T, K, marked, max_vertices=None, max_elems=None):
    """Host arrays in and out around mk_refine (X [nv, 3], T [E, 4] in bisection order, K [E], marked [E] bool):
    returns (X', T', K', parent, rounds)."""
    import torch
    nv, E = X.shape[0], T.shape[0]
    max_v = max_vertices or 4 * nv + 1024
    max_e = max_elems or 8 * E + 1024
    dev = torch.device("cuda")
    Xd = torch.zeros((max_v, 3), dtype=torch.float64, device=dev)
    Xd[:nv] = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).to(dev)
    Td = torch.zeros((max_e, 4), dtype=torch.int32, device=dev)
    Td[:E] = torch.from_numpy(np.ascontiguousarray(T, dtype=np.int32)).to(dev)
    Kd = torch.zeros(max_e, dtype=torch.int8, device=dev)
    Kd[:E] = torch.from_numpy(np.ascontiguousarray(K, dtype=np.int8)).to(dev)
    Pd = torch.zeros(max_e, dtype=torch.int32, device=dev)
    Md = torch.from_numpy(np.ascontiguousarray(marked, dtype=np.uint8)).to(dev)
    nv2, E2, r = mk_refine(ctx, Xd, Td, Kd, Pd, Md, nv, E)
    torch.cuda.synchronize()
    return (Xd[:nv2].cpu().numpy(), Td[:E2].cpu().numpy(), Kd[:E2].cpu().numpy(), Pd[:E2].cpu().numpy(), r)


def mk_batch_correction_solve(ctx, meshes, mols, sigmas, rhs_list, x_list, Ns, opt=None, stream=None, allow=()):
    """Correction solves of K molecules in shared launches (see include/mk.h); returns K report dicts."""
    K = len(meshes)
    mh = (_vp * K)(*[m.h.value for m in meshes])
    ml = (mk_molecule * K)(*[mo.c for mo in mols])
    sg = (C.c_double * K)(*[float(v) for v in sigmas])
    rp = (_vp * K)(*[_ptr(r).value for r in rhs_list])
    xp = (_vp * K)(*[_ptr(x).value for x in x_list])
    lds = (C.c_int * K)(*[int(x.shape[1]) for x in x_list])
    ns = (C.c_int * K)(*[int(n) for n in Ns])
    reps = (mk_solve_report * K)()
    o = opt or opts(precision="mixed")
    code = lib().mk_batch_correction_solve(ctx.h, K, mh, ml, sg, rp, xp, lds, ns, C.byref(o), reps, _stream(stream))
    _check(code, allow)
    out = [r.to_dict() for r in reps]
    for d in out:
        d["code"] = code
    return out


def mk_mesh_set_patch_elems(mesh, pe):
    _check(lib().mk_mesh_set_patch_elems(mesh.h, int(pe)))


def mk_autotune_patches(ctx, mesh, ld):
    """(best elements per patch, [ms per application of each candidate])"""
    best = C.c_int()
    ms = (C.c_double * 4)()
    _check(lib().mk_autotune_patches(ctx.h, mesh.h, int(ld), C.byref(best), ms))
    return best.value, list(ms)


def mk_augmented_project(ctx, mesh, mol: Molecule, vq, psihat, N, AH, MH, b, c, beta, gamma, gramA=None, gramM=None,
                         stream=None):
    ld = psihat.shape[1] if psihat.dim() == 2 else 1
    _check(lib().mk_augmented_project(ctx.h, mesh.h, C.byref(mol.c), _ptr(vq), _ptr(psihat), ld, N, _ptr(AH),
                                      _ptr(MH), _ptr(b), _ptr(c), _ptr(beta), _ptr(gamma), _ptr(gramA), _ptr(gramM),
                                      _stream(stream)))


def mk_small_eigensolve(ctx, NH, N, AH, MH, b, c, beta, gamma, lam, coef, status, stream=None):
    _check(lib().mk_small_eigensolve(ctx.h, NH, N, _ptr(AH), _ptr(MH), _ptr(b), _ptr(c), _ptr(beta), _ptr(gamma),
                                     _ptr(lam), _ptr(coef), _ptr(status), _stream(stream)))


def mk_operator_apply(ctx, mesh, mol: Molecule, sigma, x, y, stream=None, pairs=False):
    """y = (K/2 + M_Vext + sigma M) x, or y = K x (the Poisson operator) with mol None and sigma 0; float32 tensors
    select the FP32 operator, float64 the FP64 one (pairs=True: FP64 operands, products on FP32 pairs)."""
    import torch
    prec = MK_PREC_MIXED if x.dtype == torch.float32 else (MK_PREC_PAIRS if pairs else MK_PREC_FP64)
    assert y.dtype == x.dtype
    ld = x.shape[1] if x.dim() == 2 else 1
    _check(lib().mk_operator_apply(ctx.h, mesh.h, None if mol is None else C.byref(mol.c), float(sigma), prec,
                                   _ptr(x), _ptr(y), ld, _stream(stream)))


def mk_coarse_pencil(ctx, mesh, mol: Molecule, vq, AH, MH, stream=None):
    _check(lib().mk_coarse_pencil(ctx.h, mesh.h, C.byref(mol.c), _ptr(vq), _ptr(AH), _ptr(MH), _stream(stream)))


def mk_coarse_decompose(ctx, mesh, AH, d, V, stream=None):
    _check(lib().mk_coarse_decompose(ctx.h, mesh.h, _ptr(AH), _ptr(d), _ptr(V), _stream(stream)))


def mk_decompose_info(ctx):
    """Sweeps of the FP32 and FP64 phases of the context's most recent decomposition (synchronises)."""
    s32, s64 = C.c_int(0), C.c_int(0)
    _check(lib().mk_decompose_info(ctx.h, C.byref(s32), C.byref(s64)))
    return {"sweeps32": s32.value, "sweeps64": s64.value}


def mk_coarse_decompose_warm(ctx, NH, AH, V0, d, V, stream=None):
    _check(lib().mk_coarse_decompose_warm(ctx.h, NH, _ptr(AH), _ptr(V0), _ptr(d), _ptr(V), _stream(stream)))


def mk_small_eigensolve_shared(ctx, NH, N, d, V, b, c, beta, gamma, lam, coef, status, stream=None):
    _check(lib().mk_small_eigensolve_shared(ctx.h, NH, N, _ptr(d), _ptr(V), _ptr(b), _ptr(c), _ptr(beta),
                                            _ptr(gamma), _ptr(lam), _ptr(coef), _ptr(status), _stream(stream)))


def mk_small_eigensolve_static(NH, N, d, V, b, c, beta, gamma, lam, coef, status, stream=None):
    """Allocation-free variant (fixed library workspace; N_H <= 512, N <= 16); returns the status code."""
    return lib().mk_small_eigensolve_static(NH, N, _ptr(d), _ptr(V), _ptr(b), _ptr(c), _ptr(beta), _ptr(gamma),
                                            _ptr(lam), _ptr(coef), _ptr(status), _stream(stream))


def mk_joint_ritz(ctx, NH, N, k, d, V, b, c, gramA, gramM, lam, X, stream=None):
    """Lowest k Ritz pairs of the joint augmented space; returns the number of correction directions kept."""
    kept = C.c_int()
    _check(lib().mk_joint_ritz(ctx.h, NH, N, k, _ptr(d), _ptr(V), _ptr(b), _ptr(c), _ptr(gramA), _ptr(gramM),
                               _ptr(lam), _ptr(X), C.byref(kept), _stream(stream)))
    return kept.value


def mk_joint_assemble(ctx, mesh, k, N, X, psihat, u, psi, stream=None):
    ld = psihat.shape[1] if psihat.dim() == 2 else 1
    _check(lib().mk_joint_assemble(ctx.h, mesh.h, k, N, _ptr(X), _ptr(psihat), _ptr(u), ld, _ptr(psi),
                                   _stream(stream)))


def mk_orbital_assemble(ctx, mesh, coef, psihat, u, N, psi, stream=None):
    ld = psihat.shape[1] if psihat.dim() == 2 else 1
    _check(lib().mk_orbital_assemble(ctx.h, mesh.h, _ptr(coef), _ptr(psihat), _ptr(u), ld, N, _ptr(psi),
                                     _stream(stream)))


def mk_lowest_ritz(ctx, mesh, mol: Molecule, v0, steps=60, stream=None):
    v, vp = _host_f64(v0)
    th = C.c_double()
    _check(lib().mk_lowest_ritz(ctx.h, mesh.h, C.byref(mol.c), vp, steps, C.byref(th), _stream(stream)))
    return th.value


def mk_correction_shift(ctx, mesh, mol: Molecule, v0, steps=60, stream=None):
    """(theta, sigma): the lowest Ritz value and the shift the library derives from it."""
    v, vp = _host_f64(v0)
    th, sg = C.c_double(), C.c_double()
    _check(lib().mk_correction_shift(ctx.h, mesh.h, C.byref(mol.c), vp, steps, C.byref(th), C.byref(sg),
                                     _stream(stream)))
    return th.value, sg.value
