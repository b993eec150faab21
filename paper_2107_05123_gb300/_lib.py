"""ctypes binding of the C ABI in include/chns.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but convert
arguments (numpy host arrays, torch device tensors or raw integer pointers) and raise ChnsError
on a non-zero status. All computation happens in libchns.so. Importing this module fails loudly
when the compiled library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchns.so")

MAXD = 20
GMRES_MAX_RESTART = 40

# chns_status
OK, EINVAL, EUNBALANCED, ENOMEM, ECUDA, ENOTCONV, EBREAKDOWN, ENAN = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "EUNBALANCED", 3: "ENOMEM", 4: "ECUDA", 5: "ENOTCONV",
                6: "EBREAKDOWN", 7: "ENAN"}
# chns_precision
FP64, FP32, FP32_BF16COEF, FP64_DF = 0, 1, 2, 3
# chns_operator
OP_POISSON, OP_MASS, OP_CH, OP_MOMENTUM = 0, 1, 2, 3
OP_NCOMP = {OP_POISSON: 1, OP_MASS: 3, OP_CH: 2, OP_MOMENTUM: 3}
# chns_ksp / chns_pc
KSP_CG, KSP_GMRES, KSP_FCG = 0, 1, 2
APPLY_AUTO, APPLY_PATCH, APPLY_STREAM = 0, 1, 2
PC_NONE, PC_JACOBI, PC_LEARNED, PC_CHEBYSHEV, PC_SCHUR, PC_MULTIGRID = 0, 1, 2, 3, 4, 5
# chns_mg_operator
MG_POISSON, MG_SHIFTED = 0, 1


class ChnsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class chns_mesh_info(C.Structure):
    _fields_ = [("n_elem", C.c_int64), ("n_nodes", C.c_int64), ("n_hanging", C.c_int64),
                ("n_boundary", C.c_int64), ("min_level", C.c_int32), ("max_level", C.c_int32),
                ("extent", C.c_double * 3)]


class chns_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("Re", "We", "Cn", "Pe", "Fr", "rho_ratio", "eta_ratio", "dt", "C_I")]


class chns_coef(C.Structure):
    _fields_ = [("phi_tilde", C.c_void_p), ("u_adv", C.c_void_p * 3), ("mu_tilde", C.c_void_p)]


class chns_solver_params(C.Structure):
    _fields_ = [("ksp", C.c_int32), ("pc", C.c_int32), ("rtol", C.c_double),
                ("max_it", C.c_int32), ("restart", C.c_int32), ("inner_precision", C.c_int32),
                ("inner_rtol", C.c_double), ("max_refine", C.c_int32),
                ("check_every", C.c_int32), ("learned", C.c_void_p), ("inner_its", C.c_int32),
                ("mg", C.c_void_p), ("mass_its", C.c_int32), ("fp64_apply", C.c_int32)]


class chns_mg_params(C.Structure):
    _fields_ = [("coarsest_level", C.c_int32), ("degree", C.c_int32), ("power_its", C.c_int32),
                ("smooth_range", C.c_double), ("lmax_factor", C.c_double)]


class chns_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refinements", C.c_int32),
                ("rel_residual", C.c_double), ("b_norm", C.c_double), ("status", C.c_int32),
                ("ms", C.c_float), ("escalations", C.c_int32), ("final_precision", C.c_int32),
                ("fallbacks", C.c_int32)]


class chns_state(C.Structure):
    _fields_ = [("phi", C.c_void_p), ("mu", C.c_void_p), ("u", C.c_void_p * 3),
                ("u_old", C.c_void_p * 3), ("p", C.c_void_p)]


class chns_step_params(C.Structure):
    _fields_ = [("ch", chns_solver_params), ("vp", chns_solver_params),
                ("pp", chns_solver_params), ("vu", chns_solver_params),
                ("newton_rtol", C.c_double), ("newton_atol", C.c_double),
                ("newton_max_it", C.c_int32), ("blocks", C.c_int32),
                ("collect", C.c_void_p), ("collect_every", C.c_int32),
                ("collect_max", C.c_int32), ("collect_with_net", C.c_int32),
                ("u_bc", C.c_void_p * 3)]


class chns_step_stats(C.Structure):
    _fields_ = [("newton_its", C.c_int32 * 2), ("ch", chns_solve_stats * 2),
                ("vp", chns_solve_stats * 2), ("pp", chns_solve_stats * 2),
                ("vu", chns_solve_stats * 2), ("phi_mass_before", C.c_double),
                ("phi_mass_after", C.c_double), ("ms_ch", C.c_float), ("ms_vp", C.c_float),
                ("ms_pp", C.c_float), ("ms_vu", C.c_float), ("ms_total", C.c_float)]


_P = C.c_void_p
_PP3 = C.POINTER(C.c_void_p)
_SIGS = {
    "chns_mesh_create": ([_P, _P, C.c_int64, C.POINTER(C.c_double), _P, C.POINTER(_P)], C.c_int),
    "chns_mesh_get_info": ([_P, C.POINTER(chns_mesh_info)], C.c_int),
    "chns_mesh_node_coords": ([_P, _P], C.c_int),
    "chns_mesh_boundary": ([_P, _P], C.c_int),
    "chns_mesh_destroy": ([_P], None),
    "chns_mesh_set_apply_config": ([_P, C.c_int, C.c_int64], C.c_int),
    "chns_apply_poisson": ([_P, C.POINTER(chns_params), C.POINTER(chns_coef), _P, _P, C.c_int, _P], C.c_int),
    "chns_apply_mass": ([_P, C.POINTER(chns_params), C.POINTER(chns_coef), _P, _P, C.c_int, _P], C.c_int),
    "chns_apply_ch": ([_P, C.POINTER(chns_params), C.POINTER(chns_coef), _P, _P, C.c_int, _P], C.c_int),
    "chns_apply_momentum": ([_P, C.POINTER(chns_params), C.POINTER(chns_coef), _P, _P, C.c_int, _P], C.c_int),
    "chns_operator_diagonal": ([_P, C.c_int, C.POINTER(chns_params), C.POINTER(chns_coef), _P, C.c_int, _P], C.c_int),
    "chns_residual_ch": ([_P, C.POINTER(chns_params), _P, _P, _P, _P, _PP3, _P, _P], C.c_int),
    "chns_rhs_momentum": ([_P, C.POINTER(chns_params), C.POINTER(chns_coef), _PP3, _P, _P, _P], C.c_int),
    "chns_rhs_poisson": ([_P, C.POINTER(chns_params), C.POINTER(chns_coef), _PP3, _PP3, _P, _P, _P], C.c_int),
    "chns_rhs_velocity_update": ([_P, C.POINTER(chns_params), C.POINTER(chns_coef), _PP3, _PP3, _P, _P, _P, _P], C.c_int),
    "chns_phi_mass": ([_P, _P, C.POINTER(C.c_double), _P], C.c_int),
    "chns_phi_mass_noalloc": ([_P, _P, _P, _P], C.c_int),
    "chns_krylov_solve": ([_P, C.c_int, C.POINTER(chns_params), C.POINTER(chns_coef), _P, _P,
                           C.POINTER(chns_solver_params), C.POINTER(chns_solve_stats), _P], C.c_int),
    "chns_step": ([_P, C.POINTER(chns_state), C.POINTER(chns_params), C.POINTER(chns_step_params),
                   C.POINTER(chns_step_stats), _P], C.c_int),
    "chns_learned_create": ([C.c_int32, C.c_int32, C.c_uint64, _P, C.POINTER(_P)], C.c_int),
    "chns_learned_destroy": ([_P], None),
    "chns_learned_num_params": ([_P], C.c_int64),
    "chns_learned_get_params": ([_P, _P], C.c_int),
    "chns_learned_set_params": ([_P, _P], C.c_int),
    "chns_learned_set_output_scale": ([_P, C.c_double], C.c_int),
    "chns_learned_output_scale": ([_P], C.c_double),
    "chns_learned_forward": ([_P, _P, _P, _P], C.c_int),
    "chns_learned_backward": ([_P, _P, _P, _P], C.c_int),
    "chns_learned_adam": ([_P, _P, C.c_double, _P], C.c_int),
    "chns_learned_inputs": ([_P, _P, C.POINTER(chns_params), C.POINTER(chns_coef), _P, _P,
                             C.POINTER(C.c_double), _P], C.c_int),
    "chns_learned_prolong": ([_P, _P, _P, _P, _P], C.c_int),
    "chns_learned_add_sample": ([_P, _P, C.POINTER(chns_params), C.POINTER(chns_coef), _P, _P],
                                C.c_int),
    "chns_learned_collect": ([_P, _P, C.POINTER(chns_params), C.POINTER(chns_coef), _P,
                              C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32), _P], C.c_int),
    "chns_learned_num_samples": ([_P], C.c_int32),
    "chns_learned_train": ([_P, _P, C.POINTER(chns_params), C.c_int32, C.c_double, C.c_uint64, _P,
                            _P], C.c_int),
    "chns_mg_create": ([_P, C.POINTER(chns_mg_params), _P, C.POINTER(_P)], C.c_int),
    "chns_mg_destroy": ([_P], None),
    "chns_mg_levels": ([_P, C.POINTER(C.c_int32), _P, _P], C.c_int),
    "chns_mg_setup": ([_P, C.POINTER(chns_params), _P, C.c_int, _P], C.c_int),
    "chns_mg_setup_shifted": ([_P, C.POINTER(chns_params), C.c_double, C.c_double, C.c_int, _P],
                              C.c_int),
    "chns_mg_lambda": ([_P, C.c_int32, C.c_int, _P], C.c_int),
    "chns_mg_vcycle": ([_P, C.c_int32, _P, _P, C.c_int, _P], C.c_int),
    "chns_mg_prolong": ([_P, C.c_int32, _P, _P, _P], C.c_int),
    "chns_mg_restrict": ([_P, C.c_int32, _P, _P, _P], C.c_int),
    "chns_mg_coefficient": ([_P, C.c_int32, _P, _P], C.c_int),
    "chns_remesh_flags": ([_P, _P, C.c_double, C.c_int32, C.c_int32, _P, _P], C.c_int),
    "chns_mesh_leaves": ([_P, _P, _P], C.c_int),
    "chns_mesh_remesh": ([_P, _P, C.c_double, C.c_int32, C.c_int32, _P, C.POINTER(_P)], C.c_int),
    "chns_transfer": ([_P, _P, C.c_int32, _P, _P, _P], C.c_int),
    "chns_last_error": ([], C.c_char_p),
    "chns_version": ([], C.c_char_p),
    "chns_kernel_launches": ([], C.c_uint64),
}
DECLARED = tuple(_SIGS)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2107_05123_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()


def _check(st: int, where: str):
    if st != OK:
        raise ChnsError(st, where, LIB.chns_last_error().decode())


def _ptr(x):
    """Device/host pointer of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _ptr3(xs):
    arr = (C.c_void_p * 3)(*[_ptr(x) for x in xs])
    return C.cast(arr, _PP3), arr


def make_params(d) -> chns_params:
    return chns_params(*[float(d[k]) for k in
                         ("Re", "We", "Cn", "Pe", "Fr", "rho_ratio", "eta_ratio", "dt", "C_I")])


def make_coef(phi=None, u=(None, None, None), mu=None) -> chns_coef:
    """The C struct holds raw pointers; the returned object also keeps the arrays alive."""
    c = chns_coef(_ptr(phi), (C.c_void_p * 3)(*[_ptr(x) for x in u]), _ptr(mu))
    c._keep = (phi, tuple(u), mu)
    return c


def make_solver(ksp=KSP_CG, pc=PC_JACOBI, rtol=1e-8, max_it=10000, restart=30,
                inner_precision=FP64, inner_rtol=1e-3, max_refine=20, check_every=1,
                learned=None, inner_its=0, mg=None, mass_its=0, fp64_apply=FP64):
    return chns_solver_params(ksp, pc, rtol, max_it, restart, inner_precision, inner_rtol,
                              max_refine, check_every, learned, inner_its, mg, mass_its,
                              fp64_apply)


# ------------------------------------------------------------------ mesh
def chns_mesh_create(anchors, levels, extent=(1.0, 1.0, 1.0), stream=None):
    a = np.ascontiguousarray(anchors, dtype=np.uint32).reshape(-1, 3)
    lv = np.ascontiguousarray(levels, dtype=np.uint8).reshape(-1)
    ext = (C.c_double * 3)(*[float(e) for e in extent])
    out = C.c_void_p()
    _check(LIB.chns_mesh_create(a.ctypes.data, lv.ctypes.data, len(lv), ext, _stream(stream),
                                C.byref(out)), "chns_mesh_create")
    return out.value


def chns_remesh_flags(mesh, phi, threshold, lmin, lmax, flags, stream=None):
    """flags: int8 device buffer of n_elem."""
    _check(LIB.chns_remesh_flags(mesh, _ptr(phi), float(threshold), int(lmin), int(lmax),
                                 _ptr(flags), _stream(stream)), "chns_remesh_flags")


def chns_mesh_leaves(mesh, n_elem):
    """(anchors (n_elem, 3) uint32, levels (n_elem,) uint8) of a mesh, Morton order."""
    a = np.zeros((n_elem, 3), dtype=np.uint32)
    lv = np.zeros(n_elem, dtype=np.uint8)
    _check(LIB.chns_mesh_leaves(mesh, a.ctypes.data, lv.ctypes.data), "chns_mesh_leaves")
    return a, lv


def chns_mesh_remesh(mesh, phi, threshold, lmin, lmax, stream=None):
    out = C.c_void_p()
    _check(LIB.chns_mesh_remesh(mesh, _ptr(phi), float(threshold), int(lmin), int(lmax),
                                _stream(stream), C.byref(out)), "chns_mesh_remesh")
    return out.value


def chns_transfer(src_mesh, dst_mesh, src, dst, stream=None):
    """src, dst: equal-length lists of FP64 device buffers (src_mesh / dst_mesh n_nodes)."""
    n = len(src)
    if n != len(dst):
        raise ValueError("chns_transfer: src and dst differ in length")
    sp = (C.c_void_p * n)(*[_ptr(x) for x in src])
    dp = (C.c_void_p * n)(*[_ptr(x) for x in dst])
    _check(LIB.chns_transfer(src_mesh, dst_mesh, n, sp, dp, _stream(stream)), "chns_transfer")


def chns_mesh_get_info(mesh) -> chns_mesh_info:
    info = chns_mesh_info()
    _check(LIB.chns_mesh_get_info(mesh, C.byref(info)), "chns_mesh_get_info")
    return info


def chns_mesh_node_coords(mesh, n_nodes: int) -> np.ndarray:
    out = np.zeros((n_nodes, 3), dtype=np.uint32)
    _check(LIB.chns_mesh_node_coords(mesh, out.ctypes.data), "chns_mesh_node_coords")
    return out


def chns_mesh_boundary(mesh, n_nodes: int) -> np.ndarray:
    out = np.zeros(n_nodes, dtype=np.uint8)
    _check(LIB.chns_mesh_boundary(mesh, out.ctypes.data), "chns_mesh_boundary")
    return out


def chns_mesh_set_apply_config(mesh, kernel: int, max_ctas: int = 0):
    _check(LIB.chns_mesh_set_apply_config(mesh, int(kernel), int(max_ctas)),
           "chns_mesh_set_apply_config")


def chns_mesh_destroy(mesh):
    LIB.chns_mesh_destroy(mesh)


# ------------------------------------------------------------------ operators
def _apply(name, mesh, prm, coef, x, y, prec, stream):
    _check(getattr(LIB, name)(mesh, C.byref(prm), C.byref(coef), _ptr(x), _ptr(y), prec,
                              _stream(stream)), name)


def chns_apply_poisson(mesh, prm, coef, x, y, prec=FP64, stream=None):
    _apply("chns_apply_poisson", mesh, prm, coef, x, y, prec, stream)


def chns_apply_mass(mesh, prm, coef, x, y, prec=FP64, stream=None):
    _apply("chns_apply_mass", mesh, prm, coef, x, y, prec, stream)


def chns_apply_ch(mesh, prm, coef, x, y, prec=FP64, stream=None):
    _apply("chns_apply_ch", mesh, prm, coef, x, y, prec, stream)


def chns_apply_momentum(mesh, prm, coef, x, y, prec=FP64, stream=None):
    _apply("chns_apply_momentum", mesh, prm, coef, x, y, prec, stream)


def chns_operator_diagonal(mesh, op, prm, coef, d, prec=FP64, stream=None):
    _check(LIB.chns_operator_diagonal(mesh, op, C.byref(prm), C.byref(coef), _ptr(d), prec,
                                      _stream(stream)), "chns_operator_diagonal")


def chns_residual_ch(mesh, prm, phi, mu, phik, muk, u, f, stream=None):
    up, keep = _ptr3(u)
    _check(LIB.chns_residual_ch(mesh, C.byref(prm), _ptr(phi), _ptr(mu), _ptr(phik), _ptr(muk),
                                up, _ptr(f), _stream(stream)), "chns_residual_ch")


def chns_rhs_momentum(mesh, prm, coef, uk, pk, b, stream=None):
    up, keep = _ptr3(uk)
    _check(LIB.chns_rhs_momentum(mesh, C.byref(prm), C.byref(coef), up, _ptr(pk), _ptr(b),
                                 _stream(stream)), "chns_rhs_momentum")


def chns_rhs_poisson(mesh, prm, coef, v, uk, pk, b, stream=None):
    vp, k1 = _ptr3(v)
    up, k2 = _ptr3(uk)
    _check(LIB.chns_rhs_poisson(mesh, C.byref(prm), C.byref(coef), vp, up, _ptr(pk), _ptr(b),
                                _stream(stream)), "chns_rhs_poisson")


def chns_rhs_velocity_update(mesh, prm, coef, v, uk, pk, pn, b, stream=None):
    vp, k1 = _ptr3(v)
    up, k2 = _ptr3(uk)
    _check(LIB.chns_rhs_velocity_update(mesh, C.byref(prm), C.byref(coef), vp, up, _ptr(pk),
                                        _ptr(pn), _ptr(b), _stream(stream)),
           "chns_rhs_velocity_update")


def chns_phi_mass(mesh, phi, stream=None) -> float:
    out = C.c_double()
    _check(LIB.chns_phi_mass(mesh, _ptr(phi), C.byref(out), _stream(stream)), "chns_phi_mass")
    return out.value


def chns_phi_mass_noalloc(mesh, phi, out, stream=None):
    """Writes the integral to the device double `out`; allocates nothing (see include/chns.h)."""
    _check(LIB.chns_phi_mass_noalloc(mesh, _ptr(phi), _ptr(out), _stream(stream)),
           "chns_phi_mass_noalloc")


def chns_krylov_solve(mesh, op, prm, coef, b, x, solver, stream=None, check=True):
    st = chns_solve_stats()
    rc = LIB.chns_krylov_solve(mesh, op, C.byref(prm), C.byref(coef), _ptr(b), _ptr(x),
                               C.byref(solver), C.byref(st), _stream(stream))
    if check:
        _check(rc, "chns_krylov_solve")
    return st


def chns_step(mesh, state: chns_state, prm, step_params, stream=None) -> chns_step_stats:
    """On failure the raised ChnsError carries the partial statistics as .stats."""
    st = chns_step_stats()
    rc = LIB.chns_step(mesh, C.byref(state), C.byref(prm), C.byref(step_params), C.byref(st),
                       _stream(stream))
    if rc != OK:
        err = ChnsError(rc, "chns_step", LIB.chns_last_error().decode())
        err.stats = st
        raise err
    return st


# ------------------------------------------------------------------ learned preconditioner
# ------------------------------------------------------------------ geometric multigrid
def chns_mg_create(mesh, coarsest_level=2, degree=3, power_its=12, smooth_range=15.0,
                   lmax_factor=1.1, stream=None):
    p = chns_mg_params(coarsest_level, degree, power_its, smooth_range, lmax_factor)
    out = C.c_void_p()
    _check(LIB.chns_mg_create(mesh, C.byref(p), _stream(stream), C.byref(out)), "chns_mg_create")
    return out.value


def chns_mg_destroy(mg):
    LIB.chns_mg_destroy(mg)


def chns_mg_levels(mg):
    """(n_nodes, n_elem) per level, fine first, as int64 numpy arrays."""
    n = C.c_int32()
    _check(LIB.chns_mg_levels(mg, C.byref(n), None, None), "chns_mg_levels")
    nodes = np.zeros(n.value, dtype=np.int64)
    elems = np.zeros(n.value, dtype=np.int64)
    _check(LIB.chns_mg_levels(mg, C.byref(n), _ptr(nodes), _ptr(elems)), "chns_mg_levels")
    return nodes, elems


def chns_mg_setup(mg, prm, phi, prec=FP64, stream=None):
    _check(LIB.chns_mg_setup(mg, C.byref(prm), _ptr(phi), prec, _stream(stream)), "chns_mg_setup")


def chns_mg_setup_shifted(mg, prm, sa, sb, prec=FP64, stream=None):
    _check(LIB.chns_mg_setup_shifted(mg, C.byref(prm), sa, sb, prec, _stream(stream)),
           "chns_mg_setup_shifted")


def chns_mg_lambda(mg, n_levels, prec=FP64, op=MG_POISSON) -> np.ndarray:
    out = np.zeros(n_levels, dtype=np.float64)
    _check(LIB.chns_mg_lambda(mg, op, prec, _ptr(out)), "chns_mg_lambda")
    return out


def chns_mg_vcycle(mg, r, z, prec=FP64, stream=None, op=MG_POISSON):
    _check(LIB.chns_mg_vcycle(mg, op, _ptr(r), _ptr(z), prec, _stream(stream)), "chns_mg_vcycle")


def chns_mg_prolong(mg, level, xc, xf, stream=None):
    _check(LIB.chns_mg_prolong(mg, level, _ptr(xc), _ptr(xf), _stream(stream)), "chns_mg_prolong")


def chns_mg_restrict(mg, level, xf, xc, stream=None):
    _check(LIB.chns_mg_restrict(mg, level, _ptr(xf), _ptr(xc), _stream(stream)),
           "chns_mg_restrict")


def chns_mg_coefficient(mg, level, phi, stream=None):
    _check(LIB.chns_mg_coefficient(mg, level, _ptr(phi), _stream(stream)), "chns_mg_coefficient")


def chns_learned_create(D, capacity=0, seed=0, stream=None):
    out = C.c_void_p()
    _check(LIB.chns_learned_create(int(D), int(capacity), int(seed), _stream(stream),
                                   C.byref(out)), "chns_learned_create")
    return out.value


def chns_learned_destroy(net):
    LIB.chns_learned_destroy(net)


def chns_learned_num_params(net) -> int:
    return int(LIB.chns_learned_num_params(net))


def chns_learned_get_params(net) -> np.ndarray:
    out = np.zeros(chns_learned_num_params(net), dtype=np.float32)
    _check(LIB.chns_learned_get_params(net, out.ctypes.data), "chns_learned_get_params")
    return out


def chns_learned_set_params(net, params):
    v = np.ascontiguousarray(params, dtype=np.float32)
    if v.size != chns_learned_num_params(net):
        raise ValueError("parameter vector has the wrong length")
    _check(LIB.chns_learned_set_params(net, v.ctypes.data), "chns_learned_set_params")


def chns_learned_set_output_scale(net, scale):
    _check(LIB.chns_learned_set_output_scale(net, float(scale)), "chns_learned_set_output_scale")


def chns_learned_output_scale(net) -> float:
    return float(LIB.chns_learned_output_scale(net))


def chns_learned_forward(net, x, out, stream=None):
    _check(LIB.chns_learned_forward(net, _ptr(x), _ptr(out), _stream(stream)),
           "chns_learned_forward")


def chns_learned_backward(net, gout, grad, stream=None):
    _check(LIB.chns_learned_backward(net, _ptr(gout), _ptr(grad), _stream(stream)),
           "chns_learned_backward")


def chns_learned_adam(net, grad, lr, stream=None):
    _check(LIB.chns_learned_adam(net, _ptr(grad), float(lr), _stream(stream)), "chns_learned_adam")


def chns_learned_inputs(net, mesh, prm, coef, r, x, stream=None) -> float:
    s = C.c_double()
    _check(LIB.chns_learned_inputs(net, mesh, C.byref(prm), C.byref(coef), _ptr(r), _ptr(x),
                                   C.byref(s), _stream(stream)), "chns_learned_inputs")
    return s.value


def chns_learned_prolong(net, mesh, grid, y, stream=None):
    _check(LIB.chns_learned_prolong(net, mesh, _ptr(grid), _ptr(y), _stream(stream)),
           "chns_learned_prolong")


def chns_learned_add_sample(net, mesh, prm, coef, e, stream=None):
    _check(LIB.chns_learned_add_sample(net, mesh, C.byref(prm), C.byref(coef), _ptr(e),
                                       _stream(stream)), "chns_learned_add_sample")


def chns_learned_collect(net, mesh, prm, coef, b, every, max_samples, with_net=False,
                         stream=None) -> int:
    added = C.c_int32()
    _check(LIB.chns_learned_collect(net, mesh, C.byref(prm), C.byref(coef), _ptr(b), int(every),
                                    int(max_samples), int(bool(with_net)), C.byref(added),
                                    _stream(stream)), "chns_learned_collect")
    return added.value


def chns_learned_num_samples(net) -> int:
    return int(LIB.chns_learned_num_samples(net))


def chns_learned_train(net, mesh, prm, iterations, lr, seed=0, stream=None) -> np.ndarray:
    loss = np.zeros(max(int(iterations), 1), dtype=np.float32)
    _check(LIB.chns_learned_train(net, mesh, C.byref(prm), int(iterations), float(lr), int(seed),
                                  loss.ctypes.data, _stream(stream)), "chns_learned_train")
    return loss[:int(iterations)]


def chns_version() -> str:
    return LIB.chns_version().decode()


def chns_kernel_launches() -> int:
    return int(LIB.chns_kernel_launches())
