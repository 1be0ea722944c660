"""Python binding of the C ABI in include/biot_pint.h (argument marshalling only).

Every function here forwards to the CUDA library libbiot_pint.so built in-tree
by paper_2310_10430_gb300/build.py; nothing is computed in Python. Importing the
module does not load the library; the first call does, and raises
``BiotLibraryMissing`` when it has not been built (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbiot_pint.so")

BIOT_OK, BIOT_E_INVALID, BIOT_E_OOM, BIOT_E_CUDA, BIOT_E_STATE, BIOT_E_NOT_CONVERGED, BIOT_E_DIVERGED, \
    BIOT_E_TIMEOUT = range(8)
STATUS_NAMES = ["BIOT_OK", "BIOT_E_INVALID", "BIOT_E_OOM", "BIOT_E_CUDA", "BIOT_E_STATE",
                "BIOT_E_NOT_CONVERGED", "BIOT_E_DIVERGED", "BIOT_E_TIMEOUT"]
BIOT_PRECOND_TRI, BIOT_PRECOND_DIAG = 1, 2
BIOT_FP64, BIOT_FP32, BIOT_BF16VAL_FP32ACC = 0, 1, 2
BIOT_TERZAGHI, BIOT_MMS_TRIG, BIOT_BARRY_MERCER, BIOT_MANDEL = 0, 1, 2, 3
BIOT_BETA_H2, BIOT_BETA_H, BIOT_BETA_NONE = 0, 1, 2
BIOT_SCHED_TOL, BIOT_SCHED_PAPER, BIOT_SCHED_EAGER = 0, 1, 2
BIOT_INNER_EXACT, BIOT_INNER_GMG = 0, 1
BIOT_KC_RESIDUAL, BIOT_KC_SPMM, BIOT_KC_BAND_SOLVE = 0, 1, 2


class BiotParams(ctypes.Structure):
    _fields_ = [
        ("E", ctypes.c_double), ("nu", ctypes.c_double), ("alpha", ctypes.c_double),
        ("kappa_const", ctypes.c_double), ("kappa_elem", ctypes.POINTER(ctypes.c_double)),
        ("tau", ctypes.c_double), ("n_t", ctypes.c_int32), ("problem", ctypes.c_int32),
        ("beta_mode", ctypes.c_int32), ("load", ctypes.c_double), ("n_iter", ctypes.c_int32),
        ("window", ctypes.c_int32), ("schedule", ctypes.c_int32), ("precision", ctypes.c_int32),
    ]


class BiotInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("n_nodes", ctypes.c_int32), ("n_dof", ctypes.c_int32),
        ("nnz", ctypes.c_int64), ("n_pairs", ctypes.c_int32), ("n_t", ctypes.c_int32),
        ("window_cap", ctypes.c_int32), ("band_u", ctypes.c_int32), ("band_p", ctypes.c_int32),
        ("precond", ctypes.c_int32), ("precision", ctypes.c_int32), ("beta", ctypes.c_double),
        ("device_bytes", ctypes.c_int64), ("inner", ctypes.c_int32), ("gmg_levels", ctypes.c_int32),
        ("gmg_lam_u", ctypes.c_double), ("gmg_lam_p", ctypes.c_double),
    ]


class BiotTuning(ctypes.Structure):
    _fields_ = [
        ("variant_u", ctypes.c_int32), ("variant_p", ctypes.c_int32),
        ("tma_u", ctypes.c_int32), ("nb_u", ctypes.c_int32), ("threads_u", ctypes.c_int32),
        ("tma_p", ctypes.c_int32), ("nb_p", ctypes.c_int32), ("threads_p", ctypes.c_int32),
        ("ms_u", ctypes.c_double), ("ms_p", ctypes.c_double),
        ("ms_u_default", ctypes.c_double), ("ms_p_default", ctypes.c_double),
        ("from_cache", ctypes.c_int32), ("strips", ctypes.c_int32),
        ("variant_sep_u", ctypes.c_int32), ("variant_sep_p", ctypes.c_int32),
        ("ms_sep_u", ctypes.c_double), ("ms_sep_p", ctypes.c_double),
        ("spmm_variant", ctypes.c_int32), ("ms_spmm", ctypes.c_double), ("ms_spmm_default", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BiotLibraryMissing(RuntimeError):
    pass


class BiotError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {message}")


_lib: Optional[ctypes.CDLL] = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)

_SIGNATURES = {
    "biot_mesh_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_double, _P, ctypes.POINTER(_P)]),
    "biot_assemble": (ctypes.c_int, [_P, ctypes.POINTER(BiotParams)]),
    "biot_precond_setup": (ctypes.c_int, [_P, ctypes.c_int32]),
    "biot_set_substructure": (ctypes.c_int, [_P, ctypes.c_int32]),
    "biot_pint_solve": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int32, _I32, _D]),
    "biot_set_schedule": (ctypes.c_int, [_P, ctypes.c_int32]),
    "biot_set_inner_solver": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "biot_sweep": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D]),
    "biot_batch_solve": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                        ctypes.c_int32, _I32, _D]),
    "biot_residual_norms": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D]),
    "biot_get_solution": (ctypes.c_int, [_P, ctypes.c_int32, _D]),
    "biot_get_state": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D]),
    "biot_set_state": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D]),
    "biot_get_csr": (ctypes.c_int, [_P, _I32, _I32, _D, _D, _I64]),
    "biot_get_rhs": (ctypes.c_int, [_P, _D]),
    "biot_get_residual": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _D]),
    "biot_precond_apply": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D]),
    "biot_get_info": (ctypes.c_int, [_P, ctypes.POINTER(BiotInfo)]),
    "biot_timing_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "biot_timing_read": (ctypes.c_int, [_P, ctypes.c_int32, _D, _I64]),
    "biot_residual_norms_noalloc": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _P, _P]),
    "biot_tune": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(BiotTuning)]),
    "biot_launch_count": (ctypes.c_int64, []),
    "biot_debug_set_wait_budget": (ctypes.c_int, [ctypes.c_int64]),
    "biot_last_error": (ctypes.c_char_p, [_P]),
    "biot_destroy": (None, [_P]),
}


def lib() -> ctypes.CDLL:
    """Load libbiot_pint.so (once) and declare the signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise BiotLibraryMissing(f"{LIB_PATH} not built; run __graft_entry__.build() or "
                                     "python paper_2310_10430_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _check(status: int, ctx, where: str):
    if status != BIOT_OK:
        msg = lib().biot_last_error(ctx).decode()
        raise BiotError(status, where, msg)


def _stream_handle(stream) -> Optional[int]:
    """Accept None, an int handle, or a torch.cuda.Stream."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---- one wrapper per ABI entry point ---------------------------------------

def biot_mesh_create(n: int, Lx: float = 1.0, Ly: float = 1.0, stream=None):
    out = _P()
    st = lib().biot_mesh_create(int(n), float(Lx), float(Ly), _stream_handle(stream), ctypes.byref(out))
    _check(st, None, "biot_mesh_create")
    return out


def make_params(E, nu, alpha, kappa, tau, n_t, problem=BIOT_TERZAGHI, beta_mode=BIOT_BETA_H2, load=1.0,
                n_iter=10, window=0, schedule=BIOT_SCHED_TOL, precision=BIOT_FP64):
    """BiotParams plus the array that owns kappa_elem (keep both alive until biot_assemble returns)."""
    p = BiotParams()
    p.E, p.nu, p.alpha, p.tau = float(E), float(nu), float(alpha), float(tau)
    keep = None
    if np.isscalar(kappa):
        p.kappa_const = float(kappa)
        p.kappa_elem = None
    else:
        keep = np.ascontiguousarray(kappa, dtype=np.float64)
        p.kappa_const = 0.0
        p.kappa_elem = keep.ctypes.data_as(_D)
    p.n_t, p.problem, p.beta_mode, p.load = int(n_t), int(problem), int(beta_mode), float(load)
    p.n_iter, p.window, p.schedule, p.precision = int(n_iter), int(window), int(schedule), int(precision)
    return p, keep


def biot_assemble(ctx, params: BiotParams):
    _check(lib().biot_assemble(ctx, ctypes.byref(params)), ctx, "biot_assemble")


def biot_precond_setup(ctx, kind: int):
    _check(lib().biot_precond_setup(ctx, int(kind)), ctx, "biot_precond_setup")


def biot_set_substructure(ctx, strips: int):
    _check(lib().biot_set_substructure(ctx, int(strips)), ctx, "biot_set_substructure")


def biot_set_inner_solver(ctx, kind: int, levels: int = 0, cycles: int = 1, smooth: int = 2):
    _check(lib().biot_set_inner_solver(ctx, int(kind), int(levels), int(cycles), int(smooth)), ctx,
           "biot_set_inner_solver")


def biot_set_schedule(ctx, schedule: int):
    _check(lib().biot_set_schedule(ctx, int(schedule)), ctx, "biot_set_schedule")


def biot_pint_solve(ctx, tol: float, max_outer: int, allow_not_converged: bool = False):
    """Returns (status, sweeps_done, final_rel_res)."""
    sw = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = lib().biot_pint_solve(ctx, float(tol), int(max_outer), ctypes.byref(sw), ctypes.byref(rr))
    if not (st == BIOT_OK or (allow_not_converged and st == BIOT_E_NOT_CONVERGED)):
        _check(st, ctx, "biot_pint_solve")
    return st, sw.value, rr.value


def biot_batch_solve(ctxs, tol: float, max_outer: int, use_graph: bool = True, allow_not_converged: bool = False):
    """Returns (status, sweeps_done[count], final_rel_res[count])."""
    count = len(ctxs)
    arr = (_P * count)(*[c.value if isinstance(c, _P) else c for c in ctxs])
    sw = np.zeros(count, dtype=np.int32)
    rr = np.zeros(count)
    st = lib().biot_batch_solve(arr, count, float(tol), int(max_outer), 1 if use_graph else 0,
                                sw.ctypes.data_as(_I32), _dptr(rr))
    if not (st == BIOT_OK or (allow_not_converged and st == BIOT_E_NOT_CONVERGED)):
        _check(st, None, "biot_batch_solve")
    return st, sw, rr


def biot_sweep(ctx, lo: int, hi: int, want_rel: bool = True):
    rel = np.zeros(hi - lo + 1) if want_rel else None
    _check(lib().biot_sweep(ctx, int(lo), int(hi), _dptr(rel)), ctx, "biot_sweep")
    return rel


def biot_residual_norms(ctx, lo: int, hi: int):
    rel = np.zeros(hi - lo + 1)
    _check(lib().biot_residual_norms(ctx, int(lo), int(hi), _dptr(rel)), ctx, "biot_residual_norms")
    return rel


def biot_get_info(ctx) -> BiotInfo:
    info = BiotInfo()
    _check(lib().biot_get_info(ctx, ctypes.byref(info)), ctx, "biot_get_info")
    return info


def biot_get_solution(ctx, step: int) -> np.ndarray:
    out = np.zeros(biot_get_info(ctx).n_dof)
    _check(lib().biot_get_solution(ctx, int(step), _dptr(out)), ctx, "biot_get_solution")
    return out


def biot_get_state(ctx, lo: int, hi: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    nd = biot_get_info(ctx).n_dof
    if out is None:
        out = np.zeros((hi - lo + 1, nd))
    _check(lib().biot_get_state(ctx, int(lo), int(hi), _dptr(out)), ctx, "biot_get_state")
    return out


def biot_set_state(ctx, lo: int, hi: int, host: np.ndarray):
    host = np.ascontiguousarray(host, dtype=np.float64)
    _check(lib().biot_set_state(ctx, int(lo), int(hi), _dptr(host)), ctx, "biot_set_state")


def biot_get_csr(ctx, values: bool = True):
    info = biot_get_info(ctx)
    rowptr = np.zeros(info.n_dof + 1, dtype=np.int32)
    col = np.zeros(info.nnz, dtype=np.int32)
    val = np.zeros(info.nnz) if values else None
    ap = np.zeros(info.n_pairs) if values else None
    nnz = ctypes.c_int64(0)
    st = lib().biot_get_csr(ctx, rowptr.ctypes.data_as(_I32), col.ctypes.data_as(_I32), _dptr(val), _dptr(ap),
                            ctypes.byref(nnz))
    _check(st, ctx, "biot_get_csr")
    return rowptr, col, val, ap


def biot_get_rhs(ctx) -> np.ndarray:
    info = biot_get_info(ctx)
    out = np.zeros((info.n_t + 1, info.n_dof))
    _check(lib().biot_get_rhs(ctx, _dptr(out)), ctx, "biot_get_rhs")
    return out


def biot_get_residual(ctx, lo: int, hi: int) -> np.ndarray:
    out = np.zeros((hi - lo + 1, biot_get_info(ctx).n_dof))
    _check(lib().biot_get_residual(ctx, int(lo), int(hi), _dptr(out)), ctx, "biot_get_residual")
    return out


def biot_precond_apply(ctx, vin: np.ndarray) -> np.ndarray:
    vin = np.ascontiguousarray(np.atleast_2d(vin), dtype=np.float64)
    out = np.zeros_like(vin)
    _check(lib().biot_precond_apply(ctx, vin.shape[0], _dptr(vin), _dptr(out)), ctx, "biot_precond_apply")
    return out


def biot_timing_enable(ctx, enable: bool = True):
    _check(lib().biot_timing_enable(ctx, 1 if enable else 0), ctx, "biot_timing_enable")


def biot_timing_read(ctx, kernel_class: int):
    """(total_ms, launches) recorded for one kernel class."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(lib().biot_timing_read(ctx, int(kernel_class), ctypes.byref(ms), ctypes.byref(n)), ctx, "biot_timing_read")
    return ms.value, n.value


def biot_residual_norms_noalloc(n_nodes, nodeptr, nbr, rowptr, val, ap_pp, dscale, X, F, ldx, lo, ncols, R, ldr,
                                rel, stream=None):
    """Allocation-free window residual norms; every array argument is a device
    pointer (int) owned by the caller, e.g. torch_tensor.data_ptr()."""
    st = lib().biot_residual_norms_noalloc(int(n_nodes), nodeptr, nbr, rowptr, val, ap_pp, dscale, X, F, int(ldx),
                                           int(lo), int(ncols), R, int(ldr), rel, _stream_handle(stream))
    _check(st, None, "biot_residual_norms_noalloc")


def biot_tune(ctx, cache_path: Optional[str] = None) -> BiotTuning:
    out = BiotTuning()
    _check(lib().biot_tune(ctx, cache_path.encode() if cache_path else None, ctypes.byref(out)), ctx, "biot_tune")
    return out


def biot_launch_count() -> int:
    return int(lib().biot_launch_count())


def biot_debug_set_wait_budget(cycles: int):
    """Failure-detection test hook: budget (SM cycles) of the first bounded wait of every
    band-solve block on the current device; cycles <= 0 restores the default."""
    _check(lib().biot_debug_set_wait_budget(int(cycles)), None, "biot_debug_set_wait_budget")


def biot_last_error(ctx=None) -> str:
    return lib().biot_last_error(ctx).decode()


def biot_destroy(ctx):
    lib().biot_destroy(ctx)


# ---- convenience: a context built from a workload description ---------------

_PROBLEMS = {"terzaghi": BIOT_TERZAGHI, "mms": BIOT_MMS_TRIG, "barry_mercer": BIOT_BARRY_MERCER,
             "mandel": BIOT_MANDEL}
_BETA = {"h2": BIOT_BETA_H2, "h": BIOT_BETA_H, "none": BIOT_BETA_NONE}
_PRECOND = {"tri": BIOT_PRECOND_TRI, "diag": BIOT_PRECOND_DIAG}
_PRECISION = {"fp64": BIOT_FP64, "fp32": BIOT_FP32, "bf16": BIOT_BF16VAL_FP32ACC}


class Context:
    """Owns one biot_ctx built from an object with the attributes of workloads.BiotCase."""

    def __init__(self, case, stream=None, window: int = 0, schedule: int = BIOT_SCHED_TOL,
                 precision: str = "fp64", precond: Optional[str] = None, strips: Optional[int] = None,
                 gmg: Optional[dict] = None):
        self.case = case
        self.ctx = biot_mesh_create(case.n, case.Lx, case.Ly, stream)
        try:
            kappa = case.kappa if np.isscalar(case.kappa) else np.asarray(case.kappa, dtype=np.float64)
            p, keep = make_params(case.E, case.nu, case.alpha, kappa, case.tau, case.n_t,
                                  _PROBLEMS[case.problem], _BETA[case.beta_mode], case.load, case.n_iter,
                                  window, schedule, _PRECISION[precision])
            biot_assemble(self.ctx, p)
            del keep
            if strips is not None:
                biot_set_substructure(self.ctx, strips)
            if gmg is not None:  # multigrid block solves: dict(levels=, cycles=, smooth=)
                biot_set_inner_solver(self.ctx, BIOT_INNER_GMG, **gmg)
            biot_precond_setup(self.ctx, _PRECOND[precond or case.precond])
        except Exception:
            biot_destroy(self.ctx)
            self.ctx = None
            raise

    @property
    def info(self) -> BiotInfo:
        return biot_get_info(self.ctx)

    def close(self):
        if self.ctx is not None:
            biot_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
