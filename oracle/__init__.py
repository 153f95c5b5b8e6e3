"""ctypes binding of the plain FP64 CPU oracle (arXiv 2502.19342, Sec. 2-3).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path.

A *problem* is a plain dict:
    dims  int32 (n_domains, 3)     elements per direction of each periodic box
    lo,hi float64 (n_domains, 3)   box corners
    n_fv  int                      FV sub-cells per direction
    gamma, Rgas, mu, Pr, Dk        float64 (n_species,) species properties
    riemann int                    0 = local Lax-Friedrichs, 1 = Roe + Harten-Hyman, 2 = Roe-HH between
                                   DG elements, LLF on faces touching FV data (Sec. 5.1)
    N     int8 (n_elem,)           DG degree per element
    fv    uint8 (n_elem,)          1 for FV sub-cell elements
    chain int (optional)           1: domains glued in order along x, conforming or mortar
                                   interfaces between them (Sec. 3.2.3)
    fv_own_n int (optional)        1: an FV element of degree N has N+1 sub-cells per direction
                                   (the per-element variant; n_fv unused; not with chain)
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_i8p = C.POINTER(C.c_int8)
_u8p = C.POINTER(C.c_uint8)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_dp = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [
        ("n_domains", C.c_int), ("dims", _i32p), ("lo", _dp), ("hi", _dp), ("n_fv", C.c_int),
        ("n_species", C.c_int), ("gamma", _dp), ("Rgas", _dp), ("mu", _dp), ("Pr", _dp),
        ("Dk", _dp), ("riemann", C.c_int), ("N", _i8p), ("fv", _u8p), ("nodes", C.c_int), ("split", C.c_int),
        ("sutherland", C.c_int), ("T_ref", C.c_double), ("S_sutherland", C.c_double), ("indicator_vars", C.c_int),
        ("pp_limiter", C.c_int), ("pp_eps", C.c_double), ("chain_x", C.c_int), ("fv_own_n", C.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER(_Problem)
        L.oracle_state_size.restype = C.c_int64
        L.oracle_state_size.argtypes = [P]
        L.oracle_elem_offsets.argtypes = [P, _i64p]
        L.oracle_eval_rhs.argtypes = [P, _dp, _dp]
        L.oracle_eval_rhs_jvp.argtypes = [P, _dp, _dp, _dp, _dp]
        L.oracle_eval_rhs_extended.argtypes = [P, _dp, _dp]
        L.oracle_eval_rhs_jvp_extended.argtypes = [P, _dp, _dp, _dp, _dp]
        L.oracle_adjoint_columns.argtypes = [P, _dp, _dp, C.c_int, _dp]
        L.oracle_count_flops.argtypes = [P, _dp, _dp]
        L.oracle_dt.argtypes = [P, _dp, C.c_double, C.c_double, _dp]
        L.oracle_rk3.argtypes = [P, _dp, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        L.oracle_lsrk4.argtypes = [P, _dp, C.c_int, C.c_double, C.c_double, C.c_double, _dp]
        L.oracle_lsrk4_scalar.restype = C.c_double
        L.oracle_lsrk4_scalar.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        L.oracle_set_threads.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_pp_limit.restype = C.c_int64
        L.oracle_pp_limit.argtypes = [P, _dp, C.c_double]
        L.oracle_rk3_scalar_linear.restype = C.c_double
        L.oracle_rk3_scalar_linear.argtypes = [C.c_double, C.c_double, C.c_double]
        L.oracle_indicator.argtypes = [P, _dp, _dp, _dp]
        L.oracle_adapt_decide.argtypes = [P, _dp, _dp, _dp, C.c_int, C.c_int, _i8p, _u8p]
        L.oracle_remap.argtypes = [P, _i8p, _u8p, _dp, _dp]
        L.oracle_basis.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, C.c_int]
        L.oracle_vmap.argtypes = [C.c_int, C.c_int, _dp, C.c_int]
        L.oracle_dg2fv.argtypes = [C.c_int, C.c_int, _dp, C.c_int]
        L.oracle_fv2dg.argtypes = [C.c_int, C.c_int, _dp, C.c_int]
        L.oracle_fv_overlap.argtypes = [C.c_int, C.c_int, _dp]
        L.oracle_leg_vandermonde.argtypes = [C.c_int, _dp, C.c_int]
        L.oracle_mortar.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _dp, C.c_int]
        L.oracle_flux.argtypes = [P, _dp, _dp, C.c_int, _dp, _dp]
        L.oracle_riemann.argtypes = [P, _dp, _dp, C.c_int, _dp]
        L.oracle_primitives.argtypes = [P, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t)


class _Bound:
    """Keeps the numpy arrays behind a ctypes problem alive."""

    def __init__(self, prob, N=None, fv=None):
        self.dims = np.ascontiguousarray(prob["dims"], dtype=np.int32).reshape(-1, 3)
        self.lo = np.ascontiguousarray(prob["lo"], dtype=np.float64).reshape(-1, 3)
        self.hi = np.ascontiguousarray(prob["hi"], dtype=np.float64).reshape(-1, 3)
        sp = [np.ascontiguousarray(prob[k], dtype=np.float64) for k in ("gamma", "Rgas", "mu", "Pr", "Dk")]
        self.sp = sp
        n_elem = int(np.prod(self.dims, axis=1).sum())
        NN = prob.get("N") if N is None else N
        FF = prob.get("fv") if fv is None else fv
        if NN is None:
            NN = np.full(n_elem, 1, np.int8)
        if FF is None:
            FF = np.zeros(n_elem, np.uint8)
        self.N = np.ascontiguousarray(NN, dtype=np.int8)
        self.fv = np.ascontiguousarray(FF, dtype=np.uint8)
        assert self.N.size == n_elem and self.fv.size == n_elem
        self.n_elem = n_elem
        self.c = _Problem(
            self.dims.shape[0], _ptr(self.dims, _i32p), _ptr(self.lo, _dp), _ptr(self.hi, _dp),
            int(prob["n_fv"]), len(sp[0]), _ptr(sp[0], _dp), _ptr(sp[1], _dp), _ptr(sp[2], _dp),
            _ptr(sp[3], _dp), _ptr(sp[4], _dp), int(prob.get("riemann", 0)),
            _ptr(self.N, _i8p), _ptr(self.fv, _u8p), int(prob.get("nodes", 0)), int(prob.get("split", 0)),
            int(prob.get("sutherland", 0)), float(prob.get("T_ref", 1.0)), float(prob.get("S_sutherland", 0.0)),
            int(prob.get("indicator_vars", 0)), int(prob.get("pp_limiter", 0)), float(prob.get("pp_eps", 1e-10)),
            int(prob.get("chain", 0)), int(prob.get("fv_own_n", 0)))

    @property
    def ref(self):
        return C.byref(self.c)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed ({rc})")


def state_size(prob):
    b = _Bound(prob)
    n = lib().oracle_state_size(b.ref)
    if n < 0:
        raise RuntimeError("malformed problem")
    return int(n)


def elem_offsets(prob):
    b = _Bound(prob)
    off = np.zeros(b.n_elem, np.int64)
    _check(lib().oracle_elem_offsets(b.ref, _ptr(off, _i64p)), "elem_offsets")
    return off


def eval_rhs(prob, U):
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.size == state_size(prob)
    R = np.zeros_like(U)
    _check(lib().oracle_eval_rhs(b.ref, _ptr(U, _dp), _ptr(R, _dp)), "eval_rhs")
    return R


def eval_rhs_extended(prob, U):
    """R(U) evaluated in long double arithmetic (rounding-error reference)."""
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    R = np.zeros_like(U)
    _check(lib().oracle_eval_rhs_extended(b.ref, _ptr(U, _dp), _ptr(R, _dp)), "eval_rhs_extended")
    return R


def eval_rhs_jvp(prob, U, dU):
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    dU = np.ascontiguousarray(dU, dtype=np.float64)
    R = np.zeros_like(U)
    dR = np.zeros_like(U)
    _check(lib().oracle_eval_rhs_jvp(b.ref, _ptr(U, _dp), _ptr(dU, _dp), _ptr(R, _dp), _ptr(dR, _dp)), "jvp")
    return R, dR


def eval_rhs_jvp_extended(prob, U, dU):
    """eval_rhs_jvp carried in long double: the FP64 tangent's rounding reference."""
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    dU = np.ascontiguousarray(dU, dtype=np.float64)
    R = np.zeros_like(U)
    dR = np.zeros_like(U)
    _check(lib().oracle_eval_rhs_jvp_extended(b.ref, _ptr(U, _dp), _ptr(dU, _dp), _ptr(R, _dp), _ptr(dR, _dp)),
           "jvp (extended)")
    return R, dR


def adjoint_columns(prob, U, Rbar, extended=False):
    """R'(U)^T R_bar entry by entry from tangents along the unit vectors (tiny
    meshes); extended=True carries tangent and sums in long double."""
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    Rbar = np.ascontiguousarray(Rbar, dtype=np.float64)
    Ub = np.zeros_like(U)
    _check(lib().oracle_adjoint_columns(b.ref, _ptr(U, _dp), _ptr(Rbar, _dp), int(extended), _ptr(Ub, _dp)),
           "adjoint columns")
    return Ub


STEPS = {1: "face values", 2: "FV sub-cells", 3: "lifting value", 4: "DG lifting + volume",
         5: "face flux", 6: "surface"}


def count_flops(prob, U):
    """Counted operations of one R(U): dict add, mul, div, sqrt, and 'steps':
    {step: {add, mul, div, sqrt}} for the six steps of the evaluation."""
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(40)
    _check(lib().oracle_count_flops(b.ref, _ptr(U, _dp), _ptr(out, _dp)), "count_flops")
    keys = ("add", "mul", "div", "sqrt")
    steps = {s: dict(zip(keys, out[8 + 4 * s:12 + 4 * s])) for s in range(1, 7)}
    return {"add": out[0], "mul": out[1], "div": out[2], "sqrt": out[3], "steps": steps}


def dt(prob, U, cfl_c, cfl_v):
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(3)
    _check(lib().oracle_dt(b.ref, _ptr(U, _dp), cfl_c, cfl_v, _ptr(out, _dp)), "dt")
    return float(out[0]), float(out[1]), float(out[2])


def rk3(prob, U, n_steps, dt_fixed=-1.0, cfl_c=0.5, cfl_v=0.5):
    """n_steps SSP-RK3 steps; returns (U_final, dts)."""
    b = _Bound(prob)
    X = np.array(U, dtype=np.float64, copy=True)
    dts = np.zeros(max(n_steps, 1))
    _check(lib().oracle_rk3(b.ref, _ptr(X, _dp), n_steps, dt_fixed, cfl_c, cfl_v, _ptr(dts, _dp)), "rk3")
    return X, dts[:n_steps]


def rk3_scalar_linear(lam, dt_, u0):
    return lib().oracle_rk3_scalar_linear(lam, dt_, u0)


def lsrk4(prob, U, n_steps, dt_fixed=-1.0, cfl_c=0.5, cfl_v=0.5):
    """n_steps steps of the five-stage low-storage RK4; returns (U_final, dts)."""
    b = _Bound(prob)
    X = np.array(U, dtype=np.float64, copy=True)
    dts = np.zeros(max(n_steps, 1))
    _check(lib().oracle_lsrk4(b.ref, _ptr(X, _dp), n_steps, dt_fixed, cfl_c, cfl_v, _ptr(dts, _dp)), "lsrk4")
    return X, dts[:n_steps]


def set_threads(n=0):
    """Host threads of the oracle's loops (n > 0 sets them); returns the number in use."""
    return int(lib().oracle_set_threads(int(n)))


def pp_limit(prob, U, eps=1e-10):
    """Positivity limiter (Sec. 3.5) applied once; returns (U_limited, elements changed)."""
    b = _Bound(prob)
    X = np.array(U, dtype=np.float64, copy=True)
    n = lib().oracle_pp_limit(b.ref, _ptr(X, _dp), float(eps))
    if n < 0:
        raise RuntimeError("oracle pp_limit failed")
    return X, int(n)


def lsrk4_scalar(kind, lam, dt_, u0):
    """One low-storage RK4 step of u' = lam u (kind 0) or u' = -u^2 (kind 1)."""
    return lib().oracle_lsrk4_scalar(int(kind), lam, dt_, u0)


def indicator(prob, U):
    b = _Bound(prob)
    U = np.ascontiguousarray(U, dtype=np.float64)
    Ip = np.zeros(b.n_elem)
    Ih = np.zeros(b.n_elem)
    _check(lib().oracle_indicator(b.ref, _ptr(U, _dp), _ptr(Ip, _dp), _ptr(Ih, _dp)), "indicator")
    return Ip, Ih


def adapt_decide(prob, Ip, Ih, thresholds, N_min, N_max):
    b = _Bound(prob)
    Ip = np.ascontiguousarray(Ip, dtype=np.float64)
    Ih = np.ascontiguousarray(Ih, dtype=np.float64)
    thr = np.ascontiguousarray(thresholds, dtype=np.float64)
    Nn = np.zeros(b.n_elem, np.int8)
    fn = np.zeros(b.n_elem, np.uint8)
    _check(lib().oracle_adapt_decide(b.ref, _ptr(Ip, _dp), _ptr(Ih, _dp), _ptr(thr, _dp), N_min, N_max,
                                     _ptr(Nn, _i8p), _ptr(fn, _u8p)), "adapt_decide")
    return Nn, fn


def remap(prob, N_new, fv_new, U_old):
    b = _Bound(prob)
    Nn = np.ascontiguousarray(N_new, dtype=np.int8)
    fn = np.ascontiguousarray(fv_new, dtype=np.uint8)
    new = dict(prob, N=Nn, fv=fn)
    Unew = np.zeros(state_size(new))
    U_old = np.ascontiguousarray(U_old, dtype=np.float64)
    _check(lib().oracle_remap(b.ref, _ptr(Nn, _i8p), _ptr(fn, _u8p), _ptr(U_old, _dp), _ptr(Unew, _dp)), "remap")
    return Unew


def basis(N, nodes=0):
    """Reference operators of degree N; nodes 0 = Legendre-Gauss, 1 = Legendre-Gauss-Lobatto."""
    n = N + 1
    x, w, lm, lp = (np.zeros(n) for _ in range(4))
    D, Dh = np.zeros((n, n)), np.zeros((n, n))
    _check(lib().oracle_basis(N, _ptr(x, _dp), _ptr(w, _dp), _ptr(D, _dp), _ptr(Dh, _dp), _ptr(lm, _dp),
                              _ptr(lp, _dp), int(nodes)), "basis")
    return {"x": x, "w": w, "D": D, "Dhat": Dh, "lm": lm, "lp": lp}


def vmap(N_from, N_to, nodes=0):
    M = np.zeros((N_to + 1, N_from + 1))
    _check(lib().oracle_vmap(N_from, N_to, _ptr(M, _dp), int(nodes)), "vmap")
    return M


def dg2fv(N, n_fv, nodes=0):
    M = np.zeros((n_fv, N + 1))
    _check(lib().oracle_dg2fv(N, n_fv, _ptr(M, _dp), int(nodes)), "dg2fv")
    return M


def fv2dg(N, n_fv, nodes=0):
    M = np.zeros((N + 1, n_fv))
    _check(lib().oracle_fv2dg(N, n_fv, _ptr(M, _dp), int(nodes)), "fv2dg")
    return M


def mortar(N, half, proj=False, fv=False, nodes=0):
    """Sec. 3.2.3 mortar matrix of one direction: interpolation to the virtual small
    side of half `half` (proj=False) or L2 projection back (proj=True); on degree-N
    nodes, or (fv=True) on N sub-cells."""
    n = N if fv else N + 1
    M = np.zeros((n, n))
    _check(lib().oracle_mortar(int(N), int(half), int(bool(proj)), int(bool(fv)), _ptr(M, _dp), int(nodes)), "mortar")
    return M


def fv_overlap(n_from, n_to):
    """n_to x n_from piecewise-constant L2 projection between uniform sub-cell grids."""
    M = np.zeros((n_to, n_from))
    _check(lib().oracle_fv_overlap(n_from, n_to, _ptr(M, _dp)), "fv_overlap")
    return M


def leg_vandermonde(N, nodes=0):
    M = np.zeros((N + 1, N + 1))
    _check(lib().oracle_leg_vandermonde(N, _ptr(M, _dp), int(nodes)), "leg_vandermonde")
    return M


def _phys_only(prob):
    p = dict(prob)
    p.setdefault("dims", [[1, 1, 1]])
    p.setdefault("lo", [[0, 0, 0]])
    p.setdefault("hi", [[1, 1, 1]])
    p.setdefault("n_fv", 2)
    return _Bound(p)


def flux(prob, u, g, direction):
    b = _phys_only(prob)
    u = np.ascontiguousarray(u, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    Fc = np.zeros(u.size)
    Fv = np.zeros(u.size)
    _check(lib().oracle_flux(b.ref, _ptr(u, _dp), _ptr(g, _dp), direction, _ptr(Fc, _dp), _ptr(Fv, _dp)), "flux")
    return Fc, Fv


def riemann(prob, uL, uR, direction):
    b = _phys_only(prob)
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    F = np.zeros(uL.size)
    _check(lib().oracle_riemann(b.ref, _ptr(uL, _dp), _ptr(uR, _dp), direction, _ptr(F, _dp)), "riemann")
    return F


def primitives(prob, u):
    """rho, p, T, c, kappa, cv, cp, mu, lambda, Y_1..Y_Nk of one state."""
    b = _phys_only(prob)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(9 + len(prob["gamma"]))
    _check(lib().oracle_primitives(b.ref, _ptr(u, _dp), _ptr(out, _dp)), "primitives")
    names = ["rho", "p", "T", "c", "kappa", "cv", "cp", "mu", "lam"]
    d = {k: out[i] for i, k in enumerate(names)}
    d["Y"] = out[9:]
    return d
