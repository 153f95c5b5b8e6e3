"""Python binding of the dgfv C ABI (include/dgfv.h): argument marshalling only.

Every step of the right-hand side runs in the CUDA library
``_build/libdgfv.so``; this module has no fallback.  Device arrays are torch
tensors (float64, CUDA); streams are torch's current CUDA stream unless given.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdgfv.so")

DGFV_OK = 0
STATUS = {0: "DGFV_OK", -1: "DGFV_ERR_ARG", -2: "DGFV_ERR_CUDA", -3: "DGFV_ERR_OOM", -4: "DGFV_ERR_NONPHYSICAL",
          -5: "DGFV_ERR_NONFINITE", -6: "DGFV_ERR_TIMEOUT", -7: "DGFV_ERR_STATE"}

# every symbol the header declares
SYMBOLS = ["dgfv_init_mesh", "dgfv_num_elements", "dgfv_set_degrees", "dgfv_get_degrees", "dgfv_state_layout",
           "dgfv_set_state", "dgfv_get_state", "dgfv_set_state_host", "dgfv_get_state_host", "dgfv_eval_rhs",
           "dgfv_compute_dt", "dgfv_rk_step", "dgfv_rk_steps", "dgfv_indicator", "dgfv_adapt", "dgfv_sync_status",
           "dgfv_status_string", "dgfv_last_error", "dgfv_destroy", "dgfv_bank_entry", "dgfv_probe_dfma",
           "dgfv_profile_enable", "dgfv_profile_read", "dgfv_compute_dt_noalloc", "dgfv_rhs_vjp",
           "dgfv_rk_step_vjp", "dgfv_set_launch_mode", "dgfv_autotune", "dgfv_rk_step_save",
           "dgfv_rk_step_vjp_stages", "dgfv_probe_dmma", "dgfv_pp_limit", "dgfv_pp_count",
           "dgfv_set_fv_variant"]
KERNELS = ["prolong", "fv", "face_lift", "dg_volume", "face_flux", "surface", "dt", "indicator", "remap"]


class MeshDesc(C.Structure):
    _fields_ = [("n_domains", C.c_int), ("dims", C.POINTER(C.c_int32)), ("lo", C.POINTER(C.c_double)),
                ("hi", C.POINTER(C.c_double)), ("N_min", C.c_int), ("N_max", C.c_int), ("N_fv", C.c_int),
                ("chain_x", C.c_int)]


class Phys(C.Structure):
    _fields_ = [("n_species", C.c_int), ("gamma", C.c_double * 3), ("Rgas", C.c_double * 3),
                ("mu", C.c_double * 3), ("Pr", C.c_double * 3), ("D", C.c_double * 3), ("sutherland", C.c_int),
                ("T_ref", C.c_double), ("S", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("riemann", C.c_int), ("cfl_c", C.c_double), ("cfl_v", C.c_double), ("T_fv_on", C.c_double),
                ("T_fv_off", C.c_double), ("T_ref", C.c_double), ("T_crs", C.c_double), ("nodes", C.c_int),
                ("split_form", C.c_int), ("integrator", C.c_int), ("indicator_vars", C.c_int),
                ("pp_limiter", C.c_int), ("pp_eps", C.c_double)]


class AdaptStats(C.Structure):
    _fields_ = [("n_fv", C.c_int64), ("hist", C.c_int64 * 8), ("n_changed", C.c_int64), ("n_near", C.c_int64),
                ("mean_dofs", C.c_double)]


_lib = None


def lib():
    """Load the CUDA library; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"dgfv CUDA library missing at {LIB_PATH}: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
        L.dgfv_init_mesh.argtypes = [C.POINTER(vp), C.POINTER(MeshDesc), C.POINTER(Phys), C.POINTER(Opts)]
        L.dgfv_num_elements.restype = i64
        L.dgfv_num_elements.argtypes = [vp]
        L.dgfv_set_degrees.argtypes = [vp, C.POINTER(C.c_int8), C.POINTER(C.c_uint8), C.c_int]
        L.dgfv_get_degrees.argtypes = [vp, C.POINTER(C.c_int8), C.POINTER(C.c_uint8)]
        L.dgfv_state_layout.argtypes = [vp, C.POINTER(i64), C.POINTER(vp)]
        for f in ("dgfv_set_state", "dgfv_get_state", "dgfv_set_state_host", "dgfv_get_state_host"):
            getattr(L, f).argtypes = [vp, vp, i64, vp]
        L.dgfv_eval_rhs.argtypes = [vp, vp, vp, vp]
        L.dgfv_compute_dt.argtypes = [vp, vp, dp, vp]
        L.dgfv_compute_dt_noalloc.argtypes = [vp, vp, vp, vp]
        L.dgfv_rhs_vjp.argtypes = [vp, vp, vp, vp, vp]
        L.dgfv_set_launch_mode.argtypes = [vp, C.c_int]
        L.dgfv_set_fv_variant.argtypes = [vp, C.c_int]
        L.dgfv_autotune.argtypes = [vp, C.POINTER(C.c_int), vp]
        L.dgfv_rk_step_vjp.argtypes = [vp, vp, C.c_double, vp, vp, vp]
        L.dgfv_rk_step_save.argtypes = [vp, C.c_double, vp, vp, vp]
        L.dgfv_rk_step_vjp_stages.argtypes = [vp, C.POINTER(vp), C.c_double, vp, vp, vp]
        L.dgfv_rk_step.argtypes = [vp, C.c_double, dp, vp]
        L.dgfv_rk_steps.argtypes = [vp, C.c_int, C.c_double, dp, vp]
        L.dgfv_indicator.argtypes = [vp, vp, vp, vp, vp, vp]
        L.dgfv_adapt.argtypes = [vp, C.POINTER(AdaptStats), vp]
        L.dgfv_sync_status.argtypes = [vp, vp]
        L.dgfv_status_string.restype = C.c_char_p
        L.dgfv_status_string.argtypes = [C.c_int]
        L.dgfv_last_error.restype = C.c_char_p
        L.dgfv_last_error.argtypes = [vp]
        L.dgfv_destroy.argtypes = [vp]
        L.dgfv_destroy.restype = None
        L.dgfv_bank_entry.restype = i64
        L.dgfv_bank_entry.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp, i64]
        L.dgfv_probe_dfma.restype = C.c_double
        L.dgfv_probe_dfma.argtypes = [C.c_int, vp]
        L.dgfv_pp_limit.argtypes = [vp, vp, C.POINTER(i64), vp]
        L.dgfv_pp_count.argtypes = [vp, C.POINTER(i64), C.c_int, vp]
        L.dgfv_probe_dmma.restype = C.c_double
        L.dgfv_probe_dmma.argtypes = [C.c_int, vp]
        L.dgfv_profile_enable.argtypes = [vp, C.c_int]
        L.dgfv_profile_read.argtypes = [vp, dp, C.POINTER(i64), C.c_int]
        _lib = L
    return _lib


class DgfvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_dev(t, n=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")


class Context:
    """One dgfv context (mesh, species, options, degree pattern, state)."""

    def __init__(self, problem, N_min=None, N_max=None, opts=None):
        L = lib()
        dims = np.ascontiguousarray(problem["dims"], np.int32).reshape(-1, 3)
        lo = np.ascontiguousarray(problem["lo"], np.float64).reshape(-1, 3)
        hi = np.ascontiguousarray(problem["hi"], np.float64).reshape(-1, 3)
        Ns = np.asarray(problem["N"])
        N_min = int(Ns.min()) if N_min is None else int(N_min)
        N_max = int(Ns.max()) if N_max is None else int(N_max)
        self._keep = (dims, lo, hi)
        mesh = MeshDesc(dims.shape[0], dims.ctypes.data_as(C.POINTER(C.c_int32)),
                        lo.ctypes.data_as(C.POINTER(C.c_double)), hi.ctypes.data_as(C.POINTER(C.c_double)),
                        N_min, N_max, 0 if problem.get("fv_own_n", 0) else int(problem["n_fv"]),
                        int(problem.get("chain", 0)))
        nk = len(problem["gamma"])
        ph = Phys()
        ph.n_species = nk
        for k in range(nk):
            ph.gamma[k] = float(problem["gamma"][k])
            ph.Rgas[k] = float(problem["Rgas"][k])
            ph.mu[k] = float(problem["mu"][k])
            ph.Pr[k] = float(problem["Pr"][k])
            ph.D[k] = float(problem["Dk"][k])
        ph.sutherland = int(problem.get("sutherland", 0))
        ph.T_ref = float(problem.get("T_ref", 1.0))
        ph.S = float(problem.get("S_sutherland", 0.0))
        o = dict(cfl_c=0.5, cfl_v=0.5, thresholds=(1.0, 1.6, 3.0, 7.0))
        o.update(opts or {})
        thr = o["thresholds"]
        op = Opts(int(problem.get("riemann", 0)), float(o["cfl_c"]), float(o["cfl_v"]), *[float(x) for x in thr],
                  int(problem.get("nodes", 0)), int(problem.get("split", 0)), int(o.get("integrator", 0)),
                  int(problem.get("indicator_vars", 0)), int(problem.get("pp_limiter", 0)),
                  float(problem.get("pp_eps", 1e-10)))
        h = C.c_void_p()
        rc = L.dgfv_init_mesh(C.byref(h), C.byref(mesh), C.byref(ph), C.byref(op))
        if rc != 0:
            raise DgfvError(rc, "dgfv_init_mesh failed")
        self.h = h
        self.n_elem = int(L.dgfv_num_elements(h))
        self.V = nk + 4
        self.set_degrees(problem["N"], problem.get("fv"), remap=False)

    def _rc(self, rc, what):
        if rc != 0:
            msg = lib().dgfv_last_error(self.h)
            raise DgfvError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            lib().dgfv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- pattern / layout
    def set_degrees(self, N, fv=None, remap=True):
        N = np.ascontiguousarray(N, np.int8)
        f = np.zeros(self.n_elem, np.uint8) if fv is None else np.ascontiguousarray(fv, np.uint8)
        self._rc(lib().dgfv_set_degrees(self.h, N.ctypes.data_as(C.POINTER(C.c_int8)),
                                        f.ctypes.data_as(C.POINTER(C.c_uint8)), int(remap)), "set_degrees")

    def get_degrees(self):
        N = np.zeros(self.n_elem, np.int8)
        f = np.zeros(self.n_elem, np.uint8)
        self._rc(lib().dgfv_get_degrees(self.h, N.ctypes.data_as(C.POINTER(C.c_int8)),
                                        f.ctypes.data_as(C.POINTER(C.c_uint8))), "get_degrees")
        return N, f

    def state_layout(self):
        n = C.c_int64()
        p = C.c_void_p()
        self._rc(lib().dgfv_state_layout(self.h, C.byref(n), C.byref(p)), "state_layout")
        return int(n.value), p.value

    @property
    def state_size(self):
        return self.state_layout()[0]

    # --------------------------------------------------------------- state
    def set_state(self, U, stream=None):
        _check_dev(U, self.state_size)
        self._rc(lib().dgfv_set_state(self.h, _ptr(U), U.numel(), _stream(stream)), "set_state")

    def get_state(self, out=None, stream=None):
        import torch
        n = self.state_size
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device="cuda")
        _check_dev(out, n)
        self._rc(lib().dgfv_get_state(self.h, _ptr(out), n, _stream(stream)), "get_state")
        return out

    def set_state_host(self, U, stream=None):
        """U: host float64 array or CPU tensor (pinned memory gives asynchronous copies)."""
        import torch
        if isinstance(U, np.ndarray):
            U = torch.from_numpy(np.ascontiguousarray(U, np.float64))
        assert U.device.type == "cpu" and U.dtype == torch.float64 and U.is_contiguous()
        self._rc(lib().dgfv_set_state_host(self.h, _ptr(U), U.numel(), _stream(stream)), "set_state_host")

    def get_state_host(self, out=None, stream=None):
        import torch
        n = self.state_size
        if out is None:
            out = torch.empty(n, dtype=torch.float64)
        self._rc(lib().dgfv_get_state_host(self.h, _ptr(out), n, _stream(stream)), "get_state_host")
        return out

    # --------------------------------------------------------------- operator
    def eval_rhs(self, U, R=None, stream=None):
        import torch
        n = self.state_size
        _check_dev(U, n)
        if R is None:
            R = torch.empty(n, dtype=torch.float64, device="cuda")
        _check_dev(R, n)
        self._rc(lib().dgfv_eval_rhs(self.h, _ptr(U), _ptr(R), _stream(stream)), "eval_rhs")
        return R

    def rhs_vjp(self, U, Rbar, Ubar=None, stream=None):
        """(dR/dU)^T Rbar at U (DG patterns, local Lax-Friedrichs flux)."""
        import torch
        n = self.state_size
        _check_dev(U, n)
        _check_dev(Rbar, n)
        if Ubar is None:
            Ubar = torch.empty(n, dtype=torch.float64, device="cuda")
        _check_dev(Ubar, n)
        self._rc(lib().dgfv_rhs_vjp(self.h, _ptr(U), _ptr(Rbar), _ptr(Ubar), _stream(stream)), "rhs_vjp")
        return Ubar

    def rk_step_vjp(self, U0, dt, Ubar_next, Ubar=None, stream=None):
        """Adjoint of one SSP-RK3 step of size dt from U0 (stages recomputed)."""
        import torch
        n = self.state_size
        _check_dev(U0, n)
        _check_dev(Ubar_next, n)
        if Ubar is None:
            Ubar = torch.empty(n, dtype=torch.float64, device="cuda")
        _check_dev(Ubar, n)
        self._rc(lib().dgfv_rk_step_vjp(self.h, _ptr(U0), float(dt), _ptr(Ubar_next), _ptr(Ubar), _stream(stream)),
                 "rk_step_vjp")
        return Ubar

    def rk_step_save(self, dt, stage1, stage2, stream=None):
        """One RK step of size dt; the two intermediate stage states go to stage1, stage2."""
        n = self.state_size
        _check_dev(stage1, n)
        _check_dev(stage2, n)
        self._rc(lib().dgfv_rk_step_save(self.h, float(dt), _ptr(stage1), _ptr(stage2), _stream(stream)),
                 "rk_step_save")

    def rk_step_vjp_stages(self, stages, dt, Ubar_next, Ubar=None, stream=None):
        """Adjoint of one RK step from the stored stage states (U0, U1, U2)."""
        import torch
        n = self.state_size
        for t in stages:
            _check_dev(t, n)
        _check_dev(Ubar_next, n)
        if Ubar is None:
            Ubar = torch.empty(n, dtype=torch.float64, device="cuda")
        arr = (C.c_void_p * 3)(*[t.data_ptr() for t in stages])
        self._rc(lib().dgfv_rk_step_vjp_stages(self.h, arr, float(dt), _ptr(Ubar_next), _ptr(Ubar), _stream(stream)),
                 "rk_step_vjp_stages")
        return Ubar

    def pp_limit(self, U, stream=None):
        """Positivity limiter (Sec. 3.5) applied once to U in place; returns the elements changed."""
        _check_dev(U, self.state_size)
        n = C.c_int64(0)
        self._rc(lib().dgfv_pp_limit(self.h, _ptr(U), C.byref(n), _stream(stream)), "pp_limit")
        return int(n.value)

    def pp_count(self, reset=False, stream=None):
        """Element limitings by the stage limiter since the last reset."""
        n = C.c_int64(0)
        self._rc(lib().dgfv_pp_count(self.h, C.byref(n), int(bool(reset)), _stream(stream)), "pp_count")
        return int(n.value)

    def compute_dt(self, U, stream=None):
        _check_dev(U, self.state_size)
        out = (C.c_double * 3)()
        self._rc(lib().dgfv_compute_dt(self.h, _ptr(U), out, _stream(stream)), "compute_dt")
        return tuple(out)

    def compute_dt_noalloc(self, U, out3, stream=None):
        """Time step into the caller's device tensor out3 (3 float64), through
        the allocation-free entry point; does not synchronise."""
        _check_dev(U, self.state_size)
        _check_dev(out3, 3)
        self._rc(lib().dgfv_compute_dt_noalloc(self.h, _ptr(U), _ptr(out3), _stream(stream)), "compute_dt_noalloc")
        return out3

    def rk_step(self, dt=-1.0, want_dt=True, stream=None):
        out = C.c_double(0.0)
        self._rc(lib().dgfv_rk_step(self.h, float(dt), C.byref(out) if want_dt else None, _stream(stream)),
                 "rk_step")
        return out.value if want_dt else None

    def rk_steps(self, n_steps, dt=-1.0, want_dt=True, stream=None):
        out = C.c_double(0.0)
        self._rc(lib().dgfv_rk_steps(self.h, int(n_steps), float(dt), C.byref(out) if want_dt else None,
                                     _stream(stream)), "rk_steps")
        return out.value if want_dt else None

    def indicator(self, U, stream=None):
        import torch
        _check_dev(U, self.state_size)
        Ip = torch.empty(self.n_elem, dtype=torch.float64, device="cuda")
        Ih = torch.empty(self.n_elem, dtype=torch.float64, device="cuda")
        dec = torch.empty(self.n_elem, dtype=torch.uint8, device="cuda")
        self._rc(lib().dgfv_indicator(self.h, _ptr(U), _ptr(Ip), _ptr(Ih), _ptr(dec), _stream(stream)), "indicator")
        return Ip, Ih, dec

    def adapt(self, stream=None):
        st = AdaptStats()
        self._rc(lib().dgfv_adapt(self.h, C.byref(st), _stream(stream)), "adapt")
        return dict(n_fv=st.n_fv, hist=list(st.hist), n_changed=st.n_changed, n_near=st.n_near,
                    mean_dofs=st.mean_dofs)

    def sync_status(self, stream=None):
        self._rc(lib().dgfv_sync_status(self.h, _stream(stream)), "device status")

    def set_fv_variant(self, variant):
        """FV sub-cell kernel layout: 0 automatic, 1 gradients recomputed at each face, 2 gradients kept,
        3 gradients kept with the z faces in a second pass (two CTAs per SM)."""
        self._rc(lib().dgfv_set_fv_variant(self.h, int(variant)), "set_fv_variant")

    def set_launch_mode(self, mode):
        """0 (or False): one launch per kernel over all degrees; 1 (or True): one
        launch per degree bin; 2: as 0 with the persistent volume kernel."""
        self._rc(lib().dgfv_set_launch_mode(self.h, int(mode)), "set_launch_mode")

    def autotune(self, stream=None):
        """Time launch variants and tile sizes of the volume kernel on the current
        state; returns {"variant": v, N: elements per tile, ...}."""
        out = (C.c_int * 9)()
        self._rc(lib().dgfv_autotune(self.h, out, _stream(stream)), "autotune")
        res = {"variant": int(out[0])}
        res.update({n - 1: out[n] for n in range(1, 9) if out[n] > 0})
        return res

    def profile_enable(self, on=True):
        self._rc(lib().dgfv_profile_enable(self.h, int(on)), "profile_enable")

    def profile_read(self):
        """{kernel: (milliseconds, launches)} since the last profile_enable."""
        ms = (C.c_double * len(KERNELS))()
        nl = (C.c_int64 * len(KERNELS))()
        n = lib().dgfv_profile_read(self.h, ms, nl, len(KERNELS))
        if n < 0:
            self._rc(n, "profile_read")
        return {KERNELS[k]: (ms[k], int(nl[k])) for k in range(n)}

    def bank_entry(self, which, N, M=0):
        buf = np.zeros(4096)
        n = lib().dgfv_bank_entry(self.h, which, N, M, buf.ctypes.data_as(C.POINTER(C.c_double)), buf.size)
        if n < 0:
            raise DgfvError(int(n), "bank_entry")
        return buf[:n].copy()


def init_mesh(problem, N_min=None, N_max=None, opts=None):
    return Context(problem, N_min, N_max, opts)


def probe_dfma(iters=1 << 16, stream=None):
    """Measured FP64 FMA throughput (flop/s, 2 per DFMA) of this GPU."""
    return float(lib().dgfv_probe_dfma(int(iters), _stream(stream)))


def probe_dmma(iters=1 << 12, stream=None):
    """Measured FP64 tensor-core (mma.sync m8n8k4) throughput (flop/s) of this GPU."""
    return float(lib().dgfv_probe_dmma(int(iters), _stream(stream)))


def rhs_function():
    """torch.autograd.Function computing R(U) on the CUDA path, with the
    hand-written adjoint as its backward (degree pattern frozen).
    Usage: R = rhs_function().apply(U, ctx)."""
    import torch

    class RHS(torch.autograd.Function):
        @staticmethod
        def forward(fctx, U, ctx):
            fctx.ctx = ctx
            fctx.save_for_backward(U)
            return ctx.eval_rhs(U.contiguous())

        @staticmethod
        def backward(fctx, Rbar):
            (U,) = fctx.saved_tensors
            return fctx.ctx.rhs_vjp(U, Rbar.contiguous()), None

    return RHS


def rk_step_function():
    """torch.autograd.Function of one Runge-Kutta step of fixed size on the
    CUDA path, in the context's scheme (SSP-RK3, or the low-storage RK4 with
    opts integrator 1): forward U1 = step(U0) through the context, backward
    the step's hand-written adjoint with its stage states recomputed from the
    saved U0 (degree pattern frozen).  A rollout is a chain of applications, so autograd
    keeps one state per step.  Usage: U1 = rk_step_function().apply(U0, ctx, dt).
    The context's state is U1 after the forward."""
    import torch

    class RKStep(torch.autograd.Function):
        @staticmethod
        def forward(fctx, U0, ctx, dt):
            fctx.ctx, fctx.dt = ctx, float(dt)
            U0 = U0.detach().contiguous()
            fctx.save_for_backward(U0)
            ctx.set_state(U0)
            ctx.rk_step(float(dt), want_dt=False)
            return ctx.get_state()

        @staticmethod
        def backward(fctx, U1bar):
            (U0,) = fctx.saved_tensors
            return fctx.ctx.rk_step_vjp(U0, fctx.dt, U1bar.contiguous()), None, None

    return RKStep


def rollout_gradient(ctx, U0, n_steps, dt, loss_grad, keep_stages=False, checkpoint_every=1):
    """Gradient of a loss of the state after n_steps Runge-Kutta steps of size
    dt (the context's scheme; keep_stages needs SSP-RK3) with respect to the
    initial state, by the adjoint of every step.
    keep_stages=False keeps one checkpoint every `checkpoint_every` steps: with
    1 (the default) the state at the start of every step, whose stage states
    the backward pass recomputes; with k > 1 every k-th state, the backward
    pass stepping each segment forward again from its checkpoint to recover
    its step states (n_steps/k + k states in memory instead of n_steps, for one
    more forward pass; the forward is deterministic, so the gradient is bitwise
    the same).  keep_stages=True keeps all three stage states per step (three
    times the memory of k = 1, no recomputation).
    loss_grad(U_final) returns dLoss/dU_final.  Returns (gradient, U_final);
    the context's state is U_final afterwards."""
    import torch
    k = int(checkpoint_every)
    if k < 1 or (keep_stages and k != 1):
        raise ValueError("checkpoint_every must be >= 1 (and 1 with keep_stages)")
    ctx.set_state(U0)
    ckpt = []
    for s in range(n_steps):
        if keep_stages:
            U = ctx.get_state()
            s1, s2 = torch.empty_like(U), torch.empty_like(U)
            ctx.rk_step_save(dt, s1, s2)
            ckpt.append((U, s1, s2))
        else:
            if s % k == 0:
                ckpt.append(ctx.get_state())
            ctx.rk_step(dt, want_dt=False)
    Uf = ctx.get_state()
    lam = loss_grad(Uf)
    if keep_stages:
        for s in range(n_steps - 1, -1, -1):
            lam = ctx.rk_step_vjp_stages(ckpt[s], dt, lam)
    else:
        for seg in range((n_steps - 1) // k if n_steps else -1, -1, -1):
            first, last = seg * k, min(seg * k + k, n_steps)
            states = [ckpt[seg]]
            if last - first > 1:
                ctx.set_state(ckpt[seg])
                for _ in range(first, last - 1):
                    ctx.rk_step(dt, want_dt=False)
                    states.append(ctx.get_state())
            for s in range(last - 1, first - 1, -1):
                lam = ctx.rk_step_vjp(states[s - first], dt, lam)
    ctx.set_state(Uf)
    return lam, Uf
