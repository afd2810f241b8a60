"""Thin Python binding of libstc (include/stc.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts numpy
arrays to the C ABI's fp64 host buffers and back.  It raises if libstc.so is
missing -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstc.so")

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
P_double = ctypes.POINTER(ctypes.c_double)
P_int = ctypes.POINTER(ctypes.c_int)

FIELDS = dict(V=0, PBAR=1, U=2, P=3, RES_V=4, RES_PBAR=5, RES_U=6, RES_P=7, Z=8, VSTAR=9, LAMBDA=10,
              RHO=11, MU=12, W=13, Y=14, KKT_U=15, KKT_G=16, MTERM=17, RES_IN_V=18, RES_IN_PBAR=19,
              RES_IN_U=20, RES_IN_P=21, XOLD_V=22, XOLD_PBAR=23, XOLD_U=24, XOLD_P=25,
              SIM_GRAD_RHO=26, SIM_GRAD_U=27, SIM_ADJ_V0=28, SIM_ADJ_RHO0=29, SIM_ADJ_VN=30)

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "DIVERGED",
          6: "UNSUPPORTED", 7: "BUSY"}


class StcParams(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("num_steps", c_int), ("dt", c_double), ("r", c_double),
                ("K", c_double), ("beta", c_double), ("precision", c_int), ("ao_iters", c_int),
                ("pre", c_int), ("post", c_int), ("coarse_sweeps", c_int), ("coarsest_n", c_int),
                ("taylor_tol", c_double), ("taylor_kmax", c_int), ("eps_stfas", c_double),
                ("eps_admm", c_double), ("max_vcycles", c_int), ("metric_levels", c_int),
                ("metric_sigma0", c_double), ("scgs_omega", c_double), ("lm_shift", c_double),
                ("poisson_vcycles", c_int), ("self_advection", c_int), ("ao_halvings", c_int),
                ("cgc_guard", c_int), ("lm_adapt", c_int), ("al_threshold", c_double), ("time_coarsen", c_int),
                ("nz", c_int), ("boundary", c_int), ("scgs_cta_cells", c_int),
                ("ao_trials", c_int), ("k_adapt", c_int)]


class StcReport(ctypes.Structure):
    _fields_ = [("admm_iters", c_int), ("vcycles", c_int), ("kkt_rel", c_double), ("kkt_abs", c_double),
                ("f_inf", c_double), ("drho", c_double), ("seconds", c_double),
                ("seconds_to_1e4", c_double), ("rejected_vcycles", c_int), ("lm_shift", c_double),
                ("density_stop_iter", c_int), ("seconds_to_density_stop", c_double), ("objective", c_double),
                ("lambda_updates", c_int), ("seconds_to_1e2", c_double), ("seconds_to_1e3", c_double),
                ("seconds_to_1e6", c_double), ("K_final", c_double)]


class ServerParams(ctypes.Structure):
    _fields_ = [("budget_bytes", c_size_t), ("workers", c_int), ("backend", c_int), ("device", c_int),
                ("max_bypass", c_int), ("mode", c_int), ("stream", c_void_p), ("max_resident", c_int),
                ("kkt_rel_tol", c_double), ("max_admm", c_int)]


class Request(ctypes.Structure):
    _fields_ = [("params", ctypes.POINTER(StcParams)), ("rho0", P_double), ("v0", P_double),
                ("nkeys", c_int), ("key_steps", P_int), ("key_rho", P_double), ("key_c", P_double),
                ("kkt_rel_tol", c_double), ("max_admm", c_int), ("sim_seconds", c_double),
                ("sim_status", c_int)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("state", c_int), ("status", c_int), ("bytes", c_size_t), ("t_submit", c_double),
                ("t_admit", c_double), ("t_done", c_double), ("report", StcReport),
                ("error", ctypes.c_char * 160)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", c_int), ("running", c_int), ("done", c_int), ("failed", c_int),
                ("cancelled", c_int), ("bytes_in_use", c_size_t), ("peak_bytes", c_size_t)]


P_server = c_void_p
P_ll = ctypes.POINTER(ctypes.c_longlong)

# name -> (restype, argtypes)
SIGNATURES = {
    "stc_default_params": (None, [ctypes.POINTER(StcParams), c_int, c_int, c_int]),
    "stc_create_problem": (c_int, [ctypes.POINTER(StcParams), P_double, P_double, c_void_p,
                                   ctypes.POINTER(c_void_p)]),
    "stc_set_keyframes": (c_int, [c_void_p, c_int, P_int, P_double, P_double]),
    "stc_vcycle": (c_int, [c_void_p, c_int, P_double]),
    "stc_solve": (c_int, [c_void_p, c_double, c_int, ctypes.POINTER(StcReport)]),
    "stc_get_forces": (c_int, [c_void_p, P_double, c_size_t]),
    "stc_get_density": (c_int, [c_void_p, P_double, c_size_t]),
    "stc_get_velocity": (c_int, [c_void_p, P_double, c_size_t]),
    "stc_destroy_problem": (c_int, [c_void_p]),
    "stc_last_error": (ctypes.c_char_p, []),
    "stc_get_field": (c_int, [c_void_p, c_int, c_int, P_double, c_size_t]),
    "stc_set_field": (c_int, [c_void_p, c_int, c_int, P_double, c_size_t]),
    "stc_level_info": (c_int, [c_void_p, P_int, c_int, P_int, P_int]),
    "stc_level_steps": (c_int, [c_void_p, c_int, P_int, P_double]),
    "stc_level_dims": (c_int, [c_void_p, c_int, P_int, P_int, P_int]),
    "stc_simulate": (c_int, [c_void_p, c_double, c_int, P_int]),
    "stc_simulate_adjoint": (c_int, [c_void_p, c_double, c_int, c_int, P_int]),
    "stc_copy_field_device": (c_int, [c_void_p, c_int, c_int, c_void_p, c_size_t, c_int, c_int, c_double]),
    "stc_advect": (c_int, [c_void_p, c_int]),
    "stc_get_taylor_orders": (c_int, [c_void_p, P_int, c_size_t]),
    "stc_metric_terms": (c_int, [c_void_p]),
    "stc_adjoint": (c_int, [c_void_p, c_int, c_double, c_double]),
    "stc_project": (c_int, [c_void_p, c_int, c_int, c_int]),
    "stc_ao": (c_int, [c_void_p, c_int, c_int]),
    "stc_ao_trace": (c_int, [c_void_p, P_int, c_size_t, P_int]),
    "stc_prepare_targets": (c_int, [c_void_p]),
    "stc_nso_residual": (c_int, [c_void_p, c_int, P_double]),
    "stc_smooth": (c_int, [c_void_p, c_int, c_int]),
    "stc_problem_bytes": (c_int, [ctypes.POINTER(StcParams), c_int, ctypes.POINTER(c_size_t)]),
    "stc_dct_tables": (c_int, [c_int, c_int, P_double, c_size_t]),
    "stc_server_default_params": (None, [ctypes.POINTER(ServerParams), c_size_t]),
    "stc_server_create": (c_int, [ctypes.POINTER(ServerParams), ctypes.POINTER(c_void_p)]),
    "stc_server_submit": (c_int, [P_server, ctypes.POINTER(Request), P_ll]),
    "stc_server_submit_problem": (c_int, [P_server, c_void_p, P_ll]),
    "stc_server_step": (c_int, [P_server, P_int]),
    "stc_server_poll": (c_int, [P_server, ctypes.c_longlong, ctypes.POINTER(TicketInfo)]),
    "stc_server_wait": (c_int, [P_server, ctypes.c_longlong, c_double, ctypes.POINTER(TicketInfo)]),
    "stc_server_cancel": (c_int, [P_server, ctypes.c_longlong]),
    "stc_server_get_forces": (c_int, [P_server, ctypes.c_longlong, P_double, c_size_t]),
    "stc_server_release": (c_int, [P_server, ctypes.c_longlong]),
    "stc_server_stats_get": (c_int, [P_server, ctypes.POINTER(ServerStats)]),
    "stc_server_destroy": (c_int, [P_server]),
    "stc_nso_solve": (c_int, [c_void_p, c_double, c_int, P_int, P_double]),
    "stc_lm_info": (c_int, [c_void_p, P_double, P_int]),
    "stc_restrict": (c_int, [c_void_p, c_int]),
    "stc_prolong_correct": (c_int, [c_void_p, c_int]),
    "stc_kkt_residual": (c_int, [c_void_p, P_double]),
    "stc_admm_update": (c_int, [c_void_p, P_double]),
    "stc_set_penalty": (c_int, [c_void_p, c_double, c_double]),
    "stc_solve_history": (c_int, [c_void_p, P_double, c_size_t, P_int]),
    "stc_solve_begin": (c_int, [c_void_p, c_double, c_int]),
    "stc_solve_phase": (c_int, [c_void_p, P_int, P_int]),
    "stc_solve_head": (c_int, [c_void_p]),
    "stc_solve_tail": (c_int, [c_void_p]),
    "stc_solve_report": (c_int, [c_void_p, ctypes.POINTER(StcReport), P_int]),
    "stc_batch_create": (c_int, [c_void_p, ctypes.POINTER(c_void_p)]),
    "stc_batch_nso_cycle": (c_int, [c_void_p, ctypes.POINTER(c_void_p), c_int, P_int, P_int]),
    "stc_batch_destroy": (c_int, [c_void_p]),
    "stc_launch_count": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "stc_set_kernel_timing": (c_int, [c_void_p, c_int]),
    "stc_kernel_timing": (c_int, [c_void_p, P_double, ctypes.POINTER(ctypes.c_longlong)]),
    "stc_kernel_timing_of": (c_int, [c_void_p, c_int, P_double, ctypes.POINTER(ctypes.c_longlong)]),
    "stc_measure_fp32_peak": (c_int, [c_void_p, P_double]),
    "stc_memory_bytes": (c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "stc_adjoint_sweep_noalloc": (c_int, [c_int, c_int, c_int, c_double, c_int, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_double, c_double, c_void_p,
                                          c_void_p]),
}

_lib = None


def load(path=None):
    """Load libstc.so (built by ``paper_1608_01102_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libstc.so not built (%s): run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class StcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def _check(code):
    if code != 0:
        raise StcError(code, load().stc_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(P_double)


def grid_sizes(nx, ny, nz=0):
    """(faces, cells) of the 2D grid nx x ny (nz = 0) or the 3D grid nx x ny x nz."""
    if nz:
        return nz * ny * (nx + 1) + nz * (ny + 1) * nx + (nz + 1) * ny * nx, nx * ny * nz
    return ny * (nx + 1) + (ny + 1) * nx, nx * ny


def default_params(nx, ny, N, **overrides):
    p = StcParams()
    load().stc_default_params(ctypes.byref(p), nx, ny, N)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Problem:
    """One control problem resident on the current CUDA device."""

    def __init__(self, params, rho0, v0=None, stream=None):
        self.lib = load()
        self.params = params
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64).ravel()
        v0p = None
        if v0 is not None:
            self._v0 = np.ascontiguousarray(v0, dtype=np.float64).ravel()
            v0p = _dptr(self._v0)
        h = c_void_p()
        st = c_void_p(int(stream)) if stream is not None else None
        _check(self.lib.stc_create_problem(ctypes.byref(params), _dptr(rho0), v0p, st, ctypes.byref(h)))
        self.h = h
        self.nx, self.ny, self.N = params.nx, params.ny, params.num_steps
        self.nz = params.nz

    # sizes --------------------------------------------------------------
    def level_shape(self, level):
        """(nx, ny) of a 2D level, (nx, ny, nz) of a 3D one."""
        nx, ny, nz = c_int(), c_int(), c_int()
        _check(self.lib.stc_level_dims(self.h, level, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(nz)))
        return (nx.value, ny.value, nz.value) if nz.value else (nx.value, ny.value)

    def num_levels(self):
        nl = c_int()
        _check(self.lib.stc_level_info(self.h, ctypes.byref(nl), 0, None, None))
        return nl.value

    def level_steps(self, level=0):
        n, dt = c_int(), c_double()
        _check(self.lib.stc_level_steps(self.h, level, ctypes.byref(n), ctypes.byref(dt)))
        return n.value, dt.value

    def field_shape(self, name, level=0):
        F, C = grid_sizes(*self.level_shape(level))
        N = self.level_steps(level)[0] if level > 0 else self.N
        face_np1 = ("V", "RES_V", "RES_IN_V", "XOLD_V", "KKT_G")
        cell_np1 = ("PBAR", "RES_PBAR", "RES_IN_PBAR", "XOLD_PBAR", "RHO", "MTERM", "SIM_GRAD_RHO")
        face_n = ("U", "RES_U", "RES_IN_U", "XOLD_U", "Z", "VSTAR", "LAMBDA", "W", "Y", "KKT_U", "SIM_GRAD_U")
        cell_n = ("P", "RES_P", "RES_IN_P", "XOLD_P", "MU")
        if name in ("SIM_ADJ_V0", "SIM_ADJ_VN"):
            return (1, F)
        if name == "SIM_ADJ_RHO0":
            return (1, C)
        if name in face_np1:
            return (N + 1, F)
        if name in cell_np1:
            return (N + 1, C)
        if name in face_n:
            return (N, F)
        if name in cell_n:
            return (N, C)
        raise KeyError(name)

    # field access -----------------------------------------------------------
    def get(self, name, level=0):
        shape = self.field_shape(name, level)
        out = np.empty(shape, dtype=np.float64)
        _check(self.lib.stc_get_field(self.h, FIELDS[name], level, _dptr(out), out.size))
        return out

    def set(self, name, arr, level=0):
        shape = self.field_shape(name, level)
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(shape)
        _check(self.lib.stc_set_field(self.h, FIELDS[name], level, _dptr(a), a.size))

    def set_state(self, x, level=0):
        for k, name in (("v", "V"), ("pbar", "PBAR"), ("u", "U"), ("p", "P")):
            self.set(name, x[k], level)

    def get_state(self, level=0, prefix=""):
        return {k: self.get(prefix + name, level)
                for k, name in (("v", "V"), ("pbar", "PBAR"), ("u", "U"), ("p", "P"))}

    # method steps -------------------------------------------------------------
    def set_keyframes(self, keyframes):
        """keyframes: dict step -> (rho_star (C,), c)."""
        steps = sorted(keyframes)
        st = (c_int * len(steps))(*steps)
        stars = np.ascontiguousarray(np.array([keyframes[s][0] for s in steps]).reshape(len(steps), -1),
                                     dtype=np.float64)
        cs = np.array([keyframes[s][1] for s in steps], dtype=np.float64)
        _check(self.lib.stc_set_keyframes(self.h, len(steps), st, _dptr(stars), _dptr(cs)))

    def vcycle(self, n=1):
        f = c_double()
        _check(self.lib.stc_vcycle(self.h, n, ctypes.byref(f)))
        return f.value

    def solve(self, tol=1e-4, max_admm=50, allow_not_converged=True):
        rep = StcReport()
        code = self.lib.stc_solve(self.h, tol, max_admm, ctypes.byref(rep))
        if code != 0 and not (allow_not_converged and code == 4):
            _check(code)
        return {k: getattr(rep, k) for k, _ in StcReport._fields_}

    def solve_history(self):
        """[(kkt_rel, seconds, K)] per ADMM iteration of the last solve."""
        n = c_int()
        _check(self.lib.stc_solve_history(self.h, None, 0, ctypes.byref(n)))
        buf = np.zeros(3 * n.value)
        if n.value:
            _check(self.lib.stc_solve_history(self.h, _dptr(buf), buf.size, ctypes.byref(n)))
        return [tuple(buf[3 * k:3 * k + 3]) for k in range(n.value)]

    # the ADMM loop as resumable phases (stc_solve_begin / _head / _tail) ---------
    def solve_begin(self, tol=1e-4, max_admm=50):
        _check(self.lib.stc_solve_begin(self.h, tol, max_admm))

    def solve_phase(self):
        """(phase, wants_cycle): phase 0 = AO due, 1 = NSO cycles, 2 = finished."""
        ph, w = c_int(), c_int()
        _check(self.lib.stc_solve_phase(self.h, ctypes.byref(ph), ctypes.byref(w)))
        return ph.value, bool(w.value)

    def solve_head(self):
        _check(self.lib.stc_solve_head(self.h))

    def solve_tail(self):
        _check(self.lib.stc_solve_tail(self.h))

    def solve_report(self):
        rep, conv = StcReport(), c_int()
        _check(self.lib.stc_solve_report(self.h, ctypes.byref(rep), ctypes.byref(conv)))
        out = {k: getattr(rep, k) for k, _ in StcReport._fields_}
        out["converged"] = bool(conv.value)
        return out

    def advect(self, source="VSTAR"):
        _check(self.lib.stc_advect(self.h, FIELDS[source]))

    def taylor_orders(self):
        K = (c_int * self.N)()
        _check(self.lib.stc_get_taylor_orders(self.h, K, self.N))
        return np.array(list(K))

    def metric_terms(self):
        _check(self.lib.stc_metric_terms(self.h))

    def adjoint(self, source="VSTAR", alpha=1.0, beta=1.0):
        _check(self.lib.stc_adjoint(self.h, FIELDS[source], alpha, beta))

    def project(self, name, first, count):
        _check(self.lib.stc_project(self.h, FIELDS[name], first, count))

    def ao(self, iters=2, warm=False):
        _check(self.lib.stc_ao(self.h, iters, 1 if warm else 0))

    def ao_trace(self):
        buf = np.zeros(256, dtype=np.int32)
        n = c_int()
        _check(self.lib.stc_ao_trace(self.h, buf.ctypes.data_as(P_int), buf.size, ctypes.byref(n)))
        return [int(a) for a in buf[:min(n.value, buf.size)]]

    def prepare_targets(self):
        _check(self.lib.stc_prepare_targets(self.h))

    def nso_residual(self, level=0):
        f = c_double()
        _check(self.lib.stc_nso_residual(self.h, level, ctypes.byref(f)))
        return f.value

    def nso_solve(self, f_target, max_cycles=20):
        c = c_int()
        f = c_double()
        _check(self.lib.stc_nso_solve(self.h, f_target, max_cycles, ctypes.byref(c), ctypes.byref(f)))
        return f.value, c.value

    def lm_info(self):
        lm, rej = c_double(), c_int()
        _check(self.lib.stc_lm_info(self.h, ctypes.byref(lm), ctypes.byref(rej)))
        return lm.value, rej.value

    def smooth(self, level=0, sweeps=1):
        _check(self.lib.stc_smooth(self.h, level, sweeps))

    def restrict(self, level=0):
        _check(self.lib.stc_restrict(self.h, level))

    def prolong_correct(self, level=0):
        _check(self.lib.stc_prolong_correct(self.h, level))

    def kkt_residual(self):
        f = c_double()
        _check(self.lib.stc_kkt_residual(self.h, ctypes.byref(f)))
        return f.value

    def admm_update(self):
        f = c_double()
        _check(self.lib.stc_admm_update(self.h, ctypes.byref(f)))
        return f.value

    def set_penalty(self, K, beta=1.0):
        _check(self.lib.stc_set_penalty(self.h, K, beta))

    def forces(self):
        return self.get("U")

    # forward simulation and its adjoint ------------------------------------
    def simulate(self, tol=1e-6, max_iter=100):
        """stc_simulate: v_1..v_N and rho_1..rho_N from v_0, rho_0 and U;
        returns the Picard iterations used."""
        it = c_int()
        _check(self.lib.stc_simulate(self.h, tol, max_iter, ctypes.byref(it)))
        return it.value

    def simulate_adjoint(self, tol=1e-6, max_iter=100, with_step0=False):
        it = c_int()
        _check(self.lib.stc_simulate_adjoint(self.h, tol, max_iter, 1 if with_step0 else 0, ctypes.byref(it)))
        return it.value

    def copy_device(self, name, ptr, count, is_double, to_field, scale=1.0, level=0):
        """Device-to-device copy between a field and the buffer at device address ptr."""
        _check(self.lib.stc_copy_field_device(self.h, FIELDS[name], level, c_void_p(int(ptr)), count,
                                              1 if is_double else 0, 1 if to_field else 0, float(scale)))

    def launch_count(self):
        n = ctypes.c_longlong()
        _check(self.lib.stc_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def set_kernel_timing(self, on=True):
        _check(self.lib.stc_set_kernel_timing(self.h, 1 if on else 0))

    def kernel_timing(self, kind=0):
        """(summed ms, launches) of the timed finest-level launches: kind 0 =
        SCGS colour, 1 = colour residual."""
        ms, n = c_double(), ctypes.c_longlong()
        _check(self.lib.stc_kernel_timing_of(self.h, kind, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def taylor_kmax(self):
        return self.params.taylor_kmax

    def memory_bytes(self):
        b = c_size_t()
        _check(self.lib.stc_memory_bytes(self.h, ctypes.byref(b)))
        return b.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.stc_destroy_problem(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adjoint_sweep_noalloc(nx, ny, N, dt, taylor_kmax, vel, rho, K, mterm, mu, base, alpha, beta, out,
                          stream=None):
    """stc_adjoint_sweep_noalloc on device pointers (ints, e.g. tensor.data_ptr()).

    For callers that cannot allocate device memory at the call (a fixed,
    pre-reserved device-memory budget, or no tolerance for cudaMalloc's implicit
    synchronisation): the library allocates nothing here; its only scratch is a
    fixed 4 MiB device array shared by all calls, so overlapping calls race."""
    lib = load()
    vp = lambda p: c_void_p(int(p)) if p else None
    _check(lib.stc_adjoint_sweep_noalloc(nx, ny, N, dt, taylor_kmax, vp(vel), vp(rho), vp(K), vp(mterm), vp(mu),
                                         vp(base), alpha, beta, vp(out), vp(stream)))


class Batch:
    """stc_batch: NSO V-cycles of many problems in one CUDA graph launch."""

    def __init__(self, stream=None):
        self.lib = load()
        h = c_void_p()
        _check(self.lib.stc_batch_create(c_void_p(int(stream)) if stream else None, ctypes.byref(h)))
        self.h = h

    def nso_cycle(self, problems):
        """One V-cycle for every problem that wants one; returns (cycled, statuses)."""
        n = len(problems)
        arr = (c_void_p * max(n, 1))(*[p.h for p in problems])
        st = (c_int * max(n, 1))()
        c = c_int()
        _check(self.lib.stc_batch_nso_cycle(self.h, arr, n, ctypes.byref(c), st))
        return c.value, [int(st[k]) for k in range(n)]

    def close(self):
        if self.h:
            self.lib.stc_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_peak(stream=None):
    """stc_measure_fp32_peak: the device's FP32 FMA throughput in GFLOP/s."""
    g = c_double()
    _check(load().stc_measure_fp32_peak(c_void_p(int(stream)) if stream else None, ctypes.byref(g)))
    return g.value


def problem_bytes(params, nkeys=1):
    """Device bytes of a problem with these parameters and nkeys keyframes
    (stc_problem_bytes: host arithmetic, no device needed)."""
    b = c_size_t()
    _check(load().stc_problem_bytes(ctypes.byref(params), nkeys, ctypes.byref(b)))
    return b.value


def dct_tables(nx, ny):
    """The exact 2D projection's tables (stc_dct_tables: host arithmetic, no
    device needed): dict with Cx, CxT, Cy, CyT (square) and inv_lam (ny x nx)."""
    n = 2 * nx * nx + 2 * ny * ny + nx * ny
    out = np.zeros(n)
    _check(load().stc_dct_tables(nx, ny, out.ctypes.data_as(P_double), n))
    sizes = [("Cx", (nx, nx)), ("CxT", (nx, nx)), ("Cy", (ny, ny)), ("CyT", (ny, ny)), ("inv_lam", (ny, nx))]
    res, o = {}, 0
    for name, shp in sizes:
        k = shp[0] * shp[1]
        res[name] = out[o:o + k].reshape(shp)
        o += k
    return res


TICKET_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


def _info_dict(info):
    d = {k: getattr(info, k) for k, _ in TicketInfo._fields_ if k not in ("report", "error")}
    d["state"] = TICKET_STATES[info.state]
    d["report"] = {k: getattr(info.report, k) for k, _ in StcReport._fields_}
    d["error"] = info.error.decode(errors="replace")
    return d


class Server:
    """Serving many control problems on one device (include/stc_server.h)."""

    def __init__(self, budget_bytes, workers=8, backend=0, device=0, max_bypass=8, mode=0, stream=None,
                 max_resident=16, tol=1e-4, max_admm=50):
        """mode 0: worker threads; mode 1: stepped (step() runs one batched step)."""
        self.lib = load()
        sp = ServerParams()
        self.lib.stc_server_default_params(ctypes.byref(sp), int(budget_bytes))
        sp.workers, sp.backend, sp.device, sp.max_bypass = workers, backend, device, max_bypass
        sp.mode, sp.max_resident, sp.kkt_rel_tol, sp.max_admm = mode, max_resident, tol, max_admm
        sp.stream = c_void_p(int(stream)) if stream else None
        h = c_void_p()
        _check(self.lib.stc_server_create(ctypes.byref(sp), ctypes.byref(h)))
        self.h = h
        self._sizes = {}

    def submit(self, params, rho0, keyframes=None, v0=None, tol=1e-4, max_admm=50, sim_seconds=0.0,
               sim_status=0):
        """keyframes: dict step -> (rho_star, c).  Returns the ticket."""
        keyframes = keyframes or {}
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64).ravel()
        steps = sorted(keyframes)
        ks = np.array(steps, dtype=np.int32)
        kr = np.ascontiguousarray(np.array([keyframes[k][0] for k in steps], dtype=np.float64).reshape(-1))
        kc = np.array([keyframes[k][1] for k in steps], dtype=np.float64)
        v0a = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64).ravel()
        rq = Request()
        rq.params = ctypes.pointer(params)
        rq.rho0 = _dptr(rho0)
        rq.v0 = _dptr(v0a) if v0a is not None else None
        rq.nkeys = len(steps)
        rq.key_steps = ks.ctypes.data_as(P_int) if steps else None
        rq.key_rho = _dptr(kr) if steps else None
        rq.key_c = _dptr(kc) if steps else None
        rq.kkt_rel_tol, rq.max_admm = tol, max_admm
        rq.sim_seconds, rq.sim_status = sim_seconds, sim_status
        t = ctypes.c_longlong()
        _check(self.lib.stc_server_submit(self.h, ctypes.byref(rq), ctypes.byref(t)))
        F = grid_sizes(params.nx, params.ny, params.nz)[0]
        self._sizes[t.value] = (params.num_steps, F)
        return t.value

    def submit_problem(self, problem):
        """Mode 1: queue a Problem created on the server's stream (not destroyed by the server)."""
        t = ctypes.c_longlong()
        _check(self.lib.stc_server_submit_problem(self.h, problem.h, ctypes.byref(t)))
        self._sizes[t.value] = (problem.N, problem.field_shape("U")[1])
        return t.value

    def step(self):
        """Mode 1: one serving step; returns the problems resident or queued after it."""
        a = c_int()
        _check(self.lib.stc_server_step(self.h, ctypes.byref(a)))
        return a.value

    def poll(self, ticket):
        info = TicketInfo()
        _check(self.lib.stc_server_poll(self.h, ticket, ctypes.byref(info)))
        return _info_dict(info)

    def wait(self, ticket, timeout=-1.0):
        info = TicketInfo()
        _check(self.lib.stc_server_wait(self.h, ticket, float(timeout), ctypes.byref(info)))
        return _info_dict(info)

    def cancel(self, ticket):
        _check(self.lib.stc_server_cancel(self.h, ticket))

    def forces(self, ticket):
        N, F = self._sizes[ticket]
        out = np.zeros((N, F))
        _check(self.lib.stc_server_get_forces(self.h, ticket, _dptr(out), out.size))
        return out

    def release(self, ticket):
        _check(self.lib.stc_server_release(self.h, ticket))
        self._sizes.pop(ticket, None)

    def stats(self):
        st = ServerStats()
        _check(self.lib.stc_server_stats_get(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self.lib.stc_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
