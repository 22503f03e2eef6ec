"""Thin ctypes binding of librbc.so (the C ABI declared in include/rbc.h).

Argument marshalling only: every step of the propagator, the Parareal update and
the norms runs in the CUDA library.  PyTorch provides device memory and streams.
There is no CPU fallback: if the library is missing, every entry point raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbc.so")

RBC_OK, RBC_EINVAL, RBC_ENOMEM, RBC_ECUDA, RBC_EDIVERGED, RBC_ETIMEOUT, RBC_ENOTCONVERGED = 0, -1, -2, -3, -4, -5, 1
RBC_FP64, RBC_MIXED, RBC_MIXED_BF16 = 0, 1, 2
RBC_FIXED_T, RBC_FIXED_FLUX = 0, 1
RBC_RK443, RBC_RK222, RBC_RK111 = 0, 1, 2
CRIT_FIXED, CRIT_DEFECT, CRIT_NU, CRIT_STAT = 0, 1, 2, 3

EXPORTS = [
    "rbc_last_error", "rbc_create", "rbc_destroy", "rbc_state_bytes", "rbc_workspace_bytes_per_state",
    "rbc_reserve", "rbc_set_state", "rbc_get_state", "rbc_step_batch", "rbc_check_diverged", "rbc_nusselt",
    "rbc_l2_temperature", "parareal_create", "parareal_destroy", "parareal_iterate", "rbc_profile",
    "rbc_profile_read", "rbc_launch_count", "rbc_nusselt_static", "rbc_step_batch_ra", "rbc_restrict",
    "rbc_prolong", "rbc_parareal_correct", "rbc_l2_diff", "parareal_set_schedule", "parareal_coarse_sms",
    "rbc_diag_size", "rbc_diagnostics", "rbc_set_wait_limit", "parareal_set_depth",
    "rbc_step_batch_sampled", "rbc_stat_summary", "parareal_set_sampling", "parareal_stat_means",
    "rbc_autotune", "rbc_tuned_shapes", "rbc_set_shapes",
]
KERNEL_NAMES = ["k_zinv", "k_rows", "k_zfwd", "k_solve"]


class RBCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rbc status {status}: {msg}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("bc", ctypes.c_int), ("eager", ctypes.c_int),
                ("scheme", ctypes.c_int)]


_lib = None


def load():
    """Load librbc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: build it with paper_2001_01609_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    PD, PI = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    sig = {
        "rbc_last_error": (ctypes.c_char_p, []),
        "rbc_create": (I, [D, D, D, I, I, D, ctypes.POINTER(_Opts), ctypes.POINTER(P)]),
        "rbc_destroy": (None, [P]),
        "rbc_state_bytes": (S, [P]),
        "rbc_workspace_bytes_per_state": (S, [P]),
        "rbc_reserve": (I, [P, I]),
        "rbc_set_state": (I, [P, P, PD, PD, PD]),
        "rbc_get_state": (I, [P, P, PD, PD, PD]),
        "rbc_step_batch": (I, [P, P, I, PI, P, P]),
        "rbc_check_diverged": (I, [P, P]),
        "rbc_nusselt": (I, [P, P, PD, P]),
        "rbc_l2_temperature": (I, [P, P, PD, P]),
        "parareal_create": (I, [P, P, D, D, I, I, D, ctypes.POINTER(P)]),
        "parareal_destroy": (None, [P]),
        "parareal_iterate": (I, [P, P, P, I, PI, PD, PD, P]),
        "rbc_profile": (I, [P, I]),
        "rbc_profile_read": (I, [P, PD, ctypes.POINTER(ctypes.c_longlong), PD, PD]),
        "rbc_launch_count": (ctypes.c_ulonglong, []),
        "rbc_nusselt_static": (I, [P, P, PD, P]),
        "rbc_step_batch_ra": (I, [P, P, I, PI, PD, P, P]),
        "rbc_restrict": (I, [P, P, P, P, I, P]),
        "rbc_prolong": (I, [P, P, P, P, I, P]),
        "rbc_parareal_correct": (I, [P, P, P, P, P, P, I, P]),
        "rbc_l2_diff": (I, [P, P, P, I, P, P]),
        "parareal_set_schedule": (I, [P, I, I, I, I, I]),
        "parareal_coarse_sms": (I, [P]),
        "rbc_diag_size": (S, [P]),
        "rbc_diagnostics": (I, [P, P, I, P, P]),
        "rbc_set_wait_limit": (I, [ctypes.c_longlong]),
        "parareal_set_depth": (I, [P, I]),
        "rbc_step_batch_sampled": (I, [P, P, I, I, I, P, P, P]),
        "rbc_stat_summary": (I, [I, D, D, PD, PD]),
        "parareal_set_sampling": (I, [P, I, I]),
        "parareal_stat_means": (I, [P, PD]),
        "rbc_autotune": (I, [P, I, PD, P]),
        "rbc_tuned_shapes": (I, [P, I, PI]),
        "rbc_set_shapes": (I, [P, I, PI]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status, allow=()):
    if status != RBC_OK and status not in allow:
        raise RBCError(status, load().rbc_last_error().decode())
    return status


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


class Propagator:
    """F (or G) of Eq. 20 on one grid: rbc_create(Ra, Pr, Lx, Nx, Nz, dt)."""

    def __init__(self, Ra, Pr, Lx, Nx, Nz, dt, precision=RBC_FP64, eager=False, bc=RBC_FIXED_T,
                 scheme=RBC_RK443):
        """bc: RBC_FIXED_T (Eq. 6) or RBC_FIXED_FLUX (Eq. 7, Ra = Ra_f of Eq. 8);
        scheme: RBC_RK443, or the lower-order RBC_RK222 / RBC_RK111 (Sec. 3.6)."""
        lib = load()
        self.Ra, self.Pr, self.Lx, self.Nx, self.Nz, self.dt = Ra, Pr, Lx, Nx, Nz, dt
        self.precision, self.bc, self.scheme = precision, bc, scheme
        h = ctypes.c_void_p()
        opts = _Opts(precision, bc, 1 if eager else 0, scheme)
        _check(lib.rbc_create(Ra, Pr, Lx, Nx, Nz, dt, ctypes.byref(opts), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().rbc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def state_shape(self):
        return (2, self.Nz, self.Nx // 2, 2)

    @property
    def state_bytes(self):
        return load().rbc_state_bytes(self.h)

    @property
    def workspace_bytes_per_state(self):
        return load().rbc_workspace_bytes_per_state(self.h)

    def new_states(self, B, device="cuda"):
        import torch
        return torch.zeros((B,) + self.state_shape, dtype=torch.float64, device=device)

    def reserve(self, B):
        _check(load().rbc_reserve(self.h, B))

    def set_state(self, state, T, u=None, w=None):
        T = np.ascontiguousarray(T, dtype=np.float64)
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        _check(load().rbc_set_state(self.h, _ptr(state), _dptr(T), _dptr(u), _dptr(w)))

    def get_state(self, state):
        shp = (self.Nz, self.Nx)
        T, u, w = np.empty(shp), np.empty(shp), np.empty(shp)
        _check(load().rbc_get_state(self.h, _ptr(state), _dptr(T), _dptr(u), _dptr(w)))
        return T, u, w

    def step_batch(self, states, nsteps, nu=None, stream=None, ra=None):
        """Advance states (B, *state_shape) in place; nsteps int or sequence of B ints.

        ra: optional Rayleigh number per state (sequence of B floats).
        """
        B = states.shape[0]
        ns = np.full(B, nsteps, dtype=np.int32) if np.isscalar(nsteps) else np.ascontiguousarray(nsteps, np.int32)
        assert ns.shape == (B,)
        nup = _ptr(nu) if nu is not None else None
        nsp = ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        if ra is None:
            _check(load().rbc_step_batch(self.h, _ptr(states), B, nsp, nup, _stream(stream)))
        else:
            rr = np.ascontiguousarray(ra, dtype=np.float64)
            assert rr.shape == (B,)
            _check(load().rbc_step_batch_ra(self.h, _ptr(states), B, nsp, _dptr(rr), nup, _stream(stream)))

    def check_diverged(self, stream=None):
        """RBC_OK, RBC_EDIVERGED (a non-finite state) or RBC_ETIMEOUT (a bounded
        device-side wait gave up) since the last check."""
        return _check(load().rbc_check_diverged(self.h, _stream(stream)), allow=(RBC_EDIVERGED, RBC_ETIMEOUT))

    def nusselt(self, state, stream=None):
        out = np.zeros(3)
        _check(load().rbc_nusselt(self.h, _ptr(state), _dptr(out), _stream(stream)))
        return tuple(out)

    def profile(self, enable=True, sample=False):
        """Per-kernel CUDA-event timing: all calls, or the next rbc_step_batch call only."""
        _check(load().rbc_profile(self.h, (2 if sample else 1) if enable else 0))

    def profile_read(self):
        K = len(KERNEL_NAMES)
        ms, fl, by = np.zeros(K), np.zeros(K), np.zeros(K)
        n = (ctypes.c_longlong * K)()
        _check(load().rbc_profile_read(self.h, _dptr(ms), n, _dptr(fl), _dptr(by)))
        return {KERNEL_NAMES[k]: dict(ms=ms[k], launches=n[k], flops=fl[k], bytes=by[k]) for k in range(K)}

    @property
    def diag_size(self):
        """Doubles per state written by diagnostics(): 6 + 2 Mz."""
        return load().rbc_diag_size(self.h)

    def diagnostics(self, states, out=None, stream=None):
        """rbc_diagnostics: Sec. 2.2 averages of states (B, *state_shape) into a
        (B, diag_size) FP64 device tensor, asynchronously on the stream.

        Columns: <u^2+w^2>_V, <u.lap u>_V, <wT>_V, Nu_V, Nu_b, Nu_t, then <T>_x and
        <(T - <T>_x)^2>_x at the Mz padded points z_j = cos(pi j/(Mz-1))/2.
        """
        import torch
        B = states.shape[0]
        if out is None:
            out = torch.empty((B, self.diag_size), dtype=torch.float64, device=states.device)
        assert out.shape == (B, self.diag_size) and out.dtype == torch.float64 and out.is_contiguous()
        _check(load().rbc_diagnostics(self.h, _ptr(states), B, _ptr(out), _stream(stream)))
        return out

    def step_batch_sampled(self, states, nsteps, every, stat=None, nu=None, stream=None):
        """rbc_step_batch_sampled: advance by nsteps with the Sec. 2.2 averages
        sampled every `every` steps; returns the (B, diag_size) device tensor of
        their trapezoid time integrals."""
        import torch
        B = states.shape[0]
        if stat is None:
            stat = torch.empty((B, self.diag_size), dtype=torch.float64, device=states.device)
        assert stat.shape == (B, self.diag_size) and stat.is_contiguous()
        _check(load().rbc_step_batch_sampled(self.h, _ptr(states), B, int(nsteps), int(every),
                                             _ptr(nu) if nu is not None else None, _ptr(stat), _stream(stream)))
        return stat

    def autotune(self, B, stream=None):
        """rbc_autotune: pick launch shapes for batches of B states (same results,
        timing only); returns (ms per step with the heuristics, with the pick)."""
        out = np.zeros(2)
        _check(load().rbc_autotune(self.h, int(B), _dptr(out), _stream(stream)))
        return float(out[0]), float(out[1])

    def tuned_shapes(self, B):
        """(solve modes, z-forward modes, z-forward chunks, clustered rows, row threads,
        lean row layout) kept for B."""
        out = (ctypes.c_int * 6)()
        _check(load().rbc_tuned_shapes(self.h, int(B), out))
        return tuple(out)

    def set_shapes(self, B, shapes):
        """rbc_set_shapes: keep these six launch shapes for batches of B states."""
        arr = (ctypes.c_int * 6)(*[int(v) for v in shapes])
        _check(load().rbc_set_shapes(self.h, int(B), arr))

    def l2_temperature(self, state, stream=None):
        out = np.zeros(1)
        _check(load().rbc_l2_temperature(self.h, _ptr(state), _dptr(out), _stream(stream)))
        return float(out[0])


def restrict(fine, coarse, fine_states, coarse_states, stream=None):
    _check(load().rbc_restrict(fine.h, coarse.h, _ptr(fine_states), _ptr(coarse_states), fine_states.shape[0],
                               _stream(stream)))


def prolong(fine, coarse, coarse_states, fine_states, stream=None):
    _check(load().rbc_prolong(fine.h, coarse.h, _ptr(coarse_states), _ptr(fine_states), coarse_states.shape[0],
                              _stream(stream)))


def parareal_correct(fine, coarse, F, Gnew, Gold, U, stream=None):
    """U = F + (prolong(Gnew) - prolong(Gold)) for B states (Eq. 20)."""
    _check(load().rbc_parareal_correct(fine.h, coarse.h, _ptr(F), _ptr(Gnew), _ptr(Gold), _ptr(U), F.shape[0],
                                       _stream(stream)))


def l2_diff(prop, A, Bm, out, stream=None):
    """out[b] = ||A[b] - Bm[b]||^2 (temperature, L2 over the domain); Bm may be None."""
    _check(load().rbc_l2_diff(prop.h, _ptr(A), _ptr(Bm) if Bm is not None else None, A.shape[0], _ptr(out),
                              _stream(stream)))


def set_wait_limit(polls):
    """Test hook: polls before a tensor-core mbarrier wait gives up (0: at once;
    negative: the default), on the current device."""
    _check(load().rbc_set_wait_limit(int(polls)))


STAT_SUMMARY = ("U", "Re", "NuV", "Nub", "Nut", "Nu_int", "P", "eps_U", "balance", "delta_t", "delta_T", "N_BL")


def stat_summary(Nz, Ra, Pr, means):
    """rbc_stat_summary: the Sec. 2.2 quantities from time means (6 + 2 Mz values):
    a dict of STAT_SUMMARY plus "Trms" (Mz values at the padded points)."""
    m = np.ascontiguousarray(means, dtype=np.float64)
    Mz = 3 * Nz // 2
    assert m.shape == (6 + 2 * Mz,)
    out = np.zeros(12 + Mz)
    _check(load().rbc_stat_summary(int(Nz), float(Ra), float(Pr), _dptr(m), _dptr(out)))
    d = {k: float(out[i]) for i, k in enumerate(STAT_SUMMARY)}
    d["N_BL"] = int(out[11])
    d["Trms"] = out[12:].copy()
    return d


def launch_count():
    return int(load().rbc_launch_count())


def coarse_dt(slice_length, dt_requested):
    """Largest dt <= dt_requested dividing the slice into whole steps (ceil the count)."""
    n = int(np.ceil(slice_length / dt_requested - 1e-9))
    return slice_length / n, n


class Parareal:
    """Parareal (Eq. 20) over [t0, t1] with nslices slices of F = fine, G = coarse."""

    def __init__(self, fine, coarse, t0, t1, nslices, criterion=CRIT_FIXED, tol=0.0):
        lib = load()
        self.fine, self.coarse, self.nslices = fine, coarse, nslices
        self.t0, self.t1 = t0, t1
        h = ctypes.c_void_p()
        _check(lib.parareal_create(fine.h, coarse.h, t0, t1, nslices, criterion, tol, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().parareal_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, group, first_group=None, fine_streams=2, coarse_priority=1, coarse_sms=0):
        """Fine group sizes, fine streams, coarse-stream priority and an optional SM
        partition for the coarse sweeps, of the overlapped schedule (timing only)."""
        fg = group if first_group is None else first_group
        _check(load().parareal_set_schedule(self.h, group, fg, fine_streams, coarse_priority, coarse_sms))

    def set_sampling(self, every, window_first=None):
        """Sample the Sec. 2.2 averages every `every` fine steps (and at slice
        ends) over the window of slices [window_first, nslices)."""
        wf = self.nslices // 2 if window_first is None else window_first
        _check(load().parareal_set_sampling(self.h, int(every), int(wf)))

    def stat_means(self):
        """Window means (6 + 2 Mz) of the last evaluated iteration."""
        out = np.zeros(6 + 2 * (3 * self.fine.Nz // 2))
        _check(load().parareal_stat_means(self.h, _dptr(out)))
        return out

    def set_depth(self, depth):
        """Iterations kept enqueued beyond the one being evaluated (0..6, timing only)."""
        _check(load().parareal_set_depth(self.h, depth))

    @property
    def coarse_sms(self):
        return load().parareal_coarse_sms(self.h)

    def set_group(self, group):
        """Equal fine groups of `group` slices on one stream, no partition."""
        self.set_schedule(group, group, 1, 0, 0)

    def iterate(self, U0, U, max_iters, stream=None):
        """Returns (status, k_done, defects[k], nus[k]); U (nslices+1 states) receives U^k."""
        k = ctypes.c_int(0)
        de = np.zeros(max_iters)
        nu = np.zeros(max_iters)
        st = load().parareal_iterate(self.h, _ptr(U0), _ptr(U), max_iters, ctypes.byref(k), _dptr(de), _dptr(nu),
                                     _stream(stream))
        _check(st, allow=(RBC_ENOTCONVERGED, RBC_EDIVERGED, RBC_ETIMEOUT))
        return st, k.value, de[: k.value], nu[: k.value]
