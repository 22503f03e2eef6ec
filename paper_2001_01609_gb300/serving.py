"""Serving many Parareal runs on one GPU: admission by device memory and
continuous batching of their fine and coarse sweeps (Sec. 3.1, Eq. 20).

Every request is one Parareal run: its own Rayleigh number, grid, number of
time slices and precision.  Requests that share a grid and a precision form a
class; a class owns one fine and one coarse propagator handle (their
operators do not depend on Ra, which is passed per state), a fine stream and a
coarse stream, and staging buffers for the batches.

Per request the work is the same sequence of library calls as
`parareal_iterate`: the coarse sweep U^0, then per iteration k the fine sweep
on slices n >= k-1, the serial correction sweep
U_{n+1}^k = F(U_n^{k-1}) + (G(U_n^k) - G(U_n^{k-1})), the relative L2 defect of
T and the Nu_V time average over the second half of the slices.  What differs
is how the calls are grouped:

* fine sweeps of all requests of a class that are in their fine phase are
  gathered into one staging batch and advanced together, `f_chunk` steps per
  launch, so that a request can join between chunks;
* the coarse steps of all requests of a class that are in a coarse sweep, each
  at its own slice, go into one batched coarse call per tick;
* fine and coarse batches of a class run on two streams, so the throughput-bound
  fine batch overlaps the latency-bound coarse sweeps of other requests, and
  different classes overlap each other.

The kernels reduce in an order that depends only on the grid, never on the
batch, so a request's states, defects and Nu values are bitwise the same
whether it is served alone or in any mix.  With `f_chunk` >= the fine steps per
slice they are also bitwise those of `parareal_iterate`; with smaller chunks
the states and defects still are and Nu differs only by the order of the
trapezoid sums.

Admission: a request is admitted, in arrival order, when its buffers (its
iterates, the previous iterate, the fine results and the coarse history) fit
in the memory budget next to the class buffers already held.  The budget is a
fraction of the free device memory when the engine starts, or a given limit.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import inputs, rbc

# Sec. 2.3: the paper's fit Nu = 0.135 Ra^0.286 (fixed-flux runs), used to size
# the thermal boundary layer delta_T = 1 / (2 Nu) (Sec. 2.2, with L = 1).
NU_FIT_A, NU_FIT_B = 0.135, 0.286
MIN_BL_POINTS = 6   # Sec. 2.2: at least six points in the thermal boundary layer
SERVING_GRIDS = ((64, 32), (256, 64), (512, 128), (1024, 256))


def boundary_layer_points(Ra, Nz):
    """Interior Lobatto points within delta_T = 1/(2 Nu(Ra)) of a wall."""
    nu = max(1.0, NU_FIT_A * Ra ** NU_FIT_B)
    delta = 0.5 / nu
    j = np.arange(1, Nz - 1)
    dist = 0.5 - 0.5 * np.cos(np.pi * j / (Nz - 1))   # distance from the wall
    return int(np.count_nonzero(dist <= delta))


def adequate_grids(Ra, grids=SERVING_GRIDS):
    return [g for g in grids if boundary_layer_points(Ra, g[1]) >= MIN_BL_POINTS]


def max_adequate_ra(Nz, lo=1e3, hi=1e12):
    """Largest Ra for which an Nz grid keeps MIN_BL_POINTS in the boundary layer."""
    if boundary_layer_points(lo, Nz) < MIN_BL_POINTS:
        return 0.0
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if boundary_layer_points(mid, Nz) >= MIN_BL_POINTS:
            lo = mid
        else:
            hi = mid
    return lo


def stable_dt(Nz, ra_max, c=40.0, dt0=1e-3):
    """Fine dt for a class: the explicit advective limit scales as 1 / (Nz^2 sqrt(Ra))
    (Chebyshev spacing ~ 1/Nz^2 at the walls, free-fall speed ~ sqrt(Ra) in
    diffusive units).  c is calibrated on measured stable dt (256x64 at Ra = 1e6:
    1.25e-5; 512x128 at 1e7: 7.8e-7); the value returned is the largest
    dt0 * 2^-j under that bound, as on the halving ladder of Sec. 3.5."""
    bound = c / (Nz * Nz * math.sqrt(max(ra_max, 1.0)))
    j = max(0, math.ceil(math.log2(dt0 / bound) - 1e-12))
    return dt0 * 2.0 ** (-j)


@dataclass
class ClassConfig:
    """Time stepping of one (grid, precision) class."""
    Nx: int
    Nz: int
    precision: int
    dt_fine: float
    dt_coarse: float
    nf: int            # fine steps per slice
    nc: int            # coarse steps per slice
    coarse_Nx: int
    coarse_Nz: int


def default_class_config(Nx, Nz, precision, fine_steps=200, coarse_ratio=2, ra_max=None):
    """Fine dt from the class's largest admissible Ra; coarse grid halved in x and z
    with `coarse_ratio` times the fine dt; a fixed number of fine steps per slice."""
    if ra_max is None:
        ra_max = min(1e8, max_adequate_ra(Nz))
    dtf = stable_dt(Nz, ra_max)
    nc = max(1, fine_steps // coarse_ratio)
    return ClassConfig(Nx, Nz, precision, dtf, dtf * fine_steps / nc, fine_steps, nc, Nx // 2, Nz // 2)


@dataclass
class Request:
    rid: int
    Ra: float
    Nx: int
    Nz: int
    nslices: int
    precision: int = rbc.RBC_FP64
    arrival: float = 0.0          # seconds after the start of the run
    seed: int = 0
    U0: torch.Tensor = None       # initial fine state on the device (prepared by Engine.prepare)
    # results
    status: int = None
    k_done: int = 0
    defects: list = field(default_factory=list)
    nus: list = field(default_factory=list)
    U: torch.Tensor = None        # final iterate U^k (nslices + 1 states), if kept
    t_admit: float = None
    t_done: float = None

    @property
    def key(self):
        return (self.Nx, self.Nz, self.precision)

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


class _Run:
    """Device buffers and the position in the Parareal sequence of one admitted request."""

    def __init__(self, req, cls, nchunks):
        N = req.nslices
        self.req, self.cls, self.N = req, cls, N
        dev = cls.device
        # torch.empty queues no kernel on the default stream; every element is
        # written on the class streams before it is read
        f64 = dict(dtype=torch.float64, device=dev)
        self.U = torch.empty((N + 1,) + cls.fine.state_shape, **f64)
        self.Uold = torch.empty((N + 1,) + cls.fine.state_shape, **f64)
        self.F = torch.empty((N,) + cls.fine.state_shape, **f64)
        self.Gold = torch.empty((N,) + cls.coarse.state_shape, **f64)
        self.I = torch.empty((nchunks, N), **f64)
        self.norm = torch.empty(2 * (N + 1), **f64)
        self.norm_h = cls.rt.host_buffer((2 * (N + 1),))
        self.I_h = cls.rt.host_buffer((nchunks, N))
        self.phase = "G0"    # G0 -> F -> G -> CHECK -> F ... -> DONE
        self.k = 0           # iterations completed
        self.n = 0           # slice position of the coarse sweep
        self.fdone = 0       # fine steps done in the current fine sweep
        self.chunk = 0
        self.dep = None      # event the next fine gather waits on
        self.check_ev = None
        self.nu_prev = 0.0


class CudaRuntime:
    """Streams, events and host staging of the engine (torch.cuda)."""

    def __init__(self, device):
        self.device = device

    def stream(self):
        return torch.cuda.Stream(self.device)

    def event(self):
        return torch.cuda.Event()

    def on(self, stream):
        return torch.cuda.stream(stream)

    def synchronize(self):
        torch.cuda.synchronize(self.device)

    def free_bytes(self):
        return torch.cuda.mem_get_info(self.device)[0]

    def host_buffer(self, shape):
        return torch.zeros(shape, dtype=torch.float64).pin_memory()


def run_bytes(N, Sf, Sc, nchunks):
    """Device bytes one request holds while admitted (see _Run)."""
    return (2 * (N + 1) + N) * Sf + N * Sc + (nchunks * N + 2 * (N + 1)) * 8


class _Class:
    def __init__(self, cfg, Pr, Lx, bmax, device, lib, rt):
        self.cfg, self.device, self.lib, self.rt = cfg, device, lib, rt
        ra0 = 1e4   # the handles' own Ra is unused: every call passes Ra per state
        self.fine = lib.Propagator(ra0, Pr, Lx, cfg.Nx, cfg.Nz, cfg.dt_fine, cfg.precision)
        self.coarse = lib.Propagator(ra0, Pr, Lx, cfg.coarse_Nx, cfg.coarse_Nz, cfg.dt_coarse, cfg.precision)
        self.Sf, self.Sc = self.fine.state_bytes, self.coarse.state_bytes
        self.bmax = bmax
        self.fine.reserve(bmax)
        self.coarse.reserve(bmax)
        self.fstage = self.fine.new_states(bmax, device)
        self.fnu = torch.zeros(bmax, dtype=torch.float64, device=device)
        self.gstage = self.coarse.new_states(bmax, device)
        self.sf = rt.stream()
        self.sg = rt.stream()
        self.runs = []          # admitted, in admission order
        self.f_inflight = None  # (event, [(run, steps)])
        self.g_inflight = []    # events of queued coarse ticks
        self.launches = {"f_batches": 0, "g_ticks": 0}
        rt.synchronize()   # the buffers above were zeroed on the default stream

    @staticmethod
    def held_bytes(fine_Sf, fine_W, coarse_Sc, coarse_W, bmax):
        return bmax * (2 * fine_Sf + fine_W + 8 + 2 * coarse_Sc + coarse_W)

    def close(self):
        self.fine.close()
        self.coarse.close()


class Engine:
    """Continuous-batching Parareal server on one GPU.

    criterion/tol/max_iters: stopping rule of every request (as parareal_create).
    f_chunk: fine steps per batched launch; requests join the fine batch between chunks.
    g_depth: coarse ticks queued ahead per class.
    mem_limit: device bytes for admission (default: mem_fraction of the free memory).
    lib, runtime: the propagator library (the C ABI binding) and the stream/event
    provider; both are replaceable so that the scheduling logic can be exercised
    on the host.
    """

    def __init__(self, criterion=rbc.CRIT_FIXED, tol=0.0, max_iters=2, f_chunk=50, g_depth=2, bmax=128,
                 mem_limit=None, mem_fraction=0.85, Pr=1.0, Lx=2.0, class_config=default_class_config,
                 keep_states=False, device="cuda", lib=rbc, runtime=None):
        self.criterion, self.tol, self.max_iters = criterion, tol, max_iters
        self.f_chunk, self.g_depth, self.bmax = f_chunk, g_depth, bmax
        self.Pr, self.Lx = Pr, Lx
        self.class_config = class_config
        self.keep_states = keep_states
        self.device = torch.device(device)
        self.lib = lib
        self.rt = runtime if runtime is not None else CudaRuntime(self.device)
        if mem_limit is None:
            mem_limit = int(self.rt.free_bytes() * mem_fraction)
        self.mem_limit = mem_limit
        self.committed = 0
        self.peak_committed = 0
        self.peak_active = 0
        self.classes = {}
        self.cfgs = {}

    # ---- classes and inputs -------------------------------------------------
    def config_for(self, key):
        if key not in self.cfgs:
            self.cfgs[key] = self.class_config(*key)
        return self.cfgs[key]

    def _class(self, key):
        cls = self.classes.get(key)
        if cls is None:
            cfg = self.config_for(key)
            cls = _Class(cfg, self.Pr, self.Lx, self.bmax, self.device, self.lib, self.rt)
            self.committed += _Class.held_bytes(cls.Sf, cls.fine.workspace_bytes_per_state, cls.Sc,
                                                cls.coarse.workspace_bytes_per_state, self.bmax)
            self.classes[key] = cls
        return cls

    def prepare(self, req):
        """Place the seeded initial state (Sec. 2.1 noise on the conduction profile) on the device."""
        cls = self._class(req.key)
        if not 1 <= req.nslices <= self.bmax:
            raise ValueError(f"request {req.rid}: {req.nslices} slices; the batch capacity is {self.bmax}")
        if req.U0 is None:
            U0 = cls.fine.new_states(1, self.device)
            cls.fine.set_state(U0[0], inputs.initial_temperature(req.Nx, req.Nz, req.seed, Lx=self.Lx))
            req.U0 = U0[0]
        return req

    def interval(self, req):
        cfg = self.config_for(req.key)
        return 0.0, req.nslices * cfg.nf * cfg.dt_fine

    def _nchunks(self, cfg):
        return -(-cfg.nf // self.f_chunk)

    def request_bytes(self, req):
        cfg = self.config_for(req.key)
        cls = self._class(req.key)
        return run_bytes(req.nslices, cls.Sf, cls.Sc, self._nchunks(cfg))

    # ---- the loop ---------------------------------------------------------
    def run(self, requests, on_done=None, deadline=None):
        """Serve `requests` (arrival times relative to the call); returns them with results.

        Arrivals are honoured on the host clock: a request is not admitted before
        its arrival time.  Latency = completion - arrival.  deadline: seconds
        after which the loop gives up with RuntimeError (work already queued on
        the device still completes).
        """
        for r in requests:
            self.prepare(r)
        self.rt.synchronize()
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        queue = []
        self.t0 = time.perf_counter()
        pi = 0
        active = 0
        while pi < len(pending) or queue or active:
            now = time.perf_counter() - self.t0
            if deadline is not None and now > deadline:
                self.rt.synchronize()
                raise RuntimeError(f"serving loop passed its {deadline} s deadline with {active} requests active")
            while pi < len(pending) and pending[pi].arrival <= now:
                queue.append(pending[pi])
                pi += 1
            # admission in arrival order, by device memory
            while queue:
                r = queue[0]
                need = self.request_bytes(r)
                if self.committed + need > self.mem_limit:
                    if active == 0:
                        raise RuntimeError(f"request {r.rid} needs {need} bytes; limit {self.mem_limit}, "
                                           f"{self.committed} held by class buffers")
                    break
                queue.pop(0)
                self._admit(r, need)
                active += 1
            progressed = False
            for cls in self.classes.values():
                done, prog = self._progress(cls, on_done)
                active -= done
                progressed = progressed or prog
            if not progressed:
                if active == 0 and not queue and pi < len(pending):
                    wait = pending[pi].arrival - (time.perf_counter() - self.t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                else:
                    time.sleep(2e-5)
        self.t_end = time.perf_counter() - self.t0
        return requests

    def _admit(self, r, need):
        cls = self._class(r.key)
        run = _Run(r, cls, self._nchunks(cls.cfg))
        run.bytes = need
        self.committed += need
        self.peak_committed = max(self.peak_committed, self.committed)
        self.peak_active = max(self.peak_active, sum(len(c.runs) for c in self.classes.values()) + 1)
        r.t_admit = time.perf_counter() - self.t0
        with self.rt.on(cls.sg):
            run.U[0].copy_(r.U0, non_blocking=True)   # U0 may be pinned host memory
        cls.runs.append(run)

    def _finish(self, run, status):
        cls, r = run.cls, run.req
        r.status = status
        r.t_done = time.perf_counter() - self.t0
        if self.keep_states:
            r.U = run.U
        cls.runs.remove(run)
        self.committed -= run.bytes

    # ---- one class: poll completions, queue the next batches ---------------
    def _progress(self, cls, on_done):
        cfg = cls.cfg
        finished = 0
        prog = False
        # fine batch completed?
        if cls.f_inflight is not None and cls.f_inflight[0].query():
            _, members = cls.f_inflight
            cls.f_inflight = None
            for run, steps in members:
                run.fdone += steps
                run.chunk += 1
                if run.fdone >= cfg.nf:
                    run.phase = "G"
                    run.n = 0
                    run.started_g = False
                else:
                    run.phase = "F"
            prog = True
        # checks completed?
        for run in [r for r in cls.runs if r.phase == "CHECK" and r.check_ev.query()]:
            st = self._check(run)
            if st is not None:
                self._finish(run, st)
                finished += 1
                if on_done:
                    on_done(run.req)
            prog = True
        # retire finished coarse ticks
        cls.g_inflight = [e for e in cls.g_inflight if not e.query()]
        if cls.f_inflight is None:
            prog |= self._launch_fine(cls)
        if len(cls.g_inflight) < self.g_depth:
            prog |= self._launch_coarse(cls)
        return finished, prog

    def _launch_fine(self, cls):
        cfg = cls.cfg
        members, total = [], 0
        for run in cls.runs:
            if run.phase != "F":
                continue
            cnt = run.N - run.k          # slices n >= k (this sweep is iteration k+1)
            if total + cnt > cls.bmax:
                continue
            members.append((run, cnt, total))
            total += cnt
        if not members:
            return False
        steps = [min(self.f_chunk, cfg.nf - run.fdone) for run, _, _ in members]
        nsteps = np.concatenate([np.full(cnt, s, np.int32) for (run, cnt, _), s in zip(members, steps)])
        ra = np.concatenate([np.full(cnt, run.req.Ra) for run, cnt, _ in members])
        with self.rt.on(cls.sf):
            for run, cnt, off in members:
                if run.dep is not None:
                    cls.sf.wait_event(run.dep)
                    run.dep = None
                n0 = run.k
                if run.fdone == 0:
                    run.F[n0:].copy_(run.U[n0:run.N])
                cls.fstage[off:off + cnt].copy_(run.F[n0:])
            cls.fine.step_batch(cls.fstage[:total], nsteps, nu=cls.fnu[:total], stream=cls.sf, ra=ra)
            for run, cnt, off in members:
                n0 = run.k
                run.F[n0:].copy_(cls.fstage[off:off + cnt])
                run.I[run.chunk, n0:].copy_(cls.fnu[off:off + cnt])
            ev = self.rt.event()
            ev.record(cls.sf)
        cls.f_inflight = (ev, [(run, s) for (run, _, _), s in zip(members, steps)])
        for run, _, _ in members:
            run.phase = "F-run"
        cls.launches["f_batches"] += 1
        return True

    def _launch_coarse(self, cls):
        cfg = cls.cfg
        fine, coarse, lib = cls.fine, cls.coarse, self.lib
        members = [run for run in cls.runs if run.phase in ("G0", "G")][: cls.bmax]
        if not members:
            return False
        with self.rt.on(cls.sg):
            for run in members:
                if run.phase == "G" and not run.started_g:
                    run.Uold.copy_(run.U)
                    run.started_g = True
                # iteration k+1 leaves U_n, n <= k, as it was: G(U_n) = Gold_n exactly
                while run.phase == "G" and run.n <= run.k and run.n < run.N:
                    n = run.n
                    lib.parareal_correct(fine, coarse, run.F[n:n + 1], run.Gold[n:n + 1], run.Gold[n:n + 1],
                                         run.U[n + 1:n + 2], stream=cls.sg)
                    run.n += 1
            members = [run for run in members if run.n < run.N]
            for b, run in enumerate(members):
                lib.restrict(fine, coarse, run.U[run.n:run.n + 1], cls.gstage[b:b + 1], stream=cls.sg)
            B = len(members)
            if B:
                coarse.step_batch(cls.gstage[:B], cfg.nc, stream=cls.sg, ra=[run.req.Ra for run in members])
            for b, run in enumerate(members):
                n = run.n
                if run.phase == "G0":
                    run.Gold[n].copy_(cls.gstage[b])
                    lib.prolong(fine, coarse, cls.gstage[b:b + 1], run.U[n + 1:n + 2], stream=cls.sg)
                else:
                    lib.parareal_correct(fine, coarse, run.F[n:n + 1], cls.gstage[b:b + 1], run.Gold[n:n + 1],
                                         run.U[n + 1:n + 2], stream=cls.sg)
                    run.Gold[n].copy_(cls.gstage[b])
                run.n += 1
            ev = self.rt.event()
            ev.record(cls.sg)
            for run in [r for r in cls.runs if r.phase in ("G0", "G") and r.n >= r.N]:
                if run.phase == "G0":
                    run.phase, run.k, run.fdone, run.chunk, run.dep = "F", 0, 0, 0, ev
                else:
                    N = run.N
                    lib.l2_diff(fine, run.U, run.Uold, run.norm[:N + 1], stream=cls.sg)
                    lib.l2_diff(fine, run.U, None, run.norm[N + 1:], stream=cls.sg)
                    run.norm_h.copy_(run.norm, non_blocking=True)
                    run.I_h.copy_(run.I, non_blocking=True)
                    run.check_ev = self.rt.event()
                    run.check_ev.record(cls.sg)
                    run.phase = "CHECK"
        cls.g_inflight.append(ev)
        cls.launches["g_ticks"] += 1
        return True

    def _check(self, run):
        """Defect and Nu of iteration k+1 (as parareal_iterate); None to continue."""
        r, N = run.req, run.N
        k = run.k + 1
        nrm = run.norm_h.numpy()
        defect = 0.0
        for n in range(1, N + 1):
            a, b = nrm[n], nrm[N + 1 + n]
            if not (math.isfinite(a) and math.isfinite(b)):
                return rbc.RBC_EDIVERGED
            if b > 0:
                defect = max(defect, math.sqrt(a / b))
        cfg = run.cls.cfg
        t0, t1 = self.interval(r)
        n_half = N // 2
        win = (t1 - t0) * (N - n_half) / N
        Ih = run.I_h.numpy()
        nu = 0.0
        for n in range(n_half, N):
            s = 0.0
            for c in range(Ih.shape[0]):
                s += Ih[c, n]
            nu += s
        nu /= win
        r.defects.append(defect)
        r.nus.append(nu)
        r.k_done = k
        run.k = k
        if self.criterion == rbc.CRIT_DEFECT and defect <= self.tol:
            return rbc.RBC_OK
        if self.criterion == rbc.CRIT_NU and k >= 2 and abs(nu - run.nu_prev) <= self.tol * abs(nu):
            return rbc.RBC_OK
        run.nu_prev = nu
        if k >= self.max_iters or k >= N:
            return rbc.RBC_OK if self.criterion == rbc.CRIT_FIXED else rbc.RBC_ENOTCONVERGED
        run.phase, run.fdone, run.chunk = "F", 0, 0
        return None

    def close(self):
        self.rt.synchronize()
        for cls in self.classes.values():
            cls.close()
        self.classes.clear()


def latency_stats(requests):
    lat = np.array([r.latency for r in requests if r.latency is not None])
    if lat.size == 0:
        return {}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def dof_steps(requests, engine):
    """Fine DOF-steps of the served work: sum over requests and iterations of
    2 Nx Nz x fine steps x slices advanced (slices n >= k-1 in iteration k)."""
    tot = 0
    for r in requests:
        cfg = engine.config_for(r.key)
        for k in range(1, r.k_done + 1):
            tot += 2 * r.Nx * r.Nz * cfg.nf * (r.nslices - (k - 1))
    return tot


def make_requests(n, seed, rate, grids=SERVING_GRIDS, ra_range=(1e4, 1e8), slices=(4, 64), p_mixed=0.5):
    """Synthetic request stream: Poisson arrivals at `rate` per second, Ra log-uniform,
    a grid drawn uniformly among those adequate for Ra, slices uniform, precision
    mixed with probability p_mixed; noise seed = request id."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += g.exponential(1.0 / rate) if rate > 0 else 0.0
        Ra = float(10 ** g.uniform(math.log10(ra_range[0]), math.log10(ra_range[1])))
        ok = adequate_grids(Ra, grids)
        Nx, Nz = ok[int(g.integers(len(ok)))]
        N = int(g.integers(slices[0], slices[1] + 1))
        prec = rbc.RBC_MIXED if g.uniform() < p_mixed else rbc.RBC_FP64
        out.append(Request(rid=i, Ra=Ra, Nx=Nx, Nz=Nz, nslices=N, precision=prec, arrival=t, seed=i))
    return out
