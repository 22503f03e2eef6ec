"""A host-only stand-in for the propagator library, for testing the serving
scheduler without a GPU.

The map is a toy (a damped, mode-coupled nonlinear update), not the method;
what matters is that it is deterministic, nonlinear (so Parareal needs several
iterations), depends on a per-state Rayleigh number, and that restriction,
prolongation, the correction and the norm act on the same state layout as
the library's: (2, Nz, Nx/2, 2), field 0 = T.
"""
import contextlib
import math

import torch


class FakePropagator:
    def __init__(self, Ra, Pr, Lx, Nx, Nz, dt, precision=0):
        self.Ra, self.Pr, self.Lx, self.Nx, self.Nz, self.dt = Ra, Pr, Lx, Nx, Nz, dt
        self.precision = precision
        self.steps_taken = 0
        self.batches = []

    @property
    def state_shape(self):
        return (2, self.Nz, self.Nx // 2, 2)

    @property
    def state_bytes(self):
        return 8 * math.prod(self.state_shape)

    @property
    def workspace_bytes_per_state(self):
        return 4 * self.state_bytes

    def reserve(self, B):
        pass

    def new_states(self, B, device="cpu"):
        return torch.zeros((B,) + self.state_shape, dtype=torch.float64, device=device)

    def set_state(self, state, T, u=None, w=None):
        t = torch.as_tensor(T, dtype=torch.float64)
        state.zero_()
        state[0, :, :, 0] = t[:, : self.Nx // 2]
        state[1, :, :, 1] = 0.5 * t[:, self.Nx // 2:]

    def one_step(self, X, ra):
        c = 0.5 * ra / 1e4
        return X + self.dt * (-X + c * torch.tanh(torch.roll(X, 1, dims=2)) * torch.cos(X))

    def step_batch(self, states, nsteps, nu=None, stream=None, ra=None):
        B = states.shape[0]
        ns = [int(nsteps)] * B if not hasattr(nsteps, "__len__") else [int(v) for v in nsteps]
        self.batches.append(B)
        for b in range(B):
            r = self.Ra if ra is None else float(ra[b])
            X = states[b].clone()
            s0 = float(X[0].mean())
            integral = 0.0
            for _ in range(ns[b]):
                X = self.one_step(X, r)
                s1 = float(X[0].mean())
                integral += self.dt * 0.5 * (s0 + s1)
                s0 = s1
            self.steps_taken += ns[b]
            states[b].copy_(X)
            if nu is not None:
                nu[b] = integral

    def close(self):
        pass


def _pad(coarse_states, fine):
    out = torch.zeros((coarse_states.shape[0],) + fine.state_shape, dtype=torch.float64)
    out[:, :, : coarse_states.shape[2], : coarse_states.shape[3], :] = coarse_states
    return out


def restrict(fine, coarse, fine_states, coarse_states, stream=None):
    coarse_states.copy_(fine_states[:, :, : coarse.Nz, : coarse.Nx // 2, :])


def prolong(fine, coarse, coarse_states, fine_states, stream=None):
    fine_states.copy_(_pad(coarse_states, fine))


def parareal_correct(fine, coarse, F, Gnew, Gold, U, stream=None):
    U.copy_(F + (_pad(Gnew, fine) - _pad(Gold, fine)))


def l2_diff(prop, A, Bm, out, stream=None):
    for b in range(A.shape[0]):
        d = A[b, 0] if Bm is None else A[b, 0] - Bm[b, 0]
        out[b] = float((d * d).sum())


Propagator = FakePropagator


class _Event:
    def __init__(self, done):
        self.done = done

    def record(self, stream=None):
        pass

    def query(self):
        return self.done()


class _Stream:
    def wait_event(self, ev):
        pass


class HostRuntime:
    """Streams and events for host tensors: work is done when it is queued."""

    def __init__(self, event_done=lambda: True):
        self.event_done = event_done

    def stream(self):
        return _Stream()

    def event(self):
        return _Event(self.event_done)

    def on(self, stream):
        return contextlib.nullcontext()

    def synchronize(self):
        pass

    def free_bytes(self):
        return 1 << 40

    def host_buffer(self, shape):
        return torch.zeros(shape, dtype=torch.float64)
