"""The FP64 oracle behind the propagator interface of the binding, on CPU
tensors in the C ABI's state layout, so that host drivers built on that
interface (statistics.StatisticalParareal) can be checked without a GPU.

Test infrastructure: it only moves data between the ABI layout and the
oracle's State (tests/layout.py) and calls the oracle.
"""
import numpy as np
import torch

from layout import from_abi, to_abi
from oracle.rbc import RBC
from oracle.rbc import prolong as o_prolong
from oracle.rbc import restrict as o_restrict


class OracleProp:
    def __init__(self, Ra, Pr, Lx, Nx, Nz, dt):
        self.o = RBC(Ra, Pr, Lx, Nx, Nz, dt)
        self.Ra, self.Pr, self.Lx, self.Nx, self.Nz, self.dt = Ra, Pr, Lx, Nx, Nz, dt
        self.steps_taken = 0

    @property
    def state_shape(self):
        return (2, self.Nz, self.Nx // 2, 2)

    @property
    def diag_size(self):
        return 6 + 2 * self.o.Mz

    def new_states(self, B, device="cpu"):
        return torch.zeros((B,) + self.state_shape, dtype=torch.float64)

    def set_state(self, state, T):
        state.copy_(torch.from_numpy(to_abi(self.o.from_grid(T))))

    def step_batch(self, states, nsteps, nu=None, stream=None, ra=None):
        for b in range(states.shape[0]):
            X = from_abi(states[b].numpy())
            for _ in range(int(nsteps)):
                X, _ = self.o.step(X)
            states[b].copy_(torch.from_numpy(to_abi(X)))
            self.steps_taken += int(nsteps)

    def diagnostics(self, states, out=None, stream=None):
        rows = []
        for b in range(states.shape[0]):
            d = self.o.diagnostics(from_abi(states[b].numpy()))
            rows.append(np.concatenate([[d["KE2"], d["eps"], d["wT"]], d["nu"], d["Tm"], d["Tv"]]))
        return torch.from_numpy(np.array(rows))


def restrict(fine, coarse, fine_states, coarse_states, stream=None):
    for b in range(fine_states.shape[0]):
        X = o_restrict(from_abi(fine_states[b].numpy()), coarse.Nx, coarse.Nz)
        coarse_states[b].copy_(torch.from_numpy(to_abi(X)))


def prolong(fine, coarse, coarse_states, fine_states, stream=None):
    for b in range(coarse_states.shape[0]):
        X = o_prolong(from_abi(coarse_states[b].numpy()), fine.Nx, fine.Nz)
        fine_states[b].copy_(torch.from_numpy(to_abi(X)))


def parareal_correct(fine, coarse, F, Gnew, Gold, U, stream=None):
    for b in range(F.shape[0]):
        pn = to_abi(o_prolong(from_abi(Gnew[b].numpy()), fine.Nx, fine.Nz))
        po = to_abi(o_prolong(from_abi(Gold[b].numpy()), fine.Nx, fine.Nz))
        U[b].copy_(torch.from_numpy(F[b].numpy() + (pn - po)))


def l2_diff(prop, A, Bm, out, stream=None):
    for b in range(A.shape[0]):
        X = from_abi(A[b].numpy())
        if Bm is not None:
            X = X - from_abi(Bm[b].numpy())
        out[b] = prop.o.l2_T(X) ** 2
