"""FP64 oracle of the fine/coarse propagator for 2D Rayleigh-Benard convection.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Physics (Sec. 2.1, Eqs. 3-6): Oberbeck-Boussinesq equations in a box
x in [0, Lx) (periodic), z in [-1/2, 1/2], no-slip walls, isothermal
T(-1/2) = 1, T(1/2) = 0 (Eq. 6) or with fixed flux dT/dz = -1 (Eq. 7, Ra then
being the flux Rayleigh number of Eq. 8), time in thermal-diffusion units.
Eq. 3 times Pr:

    u_t + u.grad u = -grad p + Pr Ra T z^ + Pr lap u,    div u = 0,
    T_t + u.grad T = lap T.

Reading: streamfunction form (div u = 0 exactly): u = d_z psi, w = -d_x psi,
omega = d_x w - d_z u = -lap psi.  The curl of the momentum equation gives

    lap psi_t = Pr lap^2 psi - Pr Ra d_x T + u.grad omega      (Fourier modes m >= 1)
    U_t       = Pr U_zz - <u.grad u>_x                          (mean flow, m = 0)
    T_t       = lap T - u.grad T.

Discretisation (Sec. 3.2): Fourier modes m = 0 .. Nx/2-1 in x (k = 2 pi m / Lx,
Nyquist dropped, coefficients normalised by 1/N), Chebyshev T_n(s), s = 2z,
n = 0 .. Nz-1 in z.  Products are formed on a 3/2-padded grid (Mx = 3Nx/2
uniform points, Mz = 3Nz/2 Chebyshev-Lobatto points) in advective form and
truncated back (dealiasing; the paper is silent, this is the reading).  Linear
terms (diffusion, pressure, buoyancy) are implicit (Sec. 3.2) with the
ultraspherical tau method; nonlinear terms explicit.  Time stepping: the
4-stage, 3rd-order IMEX Runge-Kutta RK443 of Ascher, Ruuth & Spiteri (Sec. 3.2,
Sec. 3.6), written M X_t = L X + F(X).  The lower-order coarse steppers that
Sec. 3.6 reports trying are read as the two smaller schemes of the same family:
ARS(2,2,2) ("RK222", 2 stages, 2nd order) and ARS(1,1,1) ("RK111",
forward-backward Euler, 1st order).  All three have an explicit first stage, a
constant implicit diagonal gamma and are stiffly accurate (X_{n+1} = last stage).

State: ``State(T, psi, U)`` with T, psi complex (Nx/2, Nz) (psi[0] unused, kept
zero) and U real (Nz,) = mean horizontal velocity.
"""
import numpy as np
import scipy.linalg as sla
from numpy.polynomial import chebyshev as C

from . import ultraspherical as us

# RK443 (Ascher, Ruuth & Spiteri 1997, the (4,4,3) scheme; Sec. 3.6).  Row i,
# column j: coefficient of stage j in stage i, stages 0..4, stage 0 explicit.
RK443_C = [0.0, 1 / 2, 2 / 3, 1 / 2, 1.0]
RK443_AI = [
    [0, 0, 0, 0, 0],
    [0, 1 / 2, 0, 0, 0],
    [0, 1 / 6, 1 / 2, 0, 0],
    [0, -1 / 2, 1 / 2, 1 / 2, 0],
    [0, 3 / 2, -3 / 2, 1 / 2, 1 / 2],
]
RK443_AE = [
    [0, 0, 0, 0, 0],
    [1 / 2, 0, 0, 0, 0],
    [11 / 18, 1 / 18, 0, 0, 0],
    [5 / 6, -5 / 6, 1 / 2, 0, 0],
    [1 / 4, 7 / 4, 3 / 4, -7 / 4, 0],
]


# ARS(2,2,2): gamma = 1 - 1/sqrt(2) (the root of gamma^2 - 2 gamma + 1/2 = 0 in
# (0, 1): second order and L-stable), delta = 1 - 1/(2 gamma).
_G2 = 1.0 - 1.0 / np.sqrt(2.0)
_D2 = 1.0 - 1.0 / (2.0 * _G2)
RK222_C = [0.0, _G2, 1.0]
RK222_AI = [
    [0, 0, 0],
    [0, _G2, 0],
    [0, 1 - _G2, _G2],
]
RK222_AE = [
    [0, 0, 0],
    [_G2, 0, 0],
    [_D2, 1 - _D2, 0],
]
# ARS(1,1,1): explicit Euler for F, implicit Euler for L.
RK111_C = [0.0, 1.0]
RK111_AI = [[0, 0], [0, 1.0]]
RK111_AE = [[0, 0], [1.0, 0]]

SCHEMES = {
    "RK443": (RK443_C, RK443_AI, RK443_AE),
    "RK222": (RK222_C, RK222_AI, RK222_AE),
    "RK111": (RK111_C, RK111_AI, RK111_AE),
}


class State:
    """Spectral state of one time slice: T-hat, psi-hat (m x n), mean flow U (n)."""

    def __init__(self, T, psi, U):
        self.T = T
        self.psi = psi
        self.U = U

    def copy(self):
        return State(self.T.copy(), self.psi.copy(), self.U.copy())

    def __add__(self, o):
        return State(self.T + o.T, self.psi + o.psi, self.U + o.U)

    def __sub__(self, o):
        return State(self.T - o.T, self.psi - o.psi, self.U - o.U)

    def arrays(self):
        return self.T, self.psi, self.U


def native_points(Nx, Nz, Lx):
    """Native collocation grid: x_i = Lx i / Nx, z_j = -cos(pi j/(Nz-1))/2 (ascending)."""
    x = Lx * np.arange(Nx) / Nx
    z = -0.5 * np.cos(np.pi * np.arange(Nz) / (Nz - 1))
    return x, z


class RBC:
    """Fine (or coarse) propagator of Sec. 3.2 on one grid with one time step."""

    def __init__(self, Ra, Pr, Lx, Nx, Nz, dt, bc="fixed_T", scheme="RK443"):
        """bc: "fixed_T" (Eq. 6: T = 1, 0 at z = -1/2, 1/2) or "fixed_flux"
        (Eq. 7: dT/dz = -1 at both walls, with Ra read as the flux Rayleigh
        number Ra_f of Eq. 8); no-slip walls in both.  scheme: the IMEX
        Runge-Kutta pair, "RK443" (the paper's) or the lower-order "RK222",
        "RK111" (Sec. 3.6)."""
        if Nx % 2 or Nx < 4 or Nz < 8 or Nz % 2 or dt <= 0:
            raise ValueError("need even Nx >= 4, even Nz >= 8, dt > 0")
        if bc not in ("fixed_T", "fixed_flux"):
            raise ValueError("bc must be fixed_T or fixed_flux")
        if scheme not in SCHEMES:
            raise ValueError("scheme must be one of " + ", ".join(SCHEMES))
        self.Ra, self.Pr, self.Lx, self.Nx, self.Nz, self.dt = Ra, Pr, Lx, Nx, Nz, dt
        self.bc = bc
        self.scheme = scheme
        self.c_rk, self.AI, self.AE = SCHEMES[scheme]
        self.stages = len(self.AI) - 1
        self.gamma = self.AI[1][1]             # the constant implicit diagonal
        self.nm = Nx // 2
        self.Mx = 3 * Nx // 2
        self.Mz = 3 * Nz // 2
        self.k = 2.0 * np.pi / Lx * np.arange(self.nm)
        Nz, Mz = self.Nz, self.Mz
        # padded Lobatto points s_j = cos(pi j/(Mz-1)); exact interpolation matrices
        sp = np.cos(np.pi * np.arange(Mz) / (Mz - 1))
        Vfull = C.chebvander(sp, Mz - 1)                     # Vfull[j, n] = T_n(s_j)
        self.Vpad = Vfull[:, :Nz]                            # coefficients -> values
        self.Wpad = np.linalg.solve(Vfull, np.eye(Mz))[:Nz]  # values -> coefficients, truncated
        intT = np.array([2.0 / (1.0 - n * n) if n % 2 == 0 else 0.0 for n in range(Mz)])
        self.cc_weights = np.linalg.solve(Vfull.T, intT)     # Clenshaw-Curtis on padded points
        self.Dz = 2.0 * us.cheb_derivative_matrix(Nz)        # d/dz = 2 d/ds on coefficients
        # ultraspherical tau operators (first Nz-lambda rows kept)
        self.S2 = us.convert_chain(2, Nz)[: Nz - 2]
        self.D2 = us.derivative(2, Nz)[: Nz - 2]
        self.S4 = us.convert_chain(4, Nz)[: Nz - 4]
        self.S4D2 = (us.convert_C(3, Nz) @ us.convert_C(2, Nz) @ us.derivative(2, Nz))[: Nz - 4]
        self.D4 = us.derivative(4, Nz)[: Nz - 4]
        self.bc_val_lo = us.value_row(Nz, -1)
        self.bc_val_hi = us.value_row(Nz, +1)
        self.bc_slope_lo = us.slope_row(Nz, -1)
        self.bc_slope_hi = us.slope_row(Nz, +1)
        # temperature boundary rows and values (d/ds rows: dT/dz = 2 dT/ds = -1)
        if bc == "fixed_T":
            self.T_bc_lo, self.T_bc_hi, self.T_bc_val = self.bc_val_lo, self.bc_val_hi, (1.0, 0.0)
        else:
            self.T_bc_lo, self.T_bc_hi, self.T_bc_val = self.bc_slope_lo, self.bc_slope_hi, (-0.5, -0.5)
        self._factor()

    # ---- linear operators, per Fourier mode (Eq. 3 x Pr and Eq. 5, d/dz = 2 d/ds) ----
    def ops_T(self, k):
        """T equation: M = S2, L = lap_k = 4 D2 - k^2 S2 (in C^(2))."""
        return self.S2, 4.0 * self.D2 - k * k * self.S2

    def ops_psi(self, k):
        """psi equation in C^(4): M = lap_k, L = Pr lap_k^2, C = -i k Pr Ra (on T)."""
        M = 4.0 * self.S4D2 - k * k * self.S4
        L = self.Pr * (16.0 * self.D4 - 8.0 * k * k * self.S4D2 + k ** 4 * self.S4)
        Cpl = -1j * k * self.Pr * self.Ra * self.S4
        return M, L, Cpl

    def ops_U(self):
        """Mean-flow equation: M = S2, L = Pr * 4 D2."""
        return self.S2, 4.0 * self.Pr * self.D2

    def _factor(self):
        """LU factors of the stage matrices (M - dt a_ii L) with boundary rows.

        Every diagonal coefficient of the implicit tableau is gamma (1/2 for
        RK443), so one matrix per Fourier mode serves all stages.
        """
        h = self.gamma * self.dt
        Nz = self.Nz
        M, L = self.ops_T(0.0)
        A = np.vstack([M - h * L, self.T_bc_lo, self.T_bc_hi])
        self.lu_T0 = sla.lu_factor(A)
        M, L = self.ops_U()
        A = np.vstack([M - h * L, self.bc_val_lo, self.bc_val_hi])
        self.lu_U = sla.lu_factor(A)
        self.lu_m = [None]
        for m in range(1, self.nm):
            k = self.k[m]
            MT, LT = self.ops_T(k)
            MP, LP, Cpl = self.ops_psi(k)
            A = np.zeros((2 * Nz, 2 * Nz), dtype=complex)
            A[: Nz - 2, :Nz] = MT - h * LT
            A[Nz - 2, :Nz] = self.T_bc_lo
            A[Nz - 1, :Nz] = self.T_bc_hi
            A[Nz : 2 * Nz - 4, :Nz] = -h * Cpl
            A[Nz : 2 * Nz - 4, Nz:] = MP - h * LP
            A[2 * Nz - 4, Nz:] = self.bc_val_lo
            A[2 * Nz - 3, Nz:] = self.bc_val_hi
            A[2 * Nz - 2, Nz:] = self.bc_slope_lo
            A[2 * Nz - 1, Nz:] = self.bc_slope_hi
            self.lu_m.append(sla.lu_factor(A))

    # ---- transforms ----
    def _spec_to_padded_grid(self, c):
        """(nm, Nz) complex coefficients -> real values on the (Mz, Mx) padded grid."""
        vz = c @ self.Vpad.T                                  # (nm, Mz)
        full = np.zeros((self.Mz, self.Mx // 2 + 1), dtype=complex)
        full[:, : self.nm] = vz.T
        return np.fft.irfft(full, n=self.Mx, axis=1) * self.Mx

    def _padded_grid_to_spec(self, g):
        """Real (Mz, Mx) values -> (nm, Nz) coefficients truncated to the kept modes."""
        h = np.fft.rfft(g, axis=1)[:, : self.nm] / self.Mx   # (Mz, nm)
        return (self.Wpad @ h).T

    def nonlinear(self, X):
        """Dealiased advection terms of the state X (Eqs. 3, 5 in advective form).

        Returns (N_T, N_omega) as (nm, Nz) Chebyshev coefficients of u.grad T and
        u.grad omega, N_U (Nz,) coefficients of the x-mean of u.grad u, and the
        x-mean of w T on the padded Lobatto points (Mz,) for Nu_V.
        """
        ik = 1j * self.k[:, None]
        dz = lambda c: c @ self.Dz.T
        u = dz(X.psi)
        u[0] = X.U
        w = -ik * X.psi
        w[0] = 0.0
        om = ik * w - dz(u)
        g = self._spec_to_padded_grid
        ug, wg = g(u), g(w)
        dxom, dzom = g(ik * om), g(dz(om))
        dxu, dzu = g(ik * u), g(dz(u))
        Tg, dxT, dzT = g(X.T), g(ik * X.T), g(dz(X.T))
        NT = self._padded_grid_to_spec(ug * dxT + wg * dzT)
        NO = self._padded_grid_to_spec(ug * dxom + wg * dzom)
        NU = self._padded_grid_to_spec(ug * dxu + wg * dzu)[0].real
        wT_mean = (wg * Tg).mean(axis=1)
        return NT, NO, NU, wT_mean

    # ---- the M X_t = L X + F(X) pieces, in tau rows ----
    def apply_M(self, X):
        T = X.T @ self.S2.T
        P = np.zeros((self.nm, self.Nz - 4), dtype=complex)
        for m in range(1, self.nm):
            P[m] = self.ops_psi(self.k[m])[0] @ X.psi[m]
        U = self.S2 @ X.U
        return State(T, P, U)

    def apply_L(self, X):
        T = np.zeros((self.nm, self.Nz - 2), dtype=complex)
        P = np.zeros((self.nm, self.Nz - 4), dtype=complex)
        for m in range(self.nm):
            T[m] = self.ops_T(self.k[m])[1] @ X.T[m]
        for m in range(1, self.nm):
            _, LP, Cpl = self.ops_psi(self.k[m])
            P[m] = LP @ X.psi[m] + Cpl @ X.T[m]
        U = self.ops_U()[1] @ X.U
        return State(T, P, U)

    def explicit(self, X):
        """F(X) in tau rows: -S2 N_T, +S4 N_omega, -S2 <N_U>; also the <wT>_x profile."""
        NT, NO, NU, wT = self.nonlinear(X)
        T = -(NT @ self.S2.T)
        P = NO @ self.S4.T
        P[0] = 0.0
        U = -(self.S2 @ NU)
        return State(T, P, U), wT

    def solve_stage(self, r):
        """Solve (M - gamma dt L) X = r in tau rows, boundary rows of Eq. 6 (or Eq. 7)."""
        Nz = self.Nz
        T = np.zeros((self.nm, Nz), dtype=complex)
        psi = np.zeros((self.nm, Nz), dtype=complex)
        b = np.concatenate([r.T[0].real, self.T_bc_val])   # the mean profile's wall values or slopes
        T[0] = sla.lu_solve(self.lu_T0, b)
        U = sla.lu_solve(self.lu_U, np.concatenate([r.U, [0.0, 0.0]]))
        for m in range(1, self.nm):
            b = np.zeros(2 * Nz, dtype=complex)
            b[: Nz - 2] = r.T[m]
            b[Nz : 2 * Nz - 4] = r.psi[m]
            x = sla.lu_solve(self.lu_m[m], b)
            T[m] = x[:Nz]
            psi[m] = x[Nz:]
        return State(T, psi, U)

    def step(self, X):
        """One step X_n -> X_{n+1} of the IMEX scheme (RK443 unless chosen
        otherwise); also returns Nu_V(t_n) (Eq. 9).

        Stage i: (M - dt a_ii L) X_i = M X_0 + dt sum_{j<i} (aE_ij F(X_j) + aI_ij L X_j);
        the schemes are stiffly accurate, X_{n+1} = X_s (s = 4, 2 or 1 stages).
        """
        dt = self.dt
        AE, AI, ns = self.AE, self.AI, self.stages
        MX0 = self.apply_M(X)
        Xs, Fs, LXs = [X], [], [None]
        nu0 = None
        for i in range(1, ns + 1):
            F, wT = self.explicit(Xs[i - 1])
            if i == 1:
                nu0 = self.nusselt_from(Xs[0], wT)[0]
            Fs.append(F)
            if i - 1 >= 1:
                LXs.append(self.apply_L(Xs[i - 1]))
            r = MX0
            for j in range(i):
                term = _scale(Fs[j], dt * AE[i][j])
                if j >= 1:
                    term = term + _scale(LXs[j], dt * AI[i][j])
                r = r + term
            Xs.append(self.solve_stage(r))
        return Xs[ns], nu0

    def run(self, X, nsteps):
        """nsteps steps; returns the end state and the trapezoid integral of Nu_V dt."""
        integ = 0.0
        for s in range(nsteps):
            X, nu = self.step(X)
            integ += (0.5 if s == 0 else 1.0) * self.dt * nu
        if nsteps > 0:
            integ += 0.5 * self.dt * self.nusselt(X)[0]
        return X, integ

    # ---- diagnostics ----
    def nusselt_from(self, X, wT_mean):
        """(Nu_V, Nu_b, Nu_t), Eqs. 9-11.

        Nu_V = <-dT/dz>_V + <wT>_V: the first term integrates exactly to the
        wall temperature difference of the mean profile (Lz = 1); <wT>_V is the
        Clenshaw-Curtis integral over the padded Lobatto points of the exact
        x-mean of w T.  Nu_b, Nu_t: -dT/dz of the mean profile at z = -1/2, 1/2.
        """
        a = X.T[0].real
        n = np.arange(self.Nz)
        cond = np.sum(a * ((-1.0) ** n - 1.0))
        adv = 0.5 * np.dot(self.cc_weights, wT_mean)
        nu_b = -2.0 * np.sum(a * (-1.0) ** (n + 1) * n * n)
        nu_t = -2.0 * np.sum(a * n * n)
        return cond + adv, nu_b, nu_t

    def nusselt(self, X):
        return self.nusselt_from(X, self.nonlinear(X)[3])

    def diagnostics(self, X):
        """Instantaneous averages behind the consistency checks of Sec. 2.2.

        Fields on the padded grid, products there, exact x-means (the 3/2 rule
        integrates products of the truncated Fourier series exactly), and the
        Clenshaw-Curtis rule over the padded Lobatto points in z (Lz = 1, so
        <f>_V = (1/2) sum_j cc_j <f>_x(s_j)):

          KE2 = <u^2 + w^2>_V        (Re from its square root, Sec. 2.2)
          eps = <u . lap u>_V         (viscous term of the energy balance, Eq. 14)
          wT  = <w T>_V               (buoyancy production P = Ra <w T>_V, Eq. 14)
          nu  = (Nu_V, Nu_b, Nu_t)    (Eqs. 9-11)
          Tm  = <T>_x (Mz,)           at the padded points s_j = cos(pi j/(Mz-1))
          Tv  = <(T - <T>_x)^2>_x (Mz,)

        lap u = (-d_z omega, d_x omega) with omega = -lap psi.
        """
        ik = 1j * self.k[:, None]
        dz = lambda c: c @ self.Dz.T
        u = dz(X.psi)
        u[0] = X.U
        w = -ik * X.psi
        w[0] = 0.0
        om = ik * w - dz(u)
        g = self._spec_to_padded_grid
        ug, wg, Tg = g(u), g(w), g(X.T)
        lap_u, lap_w = -g(dz(om)), g(ik * om)
        vol = lambda f: 0.5 * np.dot(self.cc_weights, f.mean(axis=1))
        KE2 = vol(ug * ug + wg * wg)
        eps = vol(ug * lap_u + wg * lap_w)
        wT_mean = (wg * Tg).mean(axis=1)
        Tm = Tg.mean(axis=1)
        Tv = ((Tg - Tm[:, None]) ** 2).mean(axis=1)
        return dict(KE2=KE2, eps=eps, wT=0.5 * np.dot(self.cc_weights, wT_mean),
                    nu=self.nusselt_from(X, wT_mean), Tm=Tm, Tv=Tv)

    def padded_z(self):
        """z of the padded Lobatto points, z_j = cos(pi j/(Mz-1))/2 (descending)."""
        return 0.5 * np.cos(np.pi * np.arange(self.Mz) / (self.Mz - 1))

    def l2_T(self, X):
        """||T||_{L2(Omega)}: Parseval in x, exact Chebyshev Gram matrix in z."""
        G = us.cheb_gram(self.Nz)
        tot = 0.0
        for m in range(self.nm):
            c = X.T[m]
            q = (c.conj() @ G @ c).real * 0.5                 # int over z in [-1/2, 1/2]
            tot += (1.0 if m == 0 else 2.0) * q
        return np.sqrt(self.Lx * tot)

    # ---- native grid <-> spectral ----
    def from_grid(self, Tg, ug=None, wg=None):
        """Grid values (Nz, Nx) on the native points -> State.

        psi from w (psi_m = i w_m / k, m >= 1), U from the x-mean of u.
        """
        Nx, Nz = self.Nx, self.Nz
        _, z = native_points(Nx, Nz, self.Lx)
        Vn = C.chebvander(2.0 * z, Nz - 1)

        def spec(g):
            h = np.fft.rfft(g, axis=1)[:, : self.nm] / Nx     # (Nz, nm)
            return np.linalg.solve(Vn, h).T                    # (nm, Nz)

        T = spec(Tg)
        T[0] = T[0].real
        psi = np.zeros_like(T)
        U = np.zeros(Nz)
        if wg is not None:
            wh = spec(wg)
            psi[1:] = 1j * wh[1:] / self.k[1:, None]
        if ug is not None:
            U = spec(ug)[0].real
        return State(T, psi, U)

    def to_grid(self, X):
        """State -> (T, u, w) values (Nz, Nx) on the native points."""
        Nx, Nz = self.Nx, self.Nz
        _, z = native_points(Nx, Nz, self.Lx)
        Vn = C.chebvander(2.0 * z, Nz - 1)
        ik = 1j * self.k[:, None]

        def grid(c):
            vz = c @ Vn.T                                       # (nm, Nz points)
            full = np.zeros((Nz, Nx // 2 + 1), dtype=complex)
            full[:, : self.nm] = vz.T
            return np.fft.irfft(full, n=Nx, axis=1) * Nx

        u = X.psi @ self.Dz.T
        u[0] = X.U
        w = -ik * X.psi
        w[0] = 0.0
        return grid(X.T), grid(u), grid(w)

    def zero_state(self):
        z = np.zeros((self.nm, self.Nz), dtype=complex)
        return State(z, z.copy(), np.zeros(self.Nz))


def _scale(X, a):
    return State(X.T * a, X.psi * a, X.U * a)


def restrict(X, Nx_c, Nz_c):
    """Fine -> coarse: keep modes m < Nx_c/2, n < Nz_c (reading of Sec. 3.6)."""
    mc = Nx_c // 2
    return State(X.T[:mc, :Nz_c].copy(), X.psi[:mc, :Nz_c].copy(), X.U[:Nz_c].copy())


def prolong(X, Nx, Nz):
    """Coarse -> fine: zero-pad the coefficient arrays (reading of Sec. 3.6)."""
    nm = Nx // 2
    T = np.zeros((nm, Nz), dtype=complex)
    P = np.zeros((nm, Nz), dtype=complex)
    U = np.zeros(Nz)
    mc, nc = X.T.shape
    T[:mc, :nc] = X.T
    P[:mc, :nc] = X.psi
    U[:nc] = X.U
    return State(T, P, U)
