"""The oracle's pins catch plausible mistakes.

Each test plants one mistake in the oracle (on the CPU, through monkeypatch)
and checks that the pin meant to guard against it now fails: a flipped sign,
a dropped term, a missing factor, a transposed operand, a wrong tableau entry,
a wrong quadrature weight.  A pin that still passed with the mistake in place
would not be pinning anything.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import test_oracle_diagnostics as diag
import test_oracle_fixed_flux as ff
import test_oracle_pins as pins
import test_oracle_tableau as tableau
import test_oracle_transfer as transfer
from oracle import rbc as orbc
from oracle import statistics as ost

ORIG_RESTRICT, ORIG_PROLONG = orbc.restrict, orbc.prolong

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_flipped_buoyancy_sign_fails_the_onset_pin(monkeypatch):
    orig = orbc.RBC.ops_psi

    def ops_psi(self, k):
        M, L, Cpl = orig(self, k)
        return M, L, -Cpl
    monkeypatch.setattr(orbc.RBC, "ops_psi", ops_psi)
    with pytest.raises(AssertionError):
        pins.test_P4_oracle_operators_match_collocation_growth_rate(2500.0)


def test_dropped_k2_in_the_temperature_laplacian_fails_the_diffusion_pin(monkeypatch):
    monkeypatch.setattr(orbc.RBC, "ops_T", lambda self, k: (self.S2, 4.0 * self.D2))
    with pytest.raises(AssertionError):
        pins.test_P2_temperature_diffusion_decays_by_the_stability_function()


def test_missing_prandtl_in_the_mean_flow_fails_its_decay_pin(monkeypatch):
    monkeypatch.setattr(orbc.RBC, "ops_U", lambda self: (self.S2, 4.0 * self.D2))
    with pytest.raises(AssertionError):
        pins.test_P2_mean_flow_viscous_decay_with_Pr()


def test_wrong_slope_boundary_row_fails_the_onset_pin(monkeypatch):
    orig = orbc.RBC.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        # the wall-slope row with n instead of n^2 (d T_n / ds at s = 1): a different constraint
        self.bc_slope_hi = self.bc_slope_hi / np.maximum(1.0, np.arange(self.Nz))
        self._factor()
    monkeypatch.setattr(orbc.RBC, "__init__", init)
    with pytest.raises(AssertionError):
        pins.test_P4_oracle_operators_match_collocation_growth_rate(2500.0)


def test_transposed_advection_operands_fail_the_dealiasing_pin(monkeypatch):
    orig = orbc.RBC.nonlinear

    def nonlinear(self, X):
        # u d_x T + w d_z T planted as u d_z T + w d_x T: swap T's two derivatives
        Xs = orbc.State(X.T.copy(), X.psi, X.U)
        ik = 1j * self.k[:, None]
        dzT = X.T @ self.Dz.T
        # a state whose d/dx is the true d/dz and vice versa is not available in
        # general; emulate the swap on the product by recomputing with ik and Dz exchanged
        NT, NO, NU, wT = orig(self, Xs)
        g = self._spec_to_padded_grid
        u = X.psi @ self.Dz.T
        u[0] = X.U
        w = -ik * X.psi
        w[0] = 0.0
        NT = self._padded_grid_to_spec(g(u) * g(dzT) + g(w) * g(ik * X.T))
        return NT, NO, NU, wT
    monkeypatch.setattr(orbc.RBC, "nonlinear", nonlinear)
    with pytest.raises(AssertionError):
        pins.test_P5_dealiased_products_equal_exact_truncated_convolution()


def test_wrong_tableau_entry_fails_the_order_conditions(monkeypatch):
    AE = [row[:] for row in tableau.AE]
    AE[2][1], AE[2][0] = AE[2][0], AE[2][1]           # two explicit weights of stage 2 swapped
    monkeypatch.setattr(tableau, "AE", AE)
    monkeypatch.setattr(tableau, "bE", AE[4])
    failures = 0
    for name in dir(tableau):
        if name.startswith("test_"):
            try:
                getattr(tableau, name)()
            except AssertionError:
                failures += 1
    assert failures >= 1


def test_reversed_quadrature_weights_fail_the_nusselt_pin(monkeypatch):
    orig = orbc.RBC.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        self.cc_weights = self.cc_weights[::-1] * np.linspace(0.5, 1.5, len(self.cc_weights))
    monkeypatch.setattr(orbc.RBC, "__init__", init)
    with pytest.raises(AssertionError):
        pins.test_nusselt_volume_term_against_brute_force_quadrature()


def _planted_diagnostics(monkeypatch, change):
    orig = orbc.RBC.diagnostics

    def diagnostics(self, X):
        d = dict(orig(self, X))
        change(d)
        return d
    monkeypatch.setattr(orbc.RBC, "diagnostics", diagnostics)


def test_flipped_viscous_term_fails_the_energy_budget_pin(monkeypatch):
    def change(d):
        d["eps"] = -d["eps"]
    _planted_diagnostics(monkeypatch, change)
    with pytest.raises(AssertionError):
        diag.test_D3_kinetic_energy_budget_along_the_dynamics()


def test_halved_kinetic_energy_fails_the_energy_budget_pin(monkeypatch):
    def change(d):
        d["KE2"] = 0.5 * d["KE2"]                     # (1/2)|u|^2 in place of |u|^2
    _planted_diagnostics(monkeypatch, change)
    with pytest.raises(AssertionError):
        diag.test_D3_kinetic_energy_budget_along_the_dynamics()


def test_variance_about_zero_fails_the_brute_force_variance_pin(monkeypatch):
    def change(d):
        d["Tv"] = d["Tv"] + d["Tm"] ** 2              # <T^2>_x, the plane mean not removed
    _planted_diagnostics(monkeypatch, change)
    with pytest.raises(AssertionError):
        diag.test_D5_plane_mean_and_variance_by_brute_force()


def test_left_endpoint_time_rule_fails_the_trapezoid_pin(monkeypatch):
    def run_sampled(rbc, X, nsteps, every):
        prev = ost.sample(rbc, X)
        acc = {q: 0.0 * v for q, v in prev.items()}
        s = 0
        while s < nsteps:
            c = min(every, nsteps - s)
            for _ in range(c):
                X, _ = rbc.step(X)
            for q in acc:
                acc[q] = acc[q] + c * rbc.dt * prev[q]
            prev = ost.sample(rbc, X)
            s += c
        acc["T"] = nsteps * rbc.dt
        return X, acc
    monkeypatch.setattr(ost, "run_sampled", run_sampled)
    with pytest.raises(AssertionError):
        diag.test_D7_trapezoid_integrals_of_pure_diffusion()


def _planted_flux_rows(monkeypatch, change):
    orig = orbc.RBC.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        if self.bc == "fixed_flux":
            change(self)
            self._factor()
    monkeypatch.setattr(orbc.RBC, "__init__", init)


def test_flipped_wall_flux_fails_the_fixed_flux_conduction_pin(monkeypatch):
    def change(r):
        r.T_bc_val = (0.5, 0.5)                         # dT/dz = +1: heat drawn out at the bottom
    _planted_flux_rows(monkeypatch, change)
    with pytest.raises(AssertionError):
        ff.test_FF1_conduction_is_a_fixed_point()


def test_value_rows_for_fixed_flux_fail_the_neumann_decay_pin(monkeypatch):
    def change(r):
        r.T_bc_lo, r.T_bc_hi = r.bc_val_lo, r.bc_val_hi
    _planted_flux_rows(monkeypatch, change)
    with pytest.raises(AssertionError):
        ff.test_FF2_neumann_mode_decays_by_the_stability_function(1)


def test_unmutated_oracle_passes_the_same_pins():
    pins.test_P4_oracle_operators_match_collocation_growth_rate(2500.0)
    pins.test_P2_temperature_diffusion_decays_by_the_stability_function()
    pins.test_P2_mean_flow_viscous_decay_with_Pr()
    pins.test_P5_dealiased_products_equal_exact_truncated_convolution()
    pins.test_nusselt_volume_term_against_brute_force_quadrature()
    diag.test_D3_kinetic_energy_budget_along_the_dynamics()
    diag.test_D5_plane_mean_and_variance_by_brute_force()
    diag.test_D7_trapezoid_integrals_of_pure_diffusion()
    ff.test_FF1_conduction_is_a_fixed_point()
    ff.test_FF2_neumann_mode_decays_by_the_stability_function(1)
    assert Fr(1, 2) == tableau.AI[1][1]


def _restrict_without_mean_flow(X, Nx_c, Nz_c):
    Xc = ORIG_RESTRICT(X, Nx_c, Nz_c)
    Xc.U = np.zeros_like(Xc.U)
    return Xc


def _restrict_wrong_modes(X, Nx_c, Nz_c):
    # keeps the last Fourier modes instead of the first
    mc = Nx_c // 2
    return orbc.State(X.T[-mc:, :Nz_c].copy(), X.psi[-mc:, :Nz_c].copy(), X.U[:Nz_c].copy())


@pytest.mark.parametrize("mistake", [_restrict_without_mean_flow, _restrict_wrong_modes])
def test_broken_restriction_fails_the_projection_pin(monkeypatch, mistake):
    monkeypatch.setattr(orbc, "restrict", mistake)
    with pytest.raises(AssertionError):
        transfer.test_restriction_residual_is_orthogonal_to_the_coarse_space((16, 12), (8, 8))


def test_prolongation_without_mean_flow_fails_the_point_evaluation_pin(monkeypatch):
    def prolong(X, Nx, Nz):
        Xf = ORIG_PROLONG(X, Nx, Nz)
        Xf.U = np.zeros_like(Xf.U)
        return Xf
    monkeypatch.setattr(orbc, "prolong", prolong)
    with pytest.raises(AssertionError):
        transfer.test_prolongation_represents_the_same_fields((8, 8), (16, 12))


def test_prolongation_with_shifted_chebyshev_modes_fails_the_point_evaluation_pin(monkeypatch):
    def prolong(X, Nx, Nz):
        Xf = ORIG_PROLONG(X, Nx, Nz)
        Xf.T = np.roll(Xf.T, 1, axis=1)
        return Xf
    monkeypatch.setattr(orbc, "prolong", prolong)
    with pytest.raises(AssertionError):
        transfer.test_prolongation_represents_the_same_fields((8, 8), (16, 12))


def test_swapped_explicit_weights_of_rk222_fail_its_order_pin(monkeypatch):
    import test_oracle_schemes as schemes
    c, AI, AE = orbc.SCHEMES["RK222"]
    bad = [row[:] for row in AE]
    bad[2][0], bad[2][1] = bad[2][1], bad[2][0]      # delta and 1 - delta exchanged
    monkeypatch.setitem(orbc.SCHEMES, "RK222", (c, AI, bad))
    ref = schemes._convect(0.024 / 1536, "RK443")
    with pytest.raises(AssertionError):
        schemes.test_S4_observed_order_of_convergence("RK222", ref)


@pytest.mark.parametrize("name", ["RK222", "RK111"])
def test_wrong_implicit_diagonal_fails_the_closed_form_decay_pin(monkeypatch, name):
    import test_oracle_schemes as schemes
    c, AI, AE = orbc.SCHEMES[name]
    bad = [row[:] for row in AI]
    for i in range(1, len(bad)):
        bad[i][i] = 0.9 * bad[i][i]
    monkeypatch.setitem(orbc.SCHEMES, name, (c, bad, AE))
    with pytest.raises(AssertionError):
        schemes.test_S3_temperature_mode_decays_by_the_closed_form(name)


def test_unmutated_lower_order_schemes_pass_the_same_pins():
    import test_oracle_schemes as schemes
    for name in ("RK222", "RK111"):
        schemes.test_S3_temperature_mode_decays_by_the_closed_form(name)
