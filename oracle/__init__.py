"""Plain FP64 CPU oracle of the 2D Rayleigh-Benard Parareal scheme.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call, link or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` (as a checker)
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) use it.

It is a slow, obviously-correct restatement of the method in NumPy/SciPy:

* ``ultraspherical`` - Chebyshev/ultraspherical conversion and derivative
  operators (the tau discretisation in z of the linear terms, Sec. 3.2).
* ``rbc``            - the Boussinesq equations (Eqs. 3-6) in streamfunction form,
  Fourier(x) x Chebyshev(z) collocation with 3/2-rule dealiasing, IMEX RK443
  time stepping (Sec. 3.2, Sec. 3.6; the lower-order RK222 and RK111 of the
  same family for coarse propagators), the Nusselt numbers (Eqs. 9-11).
* ``parareal``       - the Parareal iteration (Eq. 20) with the defect and
  Nusselt stopping norms (Sec. 3.7) and a statistical stopping rule.
* ``statistics``     - sampled time means and the consistency checks of
  Sec. 2.2 (Re, Nu_int, the P / eps_U balance, T_rms, delta_T, N_BL).

``rbc`` also takes fixed-flux walls (Eq. 7) and forms the instantaneous
averages of Sec. 2.2 (``RBC.diagnostics``).

Every function cites the passage of the paper it follows.  The oracle shares no
code with the CUDA library; only the seeded input generator
(``paper_2001_01609_gb300.inputs``) feeds both.
"""
