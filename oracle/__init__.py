"""FP64 CPU oracle of the phase-field lattice Boltzmann step (test infrastructure).

This package is the correctness reference for the CUDA path and nothing else:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path in
``paper_2003_06342_b300`` never imports, calls or falls back to it.

It is a plain, slow, obviously correct restatement of the method of
Verdier, Kestener & Cartalade, "Performance portability of lattice Boltzmann
methods for two-phase flows with phase change" (arXiv:2003.06342), written in
PyTorch CPU float64 ops, vectorised over lattice cells only, with every sum over
directions taken in lattice order i = 0..Q-1.  Each function cites the section
or equation it follows.

Modules
-------
lattice       D2Q9 / D3Q7 / D3Q19 tables (Sec. 3, lattice definitions).
model         one time step, initialisation, moments, streaming map and the
              global reductions (Sec. 2 model, Sec. 3 schemes, App. C).
closed_forms  Stefan solution (Sec. 4.2), layered Poiseuille (Sec. 4.1),
              Laplace law, coefficient A (App. B).
adjoint       reverse-mode gradient of a final-time phase-field misfit, by
              torch autograd through ``model.step`` (no hand derivation).

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
fully coupled film-boiling trajectory, whose parity is pinned only through its
components and invariants (the paper prints no field values for it): phase
mass balance with the source on, the enthalpy invariant of the temperature
scheme, the energy sum's hand value, stationarity of a flat interface.
"""
