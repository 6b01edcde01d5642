"""FP64 CPU oracle of the coupled level-set lattice Boltzmann method (arXiv 2601.05936).

TEST INFRASTRUCTURE ONLY.  This package is imported solely by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py``.  The CUDA library and its Python binding never import it, and it
imports nothing from them: the two implementations share no code.  The only
module both sides consume is the seeded input generator
``paper_2601_05936_gb300/workloads.py``, which holds geometry and parameter
recipes but none of the method's arithmetic (the oracle does not import it
either; tests pass its outputs in).

Everything here is plain numpy in float64, written step by step from the paper:

* ``lattice``  - velocity sets D2Q9 / D3Q19 / D3Q27 (Sec. 2.1, Fig. 1).
* ``lbm``      - moments, equilibrium, BGK + forcing, strain rate (Sec. 2.1, Eq. 1-6).
* ``levelset`` - upwind-5 / TVD-RK3 advection, hyperbolic extension,
                 constrained reinitialisation, least-squares geometry (Sec. 2.2).
* ``coupling`` - interface bounce-back with the stress jump (Sec. 2.3, Eq. bb,
                 bb_cc, Sdecomp) and refill of new cells (Sec. 2.4).
* ``amr``      - block sensor, grading, level masks, Dupuis-Chopard coupling
                 (Sec. 2.1 last paragraph, Sec. 2.6, Sec. 3.2.2).
* ``sim``      - the time step that composes all of the above.

Parity status per function is stated in each module header.  Readings of
passages that are garbled or silent are listed where they are used.
"""
