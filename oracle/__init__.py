"""FP64 CPU oracle for the fourth-order cut-cell multigrid method (arXiv 2410.05865).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is a plain, slow, obviously-correct restatement of the paper in
numpy/scipy, written independently of the CUDA path (no shared code, tables or
helpers; the only shared module is ``workloads``, which holds the seeded problem
definitions and none of the method's arithmetic).

Modules
-------
geometry        cell classification and cut-cell quadrature (Sec. 2.2, Sec. 3)
discretization  merging (Alg. CellMerging), the phi1/phi2 split, the regular
                and ghost rows (eq. regularLaplaceDiscretization and the ghost
                formulas of Sec. 2.3), FV-PLG lattices and the WLS rows
                (Sec. 2.3, Sec. 4.1), the discrete system (Sec. 2.4)
multigrid       SMO-1, SMO-2, Restrict/Prolong, Alg. VCycle, Alg. Multigrid,
                Alg. FMG (Sec. 5.3, Sec. 5.4)

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms, polynomial exactness, brute-force dense solves and convergence
rates (see the docstring of each test).
"""
