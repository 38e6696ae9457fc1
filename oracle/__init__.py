"""Plain, slow FP64 CPU oracle of the black-oil FIM linearisation.

TEST INFRASTRUCTURE ONLY.  This package is the checker that the CUDA library
is compared against.  It shares no code with the library (no kernels, headers,
helpers, tables or constant generators) and the library never imports it; only
the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import or run anything in here.

Contents:
* ``dual``       forward-mode dual numbers with a running magnitude bound;
* ``blackoil``   cell properties (PVT tables, rock, Corey, Stone II, Pc);
* ``linearize``  residual, dual-number Jacobian in block-CSR form, and the
                 vector-Jacobian products with respect to the new state, the
                 old state, ln k and porosity;
* ``spmv``       block-CSR matrix-vector products written as plain loops;
* ``newton``     a small Newton time stepper with a library sparse solve
                 (used by the Buckley-Leverett pin and the gradient checks);
* ``adjoint``    multi-step simulation and its discrete-adjoint gradient;
* ``coupling``   the adaptive subdomain coupling of Sec. 4 (marked cells,
                 coupling graph, connected components);
* ``pn``         the equations in pressure and component amounts with the
                 volume balance (Sec. 2.1, eq. 4), its explicit black-oil
                 phase split, the elimination of the volume rows, and a
                 Newton step in those unknowns;
* ``impec``      one IMPEC step in those unknowns: the pressure equation
                 from the linearised volume balance with coefficients frozen
                 at the old level, its direct solve, and the explicit update.

Parity status of each function is listed in the design notes; all of them are
pinned by the CPU tests (``tests/test_oracle_*.py``).
"""
