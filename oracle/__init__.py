"""FP64 CPU oracle for the shaped-stencil acoustic leapfrog.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library (``paper_2606_04882_gb300``); the only
common module is ``workloads`` (seeded inputs, no method arithmetic).

Contents (each function cites the passage of the paper it restates):
  * ``stencil``  - point sets of the five stencil shapes, symmetry orbits, the
                   weight systems of every scheme (SpatTE, SpecTE-theta, SpecLS,
                   DispTE, DispTE-theta, DispLS), the exact dispersion symbol and
                   the von Neumann CFL bound.
  * ``physics``  - Ricker wavelet, sponge damping profile, model padding.
  * ``wave``     - the time loop (plain C, fp64, ``wave_oracle.c``) for the
                   forward problem, receiver traces, and the discrete adjoint /
                   FWI gradient with respect to m = 1/v^2.

Pinned by ``tests/test_oracle_*.py`` against closed forms, textbook values,
exact discrete solutions and brute force (see each test's docstring).  The
least-squares weight schemes are pinned by the closed-form minimiser of the
one-unknown case, by normal equations built and solved independently for two
and three unknowns, and by the exact (50-digit) minimum of the paper's error
functional for every DispLS stencil the workloads run.  Where a design matrix
has singular values below the 1e-10 cutoff (Square(8)), the functional does not
fix the weights; the minimum-norm choice among near-minimisers is a reading of
the paper, and only that property (and the functional's value) pins it.
"""
