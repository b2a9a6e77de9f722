"""Oracle: a plain, slow, FP64 CPU restatement of the paper's method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
It shares no code with the CUDA path (``paper_1412_0464_gb300``); the only
common dependency is the seeded input generator package ``synth``.

Paper: C. C. Stolk, "An improved sweeping domain decomposition
preconditioner for the Helmholtz equation" (arXiv 1412.0464).

Contents (each module cites the passage it follows):

* ``mesh``    -- 1-D meshes, PML damping profile (Eq. 5) and the PML factors
                 alpha = 1/(1 + i sigma/omega) (below Eq. 40).
* ``fd``      -- fine 5-point (2-D) / 7-point (3-D) / 3-point (1-D) finite
                 difference operator with PML (Eq. 40), scaled by h^d.
* ``fe``      -- coarse optimised finite-element operator with PML-aware
                 coarsening (Section 4.2, Appendix A: Eqs. 43-47, 53-63,
                 Table 9), prolongation/restriction (Eqs. 41-42).
* ``dd``      -- the double-sweep domain decomposition: partitions (Eq. 17),
                 subdomains with frozen k and added PML (Eqs. 9-10),
                 transmission (Eqs. 19-20), SubdomSolve / ForwardSweep /
                 BackwardSweep / MidSolveIn / MidSolveOut (Table 2),
                 SweepingPrecUD / SweepingPrecX (Table 3).
* ``twogrid`` -- the two-grid sweeping preconditioner (Section 4).
* ``gmres``   -- restarted, right-preconditioned GMRES(m) (Section 4,
                 stopping rule of Section 6.1).
* ``problem`` -- assembles the above for a ``synth.Workload``.

Parity status: every function is pinned by ``tests/test_oracle_*.py``
except where a docstring says "parity unpinned".
"""
