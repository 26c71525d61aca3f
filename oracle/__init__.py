"""Oracle: a plain, slow, FP64 CPU restatement of the paper's solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It shares
no code with the CUDA path (no kernels, headers, tables or helpers); the only common
dependency is the seeded input generator in ``synth``.

Modules:
  wilson  -- gamma matrices, Wilson hopping term (Eq. 2), clover term (Eq. 3) and the
             Wilson-clover operator A (Eq. 1); a per-site variant for sampled checks.
  dd      -- domains and colours, block-diagonal D / coupling R split (Sec. II-D),
             even-odd Schur complement (Eq. 5), MR domain solver, multiplicative SAP
             (Table I).
  fgmres  -- flexible GMRES with deflated restarts (Table I, outer solver).
  dense   -- explicit dense A on tiny lattices, built site by site, for brute force.
  loadmodel -- domain count and load of Eqs. 6-7.

Canonical layouts (shared with the input generator): spinor complex128
(Lt, Lz, Ly, Lx, 4, 3); gauge complex128 (Lt, Lz, Ly, Lx, 4, 3, 3) with forward links.
"""
