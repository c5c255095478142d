"""FP64 CPU oracle for the Pressure Schur Complement Stokes solve (test infrastructure).

This package is the slow, plain reference that the CUDA path is checked against.  It
assembles the staggered (MAC) operators A, B and B^T as explicit sparse matrices and
runs the Krylov methods of Section 3 step by step in double precision.  It shares no
code with the CUDA library: only the seeded input generators
(``paper_2307_05266_gb300.synth``) feed both sides.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it; the product path never does.

Modules
-------
``mac``     face classification, face flags, sparse A, B, B^T, force (Section 2, eq.
            coupled_matrix, interior_boundary, MAC placement).
``krylov``  Jacobi-preconditioned CG for A and for the SIMPLE operator, and the outer
            preconditioned CG on S (Algorithm 1, eqs. schur_system, schur_rhs,
            schur_uzawa_prec, velocity_schur).
``stokes``  the whole path: RHS, outer solve, velocity recovery, permeability (eq.
            darcy_law), plus geometry statistics (eqs. porosity, s-t-v-ration,
            surface_area).
``dense``   dense Schur complements, spectra and minimum-norm solutions for tiny grids.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` against a closed form, an invariant, a value the paper
prints, or brute force.
"""
