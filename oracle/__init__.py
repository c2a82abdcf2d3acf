"""Plain FP64 CPU oracle of the real-space Kohn-Sham SCF with CheFSI (SPARC, Sec. 2-2.1).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run it.  The CUDA
library and its Python binding never import it, and it imports nothing from them: the two
share only the seeded input generators in ``workloads``.

Every function is written for clarity, not speed, in float64 (complex128 for Bloch
orbitals), following the paper's equations and the published methods the paper names:

* fd        -- high-order centred finite differences on a uniform periodic grid (Sec. 2.1)
* model     -- Gaussian pseudocharges, Kleinman-Bylander projectors, SAD guess (Sec. 2.1)
* xc        -- Perdew-Zunger LDA (Sec. 3; Perdew & Zunger, PRB 23, 5048, 1981)
* ham       -- matrix-free H.X (Eq. 1), dense H for brute force, exact discrete Poisson,
               Fermi-Dirac occupations and density (Eq. 2)
* chefsi    -- Lanczos bounds, Chebyshev filter and Rayleigh-Ritz (Sec. 2.1; Zhou et al. 2006)
* scf       -- restarted periodic Pulay mixing, free energy, forces, the SCF loop (Sec. 2.1)

Parity status of each function is stated in its docstring ("pinned by ..." naming the
tests under tests/test_oracle_*.py that tie it to closed forms, brute force or invariants).
"""
