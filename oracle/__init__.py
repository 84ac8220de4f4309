"""Plain FP64 CPU oracle for the batched quantum-trajectory TEBD hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may use it.  It shares no code with the CUDA
library; both sides receive the same seeded inputs from ``workloads.py``.

Modules
  philox   counter-based Philox4x32-10 generator (Salmon et al., SC'11), the
           one random source the trajectory method draws from (Sec. 4.1).
  model    the free-fermion chain, its jump operators and the two-site
           effective-Hamiltonian gates (Sec. 2.1, Eqs. Hamiltonian,
           EffHamiltonian; Sec. 2.3 Trotter splitting).
  tebd     the MPS quantum-trajectory integrator in Vidal-Hastings form
           (Sec. 2.3 Eq. Theta, Sec. 4.1 Eqs. QJump1, TransitionRate).
  mpdo     the vectorised density matrix (MPDO, d^2 = 4) under Liouvillian
           TEBD gates (Sec. 3.1, Eqs. Choi, LindbladChoi, Liouvillian, MPDO),
           with traces Tr(O rho) / Tr rho for the observables.
  purified the locally purified density matrix rho = X X^+ (Sec. 3.2, Eqs.
           Purified, ThetaPurified, MatrixR, NewPurified): effective-Hamiltonian
           layers on X with a Kraus index per site, then the R step per site.
  slater   the exact untruncated history of the free-fermion chain for a given
           jump record: every gate and jump maps a Slater determinant to a
           Slater determinant, so a history is N orbitals (Sec. 2.1, Sec. 4.1);
           it sizes the truncation error of the MPS histories at any L.
  dense    brute-force references: the dense Trotterised state vector, dense
           Lindblad integration of rho, and the correlation-matrix equation of
           motion (Sec. 2.1 Eqs. eqCorr, SoleqCorr; Eq. Lindblad).

All floating point is float64 / complex128.
"""
