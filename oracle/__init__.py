"""FP64 CPU oracle for MPS TE-PAI (test infrastructure only).

This package is the plain, slow and obviously correct restatement of the
method. Parity tests compare the CUDA path against it. Only the test suite,
the smoke check and the benchmark's CPU-baseline leg may import it. The
product path never calls it, and it shares no code with the CUDA library.

Modules and the passages they follow:
  planner     term list, rotation angles, PAI coefficients, sampling
              probabilities and the quasi-probability norm (App. A.3, Eq. gammas;
              App. A.6, Eq. overhead-bound; App. A.5, Eq. ap:eq_nu_infty)
  philox      the Philox4x64-10 counter-based generator (Salmon et al., SC'11)
  sampler     the TE-PAI circuit sampler (Sec. II.B protocol; App. A.3)
  gates       Pauli-rotation gates R_k(theta) = exp(-i h_k theta / 2) (App. A.3)
  statevector dense state vector, exact evolution (Eq. Trotter-Suzuki)
  mps         matrix product state with two-site SVD updates (Sec. II.A)
  estimator   signed, ||g||_1-weighted ensemble mean (App. B; Statement 2)
  enumerate   brute-force sum over all gate settings (Statement 1)
  run         one full ensemble run built from the above

Pin status: every function is pinned by a CPU test (tests/test_oracle_*.py).
None is "parity unpinned".
"""
