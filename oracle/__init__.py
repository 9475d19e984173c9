"""FP64 CPU oracle for the FFT Lippmann-Schwinger iteration of Milton's paper
"Substitution of subspace collections with nonorthogonal subspaces to
accelerate Fast Fourier Transform methods applied to conducting composites".

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything in this package: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the
CUDA path; both sides draw their inputs from the seeded generators in
``synth``.

The oracle is plain and slow on purpose: library FFTs (scipy.fft on every
host core, pinned against a brute-force DFT), the Green operator written out
per frequency from Eq. J11, the four schemes written step by step in the
paper's notation, and an exact discrete
solution by a dense direct solve whose eigen-decomposition gives the poles of
sigma_*(sigma_1).

Modules
-------
fourier    frequencies, brute-force DFT, the Green projection Gamma_1 (Eq. J11,
           Eq. J45) for the trigonometric and forward-difference symbols.
constants  scheme constants: reference media, t(sigma_1) (Eq. J3/J23), the
           vector p (Eq. J24 solved for p), E_2' (Eq. J21), J_3' (Eq. J26).
schemes    Moulinec-Suquet (Eq. J0-0, J1), Eyre-Milton (Eq. J2), and both applied
           in the substituted space H'' (Eq. J36, J42a, J43, J44), with the stop rule.
exact      dense direct solve of Eq. J12/J13, poles and weights, the pole hull
           [alpha, beta], energy and gradient identities.
lanczos    Lanczos estimate of [alpha, beta] from the Krylov space of chi Gamma chi.

Parity status: every function here is pinned by a `-m "not gpu"` test against
closed forms, invariants or brute force (see tests/test_oracle_*.py).
"""
