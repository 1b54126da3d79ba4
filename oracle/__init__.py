"""CPU oracle for RNS-CKKS public-key encryption, vanilla and Zinc (arXiv 2408.07304).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or execute anything in this package.  The GPU library never uses it, and
this package never imports the GPU library: the two share no code, tables or
constants.  Where both sides must follow the same convention (prime rule,
root rule, sampler counter layout, encoder FFT operation order) each side
implements it separately from the written definition.

Modules
-------
numtheory  primes q = 1 mod 2N, the minimal primitive 2N-th root psi, brv
philox     Philox4x32-10 counter-based generator (Salmon et al., SC'11)
sampler    R_2 (ternary), chi (rounded Gaussian, sigma = 3.2, CDT), R_q (uniform)
           -- Section "Polynomials and Distributions"
encoder    CKKS canonical-embedding encoder / decoder (FP64)
ring       definitional negacyclic NTT and schoolbook products (C, via ctypes)
ckks       Gen (Eq. 7), Enc (Eq. 8), Enc_z (Algorithm 1, Eq. 9), Dec (Eq. 10),
           the modulus-switched (special-prime) Enc
bfvbgv     BFV (Eq. 12) and BGV (Eq. 13) encryption, their Zinc forms, Dec
nttrand    Zinc with its errors generated in the NTT domain (a reading of the
           Conclusion's O(N) remark): rotations of a cached error basis

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, brute force, an invariant, or an independent library routine,
except the conventions the paper leaves open (prime choice, root choice,
counter layout, FFT operation order); those are pinned only by their written
definition and the agreement of two independent implementations.
"""
