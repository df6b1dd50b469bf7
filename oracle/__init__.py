"""FP64 CPU oracle for the Nystrom kernel filter (Nair & Chaudhury, arXiv 1901.06112).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
shares no code with the CUDA path; both sides take their inputs from the seeded
generators in ``paper_1901_06112_gb300.synth`` (which hold none of the method's
arithmetic), and this package does not import that module either.

Contents (every function cites the passage it follows):

* ``kernels``    -- the range kernel kappa and spatial kernel omega (Sec. II, Sec. IV setup)
* ``guide``      -- the nonlocal-means patch guide (Sec. II, Sec. IV "Color NLM")
* ``bruteforce`` -- the exact kernel filter, Eq. (1)
* ``rng``        -- SplitMix64 and the seeded index draws both sides implement
* ``kmeans``     -- Lloyd k-means landmark selection (Sec. III, Algorithm 1)
* ``nystrom``    -- Eqs. (9)-(12), (14)-(15) and Algorithm 1, in the paper's notation
* ``bound``      -- explicit K, K-hat and the Theorem 1 error bound (supplement proof)
* ``grad``       -- FP64 gradients of the Nystrom filter (PyTorch CPU autograd)

Everything computes in float64.  Parity status of each function is stated in
its module docstring; Proposition 1's constants c1, c2 are not given by the
paper, so Proposition 1 itself is "parity unpinned" (only its trend is tested).
"""
