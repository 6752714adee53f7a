"""FP64 CPU oracle for Scaled Block Vecchia (arxiv 2504.12004).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does,
and the oracle imports nothing from the product package.

Modules
  prng   -- SplitMix64 and Lemire's bounded draw (the random choices of RAC
            anchors, Alg. 3, and of the block order, Alg. 1 Step 2).
  sbv    -- scaling (Alg. 2), RAC + Lloyd blocking (Alg. 3), random block order,
            earlier-ordered m-NN (Alg. 4 / Eq. mmsearchingBV), the scaled Matern
            kernel (Eqs. scale, maternkernel), the batched block log-likelihood
            (Alg. 5), the total (Alg. 1 Step 5) and prediction (Sec. 4.2, 5.5).
  mlp    -- FP64 forward/backward of the surrogate network (GELU, MSE) and Adam,
            with an emulation of the GPU's BF16 operand rounding.
  mle    -- maximum-likelihood estimation over log theta (library optimiser),
            with the scale-family closed form used as a pin.
  grad   -- d l / d theta of the block terms (Gaussian log-density derivative
            of the block conditional, dense inverses and traces), pinned by
            central differences of sbv.block_loglik and a closed form.

Parity status: every function is pinned by a test in tests/test_oracle_*.py
except the blocking trajectory itself (RAC anchors, Lloyd iterations, block
order), whose exact output the paper does not fix: it is "parity unpinned"
against the paper and pinned only by invariants (each point sits in the block
of its nearest final centre, the order is a bijection, T=0 equals RAC).
"""
