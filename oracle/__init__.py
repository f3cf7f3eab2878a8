"""The oracle: plain, slow, obviously correct CPU FP64 implementations of what the
GPU engine computes.  TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check in __graft_entry__ and the CPU-baseline leg
of bench.py may import, call or link anything in this package.  The product
path (paper_2103_17226_gb300) never does, and shares no code with it: the only
module both sides use is paper_2103_17226_gb300.inputs, which builds seeded gate
lists and numbers and holds none of the method's arithmetic.

Modules
  quantum  -- textbook quantum mechanics: state-vector and density-matrix
              simulation, Kraus channels, outcome probabilities, evidence
              polynomials, marginals, Z-string expectations, exact angle
              gradients (forward mode), chain-rule sampling.  Ground truth.
  bn       -- the paper's Bayesian-network semantics (Sec. 3.1) evaluated by
              brute force over every assignment of every BN variable.
  gibbs    -- the paper's Gibbs sampler (Sec. 3.3.2) with every candidate amplitude
              recomputed by a pure-state run.
  acref    -- ctypes binding of acref.c, a plain FP64 evaluator of compiled
              ACs (upward and downward pass, gradient, chain-rule sampler),
              the timed CPU baseline.
"""
