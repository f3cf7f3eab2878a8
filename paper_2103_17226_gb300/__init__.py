"""GB300-native batched arithmetic-circuit engine for noisy variational quantum
circuits (Huang et al., "Logical Abstractions for Noisy Variational Quantum
Algorithm Simulation", ASPLOS 2021).

  inputs      seeded synthetic workloads (gate lists, graphs, angles, seeds)
  native      ctypes binding of libqkc: compile, load_ac, set_params, evaluate,
              marginals, gradient, sample
  build       in-tree build of libqkc.so for sm_103a
"""
