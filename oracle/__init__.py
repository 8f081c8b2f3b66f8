"""FP64 CPU oracle of the hybrid beamline tracking path (test infrastructure).

This package is the plain, slow, obviously correct statement of what the GPU
library computes: linear element maps, the prescribed-wake RK4 plasma stage,
the MLP surrogate with its gradient, MSE, Adam, beam moments and the adjoint
of the final moments with respect to quadrupole strengths. It is test
infrastructure: only the test suite, the smoke check and the timed CPU
baseline of the benchmark may import it. It shares no code with the CUDA
library and never imports it; both sides read the same seeded inputs from
the separate ``synth`` package.

Parity status of each part is given in the header of its module.
"""
