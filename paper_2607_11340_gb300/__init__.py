"""GB300-native CR-Solver hot path: batched tendon-driven PCC kinematics, penalised cost,
hand-written adjoint and Levenberg-Marquardt, behind a C-ABI CUDA library (libcrsolver.so).

Importing the package does not load the CUDA library; the first call into ``api`` does, and it
raises if the library is missing or was not built (there is no CPU fallback).
"""

__all__ = ["synth", "api", "lib"]
