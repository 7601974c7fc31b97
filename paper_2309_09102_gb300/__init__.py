"""GB300-native core of the CppFlow Cartesian path planner (arXiv 2309.09102).

Everything after candidate generation -- batched DH forward kinematics with
SE(3) pose error, joint-limit / pose masking, the dynamic-programming search
over the T x K x K candidate lattice, and per-waypoint Levenberg-Marquardt
refinement -- runs in hand-written sm_103a CUDA kernels behind the C ABI in
``include/cppflow.h``. ``paper_2309_09102_gb300.cppflow`` is the thin ctypes
binding; ``paper_2309_09102_gb300.synth`` draws seeded synthetic inputs.

Importing the package does not load the CUDA library; ``cppflow.lib()`` does,
and raises if the library has not been built.
"""
__all__ = ["synth", "cppflow"]
