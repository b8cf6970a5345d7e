"""B300-native GMMNLSE solver: the massively parallel algorithm (MPA) of
Wright et al., "Multimode Nonlinear Fiber Optics: Massively Parallel Numerical
Solver, Tutorial and Outlook" (arXiv:1708.05324), Sec. III.D.

The compute path is the C-ABI library libgmmnlse.so (hand-written sm_103a CUDA);
`binding` is its thin ctypes wrapper.  `inputs` makes seeded synthetic fibers and
pulses.  Importing this package does not load the library; binding.load() does.
"""
__all__ = ["binding", "inputs"]
