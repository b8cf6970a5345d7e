"""CPU FP64 oracle for the GMMNLSE massively parallel algorithm (MPA).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: it is used by tests/, by __graft_entry__.smoke() (to
check one GPU result) and by bench.py's cpu_baseline / reference leg.  It
shares no code with the CUDA library; the two meet only in the seeded input
arrays (paper_1708_05324_b300.inputs), which hold none of the method's
arithmetic.

Parity status per function: every public function in oracle.gmmnlse is pinned
by a test in tests/test_oracle_pins.py (the added Sec. IV terms in
tests/test_oracle_coupling.py, the overlap tensor in tests/test_oracle_overlap.py)
against closed forms, invariants or
brute force (see each docstring).  None is "parity unpinned".
"""
from .gmmnlse import (  # noqa: F401
    Fiber,
    circular_convolution,
    circular_convolution_direct,
    coupling_factor,
    energy_spectral,
    freq_from_time,
    integrand,
    overlap_tensor,
    iptrap_propagate,
    kerr_sum,
    length_scales,
    mpa_long_step,
    mpa_propagate,
    nonlinear_bracket,
    nonlinear_operator,
    photon_number,
    raman_sum,
    rk4ip_propagate,
    saturation_term,
    substep_schedule,
    time_from_freq,
)
