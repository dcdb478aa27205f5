"""Seeded synthetic inputs for the primal-dual susceptibility solver.

This package is the only code that both the FP64 oracle (``oracle/``) and the
CUDA path (``paper_2006_09808_gb300``) consume.  It holds none of the
solver's arithmetic: the measured field is simulated with the continuous,
pixel-integrated 2-D dipole Green's function and a *linear* (zero-padded)
convolution, not with the solver's periodic k-space kernel D(k).  The scanner
datasets of the paper's Sec. III (stent, seeds in meat, needle in a CuSO4
phantom) are not available, so these phantoms stand in for them.
"""

from .generator import (  # noqa: F401
    dipole_green_2d,
    simulate_field,
    ellipse_mask,
    disc,
    rod,
    SliceProblem,
    config1,
    volume,
    config2,
    magnitude_weight,
    echo_pair,
    config4_volumes,
    config5_arrivals,
)
