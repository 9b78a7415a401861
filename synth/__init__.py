"""Seeded synthetic inputs shaped like the paper's workloads.

This package only draws random numbers and shapes them (mixtures, value
ranges, spectra).  It holds none of the method's arithmetic: no rotation,
no partial distance, no pruning, no classifier.  Both the oracle-driven tests
and the CUDA path's tests and benchmark take their inputs from here.
"""
from .mixtures import (  # noqa: F401
    MixtureSpec,
    VmfSpec,
    power_law_spectrum,
    haar_orthogonal,
    WORKLOADS,
    workload,
)
