"""Seeded synthetic input generators shared by the oracle tests, the CUDA
parity tests and the benchmark. Holds no arithmetic of the method itself."""
from .harris import (HarrisConfig, harris_derived, make_harris, random_state,
                     sample_maxwell_juettner, boost_flip)
from .scan import splitmix64, tearing_scan, SCAN_LX, SCAN_DELTA, SCAN_SIGMA
from .harris3 import HarrisConfig3, make_harris3, random_state3

__all__ = ["HarrisConfig", "harris_derived", "make_harris", "random_state",
           "sample_maxwell_juettner", "boost_flip", "splitmix64", "tearing_scan",
           "SCAN_LX", "SCAN_DELTA", "SCAN_SIGMA", "HarrisConfig3", "make_harris3", "random_state3"]
