"""GB300 (sm_103a) engine for the Grunwald-Letnikov memory sum of the fractional
reaction-diffusion equation (Sprouse, MacDonald & Silva): full, short and adaptive
time-step memory, fused stencil / reaction / update, adjoint and batched launches.

The compute lives in libfd.so (include/fd.h); this package is its ctypes binding.
"""
from . import _lib, synth
from ._lib import FdError, FdProblem
from .frd import FRD, FRDBatch, FRDFunction, make_problem

__all__ = ["FRD", "FRDBatch", "FRDFunction", "FdError", "FdProblem", "make_problem", "synth", "_lib"]
