"""Seeded synthetic inputs (magnetograms and evaluation points) shared by tests and benchmarks.

Holds no DBIE arithmetic: only the test fields (Low & Lou, Gaussian active regions, potential
fields for tracing) and the point-set recipes."""
from .active_region import Magnetogram, active_region, monopole_field, trace_samples  # noqa: F401
from .lowlou import LowLou, box_scale, to_box  # noqa: F401
from . import workloads  # noqa: F401
