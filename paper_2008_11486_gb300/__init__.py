"""GB300 image reduction: calibration, alignment and co-adding of CCD frame sets.

The data-parallel path of Niwano et al., "GPU-accelerated Image Reduction
Pipeline" (PASJ 2020), as hand-written sm_103a CUDA kernels behind a C ABI
(include/irp.h).  This package holds the build script, the ctypes binding,
the tensor-level API, the batching/serving layers and the seeded synthetic
input generator.
"""
from ._binding import IrpError, lib  # noqa: F401

__all__ = ["IrpError", "lib"]
