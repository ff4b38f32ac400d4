"""GB300-native (sm_103a) 1d3v electrostatic PIC/MCC library for capacitively coupled rf
discharges (the kinetic method of arXiv:1608.04601). The compute path is libpic.so (CUDA);
``pic.Simulation`` marshals arguments to its C ABI (include/pic.h)."""

from . import pic, workloads, xsections  # noqa: F401

__all__ = ["pic", "workloads", "xsections"]
