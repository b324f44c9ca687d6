"""op2b: GB300-native edge loops of an edge-based finite-volume solver.

Sets, maps, dats and parallel loops with READ / WRITE / INC access (Sec. 3.1
of the paper) over hand-written sm_103a CUDA kernels.  The CUDA library is
loaded on first use by :mod:`paper_1403_7209_gb300.op2b`; importing this
package loads nothing.
"""
__all__ = ["meshgen", "op2b"]
