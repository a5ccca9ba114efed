"""GB300 (sm_103a) quasistatic LSPR boundary-element library.

Hot path of Clementi, Cooper & Barba (arXiv:1812.10722): the treecode-accelerated
matrix-vector product of the 2x2 single/double-layer system inside complex
GMRES, with FP64 near-singular corrections, the dipole moment and the
extinction cross-section.  The numerical work lives in ``_lib/liblspr_gb300.so``
(C ABI: ``include/lspr.h``); ``lspr`` is the Python binding and ``inputs`` the
seeded workload generator.  Importing the package does not load the library.
"""
__all__ = ["lspr", "inputs", "build"]
