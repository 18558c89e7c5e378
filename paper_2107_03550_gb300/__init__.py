"""GB300-native non-planar spectral BIEM time step (Romanet & Ozawa, arXiv 2107.03550).

The compute path is the C-ABI library ``libsbiem`` (hand-written sm_103a CUDA
kernels); :mod:`paper_2107_03550_gb300.sbiem` is its thin Python binding and
:mod:`paper_2107_03550_gb300.workloads` holds the seeded synthetic inputs.
Importing this package does not load the library; the binding does, and it
raises if the library is missing.
"""
__all__ = ["workloads", "sbiem"]
