"""GB300-native two-scale domain decomposition for the static Eikonal equation
(Martin & Tsai, arXiv:1805.04198).

The compute path lives in the C-ABI library ``libeik.so`` (CUDA, sm_103a); the
module :mod:`paper_1805_04198_gb300.eik` is its thin Python binding.  Importing
the package itself loads nothing, so the input generators can be used without
a GPU.
"""
__all__ = ["eik", "inputs"]
