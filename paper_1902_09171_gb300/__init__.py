"""GB300-native r-cell engine for the hierarchical FEM <-> MD coupling of
arXiv:1902.09171: QR-split deformation gradients, triclinic r-cells, batched
fixed-box MD with virial stress, and an explicit hex-8 FE update, as
hand-written sm_103a CUDA behind the C ABI of include/rcell.h.

    from paper_1902_09171_gb300 import build, rcell
    build.build()                 # nvcc -> librcell.so (sm_103a)
    ctx = rcell.rcell_create(...) # see rcell.py
"""
from . import build  # noqa: F401
