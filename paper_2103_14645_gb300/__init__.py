"""GB300-native renderer for baked Sparse Neural Radiance Grids (SNeRG, arXiv 2103.14645).

The deferred volume render of the paper's baked representation (Sec. 5.1-5.2, App. A,
Eqs. 2, 5-7) and its adjoint (Sec. 5.5) run as hand-written sm_103a CUDA kernels in
libsnerg.so behind the C ABI of include/snerg.h; `renderer` is its Python binding and
`synth` the seeded generator of synthetic scenes.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "renderer", "build"]
