"""GB300-native pseudo-flow continuous max-flow (Baxter, Rajchl, Yuan, Peters,
arXiv 1501.07844).

The solver is the C-ABI library ``libpfm`` (``include/pfm.h``), built from the
CUDA sources in ``csrc/`` for sm_103a.  This package is its thin binding:
``lib()`` exposes the C functions under their C names through ctypes, and
``Problem`` marshals torch tensors or numpy arrays into them.  Every step of
the iteration runs in the library's kernels; there is no CPU path, and the
binding raises if the library cannot be loaded.
"""
from .binding import (  # noqa: F401
    ANISO,
    AlmProblem,
    BF16,
    F16,
    Batch,
    F32,
    FUSED,
    FUSED_PLAIN,
    INPLACE,
    ISO,
    NORMALISED,
    PAPER_LITERAL,
    PfmError,
    Problem,
    lib,
    library_path,
)
