"""GB300 (sm_103a) implementation of the Compressed Randomized UTV hot path.

The computation lives in libcorutv.so (CUDA, C ABI in include/corutv.h);
`corutv` is its thin Python binding.  Importing this package loads the
library and fails if it has not been built (paper_1810_07323_gb300.build).
"""
from . import _lib as corutv  # noqa: F401

corutv.load()
