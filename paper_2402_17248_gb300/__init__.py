"""GB300 beamline tracking: Python binding of the C-ABI library libbl.so.

The compute path is the CUDA library; this package only marshals arguments
(torch tensors for device memory and streams) into the C calls declared in
include/bl.h. Importing it does not load the library; the first call does,
and fails loudly if libbl.so has not been built.
"""
from . import bl  # noqa: F401
