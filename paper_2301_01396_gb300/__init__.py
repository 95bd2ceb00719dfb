"""GB300-native differentiable XPBD (DiffXPBD, Stuyck & Chen): the forward XPBD step and
its discrete adjoint as hand-written sm_103a CUDA behind a C ABI.

Importing the package loads nothing; ``paper_2301_01396_gb300.binding`` loads the CUDA
library on first use and raises if it is missing."""
__all__ = ["scenes"]
