"""GB300 (sm_103a) implementation of the per-step update of the central-moment
pseudopotential lattice Boltzmann model for forced-convection boiling on a cylinder
(Saito et al., arXiv:1912.02018).

The compute path is the CUDA library liblbm.so (C ABI in include/lbm.h), built by
nvcc_build.py; this package only marshals arguments to it.  Importing works without a GPU;
creating a Sim needs the built library and a CUDA device and fails loudly otherwise.
The adjoint submodule (imported on demand) wraps the adjoint window in torch.autograd.
"""
from . import _native  # noqa: F401
from .sim import Batch, Sim  # noqa: F401

__all__ = ["Sim", "Batch", "build", "adjoint"]


def build(force: bool = False, verbose: bool = False) -> str:
    from .nvcc_build import build as _b

    return _b(force=force, verbose=verbose)
