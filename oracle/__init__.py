"""FP64 CPU oracle of the CM pseudopotential boiling LBM (arXiv:1912.02018).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import, call or link anything here; the product
package never does.  It shares no code with the CUDA path.

  thermo    Peng-Robinson EOS, critical point, Maxwell construction, h_fg (numpy/scipy)
  cm_defs   the collision straight from Eq. (collision): T(u), Hermite f^eq, Huang F_i
  stepper   ctypes driver of lbm_oracle.c, the full per-step update in plain C
  gradient  the step restated in FP64 PyTorch; reverse-mode autograd gives the gradient of
            the time-averaged wall heat flux (imported on demand: it needs torch)

Parity status: every function here is pinned by a -m "not gpu" test in tests/
except the long-run boiling heat flux, which the paper prints only as figures
(parity unpinned for the time-averaged Nusselt number itself).
"""
from . import cm_defs, thermo  # noqa: F401
from .stepper import Oracle, derive  # noqa: F401
