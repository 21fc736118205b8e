"""CPU oracle for the GPP self-energy summation: TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package. The product path (the CUDA library and its Python
binding) never imports it, and the two share no code; only the seeded input generator
(which holds none of the method's arithmetic) feeds both.

* :func:`sigma`, :func:`sigma_adjoint` -- plain FP64 C implementation (``gpp_oracle.c``),
  the definition of the sum written out with compensated summation.
* :func:`brute_sigma` -- an independent pure-Python implementation (``brute.py``) for
  tiny sizes, used only to cross-check the C oracle.
"""

from . import gpp  # noqa: F401
from .gpp import (OCC_ALL, OCC_OCCUPIED, Oracle, branch, build, compile_oracle,  # noqa: F401
                  default, lib_path, sigma, sigma_adjoint)
from .brute import brute_sigma  # noqa: F401
