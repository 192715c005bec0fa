"""Plain FP64 CPU oracle of the AWG preconditioned conjugate gradient method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (``paper_2106_10913_gb300``); the only common dependency is the input
generator package ``awg_inputs``, which holds none of the method's arithmetic.

Every function follows a numbered definition, theorem or equation of
Gouarin & Spillane, "Fully algebraic domain decomposition preconditioners with
adaptive spectral bounds" (arXiv 2106.10913), written densely and in the
paper's order, with NumPy/SciPy as the only library (dense ``eigh``,
Cholesky, sparse LU).
"""

from .awg_oracle import *  # noqa: F401,F403
