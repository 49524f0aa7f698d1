"""Plain, slow CPU oracle for the GIPC Gauss-Newton hot path -- TEST INFRASTRUCTURE.

This package restates the paper's method (Huang et al., "GIPC: Fast and stable
Gauss-Newton optimization of IPC barrier energy") step by step in plain Python
and numpy, with exact rational geometry and float64 arithmetic after it.  It
exists to check the CUDA path, which shares no code with it.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or execute anything
here.  The product path never routes through it.

Modules:
  jet        forward-mode derivative numbers (exact over Fractions, or float)
  geometry   stencil decoding (Sec. 7.2) and exact distances / parallel measure (Eq. 4-5, Sec. 6.1)
  barrier    barrier functions (Eq. 6, 12, 24), eigenvalue formulas (Eq. 18-19), filter (Eq. 23), mollifier (Eq. 25)
  stencil    per-stencil energy, gradient and projected Hessian (Alg. 2; Eq. 13-36)
"""
