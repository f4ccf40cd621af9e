"""B300-native multicomponent RHS / SSP-RK3 hot path of arXiv 2403.05910 (XFluids).

Submodules:
  cases -- seeded synthetic inputs (species tables, grids, primitive fields)
  xf    -- ctypes binding of the CUDA C-ABI library ``libxf.so``
"""
