"""GB300-native embedded-boundary multi-material Poisson solver.

Solves div(eps_r grad phi) = -rho/eps0 on Cartesian cut-cell grids with
electrodes, dielectric permittivity jumps and surface charge (Marskar,
arXiv:1809.03745, Sec. 2.1 and 3.1-3.3) by geometric multigrid in CUDA for
sm_103a.  ``paper_1809_03745_gb300.ebpoisson`` is the ctypes binding of the C
ABI in include/ebpoisson.h; ``workloads`` builds seeded synthetic problems.
"""
