"""GB300-native structured-grid Euler solver (FP64 MUSCL-minmod + Roe + SSP-RK3).

The compute path is the C-ABI library libfv (hand-written CUDA for sm_103a);
`paper_2306_14011_gb300.fv` is its thin Python binding.  Importing this package
does not load the library; `inputs` holds the seeded initial conditions.
"""
