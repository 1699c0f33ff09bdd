"""GB300 map-maker: maximum-likelihood CMB map-making by preconditioned conjugate
gradients with the binned, Jacobi and circulant preconditioners of Naess & Louis
(arXiv:1309.7473), as hand-written sm_103a CUDA behind a C ABI (include/cmm.h).

``paper_1309_7473_gb300.build.build()`` compiles the library in-tree;
``paper_1309_7473_gb300.cmm`` is the Python binding.
"""
