"""GB300 (sm_103a) maximum-likelihood map-making: libmm and its Python binding.

``paper_2112_03370_gb300.mm`` loads the compiled CUDA library (``libmm.so``) and fails loudly if it
is missing; ``paper_2112_03370_gb300.build.build()`` compiles it.
"""
