"""GB300-native GSP-Louvain (Sahu, arXiv 2402.11454): community detection
whose every pass splits internally-disconnected communities.

The computation lives in libgsp.so (CUDA, sm_103a) behind the C ABI of
include/gsp.h; ``gsp`` is its Python binding.  Build with
``paper_2402_11454_gb300.build.build()``.
"""
