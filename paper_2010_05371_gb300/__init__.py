"""GB300-native (sm_103a) EAPrunedDTW subsequence search.

Implements the data-parallel hot path of Herrmann & Webb, "Early Abandoning
PrunedDTW and its application to similarity search" (arXiv 2010.05371):
z-normalised sliding windows, the LB_Kim / LB_Keogh cascade and EAPrunedDTW
with a shared best-so-far, as hand-written CUDA behind a C ABI
(include/eapdtw.h).  This package holds the CUDA sources (csrc/), the build
step (build.py), the ctypes binding (api.py) and the seeded input generators
(synth.py).
"""
from .api import (  # noqa: F401
    Context,
    EapDtwError,
    eap_dtw,
    eap_dtw_host,
    header_functions,
    lib,
    release_scratch,
    strerror,
    subseq_search,
    subseq_search_host,
    version,
)
