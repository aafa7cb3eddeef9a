"""dnasa: GB300-native suffix-array DNA fragment reconstruction (arxiv 1404.3456).

The compute path is the C-ABI library ``libdnasa.so`` (hand-written sm_103a
CUDA kernels, declared in ``include/dnasa.h``); :mod:`.binding` marshals torch
tensors into it.  Importing this package does not load the library; the first
call into :mod:`.binding` does, and fails loudly if it has not been built.
"""
__all__ = ["binding", "synth"]
