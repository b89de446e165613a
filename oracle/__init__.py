"""CPU oracle (FP64, numpy/scipy) for the DDA solve -- test infrastructure.

Only tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg use
it.  It shares no code with the CUDA library and never imports it.
"""
