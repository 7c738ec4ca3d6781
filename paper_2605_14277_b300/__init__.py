"""B300-native sequence-form CFR (CFR, CFR+, DCFR, PCFR+) over flattened game trees.

``games``  seeded synthetic game trees (inputs only, no CFR arithmetic)
``cfr``    ctypes binding of libcfr.so (the CUDA path; see include/cfr.h)
``build``  compiles libcfr.so for sm_103a
"""
