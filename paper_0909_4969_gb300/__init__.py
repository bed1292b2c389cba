"""MACH (Tsourakakis, arXiv 0909.4969) on one GB300: Philox Bernoulli
sparsification of a dense tensor, then Tucker HOOI on the kept entries, in
hand-written sm_103a CUDA behind the C ABI declared in include/mach.h.

Import ``paper_0909_4969_gb300.mach`` for the binding (it loads libmach.so
and fails loudly when the library is missing).  ``synth`` holds the seeded
synthetic-input generators.
"""
