"""SPCG on one B300: the nested-SRHT sketch, the sketch-built preconditioner,
warm-started PCG on the sketched subproblems and the full-data refinement,
all in hand-written sm_103a CUDA kernels behind the C ABI of ``include/spcg.h``.

``paper_2607_25272_b300.spcg`` is the Python binding (argument marshalling
only); ``paper_2607_25272_b300.inputs`` holds the seeded synthetic problem
generators.  Importing the package does not load the CUDA library; the first
use of the binding does, and raises if the library is missing.
"""
