"""GB300 (sm_103a) Chebyshev-filtered subspace iteration for sequences of correlated
generalized Hermitian eigenproblems (Di Napoli & Berljafa, arXiv:1206.3768).

The compute path is the C-ABI library ``_lib/libchfsi.so`` (declared in include/chfsi.h);
``binding`` marshals torch tensors into it and ``inputs`` builds seeded synthetic
sequences.  Importing the package loads nothing; the library is loaded on first use.
"""
__all__ = ["binding", "inputs", "build"]
