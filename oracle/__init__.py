"""Independent FP64 CPU oracle for the FDLB simplified-Enskog solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link anything under ``oracle/``; only
the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` use it.  The oracle shares no code, tables or constants
with the GPU path: it rebuilds its own quadratures (in 200-digit decimal
arithmetic), grid metrics, stencils and projections.

Every function cites the passage of the paper (Busuioc & Sofonea, "Bounded
flows of dense gases", arXiv 2308.15407) it restates.  Where the paper is
silent, garbled or ambiguous the reading taken is stated beside the code.

Parity status: every oracle function is pinned by tests in ``tests/`` that
check it against closed forms, exact moments, library special cases,
invariants or brute force; none is "parity unpinned".
"""
