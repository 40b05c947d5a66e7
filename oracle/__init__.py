"""Oracle for the row-skipping outer-product SpMM (Rosko, arXiv 2307.03930).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct CPU
statement of what the CUDA library computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg (and its
``--impl reference`` arm) may import it.  The product path never calls it and
shares no code with it; the only module both sides use is the seeded input
generator ``paper_2307_03930_gb300.inputs``, which holds none of the method's
arithmetic (the oracle itself does not import it).

Modules
-------
pack      Alg. 1 (packing and indexing arrays) per row panel, and its inverse.
spmm      The SpMM C = A.B in FP64 / int64 over the nonzeros of A (Sec. 3,
          Alg. 2 semantics), plus the per-element normaliser sum |a||b|.
quant     BF16 round-to-nearest-even and symmetric INT8 quantisers.
features  Schedule-selector input features of a sparse A and N.
mlp       The selector's 3x64 ReLU MLP: forward, softmax cross-entropy,
          backward and one Adam step, in FP64.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against hand-derived examples, brute force, closed forms or invariants; none
is "parity unpinned".
"""
from . import pack, spmm, quant, features, mlp  # noqa: F401
