"""FP64 CPU oracle for the sketched inner-product-free Krylov method (sCMRH).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline leg and its ``--impl reference`` arm) may
import or run anything in this package.  The CUDA library never calls it and
shares no code with it: the oracle re-derives every step from the paper in
plain numpy at float64.

Modules
  sketch     sparse-sign sketch from a SplitMix64 counter hash (Sec. 2)
  operators  zero-boundary 2-D convolution, blur composites, CSR products
  scmrh      pivoted Hessenberg process + sketch + projected solve (Sec. 3)
  gmres      Arnoldi/MGS GMRES, used only as an independent pin

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (published test vectors, closed forms, library routines,
invariants or brute force); no oracle function is "parity unpinned".
"""
