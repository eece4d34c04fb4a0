"""CPU oracle of the recursive sparse LU (spaLU) method: test infrastructure only.

This package is a plain, slow, single-threaded FP64 restatement of the method, written to
be checked against the paper by eye.  It is NOT part of the product: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.  It shares
no code with the CUDA path (``paper_2408_14193_gb300``) and imports nothing from it; the
two meet only in the seeded problem generators of ``workloads``.

Modules (each function cites the passage of the paper it follows):
  philox  - Philox4x32-10 counter-based generator and the Gaussian entries of the sketch
  nd      - nested dissection of a regular grid (Sec. 3, Alg. 1) and its level structure
  dense   - Gaussian elimination with partial pivoting, column-pivoted QR and the
            interpolative decomposition (Sec. 4.1, Eqs. (RRQR 1)-(B))
  spalu   - the factorization (Sec. 4.3, Alg. 2) and the tree-ordered solve (Eq. (WV))
  gmres   - right-preconditioned restarted GMRES used for iterative refinement
"""
