"""Oracle: a plain, slow, FP64 CPU restatement of the preconditioned block BiCGGR solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this package;
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg and reference arm
use it.  It shares no code with the CUDA path: its only inputs are numpy arrays (links, sources)
produced by the seeded generators, and its arithmetic is written straight from the paper:

  * ``operator``: the O(a)-improved Wilson-Dirac matrix A of Eq. (1) (``AX = B``, Sec. 2), written
    out site by site with full 4x4 spin matrices and full 12x12 site blocks ``A_D``.  The paper
    defers the matrix structure to its Ref. [blockbicggr_app]; the conventions used here (chiral
    gamma basis, kappa normalisation, four-leaf clover) are the standard Sheikholeslami-Wohlert
    form and are pinned by closed forms and symmetries, not by the paper.
  * ``solver``: the Jacobi preconditioner (Sec. 2, the polynomial for G_k) and the preconditioned
    block BiCGGR iteration (Sec. 2, the algorithm box), in the paper's order and notation, with
    dense L x L solves by numpy's LU.

Every function cites the passage it follows.  Parity status per function is listed in the header
of each module; all functions are pinned by the ``-m "not gpu"`` tests.
"""
