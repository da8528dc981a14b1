"""ORACLE — test infrastructure, not part of the library.

A plain, slow, CPU-only FP64 restatement of the refinement method of
Terao, Ozaki, Imamura and Ogita, "Iterative Refinement for a Subset of
Eigenvectors of Symmetric Matrices via Matrix Multiplications" (Algorithms 1-4,
Section 3.1), plus a double-double evaluator of residuals, orthogonality and
angles (``dd.c``), a cyclic Jacobi eigensolver for small matrices and the
closed forms of the convergence analysis.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call, link or run anything in this directory.  It
shares no code with the CUDA library in ``paper_2602_23778_gb300``: neither
imports the other; both read inputs from ``workloads`` only.
"""
