"""FP64 CPU oracle for H-LU — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct restatement of what the CUDA path
computes, written from the paper (Börm, Christophersen, Kriemann, "Semi-Automatic Task
Graph Construction for H-Matrix Arithmetic", arXiv 1911.07531):

* ``geometry``  — kernel entries a_ij = 1/(4 pi (|x_i - x_j| + h)), h = mean
                  nearest-neighbour spacing (brute force);
* ``trees``     — cluster tree (Def 2.1), standard admissibility (§5.1) and block tree
                  (Def 2.2);
* ``dag``       — the semi-automatic task graph: task data dependencies (Table 1),
                  task relation (Def 3.2), refinement (Alg 9, Alg 10, Alg 11), removal of
                  redundant edges (Alg 12), the accumulator graphs (Table 2, §4.3);
* ``hmatrix``   — H-matrix storage (Def 2.3), assembly and compression, rounded
                  (truncated) addition, H-matrix times thin dense matrix, and the
                  fixed flop model used for GFLOP/s;
* ``hlu``       — recursive H-LU (Alg 2), lower / upper H-solves (Alg 3 and its upper
                  mirror), H-multiplication (Alg 1) with each leaf update applied at once,
                  block forward/backward substitution;
* ``accu``      — accumulator-based H-LU (Alg 4-8) in three accumulator formats, and a
                  task-by-task runner of the accumulator task graph;
* ``mixed``     — H-LU with FP32 factor products and FP64 elsewhere, and iterative
                  refinement with FP64 residuals;

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it. It shares no code with the CUDA library and never imports it.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against closed
forms, brute force on tiny inputs, library routines for special cases, and the worked
task-graph examples of Fig. 3 and Fig. 4.
"""
