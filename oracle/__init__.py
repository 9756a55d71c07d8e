"""FP64 CPU oracle for ALS-WR and ALS-NCG (arXiv 1508.03110).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the CUDA path and the CUDA path never imports it.

Parity status of each function (what pins it, see ``tests/test_oracle_pins.py``):
  loss            pinned: closed-form global minimum of the fully observed case,
                  U=M=0 value, finite differences of ``grad`` against it
  grad            pinned: central finite differences of ``loss``
  half_sweep      pinned: block gradient vanishes after each half (Eq. 3/4
                  optimality), ridge least squares via numpy lstsq
  chol_solve      pinned: numpy.linalg.solve on random SPD matrices
  ls_coeffs       pinned: Q(alpha) equals loss(x + alpha p) at five alphas,
                  c1 equals grad . p
  backtracking    pinned: Armijo acceptance/rejection invariants of Algorithm 3
  more_thuente    pinned: the same step as an independent implementation of the
                  published search (scipy's MINPACK-2 port) on random quartics;
                  strong Wolfe conditions hold at the step
  beta_bar        pinned: every form gives preconditioned CG on a convex quadratic
                  (exact line search), and plain NCG gives textbook CG
  ncg (Alg. 2)    pinned: equals textbook preconditioned CG on a convex quadratic;
                  fallback / restart branch: a failed line search reproduces ALS
                  bit for bit, a non-descent direction takes the preconditioner
                  point, beta restarts at 0 after every fallback
  als / alsncg    pinned: reach the closed-form global minimum of a fully
                  observed problem; ALS decreases f monotonically
  foldin          pinned: equals the user half-sweep row for a user already in R
  solve_rows      pinned: equals the selected rows of half_sweep
  ranking.*       pinned: the paper's worked example of the top-t metric
                  (s = 4, q = 5/9), identical and reversed rankings (q = 1, 0),
                  literal adjacent-swap counting on random permutations
"""
from .core import (  # noqa: F401
    Problem, build_problem, loss, grad, half_sweep, solve_rows, sweep, ls_coeffs, chol_solve,
    foldin, q_eval, q_deriv, backtracking, exact_step, more_thuente, beta_bar, BETA_FORMS, ncg, als,
    alsncg, set_threads, get_threads, IterRecord,
)
from . import ranking  # noqa: F401,E402
