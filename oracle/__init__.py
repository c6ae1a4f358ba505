"""FP64 CPU oracle for the perspective-relaxation lower bound (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2603_01306_gb300``) never imports, links or calls it,
and it never imports the product path.  Everything is plain numpy in float64,
written from the paper's definitions and algorithms:

* ``regularizer``: the Huber function (Eq. huber_loss_in_bnb), the implicit
  regularizer g_N by Algorithm 1 (Thm 4.4) and, independently, by a bisection
  on its defining infimum (Eq. 5); the conjugate g_N* (Lemma 4.2); the prox of
  rho*g_N* by Algorithm 2 (sort + textbook stack PAVA) and the prox of rho*g_N by
  the extended Moreau decomposition (Thm 4.5, Eq. prox:gN).
* ``losses``: least-squares and logistic F, grad F and F* (Sec. 2.4, Eq. 7).
* ``solver``: FISTA (Beck 2017, Sec. 10.7) with the duality-gap restart of
  Sec. 3.4; primal Phi (Eq. 6) and dual Psi (Eq. 7) with zeta = -grad F(X beta).
* ``brute``: exact k-sparse optimum of problem (1) by support enumeration for
  tiny p, and the ridge closed form.
* ``mlp``: the per-coordinate warm-start network (forward, MSE gradient by the
  chain rule, Adam, BF16 rounding) and its input features.
* ``variants``: the methods of the convergence study (Sec. 5.2): PGD and FISTA,
  fixed step or backtracking, gap / function-value / no restart.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py``, ``tests/test_oracle_mlp.py`` and ``tests/test_oracle_variants.py`` (worked examples, closed forms, Fenchel-Young
equalities, brute force); none is "parity unpinned".
"""
from . import regularizer, losses, solver, brute, mlp, variants  # noqa: F401
