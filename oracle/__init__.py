"""Plain FP64 CPU oracle for the multilevel BDDC hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA path.

Contents (each function cites the passage of Sistek, Mandel, Sousedik, Burda,
"Parallel implementation of Multilevel BDDC" it follows):

* ``fem``     -- Q1 element matrices (Laplace, linear elasticity), global sparse assembly,
                 sparse direct solve: the plain definition of the discrete solution u = K^{-1} f.
* ``maps``    -- interface classification into faces / edges / vertices, corner selection,
                 constraint matrices C_i, coarse numbering R_Ci, weights, pseudo-mesh of the
                 next level (Sec. 2-3, Algorithm 1).
* ``bddc``    -- the reduced interface problem (Sec. 2), the BDDC preconditioner with two and
                 more levels (Eq. psi_def, Eq. sub_cor, Algorithm 1, Algorithm 2), PCG with the
                 Lanczos condition-number estimate (Sec. 4).
* ``grad``    -- adjoint gradient of a linear functional J = sum_k w_k^T u_k with respect to the
                 right-hand side and per-element coefficients.

Readings of the paper where it is silent are listed in the module docstrings.  Parity status
of each function is stated there; the pins live in ``tests/test_oracle_*.py``.
"""
