"""CPU oracle for the matrix-free FIT operator (arXiv 1705.08849) -- TEST INFRASTRUCTURE.

This package is a plain, slow, obviously-correct restatement of what the GPU path computes:
it assembles the FIT system matrix A(w) = C^T M_nu C - w^2 M_eps + j w M_kappa explicitly as a
scipy sparse matrix (Sec. II, Eq. CP, Eq. Material, Eq. e2) and solves it with a direct solver
or a textbook Krylov method, all in float64 / complex128.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and its
``--impl reference`` arm) may import, call or execute anything in this package.  The product
path (``paper_1705_08849_gb300``) never imports it, and this package never imports the product
path: the two share no code.  The only shared module is ``fitgen`` (seeded synthetic inputs,
which holds none of the method's arithmetic).
"""
