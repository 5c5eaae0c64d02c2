"""FP64 CPU oracle for pISTA (preconditioned ISTA for the graphical lasso).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_2205_10027_gb300``) never imports it and shares no
code with it: the two sides meet only through the seeded input generators in
``paper_2205_10027_gb300/inputs.py``, which hold none of the method's arithmetic.

Modules
-------
``pista``  Algorithm 1 of the paper (Sec. 4), step by step in plain numpy FP64,
           plus the step functions the GPU kernels are checked against.
``gista``  An independent proximal-gradient solver (Sec. 2.2, H = I) used only
           to pin the oracle's final answer by brute force at small n.
``closed`` Closed-form solutions derived by hand from the optimality conditions
           (Sec. 5.1) for the diagonal, n = 1 and n = 2 cases.

Parity status: every function in ``pista`` is pinned by ``tests/test_oracle_pins.py``
(closed forms, the per-entry sub-gradient equation of App. A.2, the scalar lemma of
App. A.1, the KKT certificate, monotone decrease, and agreement with ``gista``),
except the iteration counts the paper prints (Tables 1-4), which depend on the
authors' random draws: those are "parity unpinned".
"""
