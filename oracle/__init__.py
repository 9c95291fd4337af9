"""CPU oracle for Res_y(f, g) -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct restatement of what the
resultant path computes, written from the paper's definitions:

* ``exact``  -- R(x) = det S^{(y)}(f, g) over Z[x] (Sylvester matrix of
  Section 3.1, f and g as in Eq. (2.1)), by Leibniz expansion, by
  fraction-free Bareiss over Z[x], by Kronecker substitution + integer
  Bareiss, and by exact values at integer points + exact interpolation.
* ``modp``   -- one modular image det(S(x0)) mod p by Gaussian elimination
  over Z_p (the per-(prime, point) quantity z_i^{(p)} of Section 4.1).
* ``squarefree`` -- the square-free factorisation R = c prod R_i^i over Z
  (Section 5, PROJECT) by Yun's algorithm with primitive gcds.

It shares no code with the CUDA path and must never be imported by it: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may use it.  Every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py`` and
``tests/test_oracle_squarefree.py``.
"""
