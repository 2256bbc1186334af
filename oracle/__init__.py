"""CPU oracle for the Monte Carlo integration of divergence-subtracted QED
vertex graphs without lepton loops (Volkov, arXiv:1909.08015).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is a plain, slow, independent restatement of the method.  It
shares no code, tables or helpers with the CUDA path:

* ``graphs``    -- graph set (Sec. I, footnote on arrow reversal; Table I).
* ``forest``    -- UV-divergent subgraphs, forests and R^new terms (Sec. II).
* ``philox``    -- Philox4x32-10 counter-based generator (Calc 2, Sec. V).
* ``mrg32k3a``  -- MRG32k3a with jump-ahead (Calc 1, Sec. V).
* ``sampler``   -- Deg(s), the Hepp-sector density g (Eqs. eq_pdf_final,
                   eq_pdf) and its exact sequential sampler (Sec. III.A).
* ``dirac``     -- explicit 4x4 Dirac matrices and traces with contracted
                   Lorentz indices, by explicit index summation.
* ``integrand`` -- the subtracted Feynman-parametric integrand I(z)
                   (Eq. eq_feyn_integral) assembled from per-subgraph
                   factors; graph functions in exact rational arithmetic.
* ``estimate``  -- the estimator (Eq. eq_integral_approx), sigma_down
                   (Eq. eq_sigma_down) and set sums (Eq. eq_sigma_sum).

Parity status per function is stated in each module header.
"""
