"""Plain FP64 CPU oracle of the fugacity-based free-energy lattice Boltzmann method
(Soomro, Ayala, Peng, Ayala, "A fugacity-based Lattice Boltzmann method for
multicomponent multiphase systems", arXiv:2212.10680).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, calls or links anything in this package.  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.

The package is written to be read against the paper, not to be fast:

* ``eos``    -- cubic equations of state (vdW, SRK, PR) with van der Waals mixing
                rules (Appendix C) and the density-explicit log-fugacity forms the
                paper recommends for the lattice (Section IV, Eqs. eqfugupdateVDW /
                eqfugupdateSRK / eqfugupdatePR), plus the textbook phi-forms
                (Eqs. eqfugvdW / eqfugSRK / eqfugPR).
* ``flash``  -- an independent PT flash (cubic volume roots, Wilson start,
                Rachford-Rice, successive substitution on fugacity equality), the
                pure-component (Maxwell) coexistence solver and the solver for the
                pressure at which a feed gives a prescribed vapour volume fraction.
                The paper uses flash results but does not give an algorithm; this
                is the textbook procedure.
* ``lbm``    -- the nine-step procedure of Section III.B (Implementation) on a
                periodic D2Q9 lattice, whole-grid numpy array operations in the
                paper's order, nothing fused or reordered.
* ``interface`` -- the measures of the dynamic validation (Section V.E): the
                interfacial tension of Eq. eqMCsigma, the Lamb period of Eq. eqPeriod
                and the crossing radius of a droplet profile.

Parity status of each function is stated in its module docstring.
"""
