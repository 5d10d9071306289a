"""CPU oracle for the EA-ADC(2)/(3) secular matrix, its Davidson roots and the
state-specific FNO/NAF truncation (arXiv:2511.05897).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or execute it.  It shares no code with the CUDA path;
both sides draw their inputs from the separate ``synth`` package.

Everything is plain numpy in float64:

* ``fci_isr``    - brute-force intermediate-state representation (Sec. II.A,
                   Eq. 1-6) from exact FCI wave functions, with Taylor
                   coefficients in the perturbation strength (Eq. 5).
* ``spinorb``    - the EA-ADC(n) blocks in spin-orbital form, written out
                   element by element (small systems).
* ``restricted`` - the same matrix for closed-shell doublets, with
                   density-fitted integrals (Sec. II.B, Eq. 25), as an
                   explicit matrix and as a matrix-vector product.
* ``davidson``   - a textbook Davidson eigensolver (Sec. II.A).
* ``fno``        - state-specific natural orbitals, natural auxiliary
                   functions and the truncation correction (Sec. II.C-E,
                   Eq. 9-17, 27-30).
"""
