"""Reference (oracle) implementation of ESMP2-TOP(1) -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything from this package.
The product path (the CUDA library and its Python binding) never imports, links
or executes it, and this package never imports the product.

Contents
--------
top.py   TOP (transition-orbital-pair) basis: SVD of the singles matrix C,
         Householder completion of the virtual space, orbital transforms
         (Sec. II.A, Eqs. 2-4).  numpy, float64.
jw.py    O1: the method written out literally in the determinant space of a
         tiny system: Jordan-Wigner fermion operators, H and the spin-summed Fock
         operator as explicit operators, Psi0 of Eq. psi0_tp, the D/L/S/N
         partition of Sec. II.B-C, the modified H0 of Eqs. old_H0 and
         qfq_replacement, a dense direct solve, and E2.
o2.c     O2: the same quantities for large systems from the textbook
         spin-orbital formulas (one-body operator acting on doubles and triples,
         Slater-Condon matrix elements), evaluated amplitude by amplitude through
         an accessor that encodes Eq. psi1 (shared spin-flip amplitudes, TOP
         content of the L-triples).  Plain loops, OpenMP, float64.
o2.py    ctypes binding of o2.c plus the plain conjugate-gradient driver.

Pins: tests/test_oracle_*.py check O1 against closed forms, textbook identities
and invariants, and O2 against O1 on random tiny systems.
"""
