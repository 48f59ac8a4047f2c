"""Plain FP64 CPU oracle for SBCI (arXiv 2603.06101) and the FCI sigma build.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may.  It shares no
code with the CUDA library (``paper_2603_06101_gb300/csrc``); the only module
both sides use is the seeded input generator ``paper_2603_06101_gb300.inputs``,
which holds no arithmetic of the method.

Contents (each function cites the passage it follows):

* ``strings``      alpha/beta occupation strings, addresses, excitation lists;
* ``slater_condon`` determinant-pair matrix elements (dense H, diagonal,
                   sampled rows) on spin-orbital bitmasks, plus a brute-force
                   second-quantised H applied operator by operator;
* ``sigma``        sigma = H c from the second-quantised Hamiltonian through
                   string excitation matrices (E_kl c -> (ij|kl) -> E_ij);
* ``spin``         <S^2> via S_- S_+;
* ``eigen``        dense eigh, Lanczos (eigsh) and a textbook Davidson;
* ``sbci``         SBCI1 following Algorithm 1 and Sections S1.1-S1.5.

Parity status: every function is pinned by the tests in ``tests/test_oracle_*``
(textbook values, closed forms, invariants, brute force); none is unpinned.
"""
