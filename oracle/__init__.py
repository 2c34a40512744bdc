"""FP64 CPU oracle for the pseudopotential MRT lattice Boltzmann step (arXiv:1605.01800).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the product path never does.
It shares no code with the CUDA library under ``paper_1605_01800_gb300/``.

- ``oracle.thermo``  Carnahan-Starling EOS (Eq. 15), critical point, Maxwell
  equal-area coexistence (Eq. 11), spinodals and the pseudopotential
  mechanical-stability coexistence of Eq. 9 (numpy / scipy).
- ``oracle.d2q9``    ctypes wrapper of ``d2q9_oracle.c``: the time step of
  Eq. 1-7, 13-15 in FP64, plain sweeps.
"""
