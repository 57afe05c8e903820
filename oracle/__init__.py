"""FP64 CPU oracle for noisy rotated-surface-code syndrome extraction (arXiv:2204.11404).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or execute anything in
this package.  It shares no code with the CUDA path and the CUDA path never
calls it.

It restates the method plainly: the circuit of Sec. III.A on the delayed
measurement register of Sec. II.B (or the full register, for the equivalence
pin), unrolled into one-qubit/two-qubit unitaries and measurements
(``circuit.py``), applied one by one to an FP64 state vector by a plain C loop
(``sv_core.c``), with noise drawn from its own Philox4x64-10 (``philox.py``).
Parity pins live in ``tests/test_oracle_*.py``; ``tableau.py`` is the
stabilizer-tableau simulator used to pin the Pauli-noise case.
"""
from .runner import run_trajectory, build_core  # noqa: F401
