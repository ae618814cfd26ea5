"""CPU oracle (test infrastructure).

Plain FP64 numpy/scipy restatement of the micro-continuum time step of
Maes, Soulaine & Menke (Sec. 2.2-2.4, App. B-D).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the CUDA path neither imports it nor shares code with it.
"""
