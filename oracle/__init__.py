"""Oracle for the finite-field NTT: a plain, slow, obviously correct CPU statement
of what the GPU path computes.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` (including ``bench.py --impl reference``) may
import, call, link or execute anything in this package.  The product path
(``paper_2509_22684_gb300``) shares no code with it and never imports it.

* ``oracle.field``   field constants derived from the modulus (Python ints)
* ``oracle.ntt_ref`` the transform by definition (O(n^2) DFT, single outputs),
  the paper's radix-2 Cooley-Tukey, inverse, coset and the Groth16 H sequence
* ``oracle.cpu``     ctypes loader for ``cpu_ntt.c``, an independent C NTT with
  4 x 64-bit limbs used for large full-vector parity and as the timed CPU
  baseline
"""
