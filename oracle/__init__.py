"""FP64 CPU oracle of the phase-field lattice Boltzmann method (arXiv 2311.05097).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never loads it, and it shares no code with the
CUDA path.
"""
