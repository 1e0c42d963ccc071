"""FP64 CPU oracle of randomized HALS NMF (Erichson, Mendible, Wihlborn, Kutz,
"Randomized Nonnegative Matrix Factorization", arXiv:1711.02037).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library (``paper_1711_02037_gb300``) never imports it, and the
two share no code: the oracle implements its own Philox4x32-10 (philox.py)
from the published definition, and it takes every input matrix from the
seeded generators in ``synth/`` or from its own draws, never from the GPU.

Modules:
  philox.py   - Philox4x32-10, U[0,1) and Box-Muller N(0,1) draws, Omega, W_init/H_init.
  rhals.py    - randomized QB (Section 2.3, Algorithm 1), randomized HALS sweeps
                (Section 3.2, Algorithm 1), deterministic HALS (Section 3.1),
                objectives and relative error.
  extras.py   - regularised updates (Section 3.4), projected gradient (Section 3.3),
                blocked QB over column blocks (Algorithm 2).
  adjoint.py  - reference gradient of <G, W_T H_T> through T compressed sweeps
                (float64 reverse mode by torch autograd on CPU).

Functions whose result no test pins against the paper or mathematics say
"parity unpinned" in their docstring.
"""
from . import philox, rhals  # noqa: F401
