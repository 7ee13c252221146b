"""CPU FP64 oracle for the sketch-powered power method.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py`` may import anything
here.  The CUDA library never calls into this package and shares no source with
it; the two meet only through the seeded input generators in
``paper_2605_09755_gb300.workloads``, which hold none of the method's
arithmetic.

Modules:
  philox      -- Philox4x32-10 (Salmon et al., SC'11), the counter-based generator
                 both sides implement independently.
  sketch      -- sparse sign sketch of Lemma 3.2 item 2, Gaussian Omega.
  algorithms  -- Algorithms 1, 2, 3 and the Randomized SVD finish (Section 2).

Every function is pinned by ``tests/test_oracle_pins.py`` to something other
than itself (published known-answer vectors, brute force on tiny inputs,
closed forms, exact algebraic identities stated in the paper).
"""
from . import philox, sketch, algorithms  # noqa: F401
