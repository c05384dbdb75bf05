"""CPU oracle for the ball dot product and ball matrix multiplication of Johansson,
"Faster arbitrary-precision dot product and matrix multiplication" (arXiv 1901.04289).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under ``paper_1901_04289_gb300`` never calls it and
shares no code with it: this package decodes the raw ball layout itself, does all arithmetic on plain
Python integers (exact, arbitrary size) and encodes its own expected outputs.

Modules:

* ``exact``  -- the plain definitions: the exact value of a dot product or matrix product of balls
  (Section II), the propagated radius, round-to-nearest-even to p bits, 30-bit upward radius
  arithmetic (Section III-A), and the containment / accuracy checks.
* ``alg1``   -- Algorithm 1 (Section III) restated step by step on Python integers: the fixed-point
  limb accumulator, the ulp error counter and the radius accumulator.
* ``alg2``   -- Algorithm 2 (Section IV-A): the height bound, the greedy block extraction, the
  optimal row/column scaling exponents and the exact scaled integer block products; and Section
  IV-B's suggested inner scaling with a permutation of the inner index (ordered, non-contiguous
  blocks).
"""
