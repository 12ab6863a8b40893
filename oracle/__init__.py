"""CPU FP64 oracle for CP-MDP (test infrastructure, not product code).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything in this package. The CUDA library never
calls it, and it never calls the CUDA library: the two share no code; the
only module both sides use is ``cpmdp_inputs`` (seeded instance drawing).

Modules
-------
tabular   -- the plain definitions on the expanded |S| x |S| transition
             matrices: GridWorld rules (scenario section), Definition 3
             components, Eq. 1 value iteration, exact policy iteration,
             brute-force policy enumeration, dense CP Kronecker expansion.
cpfactor  -- an FP64 CP-factor backup / VI / policy evaluation in plain C
             loops (``cpfactor.c``), one rank-1 term at a time, for grids
             far beyond tabular reach; also the timed CPU baseline.
dense     -- the dense CP backup written as one mode product per factor
             (numpy tensordot), plus a single-state evaluator for sampled
             checks at full size.

Every function cites the passage of the paper it follows (Eq. 1, the value
and policy iteration paragraphs of the background section, Definitions 1-3,
the GridWorld scenario). Parity status of each function is listed in its
module header; none is "parity unpinned".
"""
