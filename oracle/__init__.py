"""Oracle for exact multiple pattern matching (MAG/SMAG) -- TEST INFRASTRUCTURE ONLY.

Nothing in the product path may import this package: only tests/, the smoke
check and bench.py's CPU-baseline leg use it.  It shares no code with the
CUDA library.

  brute    -- the problem statement of Section 1 as Python loops (tiny inputs)
  native   -- C: naive r x n comparison and textbook Aho-Corasick (Section 1.1),
              optionally threaded over contiguous start ranges
  filter   -- the paper's filter steps (Sections 2, 3.1, 3.2, 3.3) in order
  mlp      -- the learned cost model's network, loss, gradient and Adam
              update in fp64 (textbook definitions; not from the paper)

Pins (tests/test_oracle_pins.py) tie each part to something outside itself:
the worked superimposition example and the q = 2 class example of Section 2,
the closed-form class sizes and match probabilities of the Section 2
illustration and of Section 3.2's p, the multiply trick of Section 3.3 checked
on all masked inputs, textbook Shift-Or as the k = 1, q = 1, r = 1 special case
of the AOSO scan, brute force on thousands of tiny inputs, and the
no-false-negative property of the filter.  The choice of parameters by the
autotuner or the learned cost model is not a computed result and is judged
by regret, not parity.
"""
