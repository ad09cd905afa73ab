"""CPU oracle for the hierarchical view library -- TEST INFRASTRUCTURE ONLY.

Plain, slow, sequential NumPy/Python restatements of what each step of the hot
path computes, written from the paper (Descend, arXiv 2305.03448) and from the
plain mathematical definitions.  Integers are evaluated in int64, floating
point in FP64 (or exactly, with math.fsum, where that is cheap).

Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never imports, links or calls it, and it shares no code with the CUDA
library: only the seeded input generators in ``synth`` feed both.

Modules
  views    view algebra (Section 3.2, the basic-view types listing, select,
           and the index generation of Section 5) and the access-conflict
           enumeration behind narrowing / access-safety checking (Section 3.3,
           Section 4 "access_safety_check")
  ops      reduce, inclusive scan, view copy (transpose) and the segmented
           reduce+scan (the four benchmarks of Section 5)
  matmul   FP64 product, bit-level bf16 round-to-nearest-even, 3-term split
  mlp      FP64 twin of the schedule cost model (forward, backward, Adam)

Every function here is pinned by ``tests/test_oracle_*.py`` to something other
than itself (worked examples of the paper, closed forms, brute force,
invariants, library special cases).  Functions without such a pin say
"parity unpinned" in their docstring; there are none at present.
"""
