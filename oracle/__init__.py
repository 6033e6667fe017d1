"""FP64 CPU oracle for the short-range particle-particle force step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs use it.  It shares no code with
the CUDA path (no kernels, headers, helpers, tables or constant generators);
the only common module is ``workloads`` (seeded input generators).

What it computes (the method of the paper's Sec. 2, with the short-range
force law and split filter stated by the benchmark spec, since the paper defers those
details to its HACC references):

* ``fit``        -- the Gaussian-split long-range force and the degree-5
                    polynomial in s = r^2 fitted to it (Sec. 2, force split).
* ``fp32``       -- exact emulation of the IEEE binary32 operations the
                    pair predicate is defined with.
* ``binning``    -- cells, sub-cell Morton order, 32-particle chunks, FP64
                    chunk anchors and FP32 offsets (Sec. 2.1, step 1:
                    partition into blocks).
* ``force``      -- the short-range acceleration a_i = sum_j d_ij f_SR(s_ij)
                    over pairs inside r_c, by brute force and by cell list
                    (Sec. 2, direct N^2 short-range solver), plus the
                    bit-exact FP32 in-range pair predicate and pair counts.
* ``integrate``  -- kick v += a dt, drift, the kick-drift trajectory, its
                    loss and a hand-written FP64 reverse mode.

Parity status: every function here is pinned by tests under ``tests/``
against closed forms, invariants, brute force or independent quadrature;
none is "parity unpinned".
"""
