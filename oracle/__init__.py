"""CPU oracle for the multi-path transfer library -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import or run anything in this package.  The library under
``paper_2604_22228_gb300`` never imports it, and this package imports nothing from
the library: the two share no code.  Inputs come from the separate ``payload``
module, which holds none of the method's arithmetic.

What the oracle states, in plain slow code, and where it comes from:

* ``planner``  -- the 2-D split of one message over a path set (Sec. 4.3, "horizontal"
  split by per-path share, then "vertical" cut into chunks; Algorithm 1's per-path
  chunk loop; the round-robin variant the text says the real code uses) and the
  invariants every plan must satisfy (Sec. 4.5: each chunk writes a pre-assigned,
  non-overlapping region fixed before the transfer starts).
* ``cost``     -- a latency-plus-bytes-over-bandwidth cost model stated by this
  project (the paper tunes offline by exhaustive search, Sec. 4.4, but prints no
  model) and the exhaustive search over splits on tiny messages.
* ``transfer`` -- the result every transfer must produce: ``dst == src`` byte for
  byte (a memcpy), the 64-bit order-independent digest used to compare large
  buffers, and the expected arenas of a batch of transfers.
* ``jacobi``   -- the compute-plus-communication demonstration (Sec. 5.4's Jacobi
  solver): sweeps of the undivided periodic grid, which subdomains exchanging halo
  rows over the transfer paths must reproduce exactly.

Parity of the planner is pinned by hand-derived plans and invariants, the cost model
by closed forms, and the copy is its own definition.  Nothing here is "parity
unpinned".
"""
from . import planner, cost, transfer, jacobi  # noqa: F401
