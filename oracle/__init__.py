"""FP64 CPU oracle (test infrastructure only).

Plain, slow, obviously-correct restatement of the photoacoustic forward operator, its exact
adjoint and the ISTA / FISTA / multi-grid FISTA shell of Javaherian & Holman
(arXiv:1603.02329). Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline may import this package; the product path (``paper_1603_02329_gb300``) never does,
and the two share no code.
"""
