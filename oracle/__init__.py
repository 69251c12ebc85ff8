"""Plain FP64 CPU oracle of the curvilinear LBM of arXiv:2301.01868.

TEST INFRASTRUCTURE ONLY: used by tests/, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference leg of ``bench.py``; never by the product path.
"""
