"""CPU oracle (FP64) for the semi-implicit 1D3V electron BTE step of arXiv 2502.16555.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py``. Nothing in the product path imports it.
"""
