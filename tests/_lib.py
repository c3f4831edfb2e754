"""Test helpers: make sure libbte.so exists (build it in-tree if not) before a test uses it."""
import os
import threading

_lock = threading.Lock()


def ensure_built():
    from paper_2502_16555_gb300 import build as B
    with _lock:
        if not os.path.exists(B.LIB):
            B.build()
    return B.LIB
