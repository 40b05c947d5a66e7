"""Test helpers: build the CUDA library once per session and load its binding."""
import functools
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@functools.lru_cache(maxsize=1)
def built():
    from paper_2307_03930_gb300 import build
    build.build()
    from paper_2307_03930_gb300 import rosko
    rosko.lib()
    return rosko
