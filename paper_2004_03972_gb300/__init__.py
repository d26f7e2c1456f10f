"""HQA-MD (arXiv:2004.03972) flux molecular dynamics on GB300 (sm_103a).

``instances`` holds the seeded input generators; ``hqa`` is the ctypes
binding of the CUDA library ``libhqa.so`` (built in-tree by ``build.py``).
The binding is imported lazily so the generators load without a GPU.
"""
from . import instances  # noqa: F401

__all__ = ["instances"]
