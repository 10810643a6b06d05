"""GB300-native (sm_103a) restarted reflected-Halpern PDHG for sparse LPs.

``Solver`` (in ``paper_2601_07628_gb300.dpdlp``) binds the C ABI of ``libdpdlp.so``
(include/dpdlp.h); ``build()`` (module ``buildlib``) compiles it.  ``costmodel`` holds the per-iteration
byte model of Eq. cost_model; ``autotune`` picks the iteration kernels' launch shapes.
"""
from .buildlib import build  # noqa: F401
