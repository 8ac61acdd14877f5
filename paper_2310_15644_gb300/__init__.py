"""GB300 (sm_103a) boundary-element library for the compressed PMCHWT product.

The compute lives in ``libbem.so`` (CUDA C++, C interface in ``include/bem.h``);
``paper_2310_15644_gb300.bem`` is its thin ctypes binding and ``build`` compiles
it in-tree.  Importing the binding raises if the library has not been built.
"""
from .build import build  # noqa: F401
