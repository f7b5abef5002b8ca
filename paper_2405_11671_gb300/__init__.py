"""GB300 (sm_103a) graph containers and algorithms after BYO (arXiv 2405.11671).

The work happens in ``libbyo.so`` (C ABI, ``include/byo.h``); this package is
its Python binding (``_byo``) and build script (``build``).
"""
from ._byo import *  # noqa: F401,F403
from ._byo import Graph, ByoError, load, LIB_PATH  # noqa: F401
