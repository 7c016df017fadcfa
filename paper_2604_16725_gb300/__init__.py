"""GB300-native (sm_103a) FliX: the flipped-indexing GPU ordered map (arXiv 2604.16725).

The compute lives in ``libflix.so`` (hand-written CUDA behind the C ABI of ``include/flix.h``);
``flix.Index`` is its Python binding.
"""
from .flix import (OP_DELETE, OP_INSERT, OP_LOOKUP, OP_NOP, OP_RANGE, OP_SUCC, QUEUE_BATCH_MAX, FlixError, Index,  # noqa: F401,E501
                   SIGNATURES, library_path, load)
