"""Plain FP64 CPU oracle of the streaming ST-HOSVD method (arXiv 2308.16395).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only the tests, the
smoke check in ``__graft_entry__`` and the CPU-baseline / reference legs of ``bench.py`` use it.
It shares no code with the CUDA library. See ``oracle/tucker_oracle.py`` for the algorithms
(Alg. 1-5 of the paper) and their citations.
"""

from .tucker_oracle import (  # noqa: F401
    unfold,
    fold,
    ttm,
    truncated_svd,
    sthosvd,
    isvd,
    non_streaming_update,
    StreamState,
    init_stream,
    stream_update,
    block_update,
    recompress,
    orthogonality_error,
    restore_orthogonality,
    reconstruct,
    reconstruct_slices,
)
