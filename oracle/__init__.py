"""FP64 CPU oracle of the test-time-training layer (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the product path never does.
"""
from .ttt_oracle import (  # noqa: F401
    LOSSES, NORMS, MODELS, sigmoid, silu, silu_prime, silu_second, param_count,
    unpack, pack, row_norm_count, apply, inner_gradient, row_targets, normalise,
    chain_forward, forward, chain_backward, backward,
)
from .gcm_oracle import gcm_forward, gcm_backward  # noqa: F401,E402
