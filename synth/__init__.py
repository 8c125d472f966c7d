"""Seeded synthetic CSR inputs shared by the tests, the bench and the oracle checks.

This package generates matrices only. It holds no part of the sparse product's
arithmetic: it never multiplies, merges or sorts partial products. Both the CUDA path
and the CPU oracle receive the arrays it returns.
"""

from .generators import (  # noqa: F401
    CSR,
    counter_u64,
    counter_uniform,
    identity,
    laplacian2d,
    laplacian3d,
    aggregation_prolongator,
    aggregation_restrictor,
    rmat,
    uniform_random,
    batch_job_params,
    batch_job,
    serve_stream,
    from_dense,
    random_small,
)
