"""CPU oracle for the ERX per-line step (test infrastructure only).

A plain, slow, FP64 NumPy restatement of the ERX detector of Garske et al.,
"ERX: A fast real-time anomaly detection algorithm for hyperspectral line
scanning" (Sec. III), plus an exact rational version for tiny inputs.  It
shares no code with the CUDA path and exists to check it: only the tests, the
smoke check and the benchmark's CPU-baseline leg may import it.
"""
from .srp import splitmix64_stream, srp_weights  # noqa: F401
from .erx_oracle import (  # noqa: F401
    ERXOracle,
    project,
    line_stats,
    ema_update,
    cholesky_ridge,
    mahalanobis,
    normalise,
    run_cube,
)
