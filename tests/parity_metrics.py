"""Element-wise parity measure shared by the GPU parity tests.

``emax(a, b)`` is the largest, over right-hand sides r (the trailing axis), of

    max_i |a[i, r] - b[i, r]|  /  max_i |b[i, r]|,

so every entry of every right-hand side is held to the tolerance relative to
that right-hand side's own scale: a wrong PML-edge row, a wrong layer of small
amplitude or one bad column of a batch cannot hide under the norm of the rest.
``single=True`` treats the whole array as one column.
"""
import numpy as np


def emax(a, b, single: bool = False) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, (a.shape, b.shape)
    if single or a.ndim < 2:
        a = a.reshape(-1, 1)
        b = b.reshape(-1, 1)
    else:
        a = a.reshape(-1, a.shape[-1])
        b = b.reshape(-1, b.shape[-1])
    scale = np.max(np.abs(b), axis=0)
    err = np.max(np.abs(a - b), axis=0)
    return float(np.max(err / np.maximum(scale, 1e-300)))


def rel(a, b) -> float:
    """||a - b|| / ||b|| over the whole array (reported beside emax)."""
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def record(test: str, **values) -> None:
    """Append the measured deviations of a test to the JSON-lines file named by
    the environment variable ASP_PARITY_RECORD (nothing when it is unset), so a
    run can report how far inside its tolerance each case is."""
    import json
    import os
    path = os.environ.get("ASP_PARITY_RECORD")
    if not path:
        return
    with open(path, "a") as fh:
        fh.write(json.dumps({"test": test, **{k: float(v) for k, v in values.items()}}) + "\n")
