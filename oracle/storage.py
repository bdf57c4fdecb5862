"""Rounding to the storage types of the basis (test infrastructure only).

The paper leaves mixed precision to future work (Sec. 5).  The reading
taken here: a basis vector is formed in working precision and then kept in
a storage type (FP64, FP32, BF16 or FP16), and every later use of it (the
elimination, the pivot block, the sketch, x = V_k y) reads the stored
value.  round_to gives the stored value as float64.
"""
from __future__ import annotations

import numpy as np

# unit roundoff of each storage type (round to nearest)
UNIT = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}


def round_to(a: np.ndarray, storage: str) -> np.ndarray:
    """Entries rounded (to nearest even) to a storage type, returned as float64."""
    a = np.asarray(a, dtype=np.float64)
    if storage == "f64":
        return a.copy()
    if storage == "f32":
        return a.astype(np.float32).astype(np.float64)
    if storage == "f16":
        return a.astype(np.float16).astype(np.float64)
    if storage == "bf16":
        # float64 -> float32 (nearest even) -> bfloat16 (nearest even on the
        # 16 dropped bits): the route a float32 working value takes
        u = a.astype(np.float32).view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
        return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    raise ValueError(storage)
