"""Error metrics (reading R9): NRMSE in dB and the paper-style peak-normalised error."""
import numpy as np


def nrmse_db(x, ref) -> float:
    x = np.asarray(x, dtype=np.complex128 if np.iscomplexobj(x) or np.iscomplexobj(ref) else np.float64)
    ref = np.asarray(ref)
    num = np.linalg.norm((x - ref).ravel())
    den = np.linalg.norm(np.asarray(ref).ravel())
    if den == 0:
        return -np.inf if num == 0 else np.inf
    if num == 0:
        return -np.inf
    return 20.0 * np.log10(num / den)


def peak_db(x, ref, power: bool = False) -> float:
    """max |x - ref| / max |ref| in dB (10 log10 for power images, 20 log10 for amplitude)."""
    d = np.max(np.abs(np.asarray(x) - np.asarray(ref)))
    p = np.max(np.abs(np.asarray(ref)))
    if d == 0:
        return -np.inf
    return (10.0 if power else 20.0) * np.log10(d / p)
