"""Shared test helpers: tolerances, relative L2 error, library build fixture."""
import numpy as np

TOL = {"f64": 1e-12, "f32": 1e-5}  # relative L2 bounds stated for the method's parity


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (nr if nr > 0 else 1.0))


def rel_scalar(got, ref) -> float:
    return abs(float(got) - float(ref)) / max(abs(float(ref)), 1e-300)


def f32_round(a):
    """FP32 inputs for the oracle: the FP64 draws rounded to float32, back in float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)
