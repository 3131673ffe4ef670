"""Helpers shared by the GPU tests: tensor conversion and the parity metric."""
import numpy as np

TOL = {"f64": 1e-12, "f32": 1e-5}  # relative max-norm per sweep against the FP64 oracle


def torch_dtype(dt):
    import torch

    return torch.float64 if dt == "f64" else torch.float32


def to_dev(a: np.ndarray, dt: str):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch_dtype(dt))


def to_np(t) -> np.ndarray:
    return t.detach().to("cpu").double().numpy()


def rel_max_err(got: np.ndarray, ref: np.ndarray) -> float:
    """||got - ref||_inf / ||ref||_inf (the parity metric)."""
    scale = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(got - ref))) / (scale if scale > 0 else 1.0)


def rounded(a: np.ndarray, dt: str) -> np.ndarray:
    """The FP64 value of an input as the device sees it (FP32 inputs are RN-rounded)."""
    return a.astype(np.float32).astype(np.float64) if dt == "f32" else np.asarray(a, dtype=np.float64)
