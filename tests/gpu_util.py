"""Helpers shared by the GPU tests: device tensors from the seeded generators, oracle comparisons."""
import numpy as np
import pytest
import torch

import synthetic


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_14958_gb300 import wd  # noqa: F401  (raises if the library is missing)
    return wd


def to_dev(a: np.ndarray, dtype=torch.complex128) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.complex128)


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fields(dims, eps=0.4, gseed=1, sseed=2):
    return synthetic.gauge_field(dims, eps, gseed), synthetic.gaussian_source(dims, sseed)
