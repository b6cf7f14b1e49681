"""Helpers shared by the GPU parity tests (host-side marshalling only)."""
import numpy as np
import torch

from workloads import uniform_elements


def to_dev(X: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.uint32).view(np.int32)).cuda()


def to_host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32).reshape(-1, 8)


def rand_dev(F, log_n: int, seed: int):
    X = uniform_elements(F.r, 1 << log_n, seed)
    return X, to_dev(X)


def first_mismatch(got: np.ndarray, want: np.ndarray) -> str:
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    if bad.size == 0:
        return "equal"
    return f"{bad.size} of {got.shape[0]} elements differ, first at {int(bad[0])}"
