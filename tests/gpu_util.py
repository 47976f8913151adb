"""Helpers shared by the GPU tests: numpy <-> device tensors, oracle inputs."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(a):
    """uint64 numpy array -> int64 CUDA tensor with the same bits."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64).reshape(-1)).cuda()


def to_np(t, shape=None):
    a = t.detach().cpu().numpy().view(np.uint64)
    return a.reshape(shape) if shape is not None else a
