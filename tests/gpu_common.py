"""Shared set-up of the GPU tests: build and load the library, move fields to the device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1207_2223_gb300 import build
    build.build()
    import paper_1207_2223_gb300 as lq
    lq.load()
    return lq


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
