"""Helpers for the GPU tests: a context with a gauge field loaded, and
conversion of half-lattice numpy fields to CUDA tensors."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(torch, arr):
    """numpy complex [.., 3, Vh] -> CUDA tensor of float64 (complex128) or float32 (complex64) pairs."""
    if arr.dtype == np.complex128:
        return torch.from_numpy(np.ascontiguousarray(arr).view(np.float64)).cuda()
    if arr.dtype == np.complex64:
        return torch.from_numpy(np.ascontiguousarray(arr).view(np.float32)).cuda()
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def host_complex(t):
    a = t.detach().cpu().numpy()
    if a.dtype == np.float64:
        return a.view(np.complex128)
    return a.view(np.complex64).astype(np.complex128)


def wrap_device(torch, ptr, numel):
    """A float64 CUDA tensor viewing `numel` doubles at device address ptr."""
    class _Wrap:
        __cuda_array_interface__ = {"shape": (int(numel),), "typestr": "<f8", "data": (int(ptr), False),
                                    "version": 3}
    return torch.as_tensor(_Wrap(), device="cuda")
