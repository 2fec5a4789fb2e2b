"""Helpers shared by the GPU tests: moving numpy payloads to CUDA tensors of
the same width and back, byte for byte, and calling the library through its
tensor binding."""
import numpy as np
import torch

_SIGNED = {1: np.int8, 2: np.int16, 4: np.int32, 8: np.int64}


def to_device(a: np.ndarray) -> torch.Tensor:
    """The same bytes as a CUDA tensor with the same row width."""
    a = np.ascontiguousarray(a)
    width = a.dtype.itemsize
    if a.dtype.kind in "iu" and width in _SIGNED:
        view = a.view(_SIGNED[width])
    elif a.dtype == np.float32 or a.dtype == np.float64:
        view = a
    else:
        view = a.view(np.uint8)
    return torch.from_numpy(view).cuda()


def to_host(t: torch.Tensor, like: np.ndarray) -> np.ndarray:
    host = t.cpu().numpy()
    return np.ascontiguousarray(host).view(like.dtype).reshape(like.shape)


def assert_no_device_error():
    import paper_2106_06161_gb300 as bs
    torch.cuda.synchronize()
    code = bs.get_error()
    assert code == 0, bs.error_string(code)
