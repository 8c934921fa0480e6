"""Helpers shared by the GPU parity tests: layout conversion only."""
import numpy as np


def ora_J_from_gpu(Jg, N, b):
    """GPU [7][b][b][N] -> oracle [N][7][b][b]."""
    return np.ascontiguousarray(np.asarray(Jg).reshape(7, b, b, N).transpose(3, 0, 1, 2))


def gpu_J_from_ora(Jo, N, b):
    return np.ascontiguousarray(np.asarray(Jo).reshape(N, 7, b, b).transpose(1, 2, 3, 0)).reshape(-1)


def to_cm(v, N, b):
    """oracle interleaved [N][b] -> GPU component-major [b][N]."""
    return np.ascontiguousarray(np.asarray(v).reshape(N, b).T).reshape(-1)


def to_il(v, N, b):
    return np.ascontiguousarray(np.asarray(v).reshape(b, N).T).reshape(-1)


def rel_err(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
