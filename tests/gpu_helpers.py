"""Shared helpers for the GPU parity tests (imported by tests/test_gpu_*.py)."""

import numpy as np
import pytest
import scipy.sparse as sp

import workload as wl

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def gpu_module():
    require_gpu()
    import paper_2407_01783_gb300 as sk
    return sk


def to_scipy(rp, ci, vals, shape):
    """Block CSR export -> scalar scipy CSR (rows/cols expanded by block size)."""
    nnz, br, bc = vals.shape
    rows = np.repeat(np.arange(shape[0]), np.diff(rp))
    R = (rows[:, None, None] * br + np.arange(br)[None, :, None]) + 0 * np.arange(bc)[None, None, :]
    Cc = (ci[:, None, None] * bc + np.arange(bc)[None, None, :]) + 0 * np.arange(br)[None, :, None]
    return sp.coo_matrix((vals.ravel(), (R.ravel(), Cc.ravel())),
                         shape=(shape[0] * br, shape[1] * bc)).tocsr()


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def soa(x):
    """Node-interleaved [node][3] -> component-major [3][node] (the C ABI's reduced layout)."""
    return np.ascontiguousarray(np.asarray(x).reshape(-1, 3).T).ravel()


def aos(x):
    """Component-major [3][node] -> node-interleaved [node][3]."""
    return np.ascontiguousarray(np.asarray(x).reshape(3, -1).T).ravel()


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def coarse_vertices(V, n):
    """Vertices of the n/2 mesh: the fine vertices at even logical positions."""
    nv, nc = n + 1, n // 2
    idx = np.arange(nc + 1) * 2
    K, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    return V[(I + nv * (J + nv * K)).ravel()]


def manufactured_instance(n, mu, dt, jitter, seed, rhs="manufactured"):
    inst = wl.Instance(n=n, mu=mu, dt=dt, jitter=jitter, seed=seed, rhs=rhs)
    V = inst.vertices()
    return inst, V, inst.force(V)
