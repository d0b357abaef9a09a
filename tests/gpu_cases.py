"""Shared helpers of the GPU tests: cases, device upload, and conversion of
the oracle's sparse matrices into the 27-plane form the library exports."""
import numpy as np

import oracle
import synth


def stencil_planes(K, dims):
    """[27][N] from a (full-index-space) sparse matrix K: plane s at node n is
    K[n, n + d], d = (s%3-1, s//3%3-1, s//9-1), 0 where the neighbour is off-grid."""
    Nx, Ny, Nz = dims
    N = Nx * Ny * Nz
    K = K.tocsr()
    out = np.zeros((27, N))
    k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    n = ((k * Ny + j) * Nx + i).ravel()
    for s in range(27):
        di, dj, dk = s % 3 - 1, (s // 3) % 3 - 1, s // 9 - 1
        ii, jj, kk = (i + di).ravel(), (j + dj).ravel(), (k + dk).ravel()
        ok = (ii >= 0) & (ii < Nx) & (jj >= 0) & (jj < Ny) & (kk >= 0) & (kk < Nz)
        cols = (kk * Ny + jj) * Nx + ii
        vals = np.zeros(N)
        vals[ok] = np.asarray(K[n[ok], cols[ok]]).ravel()
        out[s] = vals
    return out


def ragged_hill():
    # 150 x 44 x 7 nodes: half-rows of 75 columns span 3 warps with a ragged
    # tail, 44 rows span 11 block rows; odd cell count in x.
    return synth.single_hill(149, 43, 6, sigma=600.0, height=120.0, noise=0.3)


def small_cases():
    return {
        "hill64": synth.single_hill(),
        "ragged": ragged_hill(),
        "jitter": synth.jittered(21, 18, 5, seed=3, a=(1.0, 1.0, 1.0)),
        "aniso": synth.single_hill(40, 33, 9, sigma=300.0, height=100.0, a=(1.0, 1.0, 10.0)),
        "penalty": synth.single_hill(33, 40, 5, sigma=250.0, height=80.0, a=(2.0, 1.0, 0.5)),
    }


def to_dev(torch, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).to("cuda") for a in arrays]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
