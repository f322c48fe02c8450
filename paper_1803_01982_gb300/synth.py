"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the factorisation's arithmetic: it only builds test
matrices with prescribed singular values (the paper's Type-1 recipe of
Sec. 4.1 with the decays of the benchmark workloads), Kahan matrices (the
classical failure case of greedy column pivoting mentioned in Sec. 2.1) and
exactly low-rank matrices.  The Gaussian sketch Omega is NOT generated here:
both the CUDA library and the oracle draw it themselves from the Philox
counter stream.

Recipes (every factor orthonormal = Q of a Householder QR of a seeded Gaussian
matrix with diag(R) > 0, which makes Q unique):

* ``decayed(m, n, sigma, noise, seed)``:  A = U_r diag(sigma) V_r^T + noise*E
* ``kahan(n, c)``:                          Kahan's upper-triangular matrix
* ``rank_k(m, n, k, seed)``:                X_L X_R^T with Gaussian factors
* ``tucker(dims, core, decay, noise, seed)``: C x_1 Q_1 ... x_d Q_d + noise*E,
  C Gaussian, optionally graded by decay[r]^{i_r} along each mode
"""
from __future__ import annotations

import numpy as np


def orthonormal(rng: np.random.Generator, m: int, r: int) -> np.ndarray:
    G = rng.standard_normal((m, r))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def decayed(m: int, n: int, sigma, noise: float = 0.0, seed: int = 1,
            dtype=np.float32) -> np.ndarray:
    """A = U_r diag(sigma) V_r^T + noise * E, built in FP64, rounded once."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    rng = np.random.default_rng(seed)
    U = orthonormal(rng, m, r)
    V = orthonormal(rng, n, r)
    A = (U * sigma[None, :]) @ V.T
    if noise:
        A += noise * rng.standard_normal((m, n))
    return np.ascontiguousarray(A.astype(dtype))


def decayed_torch(m: int, n: int, sigma, noise: float, seed: int, device: str = "cuda"):
    """Same recipe as ``decayed`` for sizes too large to assemble on the host
    (20000^2): the orthonormal factors come from numpy (seeded Gaussians, QR on
    the host), the product and the noise are formed on the device in FP64 with
    torch's seeded generator, then rounded once to FP32.  Input synthesis only,
    not the factorisation path."""
    import torch
    sig = np.asarray(sigma, dtype=np.float64)
    r = sig.shape[0]
    rng = np.random.default_rng(seed)
    U = torch.from_numpy(orthonormal(rng, m, r)).to(device)
    V = torch.from_numpy(orthonormal(rng, n, r)).to(device)
    sigma = torch.from_numpy(sig).to(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    A = torch.empty(m, n, device=device, dtype=torch.float32)
    rb = 2048
    for i0 in range(0, m, rb):
        i1 = min(m, i0 + rb)
        blk = (U[i0:i1] * sigma[None, :]) @ V.T
        if noise:
            blk += noise * torch.randn(i1 - i0, n, generator=gen, device=device,
                                       dtype=torch.float64)
        A[i0:i1] = blk.to(torch.float32)
    del U, V
    return A


def kahan(n: int, c: float = 0.285, dtype=np.float64) -> np.ndarray:
    """Kahan matrix diag(1, s, ..., s^{n-1}) * (I - c * strict upper ones), s^2+c^2=1."""
    s = np.sqrt(1.0 - c * c)
    K = np.eye(n) - c * np.triu(np.ones((n, n)), 1)
    K = (s ** np.arange(n))[:, None] * K
    return np.ascontiguousarray(K.astype(dtype))


def rank_k(m: int, n: int, k: int, seed: int = 3, dtype=np.float64) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray((rng.standard_normal((m, k)) @ rng.standard_normal((k, n)))
                                .astype(dtype))


def config1(dtype=np.float64) -> np.ndarray:
    """1000 x 800, sigma_j = 0.9^j (j = 1..800), exactly that spectrum."""
    return decayed(1000, 800, 0.9 ** np.arange(1, 801), 0.0, seed=1, dtype=dtype)


def slow_decay(r: int) -> np.ndarray:
    return np.arange(1, r + 1, dtype=np.float64) ** -1.5


def fast_decay(r: int, base: float = 0.97) -> np.ndarray:
    return base ** np.arange(1, r + 1, dtype=np.float64)


def _tucker_core(rng, core, decay):
    C = rng.standard_normal(tuple(core))
    if decay is not None:
        for r, c in enumerate(decay):
            shape = [1] * len(core)
            shape[r] = core[r]
            C = C * (float(c) ** np.arange(core[r])).reshape(shape)
    return C


def tucker(dims, core, decay=None, noise: float = 0.0, seed: int = 1, dtype=np.float32) -> np.ndarray:
    """X = C x_1 Q_1 ... x_d Q_d + noise * E (row-major over the modes), built in
    FP64 and rounded once.  C (core[0] x ... x core[d-1]) is Gaussian, scaled by
    decay[r]^{i_r} along mode r when decay is given; Q_r is dims[r] x core[r]
    orthonormal.  The multilinear rank is core when noise = 0."""
    rng = np.random.default_rng(seed)
    X = _tucker_core(rng, core, decay)
    for r, (I, c) in enumerate(zip(dims, core)):
        Q = orthonormal(rng, I, c)
        X = np.moveaxis(np.tensordot(Q, X, axes=([1], [r])), 0, r)
    if noise:
        X = X + noise * rng.standard_normal(tuple(dims))
    return np.ascontiguousarray(X.astype(dtype))


def tucker_torch(dims, core, noise: float, seed: int, device: str = "cuda"):
    """``tucker`` (no grading) formed on the device in FP64 with torch's seeded
    generator for the noise, rounded once to FP32; for tensors too large to
    assemble on the host.  Input synthesis only."""
    import torch
    rng = np.random.default_rng(seed)
    X = torch.from_numpy(_tucker_core(rng, core, None)).to(device)
    for r, (I, c) in enumerate(zip(dims, core)):
        Q = torch.from_numpy(orthonormal(rng, I, c)).to(device)
        X = torch.movedim(torch.tensordot(Q, X, dims=([1], [r])), 0, r)
    X = X.contiguous()
    if noise:
        gen = torch.Generator(device=device)
        gen.manual_seed(seed)
        X += noise * torch.randn(X.shape, generator=gen, device=device, dtype=torch.float64)
    return X.to(torch.float32).contiguous()


def rpca_problem(m: int, n: int, rank: int, nnz: int, seed: int = 1, dtype=np.float32):
    """Robust PCA test matrix of Sec. 4.3.1: M = X* + E*, X* = X_L X_R^T with
    Gaussian X_L (m x rank) and X_R (n x rank), E* with nnz entries at
    uniformly random positions, values uniform in [-500, 500].  Returns
    (M, X*, E*), built in FP64 and rounded once."""
    rng = np.random.default_rng(seed)
    Xs = rng.standard_normal((m, rank)) @ rng.standard_normal((rank, n))
    Es = np.zeros((m, n))
    idx = rng.choice(m * n, size=nnz, replace=False)
    Es.flat[idx] = rng.uniform(-500.0, 500.0, size=nnz)
    M = Xs + Es
    return (np.ascontiguousarray(M.astype(dtype)), Xs.astype(dtype), Es.astype(dtype))
