"""Independent dense constructions used to pin the oracle (numpy/scipy only).

Nothing here is imported by the oracle or by the CUDA path."""
import numpy as np


def lap1d_half(m, h):
    """-1/2 d^2/dx^2 with Dirichlet ends: (1/(2h^2)) tridiag(-1, 2, -1)."""
    return (2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)) / (2.0 * h * h)


def dense_h(m, h, V, sigma=0.0):
    """Dense H_h + sigma as a Kronecker sum; flattened index p = i + m(j + m k)
    is C order over (k, j, i), so the x operator acts on the last factor."""
    T = lap1d_half(m, h)
    I = np.eye(m)
    A = np.kron(I, np.kron(I, T)) + np.kron(I, np.kron(T, I)) + np.kron(T, np.kron(I, I))
    return A + np.diag(np.asarray(V, dtype=np.float64).ravel() + sigma)


def harmonic_1d(m, lo, hi):
    h = (hi - lo) / (m + 1)
    x = lo + h * np.arange(1, m + 1)
    return lap1d_half(m, h) + np.diag(0.5 * x * x)


def separable_levels(m, lo, hi, count):
    """Lowest eigenvalues of -Delta_h/2 + |x|^2/2 in 3D as sums of three 1D
    tridiagonal eigenvalues (the operator is a Kronecker sum)."""
    mu = np.linalg.eigvalsh(harmonic_1d(m, lo, hi))
    s = (mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel()
    return np.sort(s)[:count]


def subspace_sin(A, B, w=1.0):
    """Largest sine of the principal angles between span(A) and span(B) in
    the weighted inner product w * x^T y."""
    qa, _ = np.linalg.qr(A)
    qb, _ = np.linalg.qr(B)
    s = np.linalg.svd(qa.T @ qb, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - min(s) ** 2)))
