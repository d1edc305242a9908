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
    # largest singular value of the part of span(A) outside span(B): accurate
    # for small angles, where sqrt(1 - cos^2) would stall near 1e-8
    return float(np.linalg.norm(qa - qb @ (qb.T @ qa), 2))


def sparse_h(m, h, V, sigma=0.0):
    """Sparse H_h + sigma (the same Kronecker sum as dense_h, CSR)."""
    import scipy.sparse as sp
    T = sp.csr_matrix(lap1d_half(m, h))
    I = sp.identity(m, format="csr")
    A = sp.kron(I, sp.kron(I, T)) + sp.kron(I, sp.kron(T, I)) + sp.kron(T, sp.kron(I, I))
    return (A + sp.diags(np.asarray(V, dtype=np.float64).ravel() + sigma)).tocsc()


def lowest_eigenpairs(m, V, k, lo=-6.0, hi=6.0):
    """The k lowest eigenpairs of H_h (the definition of the converged result
    of the scheme): shift-invert Lanczos (scipy eigsh) about a point below the
    spectrum.  Eigenvectors are normalised to <u,u> = h^3 u^T u = 1.  Returns
    ascending eigenvalues and the n x k vectors."""
    import scipy.sparse.linalg as spla
    h = (hi - lo) / (m + 1)
    A = sparse_h(m, h, V)
    below = float(np.min(V)) - 1.0
    lam, vec = spla.eigsh(A, k=k, sigma=below, which="LM", tol=1e-14)
    order = np.argsort(lam)
    return lam[order], vec[:, order] / np.sqrt(h ** 3)


def clusters(lam, count, gap):
    """Index groups of the first `count` sorted eigenvalues whose neighbours
    differ by less than `gap`; a group is kept only if it ends before `count`
    with a gap of at least `gap` to the next eigenvalue (complete clusters)."""
    groups, cur = [], [0]
    for i in range(1, len(lam)):
        if lam[i] - lam[i - 1] < gap:
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return [g for g in groups if g[-1] < count - 1 or (g[-1] == count - 1 and len(lam) > count
                                                        and lam[count] - lam[count - 1] >= gap)]
