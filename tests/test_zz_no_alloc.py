"""hq_gram_static, the allocation-free Gram entry point, against hq_gram.

Callers that cannot allocate device memory (inside a stream capture whose
policy forbids cudaMalloc, allocator-less plugin hosts, real-time loops that
must not allocate after start-up) use hq_gram_static, which keeps its
partial sums in a fixed device array instead of a caller workspace.  This
test calls it through the C ABI twice in a row, with different shapes, and
checks each result against the context entry point hq_gram on the same
inputs, with the tolerance the other Gram parity tests use.  It lives in its
own file, collected last, and passes alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_25149_gb300 import hq, inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _static_gram(lib, A, B, w, stream):
    import torch
    n, Na = A.shape
    Nb = B.shape[1]
    out = torch.empty((Na, Nb), dtype=torch.float64, device="cuda")
    st = lib.hq_gram_static(ctypes.c_void_p(A.data_ptr()), Na, ctypes.c_void_p(B.data_ptr()), Nb,
                            n, w, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert st == hq.OK, hq.status_string(st)
    return out


def test_static_gram_matches_context_gram_twice():
    import torch
    assert torch.cuda.is_available()
    lib = hq.load()
    m, N = 20, 24
    s = hq.Solver(m, N)
    s.set_potential(inputs.harmonic(m))
    w = inputs.grid_h(m) ** 3
    stream = s.stream.cuda_stream
    rng = np.random.default_rng(2024)
    cases = [(48, 17, False), (24, 24, True)]   # (Na, Nb, same block for A and B)
    for Na, Nb, same in cases:
        A = torch.from_numpy(rng.standard_normal((m ** 3, Na))).cuda()
        B = A if same else torch.from_numpy(rng.standard_normal((m ** 3, Nb))).cuda()
        got = _static_gram(lib, A, B, w, stream)
        ref = s.gram(A, B, w)
        torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL64 * np.abs(ref).max()


def test_static_gram_rejects_sizes_beyond_its_limit():
    import torch
    lib = hq.load()
    A = torch.zeros((8, 513), dtype=torch.float64, device="cuda")
    out = torch.empty((513, 513), dtype=torch.float64, device="cuda")
    st = lib.hq_gram_static(ctypes.c_void_p(A.data_ptr()), 513, ctypes.c_void_p(A.data_ptr()), 513,
                            8, 1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert st == 1   # HQ_ERR_ARG


def test_static_gram_resplits_points_to_fit_its_array():
    """Shapes whose planned split over grid points would not fit the fixed
    array are re-split into fewer, longer point chunks: n = 32^3 with 48 x 17
    columns (one 64 x 64 tile, 304 planned chunks against room for 128) and
    the symmetric 512 x 512 Gram (36 tiles per chunk, room for 3 chunks).
    Both are checked against hq_gram on the same inputs, twice in a row."""
    import torch
    lib = hq.load()
    m, N = 32, 256
    s = hq.Solver(m, N)
    s.set_potential(inputs.harmonic(m))
    w = inputs.grid_h(m) ** 3
    stream = s.stream.cuda_stream
    rng = np.random.default_rng(77)
    for Na, Nb, same in [(48, 17, False), (512, 512, True), (48, 17, False)]:
        A = torch.from_numpy(rng.standard_normal((m ** 3, Na))).cuda()
        B = A if same else torch.from_numpy(rng.standard_normal((m ** 3, Nb))).cuda()
        got = _static_gram(lib, A, B, w, stream)
        ref = s.gram(A, B, w)
        torch.cuda.synchronize()
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL64 * np.abs(ref).max()
