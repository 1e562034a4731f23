"""The tridiagonal entry point that allocates nothing.

hsgn_tridiag_solve_noalloc serves callers that cannot call cudaMalloc (host
loops with a latency budget, programs whose device memory belongs to another
allocator). It works in a fixed device scratch array inside the library. This
test calls it through the C ABI twice in a row (different sizes, both using the
scratch) and compares each result with the allocating entry point
hsgn_tridiag_solve within the solver tolerance of the parity tests. The file
name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_07539_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_allocating_solve_on_two_calls():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_07539_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    from paper_2510_07539_gb300 import solver

    lib = solver.load()
    f = lib.hsgn_tridiag_solve_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int32] + [ctypes.c_void_p] * 6
    f.restype = ctypes.c_int
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, periodic) in enumerate([(200_000, True), (70_001, False)]):
        a, b, c, d = (torch.tensor(v, device="cuda")
                      for v in inputs.random_tridiag(900 + call, n, periodic, coupling=5.0))
        ref = solver.tridiag_solve(a, b, c, d, periodic)
        x = torch.full_like(d, float("nan"))
        rc = f(n, int(periodic), *(ctypes.c_void_p(t.data_ptr()) for t in (a, b, c, d, x)),
               stream)
        assert rc == 0, lib.hsgn_error_string(rc)
        xr, rr = x.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(xr))
        assert np.max(np.abs(xr - rr)) <= 1e-13 * np.max(np.abs(rr)), call

    # sizes beyond the fixed scratch are rejected before any device work
    big = solver.NOALLOC_MAX_N + 1
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    assert f(big, 0, p, p, p, p, p, p, stream) == 1
    assert f(0, 0, p, p, p, p, p, p, stream) == 1
