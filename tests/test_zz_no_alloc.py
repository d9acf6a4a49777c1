"""rk_dots_noalloc: block inner products with fixed, statically allocated
scratch, for callers that must not allocate device memory while running.

Called through the C ABI and compared with rk_dots (which draws its scratch
from the context allocator) on two calls in a row — the second call reuses the
scratch the first one left behind. The two share the kernel, its grid and its
reduction order, so they must agree bit for bit; both must also meet the
tolerance of the other dot tests (|d - d_ref| <= 1e-13 ||Q_q|| ||w||) against
the exact products. Free device memory must not change across the calls that
follow the first (the one that looks up the scratch address). Collected last, so a run that
stops at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1501_03358_gb300 import native
    return native.load()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_dots_match_rk_dots_twice(lib):
    from paper_1501_03358_gb300 import native
    torch.cuda.set_device(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ctx = ctypes.c_void_p()
    native.check(lib.rk_context_create(native.ALLOC_FN(), native.FREE_FN(), None, ctypes.byref(ctx)))
    try:
        free_after_first = None
        for call, (n, nq) in enumerate([(262144, 61), (100003, 17), (5000, 64)]):
            rng = np.random.default_rng(40 + call)
            Q = rng.standard_normal((nq, n))
            w = rng.standard_normal(n)
            Qd = torch.from_numpy(Q).cuda()
            wd = torch.from_numpy(w).cuda()
            ref = torch.zeros(nq, dtype=torch.float64, device="cuda")
            got = torch.full((nq,), float("nan"), dtype=torch.float64, device="cuda")
            native.check(lib.rk_dots(ctx, n, nq, _p(Qd), n, _p(wd), _p(ref), stream))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            native.check(lib.rk_dots_noalloc(n, nq, _p(Qd), n, _p(wd), _p(got), stream))
            torch.cuda.synchronize()
            if free_after_first is None:
                free_after_first = torch.cuda.mem_get_info()[0]
            else:
                assert torch.cuda.mem_get_info()[0] == free0, call
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.array_equal(g, r), call
            bound = 1e-13 * np.linalg.norm(Q, axis=1) * np.linalg.norm(w)
            exact = Q @ w
            assert np.all(np.abs(g - exact) <= bound), call
        # nq = 0 is accepted and writes nothing, as with rk_dots
        out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
        native.check(lib.rk_dots_noalloc(1000, 0, None, 1000, _p(wd), _p(out), stream))
        assert out.item() == 7.0
    finally:
        lib.rk_context_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_1501_03358_gb300 import native
    n, nq = 1000, 65
    Qd = torch.zeros((nq, n), dtype=torch.float64, device="cuda")
    wd = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(nq, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.rk_dots_noalloc(n, nq, _p(Qd), n, _p(wd), _p(out), stream)
    assert rc == native.RK_E_INVALID
    assert b"64" in lib.rk_last_error()
