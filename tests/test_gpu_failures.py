"""Failure paths of the library, made on the host (no GPU fault, trap or
hang): an allocator that returns NULL gives RK_E_OOM and leaves the problem
usable, with the next solve equal bit for bit to the same solve on a problem
that never saw a failure; a constructed rBiCGStab breakdown (Algorithm 4's
"exit gracefully" branch) gives RK_E_BREAKDOWN after the restarts, as the
oracle does; a bounded device wait made to run out from the host gives
RK_E_DEVICE_TIMEOUT with no copy in flight, and the problem stays usable."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from problems import Grid, make_config
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1501_03358_gb300 import native
    return native.load()


class FailingAllocator:
    """Device memory from torch's caching allocator, except that every call
    from number `fail_at` on returns NULL (None) while armed."""

    def __init__(self):
        from paper_1501_03358_gb300 import native
        self.calls = 0
        self.fail_at = None
        self.failed = 0

        def alloc(size, user):
            self.calls += 1
            if self.fail_at is not None and self.calls >= self.fail_at:
                self.failed += 1
                return None
            return torch.cuda.caching_allocator_alloc(int(size))

        def free(ptr, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cb = (native.ALLOC_FN(alloc), native.FREE_FN(free))

    def arm(self, k):
        self.fail_at = self.calls + k
        self.failed = 0

    def disarm(self):
        self.fail_at = None


class FailCtx:
    """A librk context drawing memory through a FailingAllocator."""

    def __init__(self, lib, fa):
        self.lib = lib
        self._h = ctypes.c_void_p()
        from paper_1501_03358_gb300 import native
        native.check(lib.rk_context_create(fa.cb[0], fa.cb[1], None, ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def close(self):
        self.lib.rk_context_destroy(self._h)


SOLVES = {
    "rGCROT fp64": dict(mode="rGCROT", m=12, k=6),
    "rGCROT mixed": dict(mode="rGCROT", m=12, k=6, precision="mixed"),
    "rGCROT df": dict(mode="rGCROT", m=12, k=6, precision="df"),
    "rBiCGStab df": dict(mode="rBiCGStab", k=0, precision="df"),
    "left rGCROT sub-domain": dict(mode="rGCROT", m=12, k=6, precond="subdomain", precond_side="left"),
}


@pytest.mark.parametrize("name", sorted(SOLVES))
def test_allocator_failure_gives_oom_and_leaves_problem_usable(lib, name):
    from paper_1501_03358_gb300 import Context, Problem
    from paper_1501_03358_gb300.native import RKError, RK_E_OOM
    kw = dict(tol=1e-8, max_matvec=3000, **SOLVES[name])
    cfg = make_config(1, size=9)
    b = torch.from_numpy(cfg.rhs(0)).cuda()
    b2 = torch.from_numpy(cfg.rhs(1)).cuda()
    # reference: the same two solves on a problem that never sees a failure
    ref_ctx = Context()
    ref = Problem(ref_ctx, cfg.grid, torch.from_numpy(cfg.coef))
    x_ref, _ = ref.solve(b, **kw)
    x2_ref, _ = ref.solve(b2, **kw)
    x_ref, x2_ref = x_ref.cpu().numpy(), x2_ref.cpu().numpy()
    fa = FailingAllocator()
    fctx = FailCtx(lib, fa)
    try:
        k = 1
        while True:
            p = Problem(fctx, cfg.grid, torch.from_numpy(cfg.coef))
            fa.arm(k)  # the k-th allocation of the first solve on, fail
            failed = False
            try:
                p.solve(b, **kw)
            except RKError as e:
                assert e.code == RK_E_OOM, (k, e)
                failed = True
            fa.disarm()
            if failed:
                assert fa.failed >= 1
                st = p.stats()
                assert st["solves"] == 0 and st["recycle_dim"] == 0
            # usable afterwards: both solves equal the reference bit for bit
            x, info = p.solve(b, **kw) if failed else (None, None)
            if failed:
                assert info["status"] == 0
                assert np.array_equal(x.cpu().numpy(), x_ref), k
            x2, info2 = p.solve(b2, **kw)
            assert info2["status"] == 0
            assert np.array_equal(x2.cpu().numpy(), x2_ref), k
            p.close()
            if not failed:
                break  # the first solve no longer reaches an allocation: every site was covered
            k += 1
        assert k > 2  # the solve allocates several buffers; each failure point was exercised
    finally:
        fctx.close()
        ref.close()
        ref_ctx.close()


def test_allocator_failure_after_recycle_space_keeps_it(lib):
    """An allocation failure while growing the capacity (a larger m than the
    problem holds) keeps the stored recycle space: the next solve with the
    old capacity equals the solve on an undisturbed problem bit for bit."""
    from paper_1501_03358_gb300 import Context, Problem
    from paper_1501_03358_gb300.native import RKError, RK_E_OOM
    cfg = make_config(1, size=9)
    bs = [torch.from_numpy(cfg.rhs(t)).cuda() for t in range(3)]
    kw = dict(tol=1e-8, mode="rGCROT", m=12, k=6, max_matvec=3000)
    ref_ctx = Context()
    ref = Problem(ref_ctx, cfg.grid, torch.from_numpy(cfg.coef))
    ref.solve(bs[0], **kw)
    x_ref, _ = ref.solve(bs[1], **kw)
    fa = FailingAllocator()
    fctx = FailCtx(lib, fa)
    try:
        p = Problem(fctx, cfg.grid, torch.from_numpy(cfg.coef))
        p.solve(bs[0], **kw)
        k0 = p.stats()["recycle_dim"]
        assert k0 > 0
        fa.arm(1)
        with pytest.raises(RKError) as ei:
            p.solve(bs[2], **dict(kw, m=30))  # needs a larger basis: allocation fails
        assert ei.value.code == RK_E_OOM
        fa.disarm()
        assert p.stats()["recycle_dim"] == k0
        x, info = p.solve(bs[1], **kw)
        assert info["status"] == 0 and np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
        p.close()
    finally:
        fctx.close()
        ref.close()
        ref_ctx.close()


def test_rbicgstab_breakdown_matches_oracle(lib):
    """A = [[1, 2], [0, -1]] on two cells with b = [1, 1]: with the right
    point-Jacobi preconditioner the first alpha of Algorithm 4 divides by
    r~^T A M^{-1} r_0 = [1, 1] . [-1, 1] = 0 (exactly, in any rounding), and
    every restart from the same residual breaks down again. The library
    stops with RK_E_BREAKDOWN after its restarts, as the oracle does, with
    the same product count and x unchanged."""
    from paper_1501_03358_gb300 import Context, Problem
    from paper_1501_03358_gb300.native import RK_E_BREAKDOWN
    g = Grid(2, 1, 1, (False, False, False))
    coef = np.zeros((7, 2))
    coef[0] = [1.0, -1.0]
    coef[2, 0] = 2.0
    b = np.array([1.0, 1.0])
    op = oracle.Stencil(g, coef)
    with np.errstate(divide="ignore", invalid="ignore"):
        _, io = oracle.rbicgstab(op, b, tol=1e-8)
    assert io["status"] == oracle.BREAKDOWN
    ctx = Context()
    p = Problem(ctx, g, torch.from_numpy(coef))
    x, info = p.solve(torch.from_numpy(b).cuda(), tol=1e-8, mode="rBiCGStab", k=0, max_matvec=100)
    assert info["status"] == RK_E_BREAKDOWN
    assert info["matvecs"] == io["matvecs"] and info["restarts"] == io["restarts"]
    assert np.array_equal(x.cpu().numpy(), np.zeros(2))
    # the problem is still usable: a well-posed right-hand side for the same A
    # (r~^T A M^{-1} r_0 = 1 for b = [1, 0]) converges
    x, info = p.solve(torch.tensor([1.0, 0.0], dtype=torch.float64).cuda(), tol=1e-12, mode="rBiCGStab", k=0)
    assert info["status"] == 0
    assert np.allclose(oracle.dense_matrix(g, coef) @ x.cpu().numpy(), [1.0, 0.0], rtol=0, atol=1e-12)
    p.close()
    ctx.close()


def test_bounded_wait_gives_device_timeout_and_problem_stays_usable(lib):
    """The bounded waits of the bulk-copy pipeline, made to run out from the
    host (rk_problem_wait_limit, one poll): the copy producer of the
    double-float Arnoldi inner products gives up at a stage-release barrier,
    issues nothing more, and the consumers stop at the first stage it did not
    issue, so every copy they waited for had been issued and no copy is in
    flight when a block exits. The solve returns RK_E_DEVICE_TIMEOUT; with
    the limit restored the same problem solves the same system bit for bit
    like a problem that never timed out."""
    from paper_1501_03358_gb300 import Context, Problem, native
    from paper_1501_03358_gb300.native import RKError, RK_E_DEVICE_TIMEOUT
    cfg = make_config(1, size=32)  # 32^3 cells: 16 copy stages per block, so the producer waits
    b = torch.from_numpy(cfg.rhs(0)).cuda()
    kw = dict(tol=1e-8, mode="rGCROT", m=20, k=10, precision="df", max_matvec=3000)
    ctx = Context()
    ref = Problem(ctx, cfg.grid, torch.from_numpy(cfg.coef))
    x_ref, info_ref = ref.solve(b, **kw)
    assert info_ref["status"] == 0
    p = Problem(ctx, cfg.grid, torch.from_numpy(cfg.coef))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    native.check(lib.rk_problem_wait_limit(p._h, 1, stream))
    with pytest.raises(RKError) as ei:
        p.solve(b, **kw)
    assert ei.value.code == RK_E_DEVICE_TIMEOUT
    assert p.stats()["solves"] == 0 and p.stats()["recycle_dim"] == 0
    native.check(lib.rk_problem_wait_limit(p._h, 0, stream))
    x, info = p.solve(b, **kw)
    assert info["status"] == 0
    assert np.array_equal(x.cpu().numpy(), x_ref.cpu().numpy())
    assert info["matvecs"] == info_ref["matvecs"]
    p.close()
    ref.close()
    ctx.close()
