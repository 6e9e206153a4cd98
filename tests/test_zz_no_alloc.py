"""The allocation-free fit entry point, against the context-based one.

lp_fit_derivatives_noalloc serves callers that cannot allocate device memory
(allocator hooks, plug-ins whose host owns all device memory, loops that forbid
allocation). Here the test allocates the inputs and the output itself, calls
the entry point twice in a row (its shared scratch must be cleared between
calls) and compares each result with lp_fit_derivatives on the same stencils.
This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_14061_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _case(seed, n):
    # a jittered lattice plus a sparse cloud: some stencils take the QR path
    rng = np.random.default_rng(seed)
    h = 1e-3
    k = int(round((n // 2) ** (1 / 3)))
    g = (np.arange(k) + 0.5) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    lat = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + rng.uniform(-0.1 * h, 0.1 * h, (k ** 3, 3))
    cloud = rng.uniform(0, 3 * k * h, (n - k ** 3, 3)) + np.array([0, 0, 0.02])
    p = np.concatenate([lat, cloud])
    f = np.stack([np.sin(300 * p[:, 0]) * p[:, 1] * 50, np.cos(200 * p[:, 2]) + p[:, 0] * 80,
                  p[:, 2] * 40])
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), f, h


def test_noalloc_matches_context_fit_twice(dev):
    from paper_2206_14061_gb300 import capi
    ctx = capi.Context(20000, cap=64)
    for call, (seed, prec) in enumerate(((1, capi.LP_FP64), (2, capi.LP_MIXED))):
        x, y, z, f, h = _case(seed, 12000)
        X = [torch.tensor(a, device=dev) for a in (x, y, z)]
        F = [torch.tensor(a, device=dev) for a in f]
        nb = capi.lp_build_neighbors(ctx, *X, r_const=2.2 * h, mirror_mode=1, cap=64)
        ctx.sync()
        hn, hc = nb.export()
        n = x.size
        # caller-owned stencils (k-major), used by both entry points
        nbr = torch.tensor(np.ascontiguousarray(hn.T).ravel(), dtype=torch.int32, device=dev)
        cnt = torch.tensor(hc, dtype=torch.int32, device=dev)
        own = capi.Neighbors(ctx, capi.LpNeighbors(nbr.data_ptr(), cnt.data_ptr(), n, 64, 0))
        ref = capi.lp_fit_derivatives(ctx, *X, own, F, [1.0, 1.0, -1.0], h, precision=prec)
        d = ctx.sync()
        assert d["n_fallback"] > 0
        out = torch.full((n, 3, 9), np.nan, dtype=torch.float64, device=dev)
        got = capi.lp_fit_derivatives_noalloc(*X, nbr, cnt, 64, F, [1.0, 1.0, -1.0], h, out,
                                              precision=prec)
        torch.cuda.synchronize()
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        scale = np.abs(b).max(axis=0, keepdims=True)
        assert (np.abs(a - b) <= 1e-11 * scale).all(), call


def test_noalloc_rejects_oversize_on_host(dev):
    from paper_2206_14061_gb300 import capi
    L = capi.lib()
    import ctypes
    n = capi.NOALLOC_MAX_PARTICLES + 1
    fp = (ctypes.c_void_p * 1)(1)
    ms = (ctypes.c_double * 1)(1.0)
    st = L.lp_fit_derivatives_noalloc(n, 1, 1, 1, 1, 1, 64, fp, ms, 1, 1e-3, 0.0, 1, 0, None)
    assert st == capi.LP_ERR_INVALID_ARG
