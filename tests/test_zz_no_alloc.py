"""The allocation-free fit entry point, against the context-based one and the
oracle.

lp_fit_derivatives_noalloc serves callers that cannot allocate device memory
(allocator hooks, plug-ins whose host owns all device memory, loops that forbid
allocation). Here the test allocates the inputs and the output itself, calls
the entry point twice in a row (its shared scratch must be cleared between
calls) and compares each result with lp_fit_derivatives on the same stencils
and with the FP64 oracle. This file is collected last on purpose."""
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


def _field_err(got, ref, h):
    """max |diff| / max |ref| per field on h-scaled coefficients (first
    derivatives times h, second times h^2): a field whose exact second
    derivatives vanish has only rounding noise in that class, so the class
    alone is no scale."""
    sc = np.array([h] * 3 + [h * h] * 6)
    out = []
    for f in range(ref.shape[1]):
        r = ref[:, f] * sc
        out.append(np.abs((got[:, f] - ref[:, f]) * sc).max() / np.abs(r).max())
    return max(out)


def test_noalloc_matches_context_fit_and_oracle_twice(dev, orc):
    """Two calls in a row (FP64, then FP32 with one FP64 refinement): each
    result equals lp_fit_derivatives on the same stencils, and matches the
    FP64 oracle on the lattice's stencils (1e-11 per field of h-scaled
    coefficients in FP64, 1e-5 in the refined FP32 mode); the second call
    also reports its
    QR-fallback count, equal to the context fit's."""
    from paper_2206_14061_gb300 import capi
    ctx = capi.Context(20000, cap=64)
    for call, (seed, prec, tol) in enumerate(((1, capi.LP_FP64, 1e-11),
                                              (2, capi.LP_MIXED, 1e-5))):
        x, y, z, f, h = _case(seed, 12000)
        X = [torch.tensor(a, device=dev) for a in (x, y, z)]
        F = [torch.tensor(a, device=dev) for a in f]
        nb = capi.lp_build_neighbors(ctx, *X, r_const=2.2 * h, mirror_mode=1, cap=64)
        ctx.sync()
        hn, hc = nb.export()
        n = x.size
        ms = [1.0, 1.0, -1.0]
        # caller-owned stencils (k-major), used by both entry points
        nbr = torch.tensor(np.ascontiguousarray(hn.T).ravel(), dtype=torch.int32, device=dev)
        cnt = torch.tensor(hc, dtype=torch.int32, device=dev)
        own = capi.Neighbors(ctx, capi.LpNeighbors(nbr.data_ptr(), cnt.data_ptr(), n, 64, 0))
        ref = capi.lp_fit_derivatives(ctx, *X, own, F, ms, h, precision=prec)
        d = ctx.sync()
        assert d["n_fallback"] > 0
        out = torch.full((n, 3, 9), np.nan, dtype=torch.float64, device=dev)
        if call == 0:
            got = capi.lp_fit_derivatives_noalloc(*X, nbr, cnt, 64, F, ms, h, out,
                                                  precision=prec)
            torch.cuda.synchronize()
        else:
            got, counts = capi.lp_fit_derivatives_noalloc(*X, nbr, cnt, 64, F, ms, h, out,
                                                          precision=prec, diag=True)
            assert counts["n_fallback"] == d["n_fallback"]
            assert counts["flags"] == 0
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        scale = np.abs(b).max(axis=0, keepdims=True)
        assert (np.abs(a - b) <= 1e-11 * scale).all(), call
        o, rank = orc.fit(x, y, z, hn, hc, f, ms, h)
        # the jittered lattice (the first k^3 particles) has well-conditioned
        # stencils; the sparse cloud's full-rank stencils can be conditioned
        # so badly that rounding alone moves their solution
        lat = np.zeros(n, dtype=bool)
        lat[:int(round((n // 2) ** (1 / 3))) ** 3] = True
        assert (rank[lat] == 9).all() and (rank[~lat] < 9).any()
        err = _field_err(a[lat], o[lat], h)
        print(f"noalloc call {call}: max class error vs FP64 oracle = {err:.3e}")
        assert err <= tol, (call, err)


def test_noalloc_rejects_on_host(dev):
    from paper_2206_14061_gb300 import capi
    L = capi.lib()
    import ctypes
    fp = (ctypes.c_void_p * 1)(1)
    ms = (ctypes.c_double * 1)(1.0)
    n = capi.NOALLOC_MAX_PARTICLES + 1
    st = L.lp_fit_derivatives_noalloc(n, 1, 1, 1, 1, 1, 64, fp, ms, 1, 1e-3, 0.0, 1, 0, None,
                                      None)
    assert st == capi.LP_ERR_INVALID_ARG
    # the float-float mode needs per-particle workspace: not offered here
    st = L.lp_fit_derivatives_noalloc(16, 1, 1, 1, 1, 1, 64, fp, ms, 1, 1e-3, 0.0, 1,
                                      capi.LP_MIXED_FF, None, None)
    assert st == capi.LP_ERR_INVALID_ARG
