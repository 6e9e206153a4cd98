"""lp_step on host arrays: the library copies the state to the device, steps
and copies it back. Same bits as the same steps on device arrays, whether the
seven arrays are one packed block (one copy each way), separate pinned arrays
or pageable arrays; a mix of host and device arrays is rejected."""
import ctypes

import numpy as np
import pytest

from paper_2206_14061_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_14061_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def capi(dev):
    from paper_2206_14061_gb300 import capi as C
    C.lib()
    return C


def _setup():
    wl = W.cube(14)
    pd = W.param_dict(wl)
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    prm = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
               floor_z=pd["floor_z"], mirror_mode=pd["mirror_mode"], precision=2,
               rebuild_every=1, launch_mode=0, skin=0.1 * pd["h"], keep_lists=1)
    s = dict(wl.state)
    s["u"] = 20.0 * s["z"]
    return s, mui, eos, prm, pd["dt"]


def _run(capi, state, mui, eos, prm, dt, calls, stream):
    ctx = capi.Context(state["x"].numel(), cap=64)
    for _ in range(calls):
        capi.lp_step(ctx, state, mui, eos, prm, dt, 1, stream=stream)
    stream.synchronize()
    ctx.sync(stream)
    return {k: v.cpu().numpy().copy() for k, v in state.items()}


def test_host_arrays_give_the_device_bits(dev, capi):
    s0, mui, eos, prm, dt = _setup()
    stream = torch.cuda.Stream()
    ref = _run(capi, {k: torch.tensor(s0[k], device=dev) for k in capi.FIELDS}, mui, eos, prm,
               dt, 3, stream)
    block = torch.tensor(np.stack([s0[k] for k in capi.FIELDS])).pin_memory()
    variants = {
        "packed pinned": {k: block[i] for i, k in enumerate(capi.FIELDS)},
        "separate pinned": {k: torch.tensor(s0[k]).pin_memory() for k in capi.FIELDS},
        "pageable": {k: torch.tensor(s0[k]) for k in capi.FIELDS},
    }
    for name, st in variants.items():
        got = _run(capi, st, mui, eos, prm, dt, 3, stream)
        for k in capi.FIELDS:
            assert np.array_equal(got[k], ref[k]), (name, k)


def test_mixed_host_and_device_arrays_are_rejected(dev, capi):
    s0, mui, eos, prm, dt = _setup()
    n = s0["x"].size
    ctx = capi.Context(n, cap=64)
    keep = [torch.tensor(s0["x"]).pin_memory()] + [torch.tensor(s0[k], device=dev)
                                                   for k in capi.FIELDS[1:]]
    p = capi.LpParticles()
    for k, t in zip(capi.FIELDS, keep):
        setattr(p, k, t.data_ptr())
    p.n = n
    p.ncolumns = 1
    ma = (capi.LpMui * 1)(capi.mui_struct(mui))
    e, q = capi.eos_struct(eos), capi.params_struct(prm)
    st = capi.lib().lp_step(ctx.handle, ctypes.byref(p), ma, ctypes.byref(e), ctypes.byref(q),
                            float(dt), 1, None)
    assert st == capi.LP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        capi.lp_step(ctx, dict(zip(capi.FIELDS, keep)), mui, eos, prm, dt, 1)
