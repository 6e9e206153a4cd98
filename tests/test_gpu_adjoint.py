"""Adjoint of the LP step (lp_step_adjoint and its torch.autograd.Function)
against the oracle's tangent-linear run (exact derivatives of the same
frozen-stencil forward run) and against central finite differences of
lp_step."""
import numpy as np
import pytest

from paper_2206_14061_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = ("mu_s", "mu_2", "I0")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_14061_gb300 import build
    build.build()
    return torch.device("cuda:0")


def _split(pd):
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    prm = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
               floor_z=0.0, mirror_mode=pd["mirror_mode"], precision=0)
    return mui, eos, prm


def _flowing_column(R, aspect, spacing_div, U0, index):
    """Column with a radial flow u_r = U0 (r/R)(z/H): zero at the no-slip
    floor, so the mu(I) stress acts on the whole column from the first step."""
    wl = W.cylinder(R=R, aspect=aspect, spacing_div=spacing_div, index=index)
    s = dict(wl.state)
    H = aspect * R
    s["u"] = U0 * s["x"] / R * (s["z"] / H)
    s["v"] = U0 * s["y"] / R * (s["z"] / H)
    wl.state = s
    return wl


def _gpu_final(capi, ctx, state, mui, eos, prm, dt, nsteps, C, dev):
    st = {k: torch.tensor(state[k], device=dev) for k in capi.FIELDS}
    capi.lp_step(ctx, st, mui, eos, dict(prm, rebuild_every=C, launch_mode=0), dt, nsteps)
    ctx.sync()
    return st


def test_adjoint_matches_oracle_tangent_small(dev, orc):
    from paper_2206_14061_gb300 import capi
    wl = W.cube(8)
    s0 = dict(wl.state)
    s0["u"] = 20.0 * s0["z"]  # sheared column: mu(I) terms active from the start
    pd = W.param_dict(wl)
    mui, eos, prm = _split(pd)
    nsteps, C = 12, 4
    rng = np.random.default_rng(3)
    w = {k: rng.standard_normal(wl.n) for k in capi.FIELDS}
    ctx = capi.Context(wl.n, cap=64)
    init = {k: torch.tensor(s0[k], device=dev) for k in capi.FIELDS}
    seed = {k: torch.tensor(w[k], device=dev) for k in capi.FIELDS}
    dmui, gi = capi.lp_step_adjoint(ctx, init, mui, eos, prm, pd["dt"], nsteps, C, seed,
                                    want_initial=True)
    got = dmui.cpu().numpy()
    _, tan = orc.step_tangent(s0, orc.params(**pd), nsteps, rebuild_every=C)
    ref = np.array([sum((w[k] * tan[t, f]).sum() for f, k in enumerate(capi.FIELDS))
                    for t in range(3)])
    print("adjoint", got, "tangent", ref)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), (got, ref)
    # dL/d(initial u) of a few particles against central differences of lp_step
    L = lambda st: sum(float((st[k].cpu().numpy() * w[k]).sum()) for k in capi.FIELDS)
    for i in (0, 77, 300):
        for k in ("u", "z"):
            eps = 1e-7 if k == "u" else 1e-9
            sp = {q: v.copy() for q, v in s0.items()}
            sm = {q: v.copy() for q, v in s0.items()}
            sp[k][i] += eps
            sm[k][i] -= eps
            fd = (L(_gpu_final(capi, ctx, sp, mui, eos, prm, pd["dt"], nsteps, C, dev)) -
                  L(_gpu_final(capi, ctx, sm, mui, eos, prm, pd["dt"], nsteps, C, dev))) / (2 * eps)
            a = float(gi[k][i].item())
            assert abs(fd - a) <= 1e-5 * abs(a) + 1e-6, (i, k, fd, a)


@pytest.mark.parametrize("ghosts", [False, True])
def test_adjoint_keeps_whole_run_or_reruns_segments_alike(dev, orc, ghosts):
    """lp_step_adjoint with room for the whole run's data (the forward sweep
    keeps every segment; nothing is recomputed) and with none
    (lp_ctx_set_adjoint_memory(0): each segment re-run from its checkpoint),
    on the sheared 8^3 cube, 13 FP64 steps with stencils rebuilt every 4 (a
    last segment of one step), without and with ghosts: both equal the
    oracle's tangent-linear run, and each other to rounding (the reverse
    sweep's scattered sums are FP64 atomics, so not bit for bit)."""
    from paper_2206_14061_gb300 import capi
    wl = W.cube(8)
    s0 = dict(wl.state)
    s0["u"] = 20.0 * s0["z"]
    pd = W.param_dict(wl)
    mui, eos, prm = _split(pd)
    if ghosts:
        prm = dict(prm, free_surface=1)
        pd = dict(pd, free_surface=1)
    nsteps, C = 13, 4
    rng = np.random.default_rng(8)
    w = {k: rng.standard_normal(wl.n) for k in capi.FIELDS}
    init = {k: torch.tensor(s0[k], device=dev) for k in capi.FIELDS}
    seed = {k: torch.tensor(w[k], device=dev) for k in capi.FIELDS}
    _, tan = orc.step_tangent(s0, orc.params(**pd), nsteps, rebuild_every=C)
    ref = np.array([sum((w[k] * tan[t, f]).sum() for f, k in enumerate(capi.FIELDS))
                    for t in range(3)])
    out = {}
    for mode, limit in (("keep", -1), ("rerun", 0)):
        ctx = capi.Context(wl.n, cap=64)
        ctx.set_adjoint_memory(limit)
        dmui, gi = capi.lp_step_adjoint(ctx, init, mui, eos, prm, pd["dt"], nsteps, C, seed,
                                        want_initial=True)
        got = dmui.cpu().numpy()
        print(mode, "adjoint", got, "tangent", ref)
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), (mode, got, ref)
        out[mode] = (got, {k: gi[k].cpu().numpy() for k in capi.FIELDS})
    (a, ga), (b, gb) = out["keep"], out["rerun"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max(), (a, b)
    for k in capi.FIELDS:
        scale = np.abs(ga[k]).max()
        assert np.abs(ga[k] - gb[k]).max() <= 1e-12 * scale + 1e-300, k


def test_adjoint_across_all_three_regimes(dev, orc):
    """The adjoint on a sheared cube that spans the gas, inertial and
    quasi-static regimes (solid fraction 0.47 + 0.14 sin(2 pi x/L)
    cos(2 pi y/L + 0.3), soft quasi-static law beta = 0.1 m^2/s^2), 12 FP64
    steps with stencils rebuilt every 4: dL/d(mu_s, mu_2, I0) equals the
    oracle's tangent-linear run, and dL/d(initial u, V) of the most
    compacted (quasi-static), the loosest (gas) and a mid-range (inertial)
    particle match central differences of lp_step. Regimes are frozen at
    their forward values, so the steps of the differences change none."""
    from paper_2206_14061_gb300 import capi
    h = 1e-3
    x, y, z = W.lattice_box(12, 12, 12, h, 0.05, np.random.default_rng(31))
    L = 12 * h
    phi = 0.47 + 0.14 * np.sin(2 * np.pi * x / L) * np.cos(2 * np.pi * y / L + 0.3)
    s0 = dict(x=x, y=y, z=z, u=z * (1 + 0.2 * np.sin(2 * np.pi * y / L)),
              v=0.4 * z * np.cos(2 * np.pi * x / L), w=np.zeros(x.size), V=1 / phi)
    pd = dict(W.param_dict(W.cube(12)), beta=0.1, alpha=-0.1 * 0.59)
    mui, eos, prm = _split(pd)
    nsteps, C = 12, 4
    n = x.size
    rng = np.random.default_rng(5)
    w = {k: rng.standard_normal(n) for k in capi.FIELDS}
    ctx = capi.Context(n, cap=64)
    init = {k: torch.tensor(s0[k], device=dev) for k in capi.FIELDS}
    seed = {k: torch.tensor(w[k], device=dev) for k in capi.FIELDS}
    dmui, gi = capi.lp_step_adjoint(ctx, init, mui, eos, prm, pd["dt"], nsteps, C, seed,
                                    want_initial=True)
    got = dmui.cpu().numpy()
    _, tan = orc.step_tangent(s0, orc.params(**pd), nsteps, rebuild_every=C)
    ref = np.array([sum((w[k] * tan[t, f]).sum() for f, k in enumerate(capi.FIELDS))
                    for t in range(3)])
    print("three regimes: adjoint", got, "tangent", ref)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), (got, ref)
    Lf = lambda st: sum(float((st[k].cpu().numpy() * w[k]).sum()) for k in capi.FIELDS)
    picks = (int(np.argmax(phi)), int(np.argmin(phi)), int(np.argmin(np.abs(phi - 0.47))))
    assert phi[picks[0]] > 0.6 and phi[picks[1]] < 0.34
    for i in picks:
        for k, eps in (("u", 1e-7), ("V", 1e-8)):
            sp = {q: v.copy() for q, v in s0.items()}
            sm = {q: v.copy() for q, v in s0.items()}
            sp[k][i] += eps
            sm[k][i] -= eps
            fd = (Lf(_gpu_final(capi, ctx, sp, mui, eos, prm, pd["dt"], nsteps, C, dev)) -
                  Lf(_gpu_final(capi, ctx, sm, mui, eos, prm, pd["dt"], nsteps, C, dev))) / (2 * eps)
            a = float(gi[k][i].item())
            print(f"particle {i} (phi {phi[i]:.3f}) dL/d{k}: adjoint {a:.9e}, differences {fd:.9e}")
            assert abs(fd - a) <= 1e-5 * abs(a) + 1e-6, (i, k, fd, a)


def test_adjoint_column_against_finite_differences(dev, orc):
    """Column of radius 0.02 m at spacing R/25 (98,800 particles), 30 FP64
    steps, stencils rebuilt every 10 steps (the stable horizon of this column
    without free-surface ghost particles is about 40 steps)."""
    from paper_2206_14061_gb300 import capi
    from paper_2206_14061_gb300.autograd import lp_step_diff, runout_profile_loss
    R = 0.02
    wl = _flowing_column(R, 2.0, 25, 0.02, index=4)
    pd = W.param_dict(wl)
    mui, eos, prm = _split(pd)
    nsteps, C, eps = 30, 10, 1e-6
    ctx = capi.Context(wl.n, cap=64)
    init = {k: torch.tensor(wl.state[k], device=dev) for k in capi.FIELDS}
    rest = {k: pd[k] for k in ("d", "rho_s")}
    # (a) seeded linear functionals of the final state: all seven fields
    # (checked against the tangent-linear run) and the velocities alone
    # (checked against finite differences: V ~ 1.7 would put the FD round-off,
    # ulp(sum w V) / (2 eps), near 1e-7)
    rng = np.random.default_rng(20220628 + 4)
    w = {k: torch.tensor(rng.standard_normal(wl.n), device=dev) for k in capi.FIELDS}
    theta = torch.tensor([pd[k] for k in NAMES], dtype=torch.float64, requires_grad=True)
    fin = lp_step_diff(ctx, theta, init, rest, eos, prm, pd["dt"], nsteps, C)
    Lw = sum((fin[k] * w[k]).sum() for k in capi.FIELDS)
    (g_lin,) = torch.autograd.grad(Lw, theta)
    theta3 = theta.detach().clone().requires_grad_(True)
    fin3 = lp_step_diff(ctx, theta3, init, rest, eos, prm, pd["dt"], nsteps, C)
    Lu = sum((fin3[k] * w[k]).sum() for k in ("u", "v", "w"))
    (g_vel,) = torch.autograd.grad(Lu, theta3)
    # (b) runout + height-profile misfit
    _, h0 = runout_profile_loss(init, R, torch.zeros(32, dtype=torch.float64, device=dev))
    target = h0 * (1.0 + 0.05 * torch.tensor(rng.standard_normal(32), device=dev))
    theta2 = theta.detach().clone().requires_grad_(True)
    fin2 = lp_step_diff(ctx, theta2, init, rest, eos, prm, pd["dt"], nsteps, C)
    Lr, _ = runout_profile_loss(fin2, R, target)
    (g_run,) = torch.autograd.grad(Lr, theta2)
    fd_vel, fd_run = np.zeros(3), np.zeros(3)
    for t, name in enumerate(NAMES):
        vals = []
        for sgn in (1.0, -1.0):
            m = dict(mui, **{name: mui[name] + sgn * eps})
            st = _gpu_final(capi, ctx, wl.state, m, eos, prm, pd["dt"], nsteps, C, dev)
            vals.append((float(sum((st[k] * w[k]).sum() for k in ("u", "v", "w"))),
                         float(runout_profile_loss(st, R, target)[0])))
        fd_vel[t] = (vals[0][0] - vals[1][0]) / (2 * eps)
        fd_run[t] = (vals[0][1] - vals[1][1]) / (2 * eps)
    g_lin, g_run, g_vel = g_lin.numpy(), g_run.numpy(), g_vel.numpy()
    # exact derivatives of the oracle's forward run (tangent-linear)
    sf, tan = orc.step_tangent(wl.state, orc.params(**pd), nsteps, rebuild_every=C, brute=False)
    wn = {k: w[k].cpu().numpy() for k in capi.FIELDS}
    ref_lin = np.array([sum((wn[k] * tan[t, f]).sum() for f, k in enumerate(capi.FIELDS))
                        for t in range(3)])
    x, y, z = sf["x"], sf["y"], sf["z"]
    r = np.sqrt(x * x + y * y)
    i = int(np.argmax(r))
    b = np.clip((r / (3 * R / 32)).astype(int), 0, 31)
    tg = target.cpu().numpy()
    ref_run = np.zeros(3)
    for t in range(3):
        g = (x[i] * tan[t, 0, i] + y[i] * tan[t, 1, i]) / r[i]
        for kb in range(32):
            sel = np.flatnonzero(b == kb)
            if sel.size:
                j = sel[np.argmax(z[sel])]
                g += 2.0 * (z[j] - tg[kb]) * tan[t, 2, j]
        ref_run[t] = g
    print("all fields:        adjoint", g_lin, "tangent", ref_lin)
    print("velocities:        adjoint", g_vel, "FD", fd_vel)
    print("runout+profile:    adjoint", g_run, "tangent", ref_run, "FD", fd_run)
    assert np.abs(g_lin - ref_lin).max() <= 1e-9 * np.abs(ref_lin).max(), (g_lin, ref_lin)
    assert np.abs(g_run - ref_run).max() <= 1e-9 * np.abs(ref_run).max(), (g_run, ref_run)
    assert np.abs(g_vel - fd_vel).max() <= 1e-5 * np.abs(g_vel).max(), (g_vel, fd_vel)
    # FD of the runout+profile loss is limited by round-off of the positions
    # (about 2e-12 absolute at step 1e-6: ulp(0.02 m) accumulated over the run)
    assert (np.abs(g_run - fd_run) <= 1e-5 * np.abs(g_run) + 5e-12).all(), (g_run, fd_run)


def _runout_tangent(sf, tan, R, tg):
    """d(runout + profile misfit)/d(mu_s, mu_2, I0) from the oracle's tangent
    of the final positions, with the argmaxes of the final state."""
    x, y, z = sf["x"], sf["y"], sf["z"]
    r = np.sqrt(x * x + y * y)
    i = int(np.argmax(r))
    b = np.clip((r / (3 * R / 32)).astype(int), 0, 31)
    out = np.zeros(3)
    for t in range(3):
        g = (x[i] * tan[t, 0, i] + y[i] * tan[t, 1, i]) / r[i]
        for kb in range(32):
            sel = np.flatnonzero(b == kb)
            if sel.size:
                j = sel[np.argmax(z[sel])]
                g += 2.0 * (z[j] - tg[kb]) * tan[t, 2, j]
        out[t] = g
    return out


@pytest.mark.slow
def test_adjoint_column_200_steps(dev, orc):
    """The adjoint column at its stated length: radius 0.02 m, H = 2R, spacing
    R/25 (98,800 particles), 200 FP64 steps with a checkpoint every 20, loss =
    runout + squared misfit of the 32-bin height profile to a seeded target.

    The column starts at solid fraction 0.5 (the initial mean solid fraction
    implied by the paper's layer test, Sec. 4.1: 0.03 m of material expected
    to settle at phi_c = 0.6 into 0.025 m) with free-surface ghosts, which
    keeps it inside its stable horizon (about 670 steps at this spacing from
    rest, against about 50 at phi 0.585 without ghosts).

    From rest the loss does not depend on (mu_s, mu_2, I0) at all over this
    horizon: the stress is quadratic in the velocity gradient (P and tau both
    scale with |gdot|^2), so the floor's disturbance dies out within a few
    layers, and the runout particle and the top of every bin stay in exact
    free fall. The adjoint and central differences both give exactly 0 there.
    With a radial flow u_r = 0.5 m/s (r/R)(z/H) (zero at the no-slip floor)
    the whole column shears: dL/d(mu_s, mu_2, I0) from lp_step_adjoint then
    matches the oracle's tangent-linear run to 1e-9 and central differences of
    lp_step (step 1e-6) to 1e-5. (At 0.02 m/s the gradient, about 4e-9, sits
    only 200 times above the round-off of central differences, ulp(0.04 m)
    accumulated over the run divided by 2e-6: they agree to 5e-3 there.)"""
    from paper_2206_14061_gb300 import capi
    from paper_2206_14061_gb300.autograd import lp_step_diff, runout_profile_loss
    R = 0.02
    nsteps, C, eps = 200, 20, 1e-6
    for flow in (0.0, 0.5):
        wl = _flowing_column(R, 2.0, 25, flow, index=4)
        wl.state = dict(wl.state, V=np.full(wl.n, 1.0 / 0.5))
        pd = W.param_dict(wl)
        mui, eos, prm = _split(pd)
        prm = dict(prm, free_surface=1)
        ctx = capi.Context(wl.n, cap=64)
        init = {k: torch.tensor(wl.state[k], device=dev) for k in capi.FIELDS}
        rest = {k: pd[k] for k in ("d", "rho_s")}
        rng = np.random.default_rng(20220628 + 4)
        _, h0 = runout_profile_loss(init, R, torch.zeros(32, dtype=torch.float64, device=dev))
        target = h0 * (1.0 + 0.05 * torch.tensor(rng.standard_normal(32), device=dev))
        theta = torch.tensor([pd[k] for k in NAMES], dtype=torch.float64, requires_grad=True)
        fin = lp_step_diff(ctx, theta, init, rest, eos, prm, pd["dt"], nsteps, C)
        d = ctx.sync()
        assert d["n_nonfinite"] == 0
        umax = float(torch.sqrt(fin["u"] ** 2 + fin["v"] ** 2 + fin["w"] ** 2).max())
        assert umax < flow + 0.05, umax  # sane: gravity adds 0.02 m/s in 2 ms
        Lr, _ = runout_profile_loss(fin, R, target)
        (g_run,) = torch.autograd.grad(Lr, theta)
        g_run = g_run.numpy()
        fd_run = np.zeros(3)
        for t, name in enumerate(NAMES):
            vals = []
            for sgn in (1.0, -1.0):
                m = dict(mui, **{name: mui[name] + sgn * eps})
                st = _gpu_final(capi, ctx, wl.state, m, eos, prm, pd["dt"], nsteps, C, dev)
                vals.append(float(runout_profile_loss(st, R, target)[0]))
            fd_run[t] = (vals[0] - vals[1]) / (2 * eps)
        if flow == 0.0:
            print("200-step column from rest: adjoint", g_run, "FD", fd_run)
            assert (g_run == 0.0).all() and (fd_run == 0.0).all(), (g_run, fd_run)
            continue
        sf, tan = orc.step_tangent(wl.state, orc.params(**dict(pd, free_surface=1)), nsteps,
                                   rebuild_every=C, brute=False)
        ref_run = _runout_tangent(sf, tan, R, target.cpu().numpy())
        print("200-step flowing column: adjoint", g_run, "tangent", ref_run, "FD", fd_run,
              "FD relative", np.abs(g_run - fd_run) / np.abs(g_run))
        assert (np.abs(g_run) > 0).all(), g_run
        assert np.abs(g_run - ref_run).max() <= 1e-9 * np.abs(ref_run).max(), (g_run, ref_run)
        assert (np.abs(g_run - fd_run) <= 1e-5 * np.abs(g_run) + 5e-12).all(), (g_run, fd_run)
