"""The boundary's resume, Gaussian-width and memory-budget parameters, through
the C ABI, against the oracle.

* x0 (initial guess of S, Sec. 4.1 leaves GMRES's start vector open): a batch
  interrupted by the cycle cap resumes from its returned S and reaches the
  same solution as an uninterrupted solve and as the oracle.
* gauss_w (the Gaussian of G, Sec. 4.2 eq. Gchoice, read with a width): the
  plan's closed-form tables follow the width, and the solve matches the oracle
  run with the same width.
* mem_budget: the plan holds at most the budget and solves a list of k larger
  than its batch.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import dbar_oracle as orc

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def dbar(torch_cuda):
    from paper_1508_02363_gb300 import dbar as d
    return d


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-13, 1e-12), ("mixed", 1e-12, 1e-10)])
def test_interrupted_batch_resumes_from_x0(dbar, prec, tol, bar):
    w = wl.mixed_1024(N=128, nk=3, L=5.0)
    kw = dict(M=2, prec=prec, restart=8, tol=tol, max_batch=2)   # batches of 2 and 1
    capped = dbar.Plan(w.N, w.L, max_outer=1, **kw).solve(w.Q, w.k, want_m=False)
    assert capped["status"] == dbar.DBAR_ENOCONV and np.all(capped["resid"] > tol)
    plan = dbar.Plan(w.N, w.L, **kw)
    resumed = plan.solve(w.Q, w.k, x0=capped["S"])
    whole = plan.solve(w.Q, w.k)
    assert resumed["status"] == dbar.DBAR_OK and np.all(resumed["resid"] <= tol)
    # the counts restart with the resumed call: fewer cycles than from zero
    assert np.all(resumed["iters"][:, 1] >= 1) and np.all(resumed["iters"][:, 1] < whole["iters"][:, 1])
    for i in range(w.k.size):
        assert rel(resumed["S"][i], whole["S"][i]) < bar, i
        assert rel(resumed["m"][i], whole["m"][i]) < bar, i
        o = orc.solve_cgo(w.Q, w.k[i], w.N, w.L, M=2, tol=1e-14, restart=60)
        assert rel(resumed["S"][i], o["S"]) < bar, i
        assert rel(resumed["m"][i], o["m"]) < bar, i


def test_x0_on_the_device_aliasing_S_out_and_converged_start(dbar, torch_cuda):
    # FP64 plan: a device x0 that is also S_out; a start that already meets tol runs
    # no cycle and returns x0 unchanged
    torch = torch_cuda
    w = wl.plain_fp64()
    plan = dbar.Plan(w.N, w.L, M=w.M, prec="fp64", restart=8, tol=1e-13, max_batch=1)
    Qd = torch.from_numpy(w.Q).cuda()
    S = torch.zeros((1, w.N, w.N), dtype=torch.complex128, device="cuda")
    capped = dbar.Plan(w.N, w.L, M=w.M, prec="fp64", restart=4, max_iter=4, max_outer=1, tol=1e-13,
                       max_batch=1).solve_device(Qd, w.k, S)
    assert capped["status"] == dbar.DBAR_ENOCONV
    r = plan.solve_device(Qd, w.k, S, x0=S)
    assert r["status"] == dbar.DBAR_OK and r["resid"][0] <= 1e-13
    o = orc.solve_cgo(w.Q, w.k[0], w.N, w.L, M=w.M, tol=1e-14)
    assert rel(S[0].cpu().numpy(), o["S"]) < 1e-12
    S_conv = S.clone()
    r2 = plan.solve_device(Qd, w.k, S, x0=S_conv)
    assert r2["status"] == dbar.DBAR_OK and tuple(r2["iters"][0]) == (0, 0)
    assert torch.equal(S, S_conv)


def test_non_finite_x0_is_rejected(dbar):
    w = wl.plain_fp64()
    plan = dbar.Plan(w.N, w.L, prec="fp64", max_batch=1)
    x0 = np.zeros((1, w.N, w.N), complex)
    x0[0, 5, 7] = np.nan
    with pytest.raises(dbar.DbarError) as e:
        plan.solve(w.Q, w.k, x0=x0)
    assert e.value.status == dbar.DBAR_EINVAL


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-12), ("mixed", 1e-10)])
@pytest.mark.parametrize("width", [0.8, 1.5])
def test_gaussian_width_matches_oracle(dbar, prec, bar, width):
    w = wl.mixed_1024(N=128, nk=2, L=5.0)
    tol = 1e-13 if prec == "fp64" else 1e-12
    r = dbar.Plan(w.N, w.L, M=4, prec=prec, restart=24, tol=tol, max_batch=2, gauss_w=width).solve(w.Q, w.k)
    r1 = dbar.Plan(w.N, w.L, M=4, prec=prec, restart=24, tol=tol, max_batch=2).solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK
    for i in range(w.k.size):
        o = orc.solve_cgo(w.Q, w.k[i], w.N, w.L, M=4, tol=1e-14, restart=60, width=width)
        assert rel(r["S"][i], o["S"]) < bar, i
        assert rel(r["m"][i], o["m"]) < bar, i
        # on this resolved grid the regularisation is exact for either width
        assert rel(r["m"][i], r1["m"][i]) < bar, i


@pytest.mark.parametrize("width", [0.8, 1.5])
def test_gaussian_width_of_h_of_S_matches_oracle(dbar, torch_cuda, width):
    # a coarse grid (N = 64, L = 1.5) where the width changes h(S) by ~1e-3: the
    # plan's tables follow the width, to the FP64 bar
    torch = torch_cuda
    N, L, M = 64, 1.5, 2
    g = orc.Grid(N, L)
    f = np.exp(-((g.X - 0.4) ** 2 + (g.Y + 0.7) ** 2) / 0.64) * (1 + 0.3j * g.X)
    S = g.F(f)[None]
    plan = dbar.Plan(N, L, M=M, prec="fp64", max_batch=1, restart=4, gauss_w=width)
    Sd = torch.from_numpy(S).cuda()
    md = torch.empty_like(Sd)
    dbar.dbar_m_from_S(plan.handle, 1, Sd, md)
    ref = orc.h_of_S(S[0], g, M, width=width)
    assert rel(md[0].cpu().numpy(), ref) < 1e-12
    assert rel(ref, orc.h_of_S(S[0], g, M)) > 1e-4


def test_gaussian_width_of_the_convolution_route_matches_oracle(dbar):
    N, L, k = 32, 3.0, [0.4 + 0.2j]
    w = wl.small_gaussian(N, L, k[0])
    r = dbar.Plan(N, L, prec="fp64", regularisation="conv", tol=1e-13, max_batch=1, gauss_w=1.3).solve(w.Q, k)
    o = orc.solve_cgo_conv(w.Q, k[0], N, L, tol=1e-14, width=1.3)
    assert r["status"] == dbar.DBAR_OK
    assert rel(r["S"][0], o["S"]) < 1e-12 and rel(r["m"][0], o["m"]) < 1e-12


def test_memory_budget_bounds_the_plan(dbar):
    w = wl.mixed_1024(N=128, nk=5, L=5.0)
    one = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=16, max_batch=1).device_bytes
    two = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=16, max_batch=2).device_bytes
    budget = one + 2 * (two - one) + (two - one) // 2         # room for three slots, not four
    plan = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=16, tol=1e-12, mem_budget=budget)
    assert plan.max_batch == 3 and plan.device_bytes <= budget
    r = plan.solve(w.Q, w.k)                                   # batches of 3 and 2
    ref = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=16, tol=1e-12, max_batch=1).solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK and np.array_equal(r["S"], ref["S"])
    for bad in (dict(mem_budget=one - 1), dict(mem_budget=budget, max_batch=4)):
        with pytest.raises(dbar.DbarError) as e:
            dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=16, **bad)
        assert e.value.status == dbar.DBAR_ENOMEM, bad


@pytest.mark.parametrize("N,L,nk", [(256, 8.0, 5), (1024, 10.0, 3)])
def test_support_skip_gives_the_same_solution(dbar, N, L, nk):
    # A potential concentrated near the origin (narrow Gaussians): Q is exactly zero in
    # FP32 on most columns of the box, where the FP32 inner operator skips its
    # work; the solution is the same as with every column processed, value for value
    rng = np.random.default_rng(31)
    Q = wl.gaussian_mixture(N, L, rng.uniform(-1.5, 1.5, (3, 2)), rng.uniform(0.4, 0.8, 3),
                            rng.uniform(1, 3, 3) * np.exp(2j * np.pi * rng.uniform(size=3)))
    Q32 = Q.astype(np.complex64)
    cols = np.flatnonzero(np.any(Q32 != 0, axis=0))
    assert cols.size < 0.6 * N                     # the skip is in effect
    k = wl.random_k_disc(rng, nk, 3.0)
    kw = dict(M=2, prec="mixed", restart=16, tol=1e-12, max_batch=nk)
    r = dbar.Plan(N, L, **kw).solve(Q, k, want_m=False)
    r0 = dbar.Plan(N, L, support_skip=0, **kw).solve(Q, k, want_m=False)
    assert r["status"] == dbar.DBAR_OK
    assert np.array_equal(r["S"], r0["S"]) and np.array_equal(r["iters"], r0["iters"])
    if N <= 256:
        for i in range(nk):
            o = orc.solve_cgo(Q, k[i], N, L, M=2, tol=1e-14, restart=60)
            assert rel(r["S"][i], o["S"]) < 1e-10, i


def test_uneven_batches_run_concurrently_with_the_same_results(dbar, torch_cuda):
    # three grids (three plans), two potentials on one of them: one dbar_solve_batches
    # call gives each batch the bits of its own dbar_solve_cgo call
    torch = torch_cuda
    L = 4.0
    specs = [(64, 0, [0.3 + 0.1j, -0.2j, 0.5]), (128, 0, [1.1 - 0.4j, 0.2 + 0.9j]), (128, 1, [0.7j]),
             (256, 1, [2.0 + 1.0j, -1.5 + 0.5j, 0.1])]
    plans = {N: dbar.Plan(N, L, prec="mixed", restart=16, tol=1e-12, max_batch=3) for N in (64, 128, 256)}
    batch, ref = [], []
    for N, pot, k in specs:
        Q = torch.from_numpy(wl.uneven_potentials(N, L)[pot]).cuda()
        S = torch.empty((len(k), N, N), dtype=torch.complex128, device="cuda")
        batch.append({"plan": plans[N].handle, "Q": Q, "k": np.array(k), "S_out": S})
    st, sts, iters, resid = dbar.dbar_solve_batches(batch)
    assert st == dbar.DBAR_OK and all(x == dbar.DBAR_OK for x in sts)
    for (N, pot, k), bt, it, rs in zip(specs, batch, iters, resid):
        alone = torch.empty_like(bt["S_out"])
        r = plans[N].solve_device(bt["Q"], np.array(k), alone)
        assert torch.equal(alone, bt["S_out"]), (N, pot)
        assert np.array_equal(r["iters"], it) and np.all(rs <= 1e-12)


def test_uneven_batches_report_each_status(dbar, torch_cuda):
    torch = torch_cuda
    w = wl.plain_fp64()
    ok = dbar.Plan(w.N, w.L, prec="fp64", tol=1e-13, max_batch=1)
    capped = dbar.Plan(w.N, w.L, prec="fp64", tol=1e-13, restart=4, max_iter=4, max_outer=1, max_batch=1)
    Q = torch.from_numpy(w.Q).cuda()
    S1 = torch.empty((1, w.N, w.N), dtype=torch.complex128, device="cuda")
    S2 = torch.empty_like(S1)
    st, sts, _, _ = dbar.dbar_solve_batches([{"plan": ok.handle, "Q": Q, "k": w.k, "S_out": S1},
                                              {"plan": capped.handle, "Q": Q, "k": w.k, "S_out": S2}])
    assert st == dbar.DBAR_ENOCONV and sts == [dbar.DBAR_OK, dbar.DBAR_ENOCONV]
    bad = Q.clone()
    bad[3, 3] = float("nan")
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_solve_batches([{"plan": ok.handle, "Q": Q, "k": w.k, "S_out": S1},
                                 {"plan": capped.handle, "Q": bad, "k": w.k, "S_out": S2}])
    assert e.value.status == dbar.DBAR_EINVAL and "batch 1" in str(e.value)
