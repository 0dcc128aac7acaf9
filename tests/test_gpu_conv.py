"""The convolution regularisation G = S e^{-|xi|^2} (Sec. 4.2, remark after
eq. fourreg5a) through the C ABI against the CPU oracle's direct grid sum, and
against the Taylor-Gaussian route it is meant to test."""
import numpy as np
import pytest

import workloads as wl
from oracle import dbar_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbar():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_02363_gb300 import dbar as d
    return d


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _potential(N, L):
    X, Y = wl.mesh(N, L)
    return (1.3 * np.exp(-(X * X + Y * Y)) + (0.4 + 0.6j) * np.exp(-((X - 0.5) ** 2 + (Y + 0.3) ** 2) / 0.7)
            ).astype(np.complex128)


def _fields(N, L, nk, seed):
    # smooth fields on the xi-grid (transforms of shifted Gaussians times random complex factors)
    rng = np.random.default_rng(seed)
    g = orc.Grid(N, L)
    out = []
    for _ in range(nk):
        c = rng.standard_normal(2) * 0.7
        a = complex(*rng.standard_normal(2))
        out.append(a * g.F(np.exp(-((g.X - c[0]) ** 2 + (g.Y - c[1]) ** 2) / 1.5)))
    return np.stack(out)


@pytest.mark.parametrize("N,L", [(32, 2.0), (64, 3.0), (128, 4.0)])
def test_conv_h_of_S_matches_oracle(dbar, N, L):
    torch = pytest.importorskip("torch")
    nk = 3
    S = _fields(N, L, nk, 11)
    plan = dbar.Plan(N, L, prec="fp64", regularisation="conv", max_batch=nk)
    Sd = torch.from_numpy(S).cuda()
    m = torch.empty_like(Sd)
    dbar.dbar_m_from_S(plan.handle, nk, Sd, m)
    g = orc.Grid(N, L)
    ref = orc.h_of_S_conv(S, g)
    assert rel(m.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("N,L", [(32, 2.0), (64, 3.0)])
def test_conv_operator_matches_oracle(dbar, N, L):
    torch = pytest.importorskip("torch")
    Q = _potential(N, L)
    k = np.array([0.0, 0.7 + 0.4j, -1.5 + 2.0j])
    S = _fields(N, L, k.size, 5)
    plan = dbar.Plan(N, L, prec="fp64", regularisation="conv", max_batch=k.size)
    Sd = torch.from_numpy(S).cuda()
    out = torch.empty_like(Sd)
    dbar.dbar_apply(plan.handle, torch.from_numpy(Q).cuda(), k, Sd, out)
    for i in range(k.size):
        ref = orc.ConvProblem(Q, k[i], N, L).apply(S[i])
        assert rel(out[i].cpu().numpy(), ref) < 1e-13, i


@pytest.mark.parametrize("graphs,sstep", [(0, 0), (1, 0), (1, 4)])
def test_conv_solve_matches_oracle(dbar, graphs, sstep):
    # 5 k values on a 2-slot plan: two full batches and a ragged one; one vector per sweep
    # (sstep 0 means 1 on this route) and s-step blocks of whole applications
    N, L = 64, 4.0
    Q = _potential(N, L)
    k = np.array([0.0, 0.7 + 0.4j, -1.5 + 2.0j, 2.5 - 0.5j, -0.3 - 1.1j])
    plan = dbar.Plan(N, L, prec="fp64", regularisation="conv", tol=1e-13, restart=16, max_batch=2, graphs=graphs,
                     sstep=sstep)
    r = plan.solve(Q, k)
    assert r["status"] == dbar.DBAR_OK
    assert np.all(r["resid"] < 1e-13)
    for i in range(k.size):
        ref = orc.solve_cgo_conv(Q, k[i], N, L, tol=1e-14)
        assert rel(r["S"][i], ref["S"]) < 1e-11, i
        assert np.max(np.abs(r["m"][i] - ref["m"])) < 1e-11, i


def test_conv_and_taylor_routes_agree_on_the_gpu(dbar):
    # the paper's use of the convolution code: an independent test of the Taylor-Gaussian one
    N, L = 64, 4.0
    Q = _potential(N, L)
    k = np.array([0.4 - 0.2j, 1.0 + 1.0j, -2.0 + 0.5j, 3.0j])
    conv = dbar.Plan(N, L, prec="fp64", regularisation="conv", tol=1e-13, max_batch=4).solve(Q, k)
    tay = dbar.Plan(N, L, M=11, prec="fp64", tol=1e-13, max_batch=4).solve(Q, k)
    assert conv["status"] == dbar.DBAR_OK and tay["status"] == dbar.DBAR_OK
    for i in range(k.size):
        assert rel(conv["S"][i], tay["S"][i]) < 1e-11, i
        assert np.max(np.abs(conv["m"][i] - tay["m"][i])) < 1e-11, i


def test_conv_reflection_coefficient(dbar):
    # r(k) by the two-solve route (Sec. 6.1) with the convolution regularisation
    N, L = 64, 4.0
    Q = _potential(N, L)
    k = np.array([0.5 + 0.5j, -1.0 + 2.0j])
    plan = dbar.Plan(N, L, prec="fp64", regularisation="conv", tol=1e-13, max_batch=2)
    r, iters, resid, status = dbar.dbar_reflection(plan.handle, Q, k)
    assert status == dbar.DBAR_OK
    ref = np.array([orc.reflection(Q, kk, N, L, M=11, tol=1e-14)["r"] for kk in k])
    assert np.max(np.abs(r - ref)) < 1e-11 * np.max(np.abs(ref))


def test_conv_full_size_sampled_against_the_direct_definition(dbar):
    # N = 256 (the largest size of the route), one batch of the solve's launch shape:
    # h at sampled points by the oracle's definition, point by point
    torch = pytest.importorskip("torch")
    N, L, nk = 256, 6.0, 4
    S = _fields(N, L, nk, 23)
    plan = dbar.Plan(N, L, prec="fp64", regularisation="conv", max_batch=nk)
    Sd = torch.from_numpy(S).cuda()
    m = torch.empty_like(Sd)
    dbar.dbar_m_from_S(plan.handle, nk, Sd, m)
    m = m.cpu().numpy()
    g = orc.Grid(N, L)
    K = orc.conv_kernel_table(g)
    hs = 2 * np.pi * L / N
    rng = np.random.default_rng(1)
    for i in range(nk):
        s = g.Finv(S[i])
        r2 = (g.xi * np.conj(g.xi)).real
        xi = g.xi.copy()
        xi[0, 0] = 1.0
        mult = -np.expm1(-r2) / xi
        mult[0, 0] = 0.0
        u = g.Finv(S[i] * mult)
        for _ in range(6):
            y, x = rng.integers(0, N, 2)
            direct = np.sum(s * K[y:y + N, x:x + N][::-1, ::-1]) * hs * hs / (2 * np.pi)
            ref = u[y, x] + direct
            assert abs(m[i, y, x] - ref) < 1e-13 * np.max(np.abs(u)) + 1e-14, (i, y, x)


def test_conv_plan_rejects_taylor_and_fp32_calls(dbar):
    torch = pytest.importorskip("torch")
    N, L = 32, 2.0
    plan = dbar.Plan(N, L, prec="fp64", regularisation="conv", max_batch=1)
    S = torch.zeros((1, N, N), dtype=torch.complex128, device="cuda")
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_taylor(plan.handle, 1, S, 2)
    assert e.value.status == dbar.DBAR_EINVAL
    S32 = torch.zeros((1, N, N), dtype=torch.complex64, device="cuda")
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_apply(plan.handle, torch.zeros((N, N), dtype=torch.complex128, device="cuda"), [0.1], S32,
                        torch.empty_like(S32), fp32=True)
    assert e.value.status == dbar.DBAR_EINVAL
    r = plan.solve(np.zeros((N, N), np.complex128), np.zeros(0))
    assert r["S"].shape == (0, N, N)
