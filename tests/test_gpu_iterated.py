"""The iterated integral equation of Sec. 5 (eq. eqh2, shifted regularisation)
through the C ABI against the CPU oracle's literal implementation."""
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


def _mixture(N, L):
    X, Y = wl.mesh(N, L)
    return (1.3 * np.exp(-(X * X + Y * Y)) + (0.4 + 0.6j) * np.exp(-((X - 0.5) ** 2 + (Y + 0.3) ** 2) / 0.7)
            ).astype(np.complex128)


@pytest.mark.parametrize("fp32", [False, True])
def test_iterated_operator_matches_oracle(dbar, fp32):
    # 2k on the xi-grid; the last two put xi0 = 2i conj(k) at the edge of the box (xi_max = 32/L),
    # one on the Nyquist wavenumber -N/2 (held as +N/2), where the quotient by xi - xi0 must not
    # wrap periodically (eq. dbarinvShift)
    torch = pytest.importorskip("torch")
    N, L = 64, 3.0
    Q = _mixture(N, L)
    k = np.array([(2 + 1j) / (2 * L), (-3 + 5j) / (2 * L), (31 + 30j) / (2 * L), (-32 - 29j) / (2 * L)])
    plan = dbar.Plan(N, L, M=2, prec="mixed" if fp32 else "fp64", iterated=1, max_batch=k.size)
    rng = np.random.default_rng(3)
    g = orc.Grid(N, L)
    h = np.stack([g.F(np.exp(-((g.X - 0.3) ** 2 + g.Y ** 2)) * (1 + 0.5j * rng.standard_normal()))
                  for _ in range(k.size)])
    Qd = torch.from_numpy(Q).cuda()
    hd = torch.from_numpy(h.astype(np.complex64) if fp32 else h).cuda()
    out = torch.empty_like(hd)
    dbar.dbar_apply(plan.handle, Qd, k, hd, out, fp32=fp32)
    for i in range(k.size):
        ref = orc.IteratedProblem(Q, k[i], N, L).apply(h[i])
        assert rel(out[i].cpu().numpy(), ref) < (2e-6 if fp32 else 1e-13), i


@pytest.mark.parametrize("sstep", [1, 4])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-10)])
def test_iterated_solve_matches_oracle(dbar, prec, tol, sstep):
    # one vector per sweep, and s-step blocks chaining whole applications of the operator
    N, L = 64, 3.2
    Q = _mixture(N, L)
    k = np.array([0.0, (4 + 2j) / (2 * L), (-6 - 10j) / (2 * L), (12 + 0j) / (2 * L)])
    plan = dbar.Plan(N, L, M=2, prec=prec, iterated=1, tol=1e-13 if prec == "fp64" else 1e-12, max_batch=4,
                     sstep=sstep)
    r = plan.solve(Q, k, want_m=False)
    assert r["status"] == dbar.DBAR_OK
    for i in range(k.size):
        ref = orc.solve_iterated(Q, k[i], N, L, tol=1e-14)["h"]
        assert rel(r["S"][i], ref) < tol, i


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_reflection_through_the_iterated_equation(dbar, prec):
    # one solve per k; agrees with the two-solve route and the oracle, also at |k| where the
    # two-solve route no longer resolves E_{k/2} q
    N, L = 64, 3.2
    Q = _mixture(N, L)
    k = np.array([0.0, (3 - 2j) / L, (-8 + 6j) / L, (12 + 12j) / L])
    it = dbar.Plan(N, L, M=2, prec=prec, iterated=1, tol=1e-13 if prec == "fp64" else 1e-12, max_batch=4)
    r, iters, resid, status = dbar.dbar_reflection(it.handle, Q, k)
    assert status == dbar.DBAR_OK
    ref = np.array([orc.reflection_iterated(Q, kk, N, L, tol=1e-14)["r"] for kk in k])
    assert np.max(np.abs(r - ref)) < (1e-12 if prec == "fp64" else 1e-10) * np.max(np.abs(ref))
    direct = dbar.Plan(N, L, M=2, prec="fp64", tol=1e-13, max_batch=4)
    r2 = dbar.dbar_reflection(direct.handle, Q, k[:2])[0]
    assert np.max(np.abs(r[:2] - r2)) < 1e-10 * np.max(np.abs(ref))


def test_iterated_plan_rejects_k_off_the_grid_and_m_output(dbar):
    N, L = 32, 2.5
    Q = _mixture(N, L)
    plan = dbar.Plan(N, L, prec="fp64", iterated=1, max_batch=2)
    with pytest.raises(dbar.DbarError) as e:
        plan.solve(Q, [0.1234 + 0.0j], want_m=False)
    assert e.value.status == dbar.DBAR_EINVAL
    with pytest.raises(dbar.DbarError) as e:
        plan.solve(Q, [0.0], want_m=True)
    assert e.value.status == dbar.DBAR_EINVAL
    with pytest.raises(dbar.DbarError) as e:   # 2 k L = 20 beyond the grid's wavenumbers (N/2 = 16)
        plan.solve(Q, [4.0 + 0.0j], want_m=False)
    assert e.value.status == dbar.DBAR_EINVAL


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 1e-11)])
def test_iterated_solve_at_the_papers_large_k(dbar, prec, tol):
    # Sec. 5: k = 8.5936 ~ 55/6.4 at L = 3.2 (2kL = 55, xi0 at 86 % of the box edge at N = 128):
    # the GPU's h at N = 128 equals the oracle's, and refining to N = 256 leaves it unchanged
    L, k = 3.2, 55 / 6.4
    pts = [(0, 0), (3, -2), (-5, 7), (10, 0)]
    vals = {}
    for N in (128, 256):
        X, Y = wl.mesh(N, L)
        q = np.exp(-(X * X + Y * Y)).astype(np.complex128)
        plan = dbar.Plan(N, L, M=11, prec=prec, iterated=1, restart=16,
                         tol=1e-14 if prec == "fp64" else 1e-12, max_batch=1)
        r = plan.solve(q, [k], want_m=False)
        assert r["status"] == dbar.DBAR_OK
        h = r["S"][0]
        vals[N] = np.array([h[m2 % N, m1 % N] for m1, m2 in pts])
        if N == 128:
            ref = orc.solve_iterated(q, k, N, L, M=11, tol=1e-14)["h"]
            assert rel(h, ref) < tol
    assert np.max(np.abs(vals[128] - vals[256])) < tol


def test_lower_inner_taylor_order_gives_the_same_solution(dbar):
    # params.inner_M: FP32 correction solves at M = 2 under an M = 11 right-hand side and residual
    N, L = 64, 3.2
    Q = _mixture(N, L)
    k = np.array([0.0, (4 + 2j) / (2 * L), (-6 - 10j) / (2 * L)])
    full = dbar.Plan(N, L, M=11, prec="mixed", iterated=1, tol=1e-12, max_batch=3).solve(Q, k, want_m=False)
    low = dbar.Plan(N, L, M=11, prec="mixed", iterated=1, tol=1e-12, max_batch=3, inner_M=2).solve(Q, k,
                                                                                                   want_m=False)
    assert full["status"] == dbar.DBAR_OK and low["status"] == dbar.DBAR_OK
    for i in range(k.size):
        ref = orc.solve_iterated(Q, k[i], N, L, M=11, tol=1e-14)["h"]
        assert rel(low["S"][i], ref) < 1e-10, i
        assert rel(full["S"][i], ref) < 1e-10, i
    assert np.all(low["iters"][:, 1] <= full["iters"][:, 1] + 1)
