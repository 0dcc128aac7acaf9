"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is element by element on the same seeded inputs; the bar is
the relative L-infinity error max|X - X_oracle| / max|X_oracle| stated in each
test: 1e-12 for FP64 results, 1e-10 for mixed-precision results (FP32 inner
Krylov with FP64 refinement).
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


def dev(torch, a, fp32=False):
    a = np.ascontiguousarray(a)
    t = torch.from_numpy(a.astype(np.complex64 if fp32 else np.complex128)).cuda()
    return t


def rand_smooth_fourier(rng, nk, N, L):
    """Fourier fields of smooth decaying functions (random Gaussian mixtures)."""
    g = orc.Grid(N, L)
    out = np.zeros((nk, N, N), complex)
    for i in range(nk):
        c = rng.uniform(-1.5, 1.5, 2)
        w = rng.uniform(0.6, 1.4)
        amp = rng.standard_normal() + 1j * rng.standard_normal()
        out[i] = g.F(amp * np.exp(-((g.X - c[0]) ** 2 + (g.Y - c[1]) ** 2) / w ** 2) * (1 + 0.3j * g.X))
    return out


@pytest.mark.parametrize("N", [32, 64, 256, 2048])
@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft2_matches_oracle_fft(dbar, torch_cuda, N, fp32, sign):
    # 32 and 2048: the smallest and largest grids a plan accepts
    torch = torch_cuda
    rng = np.random.default_rng(N)
    nk = 3 if N < 2048 else 1   # the oracle's own FFT takes seconds per 2048^2 field
    x = rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N))
    plan = dbar.Plan(N, 4.0, prec="mixed", max_batch=4, restart=4)
    xd = dev(torch, x, fp32)
    yd = torch.empty_like(xd)
    dbar.dbar_fft2(plan.handle, nk, xd, yd, sign, fp32)
    torch.cuda.synchronize()
    ref = orc.dft2(x, sign)
    err = rel(yd.cpu().numpy(), ref)
    assert err < (3e-6 if fp32 else 2e-15 * np.log2(N) * 4), err


@pytest.mark.parametrize("fp32", [False, True])
def test_taylor_coefficients_match_oracle(dbar, torch_cuda, fp32):
    torch = torch_cuda
    N, L, M = 128, 4.0, 5
    rng = np.random.default_rng(5)
    S = rand_smooth_fourier(rng, 3, N, L)
    plan = dbar.Plan(N, L, M=M, prec="mixed", max_batch=4, restart=4)
    got = dbar.dbar_taylor(plan.handle, 3, dev(torch, S, fp32), M, fp32)
    g = orc.Grid(N, L)
    for i in range(3):
        c, d = orc.taylor_coeffs(S[i], g, M)
        ref = np.array(list(c) + [d])
        err = np.max(np.abs(got[i] - ref)) / np.max(np.abs(ref))
        assert err < (2e-5 if fp32 else 1e-12), (i, err, got[i], ref)


@pytest.mark.parametrize("zero_fill", [0, 1])
def test_m_from_S_matches_oracle(dbar, torch_cuda, zero_fill):
    torch = torch_cuda
    N, L, M = 128, 5.0, 3
    rng = np.random.default_rng(6)
    S = rand_smooth_fourier(rng, 2, N, L)
    plan = dbar.Plan(N, L, M=M, prec="fp64", max_batch=2, restart=4, zero_fill=zero_fill)
    Sd = dev(torch, S)
    md = torch.empty_like(Sd)
    dbar.dbar_m_from_S(plan.handle, 2, Sd, md)
    g = orc.Grid(N, L)
    for i in range(2):
        ref = orc.h_of_S(S[i], g, M, fill="zero" if zero_fill else "analytic")
        assert rel(md[i].cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rhs_matches_oracle(dbar, torch_cuda, prec):
    # mixed: computed and held in double-float, converted to FP64 at read-out
    torch = torch_cuda
    w = wl.mixed_1024(N=256, nk=3, L=10.0)
    plan = dbar.Plan(w.N, w.L, prec=prec, max_batch=4, restart=4)
    Qd = dev(torch, w.Q)
    bd = torch.empty((3, w.N, w.N), dtype=torch.complex128, device="cuda")
    dbar.dbar_rhs(plan.handle, Qd, w.k, bd)
    for i in range(3):
        ref = orc.CGOProblem(w.Q, w.k[i], w.N, w.L).rhs()
        assert rel(bd[i].cpu().numpy(), ref) < (1e-13 if prec == "fp64" else 5e-13)


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("N", [64, 128, 1024, 2048])
def test_operator_application_matches_oracle(dbar, torch_cuda, fp32, N):
    # 1024 and 2048: the grids of the benchmark and of the serving workload's largest class
    torch = torch_cuda
    L = 6.0
    rng = np.random.default_rng(N + fp32)
    w = wl.mixed_1024(N=N, nk=3, L=L)
    S = rand_smooth_fourier(rng, 3, N, L)
    plan = dbar.Plan(N, L, M=2, prec="mixed", max_batch=4, restart=4)
    Sd = dev(torch, S, fp32)
    ASd = torch.empty_like(Sd)
    dbar.dbar_apply(plan.handle, dev(torch, w.Q), w.k, Sd, ASd, fp32)
    for i in range(3 if N < 1024 else 1):   # one oracle operator at the largest grids
        P = orc.CGOProblem(w.Q, w.k[i], N, L, M=2)
        ref = P.apply(S[i].astype(np.complex64).astype(complex) if fp32 else S[i])
        assert rel(ASd[i].cpu().numpy(), ref) < (2e-5 if fp32 else 1e-13)


def _oracle(w, i, M=None, tol=1e-14):
    return orc.solve_cgo(w.Q, w.k[i], w.N, w.L, M=w.M if M is None else M, tol=tol, restart=60)


def test_plain_fp64_workload_matches_oracle(dbar):
    w = wl.plain_fp64()
    plan = dbar.Plan(w.N, w.L, M=w.M, prec="fp64", restart=32, tol=1e-13)
    r = plan.solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK and r["resid"][0] <= 1e-13
    o = _oracle(w, 0)
    assert rel(r["S"][0], o["S"]) < 1e-12
    assert rel(r["m"][0], o["m"]) < 1e-12


@pytest.mark.parametrize("resid_mode", ["double_float", "fp64"])
def test_mixed_precision_small_grid_matches_oracle(dbar, resid_mode):
    # FP32 inner GMRES; right-hand side and true residual in double-float or native FP64
    w = wl.mixed_1024(N=128, nk=4, L=5.0)
    plan = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=24, tol=1e-12, max_batch=4, resid_mode=resid_mode)
    r = plan.solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK
    for i in range(w.k.size):
        o = _oracle(w, i)
        assert rel(r["S"][i], o["S"]) < 1e-10, i
        assert rel(r["m"][i], o["m"]) < 1e-10, i
        assert r["iters"][i, 1] >= 2          # at least one refinement step after the first cycle


def test_batches_with_a_ragged_tail_match_single_solves(dbar):
    # 7 k values through a plan holding 3 slots: batches of 3, 3 and 1.
    w = wl.batched_fp64(N=64, nk_side=3)
    k = w.k[:7]
    plan = dbar.Plan(w.N, w.L, M=2, prec="fp64", restart=32, tol=1e-13, max_batch=3)
    r = plan.solve(w.Q, k)
    alone = dbar.Plan(w.N, w.L, M=2, prec="fp64", restart=32, tol=1e-13, max_batch=1)
    for i in range(k.size):
        ri = alone.solve(w.Q, k[i:i + 1])
        assert rel(r["S"][i], ri["S"][0]) < 1e-13
        o = orc.solve_cgo(w.Q, k[i], w.N, w.L, M=2, tol=1e-14)
        assert rel(r["S"][i], o["S"]) < 1e-12


def test_zero_potential_and_empty_batch(dbar):
    N, L = 64, 4.0
    plan = dbar.Plan(N, L, prec="mixed", max_batch=2)
    r = plan.solve(np.zeros((N, N)), [0.3 + 0.1j, -1.0j])
    assert r["status"] == dbar.DBAR_OK
    assert np.all(r["S"] == 0) and np.all(r["m"] == 0) and np.all(r["iters"] == 0)
    r0 = plan.solve(np.zeros((N, N)), np.zeros(0, complex))
    assert r0["S"].shape == (0, N, N)


def test_invalid_inputs_are_rejected(dbar):
    N, L = 64, 4.0
    plan = dbar.Plan(N, L, max_batch=1)
    Q = np.ones((N, N), complex)
    Q[3, 4] = np.nan
    with pytest.raises(dbar.DbarError) as e:
        plan.solve(Q, [0.1])
    assert e.value.status == dbar.DBAR_EINVAL
    with pytest.raises(dbar.DbarError) as e:
        plan.solve(np.ones((N, N)), [complex(np.inf, 0)])
    assert e.value.status == dbar.DBAR_EINVAL


def test_page_locked_host_output_matches_device_and_pageable_outputs(dbar, torch_cuda):
    # A page-locked host S_out of a mixed plan is written by the conversion kernel
    # itself; pageable host memory goes through a copy, device memory is written
    # in place: all three give the same bits.  With m_out requested the
    # page-locked S_out takes the copy route.
    torch = torch_cuda
    w = wl.mixed_1024(N=128, nk=3, L=5.0)
    plan = dbar.Plan(w.N, w.L, M=2, prec="mixed", tol=1e-12, max_batch=2)  # two batches: 2 + 1 k
    shape = (w.k.size, w.N, w.N)
    Sd = torch.empty(shape, dtype=torch.complex128, device="cuda")
    assert plan.solve_device(dev(torch, w.Q), w.k, Sd)["status"] == dbar.DBAR_OK
    Sp = torch.full(shape, np.nan, dtype=torch.complex128).pin_memory()
    Qp = torch.from_numpy(np.ascontiguousarray(w.Q, dtype=np.complex128)).pin_memory()
    st = dbar.dbar_solve_cgo(plan.handle, Qp.numpy(), w.k, Sp.numpy(), io_on_device=False)
    assert st == dbar.DBAR_OK
    r = plan.solve(w.Q, w.k)
    assert np.array_equal(Sp.numpy(), Sd.cpu().numpy())
    assert np.array_equal(r["S"], Sd.cpu().numpy())
    Sp2 = torch.full(shape, np.nan, dtype=torch.complex128).pin_memory()
    mp = np.zeros(shape, np.complex128)
    st = dbar.dbar_solve_cgo(plan.handle, w.Q, w.k, Sp2.numpy(), mp, io_on_device=False)
    assert st == dbar.DBAR_OK
    assert np.array_equal(Sp2.numpy(), Sd.cpu().numpy()) and np.array_equal(mp, r["m"])


def test_iteration_cap_reports_no_convergence(dbar):
    w = wl.plain_fp64()
    plan = dbar.Plan(w.N, w.L, prec="fp64", restart=4, max_iter=4, max_outer=1, tol=1e-13)
    r = plan.solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_ENOCONV
    assert r["resid"][0] > 1e-13 and r["iters"][0, 0] == 4


def test_mixed_solve_at_the_largest_grid_matches_the_fp64_solve(dbar):
    # N = 2048: the double-float residual's one-launch column pass with a radix-8 last
    # stage, the FP32 passes at their largest size.  The CPU oracle needs minutes per solve
    # here; the FP64 GPU path it pins at the smaller grids stands in (mixed bar 1e-10).
    w = wl.mixed_1024(N=2048, nk=2, L=12.0)
    r = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=32, tol=1e-12, max_batch=2).solve(w.Q, w.k, want_m=False)
    ref = dbar.Plan(w.N, w.L, M=2, prec="fp64", restart=32, tol=1e-13, max_batch=2).solve(w.Q, w.k, want_m=False)
    assert r["status"] == dbar.DBAR_OK and np.all(r["resid"] <= 1e-12)
    for i in range(w.k.size):
        assert rel(r["S"][i], ref["S"][i]) < 1e-10, i


@pytest.mark.slow
def test_full_size_mixed_workload_sampled_k_match_oracle(dbar, torch_cuda):
    # The 1024^2, 128-k mixed-precision workload in the launch configuration the
    # benchmark times; the oracle solves two sampled k values (smallest and largest |k|).
    torch = torch_cuda
    w = wl.mixed_1024()
    plan = dbar.Plan(w.N, w.L, M=2, prec="mixed", tol=1e-12)
    S = torch.empty((w.k.size, w.N, w.N), dtype=torch.complex128, device="cuda")
    r = plan.solve_device(dev(torch, w.Q), w.k, S)
    assert r["status"] == dbar.DBAR_OK and np.all(r["resid"] <= 1e-12)
    for i in (int(np.argmin(abs(w.k))), int(np.argmax(abs(w.k)))):
        o = _oracle(w, i, tol=1e-13)
        assert rel(S[i].cpu().numpy(), o["S"]) < 1e-10, i


@pytest.mark.parametrize("sstep", [2, 4])
def test_sstep_blocks_match_oracle(dbar, sstep):
    # s-step Arnoldi (chain of K = A - I per block, block Gram-Schmidt + Cholesky
    # QR): the same Krylov spaces as one vector per sweep, so the same solution and
    # about the same inner iterations (rounded up to whole blocks per cycle)
    w = wl.mixed_1024(N=128, nk=4, L=5.0)
    kw = dict(M=2, prec="mixed", restart=24, tol=1e-12, max_batch=4)
    r = dbar.Plan(w.N, w.L, sstep=sstep, **kw).solve(w.Q, w.k)
    ref = dbar.Plan(w.N, w.L, sstep=1, **kw).solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK and np.all(r["resid"] <= 1e-12)
    for i in range(w.k.size):
        o = _oracle(w, i)
        assert rel(r["S"][i], o["S"]) < 1e-10, i
        assert rel(r["m"][i], o["m"]) < 1e-10, i
    assert np.all(r["iters"][:, 0] <= ref["iters"][:, 0] + 2 * sstep * ref["iters"][:, 1])


@pytest.mark.parametrize("N,L,M", [(32, 3.0, 2), (64, 4.0, 2), (64, 4.0, 5), (256, 6.0, 2)])
def test_chain_moments_at_every_row_width_match_the_oracle(dbar, N, L, M):
    # The fused chain row pass forms the next vector's Taylor row moments from the
    # column-pass output (warp segments of N/16 threads below N = 512, several warps
    # above); wrong moments would leave the FP32 chain on another operator and cost inner
    # iterations.  The s-step solve matches the oracle and needs no more inner
    # iterations than one vector per sweep, up to the rounding to whole blocks.
    w = wl.mixed_1024(N=N, nk=2, L=L)
    kw = dict(M=M, prec="mixed", restart=24, tol=1e-12, max_batch=2)
    r = dbar.Plan(w.N, w.L, sstep=4, **kw).solve(w.Q, w.k)
    ref = dbar.Plan(w.N, w.L, sstep=1, **kw).solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK and np.all(r["resid"] <= 1e-12)
    for i in range(w.k.size):
        o = orc.solve_cgo(w.Q, w.k[i], w.N, w.L, M=M, tol=1e-14, restart=60)
        assert rel(r["S"][i], o["S"]) < 1e-10, i
    assert np.all(r["iters"][:, 0] <= ref["iters"][:, 0] + 2 * 4 * ref["iters"][:, 1])


def test_sstep_fp64_ragged_batches_match_single_solves_and_oracle(dbar):
    # FP64 s-step cycles; 7 k values through 3 slots (batches 3, 3, 1) and alone
    w = wl.batched_fp64(N=64, nk_side=3)
    k = w.k[:7]
    kw = dict(M=2, prec="fp64", restart=32, tol=1e-13, sstep=4)
    r = dbar.Plan(w.N, w.L, max_batch=3, **kw).solve(w.Q, k)
    assert r["status"] == dbar.DBAR_OK
    alone = dbar.Plan(w.N, w.L, max_batch=1, **kw)
    for i in range(k.size):
        ri = alone.solve(w.Q, k[i:i + 1])
        assert np.array_equal(r["S"][i], ri["S"][0]), i     # slots never mix
        o = orc.solve_cgo(w.Q, k[i], w.N, w.L, M=2, tol=1e-14)
        assert rel(r["S"][i], o["S"]) < 1e-12, i


@pytest.mark.parametrize("sstep", [1, 4])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_replayed_cycles_match_direct_launches(dbar, prec, sstep):
    # a Krylov cycle captured once as a CUDA graph and replayed gives the same bits
    w = wl.batched_fp64(N=64, nk_side=3)
    res = []
    for graphs in (1, 0):
        plan = dbar.Plan(w.N, w.L, M=2, prec=prec, restart=16, tol=1e-12, max_batch=5, graphs=graphs,
                         sstep=sstep)
        res.append(plan.solve(w.Q, w.k[:7]))     # batches of 5 and a ragged 2
    assert np.array_equal(res[0]["S"], res[1]["S"]) and np.array_equal(res[0]["iters"], res[1]["iters"])
    assert res[0]["status"] == dbar.DBAR_OK


def test_autotuned_column_tiles_give_identical_results(dbar):
    # every compiled tile shape of the FP32 column pass computes the same numbers
    # (an odd batch: the two-slot variant's last block holds one k)
    w = wl.mixed_1024(N=256, nk=3, L=6.0)
    res = []
    for autotune, variant in ((0, 0), (2, 1), (3, 2), (1, None)):
        plan = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=24, tol=1e-12, max_batch=3, autotune=autotune)
        res.append(plan.solve(w.Q, w.k, want_m=False))
        v, ms = dbar.dbar_plan_tuning(plan.handle)
        if variant is not None:
            assert v == variant
        else:
            assert v in (0, 1, 2) and len(ms) == dbar.COLUMN_VARIANTS and min(ms) > 0
    for r in res[1:]:
        assert np.array_equal(res[0]["S"], r["S"])
    assert res[0]["status"] == dbar.DBAR_OK


@pytest.mark.parametrize("N,nk,L", [(256, 3, 6.0), (1024, 2, 10.0)])
def test_row_pass_shapes_give_identical_results(dbar, N, nk, L):
    # every row-pass shape of the FP32 operator computes the same numbers; the autotuner
    # times them all and records its choice
    w = wl.mixed_1024(N=N, nk=nk, L=L)
    res = []
    for shape, plain in ((1, 0), (2, 0), (3, 0), (4, 0), (5, 0), (5, 2), (0, 0)):
        plan = dbar.Plan(w.N, w.L, M=2, prec="mixed", restart=24, tol=1e-12, max_batch=nk, row_shape=shape,
                         row_shape_plain=plain)
        res.append(plan.solve(w.Q, w.k, want_m=False))
        for passes in ("fused", "plain"):  # the fused chain pass and the row passes A / C
            rv, ms = dbar.dbar_plan_row_tuning(plan.handle, passes)
            pinned = plain if (passes == "plain" and plain) else shape
            if pinned:
                assert rv == pinned - 1
            else:
                assert rv in range(dbar.ROW_VARIANTS) and len(ms) == dbar.ROW_VARIANTS and min(ms) > 0
    for r in res[1:]:
        assert np.array_equal(res[0]["S"], r["S"]) and np.array_equal(res[0]["iters"], r["iters"])
    assert res[0]["status"] == dbar.DBAR_OK
