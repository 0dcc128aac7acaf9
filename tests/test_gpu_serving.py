"""Continuous-batching server: results alone vs in a mix, memory budget,
host-side fault injection, input validation."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def dbar():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_02363_gb300 import dbar as d
    return d


PARAMS = dict(prec="mixed", restart=24, tol=1e-12)


def solo(dbar, N, L, Q, k, want_m=True):
    plan = dbar.Plan(N, L, max_batch=1, **PARAMS)
    return plan.solve(Q, [k], want_m=want_m)


def test_each_result_is_the_same_alone_and_in_the_mix(dbar):
    # two grid classes, different potentials and k, all submitted at once
    srv = dbar.Server(6 << 30, **PARAMS)
    reqs = []
    for i, N in enumerate([64, 128, 64, 128, 64, 64, 128]):
        Q, k = wl.mixture_request(100 + i, N, 4.0, kmax=2.0)
        reqs.append((N, Q, k, srv.submit(N, 4.0, Q, k, want_m=(i % 2 == 0))))
    for i, (N, Q, k, t) in enumerate(reqs):
        r = srv.wait(t, timeout_s=120)
        assert r["status"] == dbar.DBAR_OK and r["resid"] <= 1e-12
        ref = solo(dbar, N, 4.0, Q, k)
        assert rel(r["S"], ref["S"][0]) <= 1e-12, i
        if i % 2 == 0:
            assert rel(r["m"], ref["m"][0]) <= 1e-12, i
        else:
            assert r["m"] is None
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["pending"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_requests_join_while_others_run(dbar):
    srv = dbar.Server(6 << 30, **PARAMS)
    first = [srv.submit(128, 4.0, *wl.mixture_request(200 + i, 128, 4.0, 2.0)) for i in range(3)]
    late = []
    for i in range(3):
        Q, k = wl.mixture_request(300 + i, 128, 4.0, 2.0)
        late.append((Q, k, srv.submit(128, 4.0, Q, k)))
    for t in first:
        assert srv.wait(t, timeout_s=120)["status"] == dbar.DBAR_OK
    for Q, k, t in late:
        r = srv.wait(t, timeout_s=120)
        assert r["status"] == dbar.DBAR_OK
        assert rel(r["S"], solo(dbar, 128, 4.0, Q, k, want_m=False)["S"][0]) <= 1e-12
    srv.close()


def test_budget_of_one_slot_still_serves_everything(dbar):
    # 2.5 MiB: the 64^2 tables (~0.8 MiB) and one 64^2 slot (~1.3 MiB) fit, a second slot
    # does not, and a 128^2 request cannot fit at all
    srv = dbar.Server(int(2.5 * (1 << 20)), **PARAMS)
    with pytest.raises(dbar.DbarError) as e:
        srv.submit(128, 4.0, np.ones((128, 128)), 0.3)
    assert e.value.status == dbar.DBAR_ENOMEM
    reqs = []
    for i in range(3):
        Q, k = wl.mixture_request(400 + i, 64, 4.0, 2.0)
        reqs.append((Q, k, srv.submit(64, 4.0, Q, k)))
    for Q, k, t in reqs:
        r = srv.wait(t, timeout_s=120)
        assert r["status"] == dbar.DBAR_OK
        assert rel(r["S"], solo(dbar, 64, 4.0, Q, k, want_m=False)["S"][0]) <= 1e-12
    srv.close()


def test_injected_lane_failure_requeues_and_recovers(dbar):
    srv = dbar.Server(6 << 30, **PARAMS)
    reqs = []
    for i in range(4):
        Q, k = wl.mixture_request(500 + i, 64, 4.0, 2.0)
        reqs.append((Q, k, srv.submit(64, 4.0, Q, k)))
    srv.inject_fault()
    for Q, k, t in reqs:
        r = srv.wait(t, timeout_s=120)
        assert r["status"] == dbar.DBAR_OK
        assert rel(r["S"], solo(dbar, 64, 4.0, Q, k, want_m=False)["S"][0]) <= 1e-12
    srv.close()


def test_invalid_requests_are_rejected_at_submit(dbar):
    srv = dbar.Server(1 << 30, **PARAMS)
    Q = np.ones((64, 64), complex)
    Q[1, 2] = np.inf
    for args in [(64, 4.0, Q, 0.1), (48, 4.0, np.ones((48, 48)), 0.1), (64, -1.0, np.ones((64, 64)), 0.1),
                 (64, 4.0, np.ones((64, 64)), complex(np.nan, 0))]:
        with pytest.raises(dbar.DbarError) as e:
            srv.submit(*args)
        assert e.value.status == dbar.DBAR_EINVAL
    srv.close()


def _oracle_S(args):
    N, L, Q, k = args
    from oracle import dbar_oracle as orc
    return orc.solve_cgo(Q, k, N, L, M=2, tol=1e-13, restart=40)["S"]


def test_served_results_match_the_oracle_at_the_serving_k_range(dbar):
    # The serving workload's grid classes and k range (L = 6, N raised until
    # N/(2L) >= 2 max(|k1|, |k2|) + 20): N = 256 at small |k|, N = 512 up to
    # max(|k1|, |k2|) = 11, N = 1024 at |k| = 20; each request its own Gaussian mixture
    # of 1-6 terms, all submitted together so that they share lanes.  Every served S
    # is compared with the FP64 CPU oracle (mixed-precision bar 1e-10).
    import concurrent.futures as cf
    import multiprocessing as mp
    L = 6.0
    cases = [(256, 0.12 + 0.05j), (256, -0.3 + 0.5j), (512, 3.7 + 2.1j), (512, -8.5 + 6.0j),
             (512, 11.0 - 10.8j), (1024, 20.0 + 0.0j)]
    reqs = []
    srv = dbar.Server(16 << 30, prec="mixed", restart=32, tol=1e-12)
    for i, (N, k) in enumerate(cases):
        rng = np.random.default_rng(900 + i)
        Q = wl.gaussian_mixture(N, L, *wl.draw_mixture(rng, int(rng.integers(1, 7))))
        reqs.append((N, Q, k, srv.submit(N, L, Q, k)))
    with cf.ProcessPoolExecutor(max_workers=len(cases), mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_oracle_S, (N, L, Q, k)) for N, Q, k, _ in reqs]
        served = [srv.wait(t, timeout_s=300) for *_, t in reqs]
        oracle = [f.result() for f in futs]
    srv.close()
    for i, (r, So) in enumerate(zip(served, oracle)):
        assert r["status"] == dbar.DBAR_OK and r["resid"] <= 1e-12, i
        assert rel(r["S"], So) <= 1e-10, (i, cases[i], rel(r["S"], So))
