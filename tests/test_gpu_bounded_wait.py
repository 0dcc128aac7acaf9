"""Device-side failure detection: the bounded mbarrier wait.

The bulk-copy block update waits on mbarriers with an iteration limit; when a
wait runs out the kernel sets an error flag, drains its own copies and returns,
and the solve reports DBAR_ETIMEOUT.  Here one CTA runs the same kind of wait
on a phase that nothing completes (a flag that nothing sets): the call must
come back with DBAR_ETIMEOUT, quickly, and the context must stay usable.  No
fault, trap or endless loop is involved.
"""
import time

import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbar():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_02363_gb300 import dbar as d
    return d


LIMIT = 1 << 18  # the sweeps' own limit of try_wait rounds


def test_completed_phase_returns_ok(dbar):
    sec = dbar.dbar_check_bounded_wait(True, LIMIT)
    assert 0.0 <= sec < 1.0


def test_wait_that_nothing_completes_times_out_and_context_survives(dbar):
    rounds = 1 << 12
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_check_bounded_wait(False, rounds)
    assert e.value.status == dbar.DBAR_ETIMEOUT
    assert "ran out after 4096 rounds" in str(e.value)
    # the wait is bounded in time: the run-out, timed on the host around the call
    # (host overheads included), scaled to the sweeps' limit stays within a few seconds
    t0 = time.perf_counter()
    with pytest.raises(dbar.DbarError):
        dbar.dbar_check_bounded_wait(False, 1 << 14)
    per_round = (time.perf_counter() - t0) / (1 << 14)
    assert per_round * LIMIT < 5.0, per_round
    # the context is still usable: a completed wait and a small solve afterwards
    assert dbar.dbar_check_bounded_wait(True, LIMIT) < 1.0
    w = wl.plain_fp64()
    r = dbar.Plan(w.N, w.L, prec="fp64", tol=1e-12).solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK and r["resid"][0] <= 1e-12


def test_rounds_are_validated(dbar):
    for bad in (0, -1, LIMIT + 1):
        with pytest.raises(dbar.DbarError) as e:
            dbar.dbar_check_bounded_wait(True, bad)
        assert e.value.status == dbar.DBAR_EINVAL


@pytest.mark.parametrize("prec,graphs", [("fp64", 1), ("mixed", 0)])
def test_block_update_wait_runs_out_inside_a_solve(dbar, prec, graphs):
    # The solve-level path: one block-update launch announces 16 bytes more on its first
    # bulk-copy stage than the copy delivers (a phase nothing completes); its waits run
    # out, the block reports through the plan's error flag and drains its copies, and
    # dbar_solve_cgo returns DBAR_ETIMEOUT.  The next solve on the same plan is correct.
    from oracle import dbar_oracle as orc
    w = wl.plain_fp64()
    tol = 1e-13 if prec == "fp64" else 1e-12
    plan = dbar.Plan(w.N, w.L, M=w.M, prec=prec, restart=8, sstep=4, tol=tol, max_batch=1, graphs=graphs)
    assert plan.solve(w.Q, w.k)["status"] == dbar.DBAR_OK      # cycle graphs (if any) captured
    dbar.dbar_plan_inject_wait_timeout(plan.handle)
    t0 = time.perf_counter()
    with pytest.raises(dbar.DbarError) as e:
        plan.solve(w.Q, w.k)
    elapsed = time.perf_counter() - t0
    assert e.value.status == dbar.DBAR_ETIMEOUT and "bounded device wait" in str(e.value)
    assert elapsed < 20.0, elapsed
    r = plan.solve(w.Q, w.k)
    assert r["status"] == dbar.DBAR_OK and r["resid"][0] <= tol
    o = orc.solve_cgo(w.Q, w.k[0], w.N, w.L, M=w.M, tol=1e-14)
    err = float(abs(r["S"][0] - o["S"]).max() / abs(o["S"]).max())
    assert err < (1e-12 if prec == "fp64" else 1e-10), err


def test_wait_hook_needs_block_sweeps(dbar):
    w = wl.plain_fp64()
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_plan_inject_wait_timeout(dbar.Plan(w.N, w.L, prec="fp64", sstep=1, max_batch=1).handle)
    assert e.value.status == dbar.DBAR_EINVAL
