"""The DS II reflection coefficient (Sec. 6.1, eq. rviah, rt) through the C ABI
against the CPU oracle and against the Gaussian Born limit."""
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


def _potential(N, L):
    X, Y = wl.mesh(N, L)
    return (1.3 * np.exp(-(X * X + Y * Y)) + (0.4 + 0.6j) * np.exp(-((X - 0.5) ** 2 + (Y + 0.3) ** 2) / 0.7)
            ).astype(np.complex128)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 1e-9)])
def test_reflection_matches_oracle(dbar, prec, tol):
    N, L = 64, 3.0
    Q = _potential(N, L)
    k = np.array([0.0, 0.6 + 0.2j, -1.1 + 0.9j, 2.0 - 1.5j, 0.3j])
    plan = dbar.Plan(N, L, M=2, prec=prec, tol=1e-13 if prec == "fp64" else 1e-12, max_batch=8)
    r, iters, resid, status = dbar.dbar_reflection(plan.handle, Q, k, t=0.0)
    assert status == dbar.DBAR_OK and np.all(iters[:, 0] > 0)
    ref = np.array([orc.reflection(Q, kk, N, L, tol=1e-14)["r"] for kk in k])
    err = np.max(np.abs(r - ref)) / np.max(np.abs(ref))
    assert err < tol, (err, r, ref)


def test_reflection_born_limit_on_the_gpu(dbar):
    # r(k) = (eps/2) e^{-|k|^2/4} + O(eps^3) for Q = eps e^{-|z|^2} (N = 128, L = 3.2 resolve it)
    N, L, eps = 128, 3.2, 1e-4
    X, Y = wl.mesh(N, L)
    k = np.array([0.5 + 0.5j, 1.5 - 2.0j, -3.0 + 1.0j])
    plan = dbar.Plan(N, L, M=2, prec="fp64", tol=1e-13, max_batch=4)
    r, _, _, status = dbar.dbar_reflection(plan.handle, eps * np.exp(-(X * X + Y * Y)), k)
    assert status == dbar.DBAR_OK
    born = 0.5 * np.exp(-np.abs(k) ** 2 / 4.0)
    np.testing.assert_allclose(r / eps, born, rtol=0, atol=1e-7)


def test_reflection_batches_time_factor_and_errors(dbar):
    N, L = 32, 2.5
    Q = _potential(N, L)
    k = np.array([0.2 + 0.1j, -0.7 + 0.4j, 1.0 - 0.5j, 0.1 - 1.2j, 0.9j])
    small = dbar.Plan(N, L, prec="mixed", max_batch=2)          # batches of 2, 2, 1
    big = dbar.Plan(N, L, prec="mixed", max_batch=8)
    r2 = dbar.dbar_reflection(small.handle, Q, k)[0]
    r8 = dbar.dbar_reflection(big.handle, Q, k)[0]
    assert np.array_equal(r2, r8)                                  # slots never mix
    t = 0.7
    rt = dbar.dbar_reflection(big.handle, Q, k, t=t)[0]
    np.testing.assert_allclose(rt, r8 * np.exp(-1j * t * (k * k + np.conj(k) ** 2) / 4.0), rtol=1e-13, atol=0)
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_reflection(big.handle, Q, k, t=float("inf"))
    assert e.value.status == dbar.DBAR_EINVAL
