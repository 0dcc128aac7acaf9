"""The allocation-free 2-D DFT entry point against the planned one.

dbar_fft2_noalloc exists for callers that cannot allocate device memory when
they need a transform (a host runtime that owns all device memory through its
own pool, loops that forbid allocator calls because they may synchronise the
device): it keeps its intermediate field and twiddle tables in the library's
own global arrays instead of plan workspaces.  This file is collected last, so
a failure here comes after every other test has run; it also passes on its own
in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_02363_gb300 import dbar
    return torch, dbar


# (2048, 1, True) and (1024, 2, False) are exactly the 32 MiB limit; 32 is the smallest grid
@pytest.mark.parametrize("N,nk,fp32", [(256, 4, False), (1024, 2, True), (64, 3, False),
                                       (32, 1, True), (2048, 1, True), (1024, 2, False)])
def test_noalloc_fft2_matches_planned_fft2_on_calls_in_a_row(env, N, nk, fp32):
    torch, dbar = env
    plan = dbar.Plan(N, 4.0, prec="mixed", max_batch=nk, restart=4)
    dtype = torch.complex64 if fp32 else torch.complex128
    tol = 3e-6 if fp32 else 2e-15 * np.log2(N) * 4          # the FFT parity tolerance of the suite
    rng = np.random.default_rng(N + nk)
    # calls in a row share the scratch; the third repeats the first one's kernels,
    # so nothing is loaded lazily during it and free device memory must not move
    for call in range(3):
        x = rng.standard_normal((nk, N, N)) + 1j * rng.standard_normal((nk, N, N))
        xd = torch.from_numpy(x).to(dtype).cuda()
        sign = -1 if call != 1 else 1
        ref = torch.empty_like(xd)
        dbar.dbar_fft2(plan.handle, nk, xd, ref, sign, fp32)
        got = torch.empty_like(xd)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        dbar.dbar_fft2_noalloc(N, nk, xd, got, sign, fp32)
        torch.cuda.synchronize()
        if call == 2:
            assert torch.cuda.mem_get_info()[0] == free0, "the call changed free device memory"
        assert _rel(got.cpu().numpy(), ref.cpu().numpy()) <= tol, (N, nk, fp32, call)


def test_noalloc_fft2_rejects_sizes_beyond_its_scratch(env):
    torch, dbar = env
    N, nk = 1024, 3                                           # 3 x 1024^2 complex128 = 48 MiB > 32 MiB
    x = torch.zeros((nk, N, N), dtype=torch.complex128, device="cuda")
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_fft2_noalloc(N, nk, x, x, -1, False)
    assert e.value.status == dbar.DBAR_EINVAL


# 64 MiB, 64 MiB, 36 MiB: just above the limit; then grids outside [32, 2048] or not powers of two
@pytest.mark.parametrize("N,nk,fp32", [(2048, 2, True), (2048, 1, False), (512, 9, False), (96, 1, True),
                                       (4096, 1, True), (16, 1, True)])
def test_noalloc_fft2_rejects_bad_sizes(env, N, nk, fp32):
    torch, dbar = env
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")  # never touched: rejected before launch
    with pytest.raises(dbar.DbarError) as e:
        dbar.dbar_fft2_noalloc(N, nk, x, x, -1, fp32)
    assert e.value.status == dbar.DBAR_EINVAL
