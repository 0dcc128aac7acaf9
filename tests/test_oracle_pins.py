"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a
closed form, a library routine, brute force, an invariant or a value the paper
states (see tests/golden/ for the paper's worked-example parameters).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import dbar_oracle as orc
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- FFT

@pytest.mark.parametrize("N", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_brute_force_dft(N, sign):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((3, N)) + 1j * rng.standard_normal((3, N))
    j = np.arange(N)
    D = np.exp(sign * 2j * np.pi * np.outer(j, j) / N)
    np.testing.assert_allclose(orc.dft_last_axis(x, sign), x @ D.T, atol=1e-13)


def test_fft_matches_library_and_parseval():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 256)) + 1j * rng.standard_normal((2, 256))
    X = orc.dft_last_axis(x, -1)
    np.testing.assert_allclose(X, np.fft.fft(x), atol=1e-11)
    np.testing.assert_allclose(np.sum(abs(X) ** 2, -1), 256 * np.sum(abs(x) ** 2, -1), rtol=1e-13)
    f = rng.standard_normal((32, 64)) + 1j * rng.standard_normal((32, 64))
    with pytest.raises(ValueError):
        orc.dft_last_axis(np.ones(12), -1)
    g = orc.Grid(32, 3.0)
    f = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    np.testing.assert_allclose(g.Finv(g.F(f)), f, atol=1e-13)


def test_discrete_transform_of_gaussian_is_closed_form():
    # F(exp(-|z|^2)) = 1/2 exp(-|xi|^2/4) with the 1/2pi convention of Sec. 1; this fixes
    # the scale 2 pi L^2/N^2 and the (-1)^{m1+m2} phase of the grid x_j = L(-pi + 2 pi j/N).
    g = orc.Grid(128, 4.0)
    f = np.exp(-abs(g.z) ** 2)
    np.testing.assert_allclose(g.F(f), 0.5 * np.exp(-abs(g.xi) ** 2 / 4), atol=1e-15)
    # shifted Gaussian centred off the origin: phase exp(-i xi.x0)
    x0 = 0.7 - 0.4j
    f = np.exp(-abs(g.z - x0) ** 2)
    ph = np.exp(-1j * (g.xi.real * x0.real + g.xi.imag * x0.imag))
    np.testing.assert_allclose(g.F(f), 0.5 * np.exp(-abs(g.xi) ** 2 / 4) * ph, atol=1e-15)


def test_Ek_shift_of_the_fourier_support():
    # Sec. 5.1, eq. S0: F(E_k Q)(xi) = Q^(xi + 2i conj(k)); for Q = exp(-|z|^2) that is
    # 1/2 exp(-|xi + 2i conj k|^2 / 4).  Fixes the sign convention of E_k.
    g = orc.Grid(128, 5.0)
    k = 0.9 - 0.6j
    Q = np.exp(-abs(g.z) ** 2)
    lhs = g.F(g.E(k) * Q)
    rhs = 0.5 * np.exp(-abs(g.xi + 2j * np.conj(k)) ** 2 / 4)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)
    assert np.allclose(abs(g.E(k)), 1.0, atol=1e-15)


# --------------------------------------------------------------------------- W_n

def test_W0_is_the_lemma_closed_form():
    z = np.array([0.3 + 0.1j, 1.0, -2.0 + 3.0j, 7.5 - 0.2j, 1e-3j])
    exact = 1j / z * -np.expm1(-abs(z) ** 2 / 4)          # eq. fourreg, written without cancellation
    np.testing.assert_allclose(orc.W(0, z), exact, rtol=1e-12)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 8])
def test_W_closed_form_equals_series(n):
    # compared where both forms are well conditioned: a = |z|^2/4 in [(n+1)/2, 3(n+1)]
    rng = np.random.default_rng(n)
    a = rng.uniform(0.5 * (n + 1), 3.0 * (n + 1), 50)
    z = 2 * np.sqrt(a) * np.exp(1j * rng.uniform(0, 2 * np.pi, 50))
    np.testing.assert_allclose(orc.W_closed(n, z), orc.W_series(n, z), rtol=1e-12)
    assert orc.W(n, np.array([0j]))[0] == 0


def test_printed_series_lacks_gaussian_factor():
    # eq. fourreg5a as printed has no e^{-|z|^2/4}; it then disagrees with eq. fourreg5.
    z = np.array([0.7 + 0.2j, 2.5 - 1.3j])
    n = 0
    a = abs(z) ** 2 / 4
    printed = 1j * (np.conj(z) / 4) * sum(a ** j / math.factorial(j + 1) for j in range(60))
    assert np.all(abs(printed - orc.W_closed(n, z)) > 1e-2)
    np.testing.assert_allclose(printed * np.exp(-a), orc.W_closed(n, z), rtol=1e-13)


@pytest.mark.parametrize("n", [0, 1, 2, 4])
def test_W_matches_bessel_quadrature(n):
    # Polar form of F^{-1}(conj(xi)^n/xi e^{-|xi|^2}):
    # W_n(z) = i^{n+1} e^{-i(n+1) arg z} int_0^inf r^n e^{-r^2} J_{n+1}(|z| r) dr.
    from scipy import integrate, special
    for z in [0.4 + 0.3j, -1.7 + 0.9j, 3.0 - 2.5j]:
        rho, phi = abs(z), np.angle(z)
        val, _ = integrate.quad(lambda r: r ** n * np.exp(-r * r) * special.jv(n + 1, rho * r),
                                0, 12, epsabs=1e-15, epsrel=1e-13, limit=200)
        ref = (1j) ** (n + 1) * np.exp(-1j * (n + 1) * phi) * val
        assert abs(orc.W(n, np.array([z]))[0] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("n", [0, 2, 5])
@pytest.mark.parametrize("w", [0.6, 1.7])
def test_W_of_a_wider_or_narrower_gaussian_matches_bessel_quadrature(n, w):
    # The defining integral with e^{-|xi|^2/w^2}, in polar form:
    # i^{n+1} e^{-i(n+1) arg z} int_0^inf r^n e^{-r^2/w^2} J_{n+1}(|z| r) dr.
    from scipy import integrate, special
    for z in [0.4 + 0.3j, -1.7 + 0.9j, 3.0 - 2.5j]:
        rho, phi = abs(z), np.angle(z)
        val, _ = integrate.quad(lambda r: r ** n * np.exp(-r * r / (w * w)) * special.jv(n + 1, rho * r),
                                0, 12 * w, epsabs=1e-15, epsrel=1e-13, limit=400)
        ref = (1j) ** (n + 1) * np.exp(-1j * (n + 1) * phi) * val
        assert abs(orc.W_width(n, np.array([z]), w)[0] - ref) <= 1e-12 * max(1.0, abs(ref))


# --------------------------------------------------------------------------- Taylor data

def test_taylor_coefficients_of_a_shifted_gaussian():
    # S = F(exp(-alpha|z - z0|^2)) = (1/2alpha) exp(-|xi|^2/4alpha - i(xi conj z0 + conj xi z0)/2),
    # so d^n S/d conj(xi)^n (0) = (1/2alpha)(-i z0/2)^n and dS/dxi(0) = (1/2alpha)(-i conj z0/2).
    g = orc.Grid(128, 4.0)
    alpha, z0 = 1.3, 0.6 - 0.35j
    S = g.F(np.exp(-alpha * abs(g.z - z0) ** 2))
    c, d = orc.taylor_coeffs(S, g, 5)
    for n in range(6):
        exact = (1 / (2 * alpha)) * (-0.5j * z0) ** n / math.factorial(n)
        assert abs(c[n] - exact) < 1e-13, (n, c[n], exact)
    assert abs(d - (1 / (2 * alpha)) * (-0.5j * np.conj(z0))) < 1e-13


# --------------------------------------------------------------------------- dbar^{-1}

def _dbartest(g, a, b, c):
    f = np.exp(-a * (g.z - b) * (np.conj(g.z) - c))
    with np.errstate(all="ignore"):
        exact = (1 / (a * (g.z - b))) * (1 - f)
    at_b = abs(g.z - b) < 1e-14
    exact[at_b] = (np.conj(g.z) - c)[at_b]
    return f, exact


def test_dbar_inverse_worked_example_reaches_machine_precision():
    with open(os.path.join(GOLDEN, "dbartest.json")) as fh:
        gold = json.load(fh)
    p = gold["parameters"]
    g = orc.Grid(p["N"], p["L"])
    f, exact = _dbartest(g, p["a"], p["b"], complex(p["c_re"], p["c_im"]))
    err = abs(orc.dbar_inverse(f, g, p["M"]) - exact).max()
    assert err < gold["claims"]["linf_error_below"], err


@pytest.mark.parametrize("w", [1.5, 2.0])
def test_dbar_inverse_worked_example_with_another_gaussian_width(w):
    # The regularisation is exact for any width of the Gaussian of G: the eq. dbartest
    # example keeps machine precision at the golden parameters with w = 1.5 and 2.
    with open(os.path.join(GOLDEN, "dbartest.json")) as fh:
        gold = json.load(fh)
    p = gold["parameters"]
    g = orc.Grid(p["N"], p["L"])
    f, exact = _dbartest(g, p["a"], p["b"], complex(p["c_re"], p["c_im"]))
    err = abs(orc.dbar_inverse(f, g, p["M"], width=w) - exact).max()
    assert err < gold["claims"]["linf_error_below"], err


def test_dbar_inverse_error_falls_with_M_and_N():
    # Fig. 1: exponential decrease in M (N = 128) and in N (M = 11); M = 11 at N = 64
    # already reaches machine precision.
    g = orc.Grid(128, 4.0)
    f, exact = _dbartest(g, 0.5, 1.0, 1j)
    errs = [abs(orc.dbar_inverse(f, g, M) - exact).max() for M in (1, 3, 5, 7, 11)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-13
    errN = []
    for N in (16, 32, 64):
        gN = orc.Grid(N, 4.0)
        fN, exN = _dbartest(gN, 0.5, 1.0, 1j)
        errN.append(abs(orc.dbar_inverse(fN, gN, 11) - exN).max())
    assert errN[0] > errN[1] > errN[2] and errN[2] < 1e-12, errN


def test_dbartest_prefactor_reading_and_fill_reading():
    # The printed prefactor a/(z-b) is not the inverse (1/a is); zero-filling the xi = 0
    # value (first-order rule) leaves an O(1e-2) error the analytic limit does not.
    g = orc.Grid(64, 4.0)
    a, b, c = 0.5, 1.0, 1j
    f, exact = _dbartest(g, a, b, c)
    num = orc.dbar_inverse(f, g, 11)
    printed = exact * a * a
    assert abs(num - printed).max() > 0.1
    assert abs(orc.dbar_inverse(f, g, 11, fill="zero") - exact).max() > 1e-3
    assert abs(num - exact).max() < 1e-12


# --------------------------------------------------------------------------- operator and solve

def test_zero_potential_gives_zero_solution():
    N, L = 16, 3.0
    P = orc.CGOProblem(np.zeros((N, N)), 0.4 + 0.1j, N, L)
    S, it, res = P.solve_gmres()
    assert np.all(S == 0) and it == 0
    assert np.all(P.h(S) == 0)


def test_operator_is_real_linear_not_complex_linear():
    w = wl.small_gaussian(16, 3.0, 0.2 + 0.3j, amp=1.5 + 0.5j)
    P = orc.CGOProblem(w.Q, w.k[0], w.N, w.L)
    rng = np.random.default_rng(2)
    S1 = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    S2 = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    np.testing.assert_allclose(P.apply(2.5 * S1), 2.5 * P.apply(S1), atol=1e-12)
    np.testing.assert_allclose(P.apply(S1 + S2), P.apply(S1) + P.apply(S2), atol=1e-12)
    assert abs(P.apply(1j * S1) - 1j * P.apply(S1)).max() > 1e-3


@pytest.mark.parametrize("N", [8, 16, 32])
def test_krylov_agrees_with_dense_direct_solve(N):
    w = wl.small_gaussian(N, 2.0, 0.5 + 0.3j, amp=1.0)
    P = orc.CGOProblem(w.Q, w.k[0], w.N, w.L)
    Sd = P.solve_dense()
    Sk, it, res = P.solve_gmres(tol=1e-14)
    assert res < 1e-13
    assert abs(Sk - Sd).max() <= 1e-12 * abs(Sd).max()


def test_gmres_resumes_from_an_initial_guess():
    # GMRES (Sec. 4.1) from a given start: the converged solution is a fixed point (no
    # iteration), and a solve capped early resumes from its iterate to the same solution.
    w = wl.small_gaussian(16, 2.0, 0.5 + 0.3j, amp=1.0)
    P = orc.CGOProblem(w.Q, w.k[0], w.N, w.L)
    Sd = P.solve_dense()
    S1, it1, res1 = P.solve_gmres(tol=1e-14, restart=4, maxiter=4)
    assert res1 > 1e-6 and it1 == 4
    S2, it2, res2 = P.solve_gmres(tol=1e-14, restart=8, x0=S1)
    assert res2 <= 1e-14 and abs(S2 - Sd).max() <= 1e-12 * abs(Sd).max()
    S3, it3, res3 = P.solve_gmres(tol=1e-12, x0=Sd)
    assert it3 == 0 and np.array_equal(S3, Sd)


@pytest.mark.slow
def test_plain_fp64_workload_krylov_vs_dense_8192_unknowns():
    w = wl.plain_fp64()
    P = orc.CGOProblem(w.Q, w.k[0], w.N, w.L, w.M)
    Sd = P.solve_dense()
    Sk, it, res = P.solve_gmres(tol=1e-14)
    assert abs(Sk - Sd).max() <= 1e-12 * abs(Sd).max()


def test_born_limit_first_and_second_order():
    # Q = eps q0, q0 = exp(-|z|^2): S = eps S0 + eps^2 S1 + O(eps^3) with
    # S0 = -i F(E_k q0) = -i/2 exp(-|xi + 2i conj k|^2/4) (eq. S0) and, re-derived from
    # S1 = K(S0) with the dbar^{-1} closed form, S1 = -i F[q0/(2(conj z - k)) (E_k e^{-|k|^2} - q0)].
    N, L, k = 128, 5.0, 0.37 + 0.21j
    g = orc.Grid(N, L)
    q0 = np.exp(-abs(g.z) ** 2)
    S0 = -0.5j * np.exp(-abs(g.xi + 2j * np.conj(k)) ** 2 / 4)
    S1 = -1j * g.F(q0 / (2 * (np.conj(g.z) - k)) * (g.E(k) * np.exp(-abs(k) ** 2) - q0))
    rem = []
    for eps in (1e-2, 1e-3):
        P = orc.CGOProblem(eps * q0, k, N, L, M=11)
        S, it, res = P.solve_gmres(tol=1e-15)
        rem.append(abs(S - eps * S0 - eps ** 2 * S1).max())
    # third-order remainder: shrinks by ~1e3 when eps shrinks by 10
    assert rem[0] < 1e-5 and 3e2 < rem[0] / rem[1] < 3e3, rem


def test_spectral_convergence_on_nested_grids():
    # x-grids of N and 2N share the points x_j^N = x_{2j}^{2N}; the discrete solutions
    # converge exponentially in N (Sec. 4.2, Fig. 1 right).
    L, k = 4.0, 0.3 + 0.2j
    ms = {}
    for N in (64, 128, 256):
        w = wl.small_gaussian(N, L, k)
        ms[N] = orc.solve_cgo(w.Q, k, N, L, M=11, tol=1e-14)["m"]
    e1 = abs(ms[64] - ms[128][::2, ::2]).max()
    e2 = abs(ms[128] - ms[256][::2, ::2]).max()
    assert e2 < 1e-4 * e1 and e2 < 1e-10, (e1, e2)


def test_decay_of_m_at_infinity():
    # Theorem 3.1 / Sec. 6: m = m1/z + O(1/z^2) with m1 = i S(0).
    N, L, k = 128, 8.0, 0.4 - 0.3j
    w = wl.small_gaussian(N, L, k)
    r = orc.solve_cgo(w.Q, k, N, L, M=11, tol=1e-14)
    g = orc.Grid(N, L)
    j0 = N // 2
    devs = []
    for dj in (24, 48):          # |z| ~ 9.4 and 18.8 along the positive x axis
        z = g.z[j0, j0 + dj]
        devs.append(abs(z * r["m"][j0, j0 + dj] - r["m1"]))
    assert devs[1] < 0.7 * devs[0], devs
    assert devs[1] < 0.05 * abs(r["m1"])


def test_dbar_equation_holds_on_a_refined_grid():
    # Non-tautological residual: zero-pad S to 2N (same L), rebuild m = h(S) on the finer
    # grid and check dbar m = (i/2) F^{-1} S against 1/2 E_k Q (conj(m) + 1) there.
    N, L, k = 256, 4.0, 0.3 + 0.2j
    w = wl.small_gaussian(N, L, k)
    r = orc.solve_cgo(w.Q, k, N, L, M=11, tol=1e-14)
    S = r["S"]
    N2 = 2 * N
    m_idx = np.where(np.arange(N) <= N // 2, np.arange(N), np.arange(N) - N)
    p2 = m_idx % N2
    S2 = np.zeros((N2, N2), complex)
    S2[np.ix_(p2, p2)] = S
    g2 = orc.Grid(N2, L)
    h2 = orc.h_of_S(S2, g2, 11)
    Q2 = np.exp(-abs(g2.z) ** 2)
    lhs = 0.5j * g2.Finv(S2)
    rhs = 0.5 * g2.E(k) * Q2 * (np.conj(h2) + 1)
    assert abs(lhs - rhs).max() < 1e-13
    # coarse-grid points of the refined m agree with the solved m
    assert abs(h2[::2, ::2] - r["m"]).max() < 1e-13


# --------------------------------------------------------------------------- reflection coefficient

@pytest.mark.parametrize("k", [0.7 + 0.4j, 2.0 - 1.0j, -1.5j])
def test_reflection_born_limit_is_the_gaussian_closed_form(k):
    # Sec. 6.1: for Q = eps exp(-|z|^2), S_pm = mp i eps F(E_{k/2} e^{-|z|^2}) + O(eps^2), and the
    # second-order terms of S_+ and S_- are equal (the conjugated term flips sign twice), so
    # r(k) = eps F(e^{-|z|^2} e^{-i(k2 x + k1 y)})(0) + O(eps^3) = (eps/2) e^{-|k|^2/4} + O(eps^3)
    # (the Gaussian integral; the Fourier convention carries 1/(2 pi)).
    N, L = 64, 3.0
    X, Y = wl.mesh(N, L)
    born = 0.5 * np.exp(-abs(k) ** 2 / 4.0)
    dev = []
    for eps in (1e-3, 2e-3):
        r = orc.reflection(eps * np.exp(-(X * X + Y * Y)), k, N, L)["r"]
        dev.append(r / eps - born)
        assert abs(r / eps - born) < 50 * eps * eps, (eps, r / eps, born)
    # the deviation is O(eps^2) in r/eps (no O(eps) term): doubling eps multiplies it by 4
    assert abs(dev[1] / dev[0] - 4.0) < 0.2, dev


def test_reflection_time_dependence_is_a_unimodular_factor():
    # eq. rt: r(k, t) = r(k, 0) exp(-i t (k^2 + conj(k)^2)/4), |r| conserved in time
    N, L = 32, 2.5
    X, Y = wl.mesh(N, L)
    Q = 0.8 * np.exp(-(X * X + Y * Y)) * (1 + 0.2j * X)
    k = 1.2 - 0.7j
    r0 = orc.reflection(Q, k, N, L, t=0.0)["r"]
    r1 = orc.reflection(Q, k, N, L, t=0.3)["r"]
    assert abs(abs(r1) - abs(r0)) < 1e-13 * abs(r0)
    ang = np.angle(r1 / r0)
    np.testing.assert_allclose(ang, -0.3 * (k * k + np.conj(k) ** 2).real / 4.0, atol=1e-12)


# --------------------------------------------------------------------------- iterated equation (Sec. 5)

def _mixture(N, L):
    X, Y = wl.mesh(N, L)
    return (1.3 * np.exp(-(X * X + Y * Y)) + (0.4 + 0.6j) * np.exp(-((X - 0.5) ** 2 + (Y + 0.3) ** 2) / 0.7)
            ).astype(np.complex128)


@pytest.mark.parametrize("m", [(0, 0), (1, 2), (-3, 1), (4, -5)])
def test_iterated_equation_reflection_matches_the_direct_route(m):
    # Sec. 6.1: r = i h(i conj k) from the single iterated solve (eq. eqh2, shifted regularisation
    # eq. dbarinvShift) equals (i/2)(S_+(0) - S_-(0)) from the two solves of the Sec. 4 method,
    # wherever the latter resolves the problem (small k): two different discrete operators.  The
    # grid resolves h to the box edge (Q's widest transform ~e^{-0.175|xi|^2} at xi_max = 21)
    N, L = 128, 3.0
    Q = _mixture(N, L)
    k = (m[0] + 1j * m[1]) / L
    a = orc.reflection(Q, k, N, L)["r"]
    b = orc.reflection_iterated(Q, k, N, L)["r"]
    assert abs(a - b) < 1e-13 * abs(a)


@pytest.mark.parametrize("m", [(10, 6), (-8, -12), (14, 0)])
def test_iterated_equation_born_limit_at_large_k(m):
    # the Gaussian Born limit r = (eps/2) e^{-|k|^2/4} + O(eps^3) through the iterated equation at
    # |k| = 3.6 .. 4.5, where E_{k/2} Q already reaches the edge of the xi-box (Nyquist 10)
    N, L = 64, 3.2
    X, Y = wl.mesh(N, L)
    k = (m[0] + 1j * m[1]) / L
    born = 0.5 * np.exp(-abs(k) ** 2 / 4.0)
    dev = []
    for eps in (1e-3, 2e-3):
        r = orc.reflection_iterated(eps * np.exp(-(X * X + Y * Y)), k, N, L)["r"]
        dev.append(r / eps - born)
        assert abs(r / eps - born) < 50 * eps * eps * born + 1e-11, (eps, r / eps, born)
    assert abs(dev[1] / dev[0] - 4.0) < 0.3, dev


def _shifted_gaussian_quotient(g, xi0):
    # F^{-1}(h/(xi - xi0)) for h = F e^{-|z|^2} = (1/2) e^{-|xi|^2/4}: with the shift theorem and
    # F^{-1}(F(f)/xi) = (i/2) dbar^{-1} f,  = e^{i xi0.x} (i/2) dbar^{-1}(e^{-i xi0.x} e^{-|z|^2}),
    # and e^{-i xi0.x} e^{-|z|^2} = e^{-|xi0|^2/4} e^{-(z-b)(conj z-c)}, b = -i xi0/2, c = -i conj(xi0)/2
    b, c = -0.5j * xi0, -0.5j * np.conj(xi0)
    w = g.z - b
    with np.errstate(all="ignore"):
        inv = (1 / w) * (1 - np.exp(-w * (np.conj(g.z) - c)))
    at = abs(w) < 1e-13
    inv[at] = (np.conj(g.z) - c)[at]
    return np.exp(1j * (xi0.real * g.X + xi0.imag * g.Y)) * 0.5j * np.exp(-abs(xi0) ** 2 / 4) * inv


@pytest.mark.parametrize("m0", [(0, 0), (10, 0), (30, -20), (64, 0), (50, 50), (-63, 40), (64, 64)])
def test_shifted_quotient_is_the_closed_form_up_to_the_box_edge(m0):
    # eq. dbarinvShift: h centred at the origin divided by xi - xi0, xi0 anywhere on the grid up to
    # its edge (xi_max = N/(2L) = 16 here), against the closed form above
    g = orc.Grid(128, 4.0)
    h = g.F(np.exp(-(g.z * np.conj(g.z)).real))
    xi0 = (m0[0] + 1j * m0[1]) / g.L
    exact = _shifted_gaussian_quotient(g, xi0)
    assert abs(orc.h_of_S_at(h, g, m0, 11) - exact).max() < 5e-14


def test_shifted_quotient_is_not_a_circular_shift_of_the_unshifted_one():
    # reading of eq. dbarinvShift: the quotient is formed at the grid points as they are.  Rolling h
    # by xi0 and dividing by xi instead wraps xi - xi0 periodically; near the edge of the box that
    # is a different (and wrong) operator, while it agrees where h's shifted support stays inside
    g = orc.Grid(128, 4.0)
    h = g.F(np.exp(-(g.z * np.conj(g.z)).real))
    for m0, agree in (((10, 0), True), ((64, 0), False)):
        xi0 = (m0[0] + 1j * m0[1]) / g.L
        rolled = np.exp(1j * (xi0.real * g.X + xi0.imag * g.Y)) * orc.h_of_S(
            np.roll(h, shift=(-m0[1], -m0[0]), axis=(0, 1)), g, 11)
        err = abs(rolled - _shifted_gaussian_quotient(g, xi0)).max()
        assert (err < 1e-13) == agree, (m0, err)
    # at xi0 = 0 the shifted route is the unshifted one
    S = g.F(np.exp(-((g.X - 0.4) ** 2 + (g.Y + 0.2) ** 2)) * (1 + 0.3j))
    assert abs(orc.h_of_S_at(S, g, (0, 0), 11) - orc.h_of_S(S, g, 11)).max() < 1e-15


def test_shift_table_of_sec5_unshifted_slow_shifted_spectral():
    # Sec. 5.1, the figure and table of the shifting argument: dbar^{-1} of a test function (eq.
    # dbartest, a = 1/2) whose transform sits at -2i conj(k) for the table's (N, L, k).  Reading:
    # f = E_k e^{-a|z|^2}, i.e. eq. dbartest with b = conj(k)/a, c = -k/a scaled by e^{-|k|^2/a}, so
    # dbar^{-1} f = (e^{-|k|^2/a} - f)/(a (z - b)).  Without the shift the error falls only like 1/N
    # (the k of the table grow with N); with it (phi = F(e^{i xi0.x} f), eq. dbarinvShift) it falls
    # spectrally to machine precision.
    t = json.load(open(os.path.join(GOLDEN, "shift_table.json")))
    a = 0.5
    for col in (2, 3):
        unshifted, shifted = [], []
        for row in t["rows"]:
            N, L, k = row[0], row[1], complex(*row[col])
            g = orc.Grid(N, L)
            f = g.E(k) * np.exp(-a * (g.z * np.conj(g.z)).real)
            b = np.conj(k) / a
            with np.errstate(all="ignore"):
                exact = (np.exp(-abs(k) ** 2 / a) - f) / (a * (g.z - b))
            at = abs(g.z - b) < 1e-12
            exact[at] = np.exp(-abs(k) ** 2 / a) * (np.conj(b) + k / a)
            unshifted.append(abs(orc.dbar_inverse(f, g, 11) - exact).max())
            m0 = orc.shift_index(k, L)
            xi0 = (m0[0] + 1j * m0[1]) / L
            mod = np.exp(1j * (xi0.real * g.X + xi0.imag * g.Y))
            sh = -2j * np.conj(mod) * orc.h_of_S_at(g.F(mod * f), g, m0, 11)
            shifted.append(abs(sh - exact).max())
        assert all(u > 0.04 for u in unshifted), unshifted
        assert all(1.7 < u1 / u2 < 2.3 for u1, u2 in zip(unshifted[2:], unshifted[3:])), unshifted
        assert all(s2 < s1 for s1, s2 in zip(shifted[:4], shifted[1:4])), shifted
        assert max(shifted[3:]) < 1e-13, shifted


def test_iterated_equation_reaches_machine_precision_at_the_papers_large_k():
    # Sec. 5: the paper's large-k case k = 8.5936, L = 3.2, N = 128 (its figure of the first two
    # Born iterates); 2kL = 55.0 to 1e-3, i.e. 2k on the xi-grid (k = 55/6.4).  Refining the grid
    # N = 128 -> 256 must not change the iterated equation's h (machine precision at N = 128 for
    # this k, as Sec. 5.3 states), while the Sec. 4 equation's S still moves by ~1e-4 there
    L, k = 3.2, 55 / 6.4
    assert abs(2 * 8.5936 * L - 55) < 1e-3
    pts = [(0, 0), (3, -2), (-5, 7), (10, 0)]
    h, S = {}, {}
    for N in (128, 256):
        X, Y = wl.mesh(N, L)
        q = np.exp(-(X * X + Y * Y)).astype(np.complex128)
        hh = orc.solve_iterated(q, k, N, L, M=11, tol=1e-14)["h"]
        SS = orc.solve_cgo(q, k, N, L, M=11, tol=1e-14)["S"]
        h[N] = np.array([hh[m2 % N, m1 % N] for m1, m2 in pts])
        S[N] = np.array([SS[m2 % N, m1 % N] for m1, m2 in pts])
    assert np.max(np.abs(h[128] - h[256])) < 1e-14
    assert np.max(np.abs(S[128] - S[256])) > 1e-5


def test_iterated_shift_requires_2k_on_the_grid():
    with pytest.raises(ValueError):
        orc.shift_index(0.1 + 0.0j, 3.0)
    assert orc.shift_index((1.5 + 2.0j) / 3.0, 3.0) == (4, 3)


# --------------------------------------------------------------------------- DS II round trip (Sec. 6.2)

@pytest.mark.parametrize("row", [0, 1])
def test_ds2_round_trip_reproduces_the_papers_reconstruction_errors(row):
    # q -> r (one iterated solve per k) -> q (one per z) for q = exp(-x^2-y^2), M = 11, at the
    # paper's (N, L) pairs: at these coarse grids the error is the method's discretisation error,
    # so it must reproduce the printed value itself (within 10 %; 7.47e-3 vs 7.09e-3 and
    # 3.193e-4 vs 3.187e-4 with the shifted regularisation read as in eq. dbarinvShift)
    t = json.load(open(os.path.join(GOLDEN, "ds2_reconstruction.json")))
    N, L, err_paper = t["rows"][row]
    M = t["M"]
    X, Y = wl.mesh(N, L)
    q = np.exp(-(X * X + Y * Y)).astype(np.complex128)
    R = orc.reflection_on_grid(q, N, L, M=M, tol=1e-14)
    qr = np.array([[orc.ds2_potential(R, X[a, b] + 1j * Y[a, b], N, L, M=M, tol=1e-14) for b in range(N)]
                   for a in range(N)])
    err = np.max(np.abs(qr - q))
    assert abs(err / err_paper - 1.0) < 0.1, (N, L, err, err_paper)


# --------------------------------------------------------------------------- convolution regularisation

def test_gaussian_convolution_is_the_closed_form():
    # F s = (1/2) e^{-|xi|^2/4} e^{-i xi.z0} for s = e^{-|z - z0|^2}, so
    # F^{-1}(F(s) e^{-|xi|^2}/xi) = (1/2) F^{-1}(e^{-(5/4)|xi|^2}/xi)(z - z0)
    #                             = (1/2) (i/(z - z0)) (1 - e^{-|z - z0|^2/5}),
    # the lemma of Sec. 3 with 1/(4 * 5/4); the direct grid sum must reach it.
    z0 = 0.4 - 0.3j
    g = orc.Grid(32, 2.0)
    w = g.z - z0
    r2 = (w * np.conj(w)).real
    s = np.exp(-r2)
    with np.errstate(all="ignore"):
        exact = 0.5j / w * (-np.expm1(-r2 / 5.0))
    exact[r2 == 0] = 0.0
    out = orc.gauss_convolution(s, g)
    assert abs(out - exact).max() < 1e-14
    # batch axes are summed independently
    out2 = orc.gauss_convolution(np.stack([s, 2j * s]), g)
    assert abs(out2[1] - 2j * exact).max() < 2e-14


def test_conv_kernel_is_W0_at_grid_differences():
    # W_0 is odd and vanishes at 0; the table's centre row is W_0 on the x-axis
    g = orc.Grid(16, 1.0)
    K = orc.conv_kernel_table(g)
    assert K.shape == (31, 31)
    assert K[15, 15] == 0
    assert abs(K + K[::-1, ::-1]).max() < 1e-15
    h = 2 * np.pi / 16
    x = h * np.arange(1, 16)
    assert abs(K[15, 16:] - 1j / x * (-np.expm1(-x * x / 4))).max() < 1e-15


def test_dbar_inverse_conv_worked_example():
    # dbartest (a = 1/2, b = 1, c = i) through G = S e^{-|xi|^2}: the smooth remainder's
    # x-space tail decays only like e^{-|z|^2/(4 + 1/a)}, so it needs the larger box
    g = orc.Grid(128, 5.0)
    f, exact = _dbartest(g, 0.5, 1.0, 1j)
    assert abs(orc.dbar_inverse_conv(f, g) - exact).max() < 1e-13
    g = orc.Grid(64, 4.0)
    f, exact = _dbartest(g, 0.5, 1.0, 1j)
    assert abs(orc.dbar_inverse_conv(f, g) - exact).max() < 1e-10


def test_conv_and_taylor_regularisations_give_the_same_cgo_solution():
    # the paper's use of the convolution code: an independent test of the Taylor-Gaussian one
    N, L, k = 64, 4.0, 0.7 + 0.4j
    g = orc.Grid(N, L)
    Q = np.exp(-(g.z * np.conj(g.z)).real).astype(np.complex128)
    a = orc.solve_cgo_conv(Q, k, N, L)
    b = orc.solve_cgo(Q, k, N, L, M=11)
    assert a["resid"] < 1e-13 and b["resid"] < 1e-13
    assert abs(a["S"] - b["S"]).max() < 1e-13 * abs(b["S"]).max()
    assert abs(a["m"] - b["m"]).max() < 1e-13
    # with M = 0 the Taylor route is only algebraically accurate: the agreement is lost
    c = orc.solve_cgo(Q, k, N, L, M=0)
    assert abs(c["m"] - a["m"]).max() > 1e-9


def test_conv_operator_krylov_agrees_with_dense_solve():
    N, L, k = 16, 2.0, -0.5 + 0.9j
    g = orc.Grid(N, L)
    Q = (1.5 - 0.5j) * np.exp(-(g.z * np.conj(g.z)).real)
    P = orc.ConvProblem(Q, k, N, L)
    Sd = P.solve_dense()
    Sg, it, res = P.solve_gmres(tol=1e-14)
    assert abs(Sd - Sg).max() < 1e-12 * abs(Sd).max()
    assert P.residual(Sd) < 1e-13
