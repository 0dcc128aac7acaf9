"""Plain FP64 CPU oracle for the spectral D-bar CGO solve.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``; the
product path (the CUDA library and its Python binding) never imports, calls
or links it, and it shares no code with that path.  It is deliberately slow
and written step by step in the paper's order so that each line can be
checked against the text by eye.

Reference: C. Klein, K. McLaughlin, "Spectral approach to D-bar problems"
(arXiv 1508.02363).

What it computes (paper notation):

* CGO problem (Sec. 1, eq:038/eq:039): m = psi e^{-kz} - 1 solves
  dbar m = 1/2 E_k Q (conj(m) + 1),  E_k = e^{conj(kz) - kz}.
* Fourier convention (Sec. 1): F f = (1/2pi) int f e^{-i xi.x};
  F^{-1} has the same 1/2pi.  xi = xi1 + i xi2 is complex.
* Unknown S = xi m^ (eq:042) solves (eq:MainEQa, Sec. 5.1 eq:MainEQDS)
  A S := S + i F(E_k Q conj(F^{-1}(S/xi))) = b := -i F(E_k Q).
* Regularisation (Sec. 4.2, eq. Sreg, Gchoice, fourreeg4, fourreg5,
  fourreg5a): G = e^{-|xi|^2} sum_{n<=M} c_n conj(xi)^n with
  n! c_n = (-i/2)^n F(z^n F^{-1} S)(0), and
  F^{-1}(G/xi) = sum c_n W_n, W_n = F^{-1}(conj(xi)^n/xi e^{-|xi|^2}).
  A Gaussian of width w (e^{-|xi|^2/w^2}; w = 1 is the paper's) changes only
  G and the closed form: substituting xi = w eta in the transform gives
  F^{-1}(conj(xi)^n/xi e^{-|xi|^2/w^2})(z) = w^{n+1} W_n(w z) (W_width); the
  c_n (Taylor data of S at 0) do not depend on w.
* The algorithm of Sec. 4.3 (for k = 0, used with Q -> E_k Q for k != 0 as
  in Sec. 5.1): GMRES on the stacked real and imaginary parts, each matrix
  application doing (a) Taylor coefficients via one inverse FFT and a
  summation at xi = 0, (b) G and sum c_n W_n, (c) h = F^{-1}((S-G)/xi) +
  sum c_n W_n, (d) A S = S + i F(E_k Q conj(h)): three 2-D FFTs.

* DS II reflection coefficient (Sec. 6.1, eq. MainEQDSpm, rviah, m1def, rt):
  r(k, t) = (i/2)(S_+(0) - S_-(0)) exp(-i t (k^2 + conj(k)^2)/4), S_pm the CGO
  solutions at the parameter k/2 with the potentials +Q and -Q (reflection()).

* Iterated integral equation (Sec. 5.2-5.3, eq. eqh2 with the shifted
  regularisation eq. dbarinvShift): h - K_0(H(h)) = -i F(q), 2k on the xi-grid
  (IteratedProblem, solve_iterated); reflection_iterated() gives r = i h(i conj k)
  from one solve per k.

* DS II potential from r (Sec. 1 eq. dbarrecA/B, qRec, rt; Sec. 6.2): the same
  formula with z and k exchanged on the k-grid of the box L' = N/(2 pi L)
  (reflection_on_grid, ds2_potential); the round trip q -> r -> q is pinned by the
  paper's reconstruction table.

* Convolution regularisation (Sec. 4.2, remark after eq. fourreg5a): G = S e^{-|xi|^2},
  so (S - G)/xi = S (1 - e^{-|xi|^2})/xi is smooth (0 at xi = 0) and goes through the
  FFT, while F^{-1}(G/xi) = (1/2pi) int F^{-1}(S)(z') W_0(z - z') d^2z' is summed
  directly over the grid, a four-dimensional sum (h_of_S_conv, ConvProblem,
  solve_cgo_conv).  The paper keeps this variant as an independent test of the
  Taylor-Gaussian code.

Discretisation (Sec. 4.1, eq. domain, xidomain):
  x_j = L(-pi + 2 pi j/N), xi_m = m/L with m in [-N/2+1, N/2] (Nyquist on
  the positive side).  With h = 2 pi L/N the Riemann sums give
    F_d f(xi_m)      = (2 pi L^2/N^2) (-1)^{m1+m2} DFT(f)[m mod N],
    F_d^{-1} g(x_j)  = (1/(2 pi L^2)) IDFT((-1)^{m1+m2} g)[j],
  with DFT = sum_j f_j e^{-2 pi i m.j/N} and IDFT unnormalised (e^{+}), so
  F_d^{-1} F_d = identity.

Readings where the paper is silent or misprinted (each pinned by a test):

* The grid contains xi = 0, where (S-G)/xi has a removable singularity.
  The value used there is the analytic limit d = dS/dxi(0)
  = (-i/2) F(conj(z) F^{-1} S)(0) ("analytic" fill); "zero" fill (the
  first-order rule of the prior method the paper reviews in Sec. 2) is
  kept as an option.
* The printed series form eq. fourreg5a lacks the factor e^{-|z|^2/4};
  the series used here carries it (it then equals the closed form
  eq. fourreg5 identically).
* The test problem eq. dbartest has prefactor 1/a, not a.
* GMRES restart length, orthogonalisation and starting guess are not
  stated: restarted GMRES with modified Gram-Schmidt, x0 = 0, relative
  2-norm of the stacked real residual.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# The oracle's own FFT: iterative radix-2 decimation in time, unnormalised.
# ---------------------------------------------------------------------------


def _bit_reverse(N: int) -> np.ndarray:
    nbits = N.bit_length() - 1
    idx = np.arange(N)
    rev = np.zeros(N, dtype=np.int64)
    for b in range(nbits):
        rev |= ((idx >> b) & 1) << (nbits - 1 - b)
    return rev


def dft_last_axis(x: np.ndarray, sign: int) -> np.ndarray:
    """sum_j x_j exp(sign * 2 pi i j p / N) along the last axis (N a power of 2).

    Radix-2 DIT: bit-reverse, then log2 N butterfly sweeps; the sub-DFT pair
    (E, O) of length m combines to X[p] = E[p] + w^p O[p],
    X[p+m] = E[p] - w^p O[p], w = exp(sign * i pi / m).
    """
    x = np.asarray(x, dtype=np.complex128)
    N = x.shape[-1]
    if N < 1 or (N & (N - 1)):
        raise ValueError("length must be a power of two")
    lead = x.shape[:-1]
    y = x[..., _bit_reverse(N)]
    m = 1
    while m < N:
        w = np.exp(sign * 1j * np.pi * np.arange(m) / m)
        y = y.reshape(lead + (N // (2 * m), 2, m))
        a = y[..., 0, :]
        b = y[..., 1, :] * w
        y = np.stack([a + b, a - b], axis=-2).reshape(lead + (N,))
        m *= 2
    return y


def dft2(f: np.ndarray, sign: int) -> np.ndarray:
    """2-D unnormalised DFT over the last two axes ([..., y, x])."""
    g = dft_last_axis(f, sign)
    g = np.swapaxes(dft_last_axis(np.swapaxes(g, -1, -2), sign), -1, -2)
    return g


# ---------------------------------------------------------------------------
# Grid and discrete transforms (Sec. 4.1, eq. domain / xidomain).
# ---------------------------------------------------------------------------


class Grid:
    def __init__(self, N: int, L: float):
        if N < 2 or (N & (N - 1)):
            raise ValueError("N must be a power of two")
        self.N, self.L = N, float(L)
        j = np.arange(N)
        x1 = L * (-np.pi + 2.0 * np.pi * j / N)            # x_j
        m = np.where(j <= N // 2, j, j - N)                 # wavenumber index of DFT slot p
        xi1 = m / L                                         # xi_m = m/L
        self.x1d, self.xi1d = x1, xi1
        self.X, self.Y = np.meshgrid(x1, x1, indexing="xy")  # [y][x]
        self.z = self.X + 1j * self.Y
        XI1, XI2 = np.meshgrid(xi1, xi1, indexing="xy")
        self.xi = XI1 + 1j * XI2                            # complex xi = xi1 + i xi2
        sgn1 = np.where(m % 2 == 0, 1.0, -1.0)
        self.sign = np.outer(sgn1, sgn1)                    # (-1)^{m1+m2}
        self.fwd_scale = 2.0 * np.pi * L * L / (N * N)
        self.inv_scale = 1.0 / (2.0 * np.pi * L * L)

    def F(self, f):
        """F_d f on the xi-grid (Riemann sum of the Sec. 1 transform)."""
        return self.fwd_scale * self.sign * dft2(f, -1)

    def Finv(self, g):
        """F_d^{-1} g on the x-grid."""
        return self.inv_scale * dft2(self.sign * g, +1)

    def F_at0(self, f):
        """F_d f at xi = 0: the transform reduces to a summation there (Sec. 4.3 remark)."""
        return self.fwd_scale * np.sum(f, axis=(-2, -1))

    def E(self, k: complex):
        """E_k = exp(conj(k z) - k z) = exp(-2i (k2 x + k1 y)) (eq:039)."""
        return np.exp(np.conj(k * self.z) - k * self.z)


# ---------------------------------------------------------------------------
# W_n = F^{-1}(conj(xi)^n / xi e^{-|xi|^2})  (Sec. 4.2, eq. fourreg, fourreg5,
# fourreg5a with the factor e^{-|z|^2/4} restored).
# ---------------------------------------------------------------------------


def W_closed(n: int, z):
    """eq. fourreg5: i (2i)^n n!/z^{n+1} {1 - e^{-a} sum_{k<=n} a^k/k!}, a = |z|^2/4."""
    z = np.asarray(z, dtype=np.complex128)
    a = (z * np.conj(z)).real / 4.0
    part = np.zeros_like(a)
    term = np.ones_like(a)
    for kk in range(n + 1):
        if kk > 0:
            term = term * a / kk
        part = part + term
    with np.errstate(divide="ignore", invalid="ignore"):
        return 1j * (2j) ** n * math.factorial(n) / z ** (n + 1) * (1.0 - np.exp(-a) * part)


def W_series(n: int, z, nterms: int = 200):
    """eq. fourreg5a with e^{-a}: i(2i)^n n! (conj z/4)^{n+1} e^{-a} sum_j a^j/(j+n+1)!."""
    z = np.asarray(z, dtype=np.complex128)
    a = (z * np.conj(z)).real / 4.0
    term = np.full(a.shape, 1.0 / math.factorial(n + 1))
    acc = np.zeros_like(a)
    for j in range(nterms):
        acc = acc + term
        term = term * a / (j + n + 2)
    return 1j * (2j) ** n * math.factorial(n) * (np.conj(z) / 4.0) ** (n + 1) * np.exp(-a) * acc


def W(n: int, z):
    """W_n to full FP64 accuracy: series where a = |z|^2/4 < n+1 (cancellation
    in the closed form near the origin, the paper's remark after eq. fourreg3),
    closed form elsewhere.  W_n(0) = 0."""
    z = np.asarray(z, dtype=np.complex128)
    a = (z * np.conj(z)).real / 4.0
    small = a < (n + 1)
    out = np.empty(z.shape, dtype=np.complex128)
    out[small] = W_series(n, z[small])
    out[~small] = W_closed(n, z[~small])
    return out


def W_width(n: int, z, w: float = 1.0):
    """F^{-1}(conj(xi)^n/xi e^{-|xi|^2/w^2}) = w^{n+1} W_n(w z) (the substitution xi = w eta
    in the inverse transform); w = 1 is W_n."""
    w = float(w)
    return w ** (n + 1) * W(n, w * np.asarray(z, dtype=np.complex128))


# ---------------------------------------------------------------------------
# The regularised F^{-1}(S/xi) (Sec. 4.3, steps 4a-4c).
# ---------------------------------------------------------------------------


def taylor_coeffs(S, g: Grid, M: int):
    """c_n, n = 0..M, with n! c_n = (-i/2)^n F(z^n F^{-1} S)(0) (eq. fourreeg4), and
    the fill value d = dS/dxi(0) = (-i/2) F(conj(z) F^{-1} S)(0).
    Literal route: one inverse FFT, then summations at xi = 0."""
    s = g.Finv(S)
    c = [(-0.5j) ** n / math.factorial(n) * g.F_at0(g.z ** n * s) for n in range(M + 1)]
    d = -0.5j * g.F_at0(np.conj(g.z) * s)
    return c, d


def h_of_S(S, g: Grid, M: int, fill: str = "analytic", Wn=None, width: float = 1.0):
    """h = F^{-1}(S/xi) = F^{-1}((S - G)/xi) + sum_n c_n W_n   (eq. Sreg, S0Taylor),
    with the Gaussian of G of the given width (e^{-|xi|^2/width^2}).

    S may carry leading batch axes.  Returns h on the x-grid."""
    c, d = taylor_coeffs(S, g, M)
    if Wn is None:
        Wn = [W_width(n, g.z, width) for n in range(M + 1)]
    gauss = np.exp(-(g.xi * np.conj(g.xi)).real / width ** 2)
    G = np.zeros_like(S)
    for n in range(M + 1):
        G = G + np.asarray(c[n])[..., None, None] * gauss * np.conj(g.xi) ** n
    xi = g.xi.copy()
    xi[0, 0] = 1.0                                # placeholder, overwritten below
    U = (S - G) / xi
    U[..., 0, 0] = d if fill == "analytic" else 0.0
    h = g.Finv(U)
    for n in range(M + 1):
        h = h + np.asarray(c[n])[..., None, None] * Wn[n]
    return h


def h_of_S_at(S, g: Grid, m0, M: int, fill: str = "analytic", Wn=None, width: float = 1.0):
    """F^{-1}(S/(xi - xi0)) with the shifted regularisation eq. dbarinvShift, xi0 = (m0[0] + i m0[1])/L
    a grid point:
      * S's quotient by xi - xi0 is formed at the grid points as they are (no periodic wrap of
        xi - xi0: S lives near the origin, xi0 may lie near the edge of the box);
      * G = e^{-|xi - xi0|^2} sum_n c_n conj(xi - xi0)^n with n! c_n = d^n_{conj xi} S(xi0)
        = (-i/2)^n F(z^n e^{-i xi0.x} F^{-1} S)(0) is Sec. 4's G moved to xi0 on the grid's torus:
        its difference xi - xi0 is taken periodically (reading: the paper is silent on a G that
        reaches the edge of the box; there its coefficients are those of S far from its support);
      * the analytic limit d = d_xi S(xi0) at xi0, and F^{-1}(G/(xi - xi0)) = e^{i xi0.x} sum_n c_n W_n.
    m0 = (0, 0) is h_of_S.  width: that of the Gaussian of G, as in h_of_S."""
    N = g.N
    xi0 = (m0[0] + 1j * m0[1]) / g.L
    s = g.Finv(S)
    ph = np.exp(-1j * (xi0.real * g.X + xi0.imag * g.Y))          # e^{-i xi0.x}
    c = [(-0.5j) ** n / math.factorial(n) * g.F_at0(g.z ** n * s * ph) for n in range(M + 1)]
    d = -0.5j * g.F_at0(np.conj(g.z) * s * ph)
    if Wn is None:
        Wn = [W_width(n, g.z, width) for n in range(M + 1)]
    at = (m0[1] % N, m0[0] % N)                                   # the grid point xi0
    dxi = g.xi - xi0                                              # plain difference
    dxi_t = np.roll(g.xi, shift=at, axis=(0, 1))                  # periodic difference on the torus
    gauss = np.exp(-(dxi_t * np.conj(dxi_t)).real / width ** 2)
    den, den_t = dxi.copy(), dxi_t.copy()
    den[at] = den_t[at] = 1.0                                     # placeholders, xi0 overwritten below
    U = S / den
    for n in range(M + 1):
        U = U - np.asarray(c[n])[..., None, None] * gauss * np.conj(dxi_t) ** n / den_t
    U[(Ellipsis,) + at] = d if fill == "analytic" else 0.0
    h = g.Finv(U)
    mod = np.conj(ph)                                             # e^{i xi0.x}
    for n in range(M + 1):
        h = h + np.asarray(c[n])[..., None, None] * mod * Wn[n]
    return h


def dbar_inverse(f, g: Grid, M: int, fill: str = "analytic", width: float = 1.0):
    """dbar^{-1} f = F^{-1}(-2i/xi F f) (Sec. 3 lemma), through the same regularisation."""
    return h_of_S(-2j * g.F(f), g, M, fill, width=width)


# ---------------------------------------------------------------------------
# Operator, right-hand side and solution (Sec. 4.3 with Q -> E_k Q, Sec. 5.1).
# ---------------------------------------------------------------------------


class CGOProblem:
    def __init__(self, Q, k: complex, N: int, L: float, M: int = 2, fill: str = "analytic", width: float = 1.0):
        self.g = Grid(N, L)
        self.Q = np.asarray(Q, dtype=np.complex128)
        self.k = complex(k)
        self.M = M
        self.fill = fill
        self.width = float(width)
        self.EQ = self.g.E(self.k) * self.Q
        self.Wn = [W_width(n, self.g.z, width) for n in range(M + 1)]

    def rhs(self):
        """b = -i F(E_k Q)  (Sec. 4.3 step 3; eq. S0)."""
        return -1j * self.g.F(self.EQ)

    def h(self, S):
        return h_of_S(S, self.g, self.M, self.fill, self.Wn, self.width)

    def apply(self, S):
        """A S = S + i F(E_k Q conj(h(S)))  (Sec. 4.3 step 4d)."""
        return S + 1j * self.g.F(self.EQ * np.conj(self.h(S)))

    # real-stacked view: x in R^{2N^2} <-> S in C^{N^2}
    def to_real(self, S):
        return np.ascontiguousarray(S).view(np.float64).reshape(S.shape[:-2] + (-1,))

    def from_real(self, x):
        N = self.g.N
        return np.ascontiguousarray(x).view(np.complex128).reshape(x.shape[:-1] + (N, N))

    def apply_real(self, x):
        return self.to_real(self.apply(self.from_real(x)))

    def dense_matrix(self, chunk: int = 256):
        """The 2N^2 x 2N^2 real matrix of the real-linear operator A, column by column
        (A applied to the real unit vectors)."""
        n = 2 * self.g.N ** 2
        A = np.empty((n, n))
        for j0 in range(0, n, chunk):
            j1 = min(n, j0 + chunk)
            E = np.zeros((j1 - j0, n))
            E[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
            A[:, j0:j1] = self.apply_real(E).T
        return A

    def solve_dense(self):
        """Direct solve of the same discrete system (LAPACK LU via numpy)."""
        A = self.dense_matrix()
        x = np.linalg.solve(A, self.to_real(self.rhs()))
        return self.from_real(x)

    def solve_gmres(self, tol=1e-13, restart=40, maxiter=2000, x0=None):
        b = self.to_real(self.rhs())
        x0 = None if x0 is None else self.to_real(np.asarray(x0, dtype=np.complex128))
        x, it, res = gmres(self.apply_real, b, tol=tol, restart=restart, maxiter=maxiter, x0=x0)
        return self.from_real(x), it, res

    def residual(self, S):
        b = self.rhs()
        r = b - self.apply(S)
        return np.linalg.norm(r) / np.linalg.norm(b)


# ---------------------------------------------------------------------------
# Restarted GMRES on a real vector space (Saad & Schultz), modified Gram-Schmidt,
# Givens rotations, x0 = 0.
# ---------------------------------------------------------------------------


def gmres(apply, b, tol=1e-13, restart=40, maxiter=2000, x0=None):
    """Returns (x, total_iterations, final true relative residual)."""
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if nb == 0.0:
        return x, 0, 0.0
    total = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta / nb <= tol or total >= maxiter:
            return x, total, beta / nb
        m = restart
        V = np.zeros((m + 1, b.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        e = np.zeros(m + 1)
        e[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = apply(V[j])
            for i in range(j + 1):
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rho = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            e[j + 1] = -sn[j] * e[j]
            e[j] = cs[j] * e[j]
            total += 1
            j_done = j + 1
            if abs(e[j + 1]) / nb <= tol * 0.5 or total >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), e[:j_done])
        x = x + V[:j_done].T @ y


def solve_cgo(Q, k, N, L, M=2, tol=1e-13, restart=40, maxiter=2000, fill="analytic", width=1.0, x0=None):
    """One CGO solve: returns dict(S, m, m1, iters, resid).  width: that of the
    Gaussian of G; x0: initial guess of S (None: S = 0)."""
    P = CGOProblem(Q, k, N, L, M, fill, width)
    S, it, res = P.solve_gmres(tol=tol, restart=restart, maxiter=maxiter, x0=x0)
    m = P.h(S)
    return {"S": S, "m": m, "m1": 1j * S[0, 0], "iters": it, "resid": res}


# ---------------------------------------------------------------------------
# Convolution regularisation (Sec. 4.2, remark after eq. fourreg5a).
# ---------------------------------------------------------------------------


def conv_kernel_table(g: Grid, width: float = 1.0):
    """W_0(z_j - z_j') at every difference of two grid points: [dy + N-1][dx + N-1]
    with z_j - z_j' = h (dx + i dy), h = 2 pi L/N, dx, dy in [-(N-1), N-1]
    (W_0 of the Gaussian of the given width)."""
    N = g.N
    h = 2.0 * np.pi * g.L / N
    d = np.arange(-(N - 1), N)
    DX, DY = np.meshgrid(d, d, indexing="xy")
    return W_width(0, h * (DX + 1j * DY), width)


def gauss_convolution(s, g: Grid, K=None):
    """(1/2pi) int s(z') W_0(z - z') d^2z' by the trapezoidal rule on the x-grid (the
    periodic box's quadrature, area h^2 per point), summed directly over every pair of
    grid points -- the four-dimensional sum of the remark after eq. fourreg5a:
        out[y][x] = (h^2/2pi) sum_{y', x'} s[y'][x'] K[y - y' + N-1][x - x' + N-1].
    s may carry leading batch axes."""
    N = g.N
    if K is None:
        K = conv_kernel_table(g)
    h = 2.0 * np.pi * g.L / N
    s = np.asarray(s, dtype=np.complex128)
    # win[a][b][y][x] = K[a + y][b + x]; the pair (y', x') uses a = N-1-y', b = N-1-x'
    win = np.lib.stride_tricks.sliding_window_view(K, (N, N))
    s_rev = s[..., ::-1, ::-1]
    out = np.einsum("...ab,abyx->...yx", s_rev, win)
    return out * (h * h / (2.0 * np.pi))


def h_of_S_conv(S, g: Grid, K=None, width: float = 1.0):
    """h = F^{-1}(S/xi) with G = S e^{-|xi|^2} (eq. Sreg):
        F^{-1}((S - G)/xi) = F^{-1}(S (1 - e^{-|xi|^2})/xi)   (smooth; 0 at xi = 0)
        F^{-1}(G/xi)       = (1/2pi) int F^{-1}(S)(z') W_0(z - z') d^2z'
    (with a width: e^{-|xi|^2/width^2} and W_0 of that Gaussian)."""
    xi = g.xi.copy()
    r2 = (xi * np.conj(xi)).real / width ** 2
    xi[0, 0] = 1.0                                # placeholder, the factor is 0 there
    mult = -np.expm1(-r2) / xi
    mult[0, 0] = 0.0
    u = g.Finv(S * mult)
    s = g.Finv(S)
    if K is None:
        K = conv_kernel_table(g, width)
    return u + gauss_convolution(s, g, K)


def dbar_inverse_conv(f, g: Grid):
    """dbar^{-1} f = F^{-1}(-2i/xi F f) (Sec. 3 lemma) through the convolution regularisation."""
    return h_of_S_conv(-2j * g.F(f), g)


class ConvProblem(CGOProblem):
    """The CGO operator of Sec. 4.3 (Q -> E_k Q) with h(S) from the convolution
    regularisation instead of the Taylor-Gaussian G; same right-hand side."""

    def __init__(self, Q, k: complex, N: int, L: float, width: float = 1.0):
        super().__init__(Q, k, N, L, M=0, width=width)
        self.K = conv_kernel_table(self.g, width)

    def h(self, S):
        return h_of_S_conv(S, self.g, self.K, self.width)


def solve_cgo_conv(Q, k, N, L, tol=1e-13, restart=40, maxiter=2000, width=1.0):
    """One CGO solve with the convolution regularisation: dict(S, m, m1, iters, resid)."""
    P = ConvProblem(Q, k, N, L, width)
    S, it, res = P.solve_gmres(tol=tol, restart=restart, maxiter=maxiter)
    return {"S": S, "m": P.h(S), "m1": 1j * S[0, 0], "iters": it, "resid": res}


# ---------------------------------------------------------------------------
# DS II reflection coefficient (Sec. 6.1, eq. MainEQDSpm, hpmdef, rviah,
# m1def; time dependence eq. rt).
# ---------------------------------------------------------------------------


def reflection(Q, k, N, L, M=2, t=0.0, tol=1e-13, restart=40, maxiter=2000):
    """r(k, t) for the potential Q (sampled on the x-grid), Sec. 6's convention
    (k replaced by k/2, so the exponential is e^{(conj(k z) - k z)/2} = E_{k/2}).

    The two equations eq. MainEQDSpm are the CGO equation of Sec. 5.1 at the
    parameter k/2 with the potentials +Q (S_+) and -Q (S_-).  By eq. m1def,
    m^(1)_pm = i S_pm(0); by eq. Sform / hpmdef, S_pm(0) = f(0) pm h(i conj k)
    with f common, so eq. rviah gives
        r(k) = i h(i conj k) = (m^(1)_+ - m^(1)_-)/2 = (i/2)(S_+(0) - S_-(0)),
    and eq. rt gives r(k, t) = r(k) exp(-i t (k^2 + conj(k)^2) / 4).
    Returns dict(r, Sp0, Sm0, iters, resid)."""
    k = complex(k)
    sp = solve_cgo(Q, k / 2.0, N, L, M=M, tol=tol, restart=restart, maxiter=maxiter)
    sm = solve_cgo(-np.asarray(Q), k / 2.0, N, L, M=M, tol=tol, restart=restart, maxiter=maxiter)
    r0 = 0.5j * (sp["S"][0, 0] - sm["S"][0, 0])
    r = r0 * np.exp(-1j * t * (k * k + np.conj(k) ** 2) / 4.0)
    return {"r": complex(r), "Sp0": complex(sp["S"][0, 0]), "Sm0": complex(sm["S"][0, 0]),
            "iters": (sp["iters"], sm["iters"]), "resid": max(sp["resid"], sm["resid"])}


# ---------------------------------------------------------------------------
# Iterated integral equation (Sec. 5.2-5.3, eq. eqh2, dbarinvShift): the
# unknown h, supported near the origin for every k, with 2k on the xi-grid.
# ---------------------------------------------------------------------------


def shift_index(k, L):
    """Grid offset (m1, m2) of xi0 = 2i conj(k) = 2 k2 + 2i k1, i.e. xi0 = (m1 + i m2)/L;
    Sec. 5.3 requires 2k on the xi-grid."""
    m1, m2 = 2.0 * k.imag * L, 2.0 * k.real * L
    r1, r2 = int(round(m1)), int(round(m2))
    if abs(m1 - r1) > 1e-9 or abs(m2 - r2) > 1e-9:
        raise ValueError("2k must lie on the xi-grid (2 k L integer in both components)")
    return r1, r2


class IteratedProblem:
    """h - K_0(H(h)) = -i F(q) (eq. eqh2) with
        H(h) = -i F(q conj(F^{-1}(h / (xi - xi0)))),  xi0 = 2i conj(k)   (Sec. 5.3 step 1)
        K_0(S) = -i F(q conj(F^{-1}(S / xi)))                            (eq. shift)
    F^{-1}(h/(xi - xi0)) by the shifted regularisation eq. dbarinvShift (h_of_S_at):
    h is supported near the origin, the quotient by xi - xi0 is formed at the grid
    points, and the singular point xi0 (which may lie near the edge of the box) is
    regularised by a Gaussian G centred there."""

    def __init__(self, q, k, N, L, M=2, fill="analytic", width=1.0):
        self.g = Grid(N, L)
        self.q = np.asarray(q, dtype=np.complex128)
        self.k = complex(k)
        self.M, self.fill, self.width = M, fill, float(width)
        # xi0 on the grid's wavenumbers (-N/2, N/2]; -N/2 is the Nyquist point, which the
        # grid holds on the positive side (eq. xidomain)
        m0 = shift_index(self.k, L)
        if not all(-N // 2 <= m <= N // 2 for m in m0):
            raise ValueError("2k L must lie within the grid's wavenumbers [-N/2, N/2]")
        self.m0 = tuple(N // 2 if m == -N // 2 else m for m in m0)
        self.Wn = [W_width(n, self.g.z, width) for n in range(M + 1)]

    def H(self, h):
        u = h_of_S_at(h, self.g, self.m0, self.M, self.fill, self.Wn, self.width)
        return -1j * self.g.F(self.q * np.conj(u))

    def K0(self, S):
        return -1j * self.g.F(self.q * np.conj(h_of_S(S, self.g, self.M, self.fill, self.Wn, self.width)))

    def rhs(self):
        return -1j * self.g.F(self.q)

    def apply(self, h):
        return h - self.K0(self.H(h))

    def solve_gmres(self, tol=1e-13, restart=40, maxiter=2000):
        to_real = lambda S: np.ascontiguousarray(S).view(np.float64).reshape(-1)
        N = self.g.N
        from_real = lambda x: np.ascontiguousarray(x).view(np.complex128).reshape(N, N)
        b = to_real(self.rhs())
        x, it, res = gmres(lambda v: to_real(self.apply(from_real(v))), b, tol=tol, restart=restart,
                           maxiter=maxiter)
        return from_real(x), it, res


def solve_iterated(q, k, N, L, M=2, tol=1e-13, restart=40, maxiter=2000):
    """h of eq. eqh2 at parameter k: dict(h, iters, resid)."""
    P = IteratedProblem(q, k, N, L, M)
    h, it, res = P.solve_gmres(tol=tol, restart=restart, maxiter=maxiter)
    return {"h": h, "iters": it, "resid": res}


def reflection_iterated(q, k, N, L, M=2, t=0.0, tol=1e-13):
    """r(k, t) through the iterated equation (Sec. 6.1 with Sec. 5.3): in Sec. 6's
    convention the equation is taken at k/2, so xi0 = i conj(k), and eq. rviah reads
    r = i h(i conj k) -- one solve per k.  Needs k on the xi-grid (k L integer)."""
    k = complex(k)
    sol = solve_iterated(q, k / 2.0, N, L, M=M, tol=tol)
    m1, m2 = shift_index(k / 2.0, L)
    h0 = sol["h"][m2 % N, m1 % N]
    r = 1j * h0 * np.exp(-1j * t * (k * k + np.conj(k) ** 2) / 4.0)
    return {"r": complex(r), "iters": sol["iters"], "resid": sol["resid"]}


# ---------------------------------------------------------------------------
# DS II potential from the reflection coefficient (Sec. 1 eq. dbarrecA/B,
# qRec, rt; Sec. 6.2).  In Sec. 6's convention (k and xi dual) r lives on the
# points m/L of a problem of box L, i.e. on the x-grid of the box
# L' = N/(2 pi L), and the D-bar problem in k is the CGO problem in the
# variable k with the potential conj(r(k, t)) at the parameter z/2:
# q(z, t) = (m~^(1)_+ - m~^(1)_-)/2, the same formula as r with z and k exchanged.
# ---------------------------------------------------------------------------


def inverse_box(N, L):
    """L' such that the x-grid of the box L' is the grid m/L of Sec. 6's k."""
    return N / (2.0 * math.pi * L)


def reflection_on_grid(q, N, L, M=2, tol=1e-13):
    """r(k, 0) at every point k of the x-grid of the box L' = inverse_box(N, L),
    [k2][k1] layout (one iterated solve per k)."""
    g = Grid(N, inverse_box(N, L))
    R = np.empty((N, N), dtype=np.complex128)
    for a in range(N):
        for b in range(N):
            R[a, b] = reflection_iterated(q, g.z[a, b], N, L, M=M, tol=tol)["r"]
    return R


def ds2_potential(R, z, N, L, M=2, t=0.0, tol=1e-13):
    """q(z, t) from r(k, 0) = R on the k-grid of the box L' = inverse_box(N, L)."""
    Lp = inverse_box(N, L)
    g = Grid(N, Lp)
    k = g.z
    Qk = np.conj(R * np.exp(-1j * t * (k * k + np.conj(k) ** 2) / 4.0))
    return reflection_iterated(Qk, complex(z), N, Lp, M=M, tol=tol)["r"]
