"""Seeded synthetic inputs for the spectral D-bar CGO solve.

This module only *generates inputs*: the potential Q sampled on the periodic
x-grid, the list of spectral parameters k and the solver settings.  It holds
none of the method's arithmetic (no transforms, no regularisation, no Krylov
step), so both the CPU oracle and the CUDA path can take their inputs from
here without sharing any computation.

Grid convention (paper Sec. 4, eq. "domain"): x_j = L(-pi + 2 pi j / N),
j = 0..N-1, identical in y.  Arrays are row-major [y][x] (axis 0 = y index,
axis 1 = x index), complex128.

Workloads (the paper's own test potentials are Gaussians, Sec. 4 test
problem and Sec. 6 initial data q0 = exp(-x^2-y^2)):

* ``plain_fp64``     N=64 on [-5pi,5pi]^2, Q = exp(-(x^2+y^2)), k = 0.5+0.3i.
* ``batched_fp64``   N=512 on [-8pi,8pi]^2, Q = 2 exp(-(x^2+y^2)/1.5^2) e^{0.7i},
                     256 k on the 16x16 grid linspace(-3,3,16)^2.
* ``mixed_1024``     N=1024 on [-10pi,10pi]^2, Q = sum of 4 Gaussians
                     c_j exp(-|z-z_j|^2/w_j^2), seed 7: centres U[-3,3]^2, widths
                     U[0.5,2], |c_j| U[0,5], arg c_j U[0,2pi); then 128 k with
                     |k| log-uniform in [0.1,8] and arg k U[0,2pi) from the same
                     generator.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    L: float
    Q: np.ndarray            # [N][N] complex128, row-major [y][x]
    k: np.ndarray            # [nk] complex128
    M: int = 2               # Taylor order of the regularising G
    tol: float = 1e-12       # relative residual target of the stacked real system
    mixed: bool = False      # FP32 inner Krylov with FP64 refinement
    description: str = ""


def x_grid(N: int, L: float) -> np.ndarray:
    """Periodic grid x_j = L(-pi + 2 pi j/N) (paper Sec. 4, eq. "domain")."""
    j = np.arange(N, dtype=np.float64)
    return L * (-np.pi + 2.0 * np.pi * j / N)


def mesh(N: int, L: float):
    """X, Y sampled on the grid, shape [N][N], X varying along axis 1."""
    x = x_grid(N, L)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return X, Y


def gaussian_mixture(N, L, centres, widths, amps):
    """Q = sum_j c_j exp(-|z - z_j|^2 / w_j^2) sampled on the grid.  Each term is the
    outer product exp(-(y - y_j)^2/w_j^2) exp(-(x - x_j)^2/w_j^2), so Q is one matrix
    product over the terms ([N][t] times [t][N])."""
    x = x_grid(N, L)
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 2)
    w2 = np.asarray(widths, dtype=np.float64).reshape(-1, 1) ** 2
    gx = np.exp(-((x[None, :] - centres[:, 0:1]) ** 2) / w2)      # [t][N], along x
    gy = np.exp(-((x[None, :] - centres[:, 1:2]) ** 2) / w2)      # [t][N], along y
    amps = np.asarray(amps, dtype=np.complex128).reshape(-1)
    return np.ascontiguousarray((gy.T * amps[None, :]) @ gx.astype(np.complex128))


def draw_mixture(rng: np.random.Generator, nterms: int):
    """Draw order: centres U[-3,3]^2, widths U[0.5,2], |c| U[0,5], arg c U[0,2pi)."""
    centres = rng.uniform(-3.0, 3.0, size=(nterms, 2))
    widths = rng.uniform(0.5, 2.0, size=nterms)
    mags = rng.uniform(0.0, 5.0, size=nterms)
    args = rng.uniform(0.0, 2.0 * np.pi, size=nterms)
    return centres, widths, mags * np.exp(1j * args)


def plain_fp64(N: int = 64) -> Workload:
    X, Y = mesh(N, 5.0)
    Q = np.exp(-(X * X + Y * Y)).astype(np.complex128)
    return Workload("plain_fp64", N, 5.0, Q, np.array([0.5 + 0.3j]), M=2, tol=1e-12,
                    mixed=False,
                    description=f"N={N} on [-5pi,5pi]^2, Q=exp(-(x^2+y^2)), k=0.5+0.3i, M=2, FP64")


def batched_fp64(N: int = 512, nk_side: int = 16) -> Workload:
    L = 8.0
    X, Y = mesh(N, L)
    Q = 2.0 * np.exp(-(X * X + Y * Y) / 2.25) * np.exp(0.7j)
    g = np.linspace(-3.0, 3.0, nk_side)
    K1, K2 = np.meshgrid(g, g, indexing="xy")
    k = (K1 + 1j * K2).ravel()
    return Workload("batched_fp64", N, L, Q, k, M=2, tol=1e-12, mixed=False,
                    description=f"N={N} on [-8pi,8pi]^2, Q=2exp(-r^2/2.25)e^(0.7i), "
                                f"{k.size} k on linspace(-3,3,{nk_side})^2, FP64")


def mixed_1024(N: int = 1024, nk: int = 128, seed: int = 7, L: float = 10.0) -> Workload:
    rng = np.random.default_rng(seed)
    centres, widths, amps = draw_mixture(rng, 4)
    Q = gaussian_mixture(N, L, centres, widths, amps)
    mod = np.exp(rng.uniform(np.log(0.1), np.log(8.0), size=nk))
    arg = rng.uniform(0.0, 2.0 * np.pi, size=nk)
    k = mod * np.exp(1j * arg)
    return Workload("mixed_1024", N, L, Q, k, M=2, tol=1e-12, mixed=True,
                    description=f"N={N} on [-{L:g}pi,{L:g}pi]^2, Q=4-Gaussian mixture (seed {seed}), "
                                f"{nk} k with |k| log-uniform [0.1,8], FP32 inner + FP64 refinement")


def small_gaussian(N: int, L: float, k: complex, amp: complex = 1.0, width: float = 1.0) -> Workload:
    """A single centred Gaussian amp*exp(-|z|^2/width^2); the paper's q0 at amp=width=1."""
    X, Y = mesh(N, L)
    Q = amp * np.exp(-(X * X + Y * Y) / (width * width)) * np.ones((N, N), np.complex128)
    return Workload(f"gauss_N{N}", N, L, Q, np.array([complex(k)]), M=2, tol=1e-12)


def random_k_disc(rng: np.random.Generator, nk: int, kmax: float) -> np.ndarray:
    r = kmax * np.sqrt(rng.uniform(0.0, 1.0, size=nk))
    t = rng.uniform(0.0, 2.0 * np.pi, size=nk)
    return r * np.exp(1j * t)


def resolved(N: int, L: float, k: complex, xi_q: float) -> bool:
    """Resolution rule for the k-shift of F(E_k Q): the Fourier support of E_k Q is
    centred at -2i conj(k) (paper Sec. 5.1), so the box half-width N/(2L) must cover
    2 max(|k1|,|k2|) plus the radius xi_q beyond which |Q^| is negligible."""
    return N / (2.0 * L) >= 2.0 * max(abs(k.real), abs(k.imag)) + xi_q


def mixture_request(seed: int, N: int, L: float, kmax: float, nterms_max: int = 6):
    """One serving request: a Gaussian mixture of 1..nterms_max terms and a k with
    |k| log-uniform in [0.1, kmax], both drawn from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    nterms = int(rng.integers(1, nterms_max + 1))
    centres, widths, amps = draw_mixture(rng, nterms)
    k = np.exp(rng.uniform(np.log(0.1), np.log(kmax))) * np.exp(1j * rng.uniform(0.0, 2.0 * np.pi))
    return gaussian_mixture(N, L, centres, widths, amps), complex(k)


SERVING_SIZES = (256, 512, 1024, 2048)


def serving_request(i: int, base_seed: int = 5, L: float = 6.0, kmax: float = 20.0, xi_q: float = 20.0,
                    sizes=SERVING_SIZES):
    """Request i of the serving stream, drawn from default_rng(base_seed + i): N uniform
    over `sizes`, then 1-6 Gaussian terms (drawn as in draw_mixture), then k with |k|
    log-uniform in [0.1, kmax] and arg k U[0, 2pi).  N is raised to the smallest size
    that resolves E_k Q: N/(2L) >= 2 max(|k1|, |k2|) + xi_q.  Returns (N, k, mixture),
    mixture = (centres, widths, amps) for gaussian_mixture."""
    rng = np.random.default_rng(base_seed + i)
    N = int(rng.choice(np.asarray(sizes)))
    nterms = int(rng.integers(1, 7))
    mixture = draw_mixture(rng, nterms)
    k = complex(np.exp(rng.uniform(np.log(0.1), np.log(kmax))) * np.exp(1j * rng.uniform(0.0, 2.0 * np.pi)))
    while N < max(sizes) and N / (2.0 * L) < 2.0 * max(abs(k.real), abs(k.imag)) + xi_q:
        N *= 2
    return N, k, mixture


def poisson_arrivals(rate: float, duration: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of `rate` per second over `duration` s."""
    rng = np.random.default_rng(seed)
    n = int(rate * duration * 1.5) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    return t[t < duration]


def uneven_potentials(N: int, L: float):
    """The two potentials of the uneven-batch workload on an N-grid: a Gaussian
    exp(-(x^2+y^2)) and exp(-(x^2+y^2)^2/4)(1 + 0.3 cos 3x)."""
    X, Y = mesh(N, L)
    r2 = X * X + Y * Y
    qa = np.exp(-r2).astype(np.complex128)
    qb = (np.exp(-r2 * r2 / 4.0) * (1.0 + 0.3 * np.cos(3.0 * X))).astype(np.complex128)
    return qa, qb


def uneven_batch(n: int = 1000, seed: int = 11, L: float = 4.0, kmax: float = 12.0,
                 xi_q=(12.5, 18.0)):
    """Uneven batch: N drawn from {128,256,512,1024,2048} with weights
    .3/.3/.2/.15/.05; request i uses potential i mod 2; k uniform in the disc
    |k| <= kmax, rejection-sampled (up to 64 draws) until the N-grid resolves the
    shifted support of F(E_k Q) (resolved(N, L, k, xi_q[potential])); when no draw
    fits, N is doubled and the draws continue (2048 resolves every k here)."""
    rng = np.random.default_rng(seed)
    sizes = np.array([128, 256, 512, 1024, 2048])
    Ns = rng.choice(sizes, size=n, p=[0.3, 0.3, 0.2, 0.15, 0.05])
    out = []
    for i in range(n):
        N = int(Ns[i])
        pot = i % 2
        tries = 0
        while True:
            k = complex(random_k_disc(rng, 1, kmax)[0])
            if resolved(N, L, k, xi_q[pot]):
                break
            tries += 1
            if tries >= 64 and N < 2048:
                N, tries = 2 * N, 0
        out.append((N, pot, k))
    return out


def reflection_grid(N: int = 128, L: float = 3.2, xi_q: float = 12.5, full: bool = False):
    """DS II reflection-coefficient workload (Sec. 6): initial data q = exp(-(x^2+y^2))
    (the paper's Sec. 6 example, N = 128 and L = 3.2 as in its reconstruction table)
    and k on the xi-grid (k and xi are dual in Sec. 6's k/2 convention), restricted to
    the k the grid resolves: E_{k/2} shifts the Fourier support of q by (k2, k1), so
    max(|k1|, |k2|) + xi_q <= N/(2L) with xi_q = 12.5 (beyond it |q^| < 1e-16 max).
    full=True: every k of the xi-grid (N^2 values; the iterated equation of Sec. 5
    resolves them all).  Returns (Q [N][N] complex128, k [nk] complex128, M = 11)."""
    X, Y = mesh(N, L)
    Q = np.exp(-(X * X + Y * Y)).astype(np.complex128)
    mmax = int(math.floor((N / (2.0 * L) - xi_q) * L))
    m = np.arange(-mmax, mmax + 1)
    if full:
        m = np.arange(-N // 2 + 1, N // 2 + 1)
    K1, K2 = np.meshgrid(m / L, m / L, indexing="xy")
    return Q, (K1 + 1j * K2).ravel(), 11


BY_NAME = {
    "plain_fp64": plain_fp64,
    "batched_fp64": batched_fp64,
    "mixed_1024": mixed_1024,
}


def describe(w: Workload) -> dict:
    return {"workload": w.name, "N": w.N, "L": w.L, "nk": int(w.k.size), "M": w.M,
            "tol": w.tol, "mixed": w.mixed, "desc": w.description,
            "box": f"[-{w.L:g}pi,{w.L:g}pi]^2", "h": 2 * math.pi * w.L / w.N}
