"""Seeded synthetic inputs for the Lax--Oleinik solver.

This module holds no arithmetic of the scheme itself: it only draws the
random trigonometric potentials V, initial data u0 and parameters (P, dx, h,
window W, step count) that both the CUDA library and the CPU oracle consume.
Every field is generated once on the host in binary64 with numpy's
``default_rng``; trigonometric series are evaluated as separable products of
complex exponentials (so a 256^3 field costs a few tensor contractions).

Workloads (shapes and distributions follow the paper's own use: smooth
periodic potentials on the torus, Sec. 3 hypothesis (iii); mechanical
Hamiltonian H = 1/2|p+P|^2 + V, eq. HPV):

  line256   1D, N=256, dx=1/256, P=0.3, V = sum_{k=1..4} a_k cos(2 pi k x + phi_k),
            a_k ~ U(-1/2,1/2)/k, phi_k ~ U(0, 2 pi); u0 = 0; h = 0.05; full
            periodic window; 200 steps.                                     seed 1
  grid1024  2D 1024^2, dx=1/1024, P=(0.3,0.1); V random real Fourier series
            over modes 0<|k|_inf<=6 (half plane, cos and sin coefficients
            ~ N(0, 0.25/|k|^2), |k| Euclidean); u0 the same law over modes <= 4;
            h = 0.02, W = 64; 1000 steps.                                   seed 2
  cube256   3D 256^3, dx=1/256, P=(0.2,-0.1,0.35); V over modes <=4 with
            coefficients ~ N(0, 0.2/|k|^2); u0 = 0; h = 0.02, W = 32; 500 steps.
                                                                            seed 3
  sweep512  512 2D instances, N_i uniform in {128,192,...,512}, dx = 1/N_i,
            P_i ~ U([-1,1]^2), V_i = sum over 0<|k|_inf<=4 (half plane) of
            a_k cos(2 pi k.x + phi_k), a_k ~ U(-1/2,1/2)/|k|, phi_k ~ U(0,2 pi);
            u0 = 0; h = 0.02; W = N_i/16; 2500 steps (T = 50).   seed [4, i]
  adjoint512 2D 512^2, dx=1/512, h = 0.02, W = 32, 2000 steps, P = (0.3,0.1);
            V = sum of 64 coefficients on the basis {cos,sin}(2 pi k1 x) *
            {cos,sin}(2 pi k2 y), k1,k2 in 1..4, initial values
            ~ N(0, 0.25/|k|^2); u0 = 0; checkpoint every 100 steps.          seed 5

  pendulum  the paper's Sec. 5.1 experiment: 1D on (0, 2 pi], 2K points
            x_i = (i+1) pi/K, P = 0, V = 1 - cos x, u0 = cos x, T = 8, time
            step tau = sqrt(dx) rounded down so that an integer number of
            steps ends at T.  Deterministic.
  tdep      the paper's Sec. 5.2 experiment: as pendulum with P = 1 and the
            time-dependent V(t, x) = cos(2x) sin(t), read at t_n = n tau for
            the step n -> n+1 (one row of V per step).  Deterministic.

Every builder takes optional overrides (grid size, steps) so the same laws
give small cases for tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["Problem", "line256", "grid1024", "cube256", "sweep512", "adjoint512",
           "adjoint_basis", "trig_field", "pendulum", "tdep", "integral128", "WORKLOADS"]


@dataclass
class Problem:
    """One instance of the scheme: grid, steps, parameters and fields."""
    name: str
    shape: tuple
    dx: tuple
    h: float
    P: tuple
    W: tuple                      # per axis; 0 = full periodic window
    nsteps: int
    u0: np.ndarray                # float64, shape `shape`
    V: np.ndarray | None          # float64, shape `shape` (time-independent), or
                                  # (nsteps, *shape) when extra["V_per_step"]
    extra: dict = field(default_factory=dict)

    @property
    def V_per_step(self) -> bool:
        return bool(self.extra.get("V_per_step", False))

    @property
    def npts(self) -> int:
        return int(np.prod(self.shape))

    @property
    def ndim(self) -> int:
        return len(self.shape)


def _half_space_modes(ndim: int, K: int) -> np.ndarray:
    """Integer modes k with 0 < |k|_inf <= K, one of each +-k pair (the first
    nonzero coordinate positive), in a fixed lexicographic order."""
    out = []
    for k in np.ndindex(*([2 * K + 1] * ndim)):
        kk = tuple(int(c) - K for c in k)
        nz = [c for c in kk if c != 0]
        if not nz or nz[0] < 0:
            continue
        out.append(kk)
    return np.array(out, dtype=np.int64).reshape(-1, ndim)


def trig_field(shape, modes: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """Real field  sum_m Re(coef_m * exp(2 pi i k_m . x)),  x_a = i_a / shape[a].

    Evaluated separably: a dense coefficient tensor over the mode box is
    contracted with one 1D exponential table per axis."""
    shape = tuple(int(s) for s in shape)
    ndim = len(shape)
    K = int(np.abs(modes).max()) if modes.size else 0
    C = np.zeros([2 * K + 1] * ndim, dtype=np.complex128)
    for k, c in zip(modes, coef):
        C[tuple(int(x) + K for x in k)] += c
    out = C
    for a in range(ndim):
        n = shape[a]
        ks = np.arange(-K, K + 1)
        E = np.exp(2j * np.pi * np.outer(ks, np.arange(n)) / n)      # (2K+1, n)
        out = np.tensordot(out, E, axes=([0], [0]))                   # moves axis to the end
    return np.ascontiguousarray(out.real)


def _fourier_gauss(rng, shape, K: int, var_num: float) -> np.ndarray:
    modes = _half_space_modes(len(shape), K)
    norm = np.sqrt((modes.astype(np.float64) ** 2).sum(axis=1))
    std = np.sqrt(var_num) / norm
    a = rng.normal(0.0, 1.0, len(modes)) * std
    b = rng.normal(0.0, 1.0, len(modes)) * std
    # a cos(t) + b sin(t) = Re((a - i b) e^{it})
    return trig_field(shape, modes, a - 1j * b)


def _fourier_phase(rng, shape, K: int) -> np.ndarray:
    modes = _half_space_modes(len(shape), K)
    norm = np.sqrt((modes.astype(np.float64) ** 2).sum(axis=1))
    amp = rng.uniform(-0.5, 0.5, len(modes)) / norm
    phi = rng.uniform(0.0, 2.0 * np.pi, len(modes))
    return trig_field(shape, modes, amp * np.exp(1j * phi))


def line256(N: int = 256, nsteps: int = 200, seed: int = 1) -> Problem:
    rng = np.random.default_rng(seed)
    k = np.arange(1, 5)
    a = rng.uniform(-0.5, 0.5, 4) / k
    phi = rng.uniform(0.0, 2.0 * np.pi, 4)
    V = trig_field((N,), k.reshape(-1, 1), a * np.exp(1j * phi))
    return Problem("line256", (N,), (1.0 / N,), 0.05, (0.3,), (0,), nsteps,
                   np.zeros(N), V)


def grid1024(N: int = 1024, nsteps: int = 1000, W: int = 64, seed: int = 2) -> Problem:
    rng = np.random.default_rng(seed)
    V = _fourier_gauss(rng, (N, N), 6, 0.25)
    u0 = _fourier_gauss(rng, (N, N), 4, 0.25)
    return Problem("grid1024", (N, N), (1.0 / N,) * 2, 0.02, (0.3, 0.1), (W, W), nsteps, u0, V)


def cube256(N: int = 256, nsteps: int = 500, W: int = 32, seed: int = 3) -> Problem:
    rng = np.random.default_rng(seed)
    V = _fourier_gauss(rng, (N, N, N), 4, 0.2)
    return Problem("cube256", (N, N, N), (1.0 / N,) * 3, 0.02, (0.2, -0.1, 0.35), (W, W, W),
                   nsteps, np.zeros((N, N, N)), V)


SWEEP_SIZES = tuple(range(128, 513, 64))


def sweep512(count: int = 512, nsteps: int = 2500, sizes=SWEEP_SIZES, seed: int = 4,
             first: int = 0) -> list[Problem]:
    out = []
    for i in range(first, first + count):
        rng = np.random.default_rng([seed, i])
        N = int(rng.choice(np.asarray(sizes)))
        P = tuple(float(x) for x in rng.uniform(-1.0, 1.0, 2))
        V = _fourier_phase(rng, (N, N), 4)
        out.append(Problem("sweep512[%d]" % i, (N, N), (1.0 / N,) * 2, 0.02, P,
                           (N // 16, N // 16), nsteps, np.zeros((N, N)), V))
    return out


def adjoint_basis(N: int) -> np.ndarray:
    """64 basis fields f_s1(2 pi k1 x) f_s2(2 pi k2 y), k1,k2 in 1..4,
    (s1,s2) in {cos,sin}^2; shape (64, N, N), order (k1, k2, s1, s2)."""
    x = np.arange(N) / N
    f = []
    for k in range(1, 5):
        f.append(np.cos(2 * np.pi * k * x))
        f.append(np.sin(2 * np.pi * k * x))
    f = np.array(f).reshape(4, 2, N)          # [k, s, x]
    B = np.einsum("asx,bty->abstxy", f, f).reshape(64, N, N)
    return np.ascontiguousarray(B)


def adjoint512(N: int = 512, nsteps: int = 2000, W: int = 32, seed: int = 5) -> Problem:
    rng = np.random.default_rng(seed)
    k1, k2 = np.meshgrid(np.arange(1, 5), np.arange(1, 5), indexing="ij")
    norm = np.sqrt(k1 ** 2 + k2 ** 2).astype(np.float64)                # (4,4)
    std = np.repeat(np.repeat((0.5 / norm)[:, :, None, None], 2, 2), 2, 3).reshape(64)
    coef = rng.normal(0.0, 1.0, 64) * std
    B = adjoint_basis(N)
    V = np.tensordot(coef, B, axes=(0, 0))
    return Problem("adjoint512", (N, N), (1.0 / N,) * 2, 0.02, (0.3, 0.1), (W, W), nsteps,
                   np.zeros((N, N)), np.ascontiguousarray(V),
                   extra={"coef": coef, "checkpoint_every": 100})


def _paper_1d(name: str, K: int, T: float, speed: float, P: float, nsteps: int | None):
    """Common grid of the two 1D experiments (Sec. 5): 2K points on (0, 2 pi],
    dx = pi/K, tau <= sqrt(dx) with n tau = T exactly, and a window of
    displacements wide enough for velocities up to `speed` (W = 0, the full
    periodic window, when that covers the torus)."""
    N = 2 * int(K)
    dx = np.pi / K
    n = int(np.ceil(T / np.sqrt(dx) - 1e-12)) if nsteps is None else int(nsteps)
    tau = T / n
    W = int(np.ceil(speed * tau / dx)) + 1
    if 2 * W + 1 >= N:
        W = 0
    x = (np.arange(N) + 1.0) * dx
    return N, dx, tau, n, W, x


def pendulum(K: int = 4096, T: float = 8.0, speed: float = 4.0, nsteps: int | None = None) -> Problem:
    N, dx, tau, n, W, x = _paper_1d("pendulum", K, T, speed, 0.0, nsteps)
    return Problem("pendulum", (N,), (dx,), tau, (0.0,), (W,), n, np.cos(x), 1.0 - np.cos(x),
                   extra={"K": K, "T": tau * n, "x": x})


def tdep(K: int = 4096, T: float = 8.0, speed: float = 4.0, nsteps: int | None = None) -> Problem:
    N, dx, tau, n, W, x = _paper_1d("tdep", K, T, speed, 1.0, nsteps)
    t = np.arange(n) * tau
    V = np.sin(t)[:, None] * np.cos(2.0 * x)[None, :]
    return Problem("tdep", (N,), (dx,), tau, (1.0,), (W,), n, np.cos(x), np.ascontiguousarray(V),
                   extra={"K": K, "T": tau * n, "x": x, "V_per_step": True})


def integral128(N: int = 128, nsteps: int = 100, W: int = 4, K: int = 2, seed: int = 6) -> Problem:
    """The first discrete semigroup's workload (eq. cost1): 2D N^2 torus,
    dx = 1/N, h = 0.02, P = (0.3, 0.1), W per axis; V a Fourier series over
    the half-plane modes 0 < |k|_inf <= K with cos and sin coefficients
    ~ N(0, 0.25/|k|^2) (the 1024^2 law's, fewer modes), stored as complex
    c_k = a_k - i b_k so that V = Re sum c_k exp(2 pi i k.x); u0 = 0."""
    rng = np.random.default_rng(seed)
    modes = _half_space_modes(2, K)
    norm = np.sqrt((modes.astype(np.float64) ** 2).sum(axis=1))
    a = rng.normal(0.0, 1.0, len(modes)) * np.sqrt(0.25) / norm
    b = rng.normal(0.0, 1.0, len(modes)) * np.sqrt(0.25) / norm
    coef = a - 1j * b
    return Problem("integral128", (N, N), (1.0 / N,) * 2, 0.02, (0.3, 0.1), (W, W), nsteps,
                   np.zeros((N, N)), None, extra={"modes": modes, "coef": coef})


WORKLOADS = {"line256": line256, "grid1024": grid1024, "cube256": cube256,
             "adjoint512": adjoint512}
