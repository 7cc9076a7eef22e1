"""Seeded synthetic snapshot generators (inputs only; none of the method's arithmetic).

These stand in for the paper's flow-field data (the Burgers solution and ERA5
surface pressure of Sec. 4.3).  The same module feeds both the CUDA library and the
FP64 oracle; parity tests generate on the CPU and hand identical bits to both.
Everything is plain PyTorch so one recipe runs on CPU (tests) or GPU (benchmark
inputs too large for host memory); the two devices draw different random bits.

Recipes (where the workload description leaves a parameter open, the reading taken is stated):

* ``low_rank``: A = U0 diag(s) V0^T + noise, U0 (M x r) and V0 (N x r) orthonormal
  from seeded Gaussian matrices + QR, s_i = 10^(-i/8) for i = 0..r-1, i.i.d.
  N(0, noise_std^2) noise.
* ``TravellingWaves``: snapshot t is sum_j a_j g_j sin(w_j t + phi_j) + noise with
  a_j = j^(-decay), g_j a periodic Gaussian random field on an (ny x nx) grid
  (white noise smoothed by a separable Gaussian kernel of std corr_len/sqrt(2),
  scaled to unit RMS, flattened row-major), w_j ~ U(0.01, 0.5) rad per snapshot,
  phi_j ~ U(0, 2 pi), noise N(0, noise_std^2) drawn per batch from (seed, batch).
* ``spectrum``: A = U0 diag(s) V0^T with a prescribed spectrum s (e.g. 1.15^-i).
* ``burgers``: the analytic viscous Burgers solution of Sec. 4.3,
  u(x, t) = (x/(t+1)) / (1 + sqrt((t+1)/t0) exp(Re x^2 / (4t+4))), t0 = exp(Re/8),
  on x = linspace(0, 1, M), t = linspace(0, 2, N), evaluated in float64.
* ``partition_sizes``: uneven row-block sizes drawn uniformly from [lo, hi].
"""
from __future__ import annotations

import math

import torch


def _gen(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def orthonormal(rows: int, cols: int, seed: int, device="cpu") -> torch.Tensor:
    """rows x cols float64 matrix with orthonormal columns (Gaussian, then QR)."""
    g = _gen(seed, device)
    X = torch.randn(rows, cols, generator=g, dtype=torch.float64, device=device)
    Q, R = torch.linalg.qr(X)
    return Q * torch.sign(torch.diagonal(R))[None, :]


def low_rank(M: int, N: int, rank: int, noise_std: float, seed: int, s=None):
    """Returns (A float64 M x N, U0, s, V0) for A = U0 diag(s) V0^T + noise."""
    U0 = orthonormal(M, rank, seed)
    V0 = orthonormal(N, rank, seed + 1)
    if s is None:
        s = torch.tensor([10.0 ** (-i / 8.0) for i in range(rank)], dtype=torch.float64)
    else:
        s = torch.as_tensor(s, dtype=torch.float64)
    A = (U0 * s[None, :]) @ V0.T
    if noise_std > 0:
        A = A + noise_std * torch.randn(M, N, generator=_gen(seed + 2), dtype=torch.float64)
    return A, U0, s, V0


def spectrum(M: int, N: int, s, seed: int):
    """A = U0 diag(s) V0^T (no noise) with a prescribed spectrum s (len <= min(M, N))."""
    s = torch.as_tensor(s, dtype=torch.float64)
    U0 = orthonormal(M, s.numel(), seed)
    V0 = orthonormal(N, s.numel(), seed + 1)
    return (U0 * s[None, :]) @ V0.T, U0, s, V0


def gaussian_random_fields(ny: int, nx: int, nmodes: int, corr_len: float, seed: int,
                           device="cpu", dtype=torch.float64) -> torch.Tensor:
    """(ny*nx) x nmodes matrix of unit-RMS periodic Gaussian random fields (row-major)."""
    g = _gen(seed, device)
    sd = corr_len / math.sqrt(2.0)
    ky = torch.fft.fftfreq(ny, device=device, dtype=torch.float64)
    kx = torch.fft.rfftfreq(nx, device=device, dtype=torch.float64)
    # Fourier transform of a unit-mass Gaussian kernel of std sd (cells)
    filt = torch.exp(-2.0 * (math.pi * sd) ** 2 * (ky[:, None] ** 2 + kx[None, :] ** 2))
    out = torch.empty(ny * nx, nmodes, device=device, dtype=dtype)
    for j in range(nmodes):
        w = torch.randn(ny, nx, generator=g, device=device, dtype=torch.float64)
        f = torch.fft.irfft2(torch.fft.rfft2(w) * filt, s=(ny, nx))
        f = f / torch.sqrt(torch.mean(f * f))
        out[:, j] = f.reshape(-1).to(dtype)
    return out


class TravellingWaves:
    """Sum of separable travelling-wave modes plus noise, batch by batch."""

    def __init__(self, ny: int, nx: int, nmodes: int, decay: float, noise_std: float,
                 seed: int, corr_len: float = 16.0, device="cpu", dtype=torch.float64):
        self.M = ny * nx
        self.nmodes = nmodes
        self.noise_std = noise_std
        self.seed = seed
        self.device = device
        self.dtype = dtype
        self.G = gaussian_random_fields(ny, nx, nmodes, corr_len, seed, device, dtype)
        g = _gen(seed + 7919)
        j = torch.arange(1, nmodes + 1, dtype=torch.float64)
        self.amp = j ** (-decay)
        self.omega = 0.01 + 0.49 * torch.rand(nmodes, generator=g, dtype=torch.float64)
        self.phase = 2.0 * math.pi * torch.rand(nmodes, generator=g, dtype=torch.float64)

    def coefficients(self, t0: int, B: int) -> torch.Tensor:
        t = torch.arange(t0, t0 + B, dtype=torch.float64)
        return self.amp[:, None] * torch.sin(self.omega[:, None] * t[None, :] + self.phase[:, None])

    def batch(self, index: int, B: int) -> torch.Tensor:
        """Snapshots index*B .. index*B+B-1 as an M x B column-major matrix."""
        Tm = self.coefficients(index * B, B).to(self.device, self.dtype)
        A = self.G @ Tm
        if self.noise_std > 0:
            gn = _gen(self.seed * 1000003 + index + 1, self.device)
            A += self.noise_std * torch.randn(self.M, B, generator=gn, device=self.device,
                                              dtype=self.dtype)
        return A.T.contiguous().T  # column-major storage: each snapshot contiguous


def burgers(M: int = 16384, N: int = 800, Re: float = 1000.0) -> torch.Tensor:
    """Analytic viscous Burgers snapshots (M x N, float64)."""
    x = torch.linspace(0.0, 1.0, M, dtype=torch.float64)[:, None]
    t = torch.linspace(0.0, 2.0, N, dtype=torch.float64)[None, :]
    t0 = math.exp(Re / 8.0)
    return (x / (t + 1.0)) / (1.0 + torch.sqrt((t + 1.0) / t0) * torch.exp(Re * x * x / (4.0 * t + 4.0)))


def partition_sizes(nparts: int, lo: int, hi: int, seed: int) -> list[int]:
    g = _gen(seed)
    return [int(v) for v in torch.randint(lo, hi + 1, (nparts,), generator=g)]


def offsets(sizes) -> list[int]:
    out = [0]
    for s in sizes:
        out.append(out[-1] + int(s))
    return out


def to_storage(A: torch.Tensor, dtype: torch.dtype) -> torch.Tensor:
    """Rounds a float64 batch to the storage dtype (float32 or bfloat16), column-major."""
    return A.to(dtype).T.contiguous().T
