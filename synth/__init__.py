"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module only draws numbers; it holds none of the arithmetic of the
reductions, scans, transposes or products that the library computes.  Both the
CUDA path and the CPU oracle are fed from here, and neither imports the other.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) in counter form.  For a (seed, stream) pair a
key is drawn once, and element i is

    z_i = key + (i + 1) * GAMMA  (mod 2^64),   u_i = mix(z_i)

with the published GAMMA and mix constants.  Everything runs as torch int64
arithmetic (two's-complement wrap, logical shifts emulated with a mask), so the
same call gives the same bits on the CPU and on a GPU.  Large draws are made in
chunks so the device never holds more than a few chunk-sized temporaries.

Value recipes (the workloads of the reduce/scan/transpose/matmul benchmarks):
  ints_pm1000      integers uniform in [-1000, 1000]: ((u >> 11) mod 2001) - 1000
  uniform_grid     FP32 uniform in [-1, 1) on the grid k * 2^-23:
                   k = (u >> 40) - 2^23, x = k * 2^-23 (exact in FP32)
  normal_f32       N(0, 1) by Box-Muller from two streams, computed in FP64
                   and rounded to FP32
  loguniform_lengths  floor(exp(U * ln(2^20 + 1))) clipped to [1, 2^20]
"""
from __future__ import annotations

import math

import torch

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
_CHUNK = 1 << 24


def _s64(c: int) -> int:
    c &= (1 << 64) - 1
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _lsr(z, 30)) * _s64(MIX1)
    z = (z ^ _lsr(z, 27)) * _s64(MIX2)
    return z ^ _lsr(z, 31)


def _mix_int(z: int) -> int:
    m = (1 << 64) - 1
    z &= m
    z = ((z ^ (z >> 30)) * MIX1) & m
    z = ((z ^ (z >> 27)) * MIX2) & m
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int = 0) -> int:
    return _mix_int(seed * GAMMA + stream)


def splitmix64(key: int, start: int, count: int, device="cpu") -> torch.Tensor:
    """u_i for i in [start, start+count) as int64 bit patterns of uint64."""
    i = torch.arange(start, start + count, dtype=torch.int64, device=device)
    z = (i + 1) * _s64(GAMMA) + _s64(key)
    return _mix(z)


def _chunked(n: int, out: torch.Tensor, fill) -> torch.Tensor:
    for s in range(0, n, _CHUNK):
        c = min(_CHUNK, n - s)
        out[s:s + c] = fill(s, c)
    return out


def ints_pm1000(n: int, seed: int, stream: int = 0, device="cpu") -> torch.Tensor:
    key = stream_key(seed, stream)
    out = torch.empty(n, dtype=torch.int32, device=device)
    return _chunked(n, out, lambda s, c: (_lsr(splitmix64(key, s, c, device), 11) % 2001 - 1000).to(torch.int32))


def uniform_grid(n: int, seed: int, stream: int = 0, device="cpu") -> torch.Tensor:
    key = stream_key(seed, stream)
    out = torch.empty(n, dtype=torch.float32, device=device)
    scale = 2.0 ** -23

    def fill(s, c):
        k = _lsr(splitmix64(key, s, c, device), 40) - (1 << 23)
        return k.to(torch.float32) * scale
    return _chunked(n, out, fill)


def _unit_f64(u: torch.Tensor) -> torch.Tensor:
    """[0, 1) with 53 random bits."""
    return _lsr(u, 11).to(torch.float64) * (2.0 ** -53)


def normal_f32(n: int, seed: int, stream: int = 0, device="cpu") -> torch.Tensor:
    ka, kb = stream_key(seed, 2 * stream + 1000), stream_key(seed, 2 * stream + 1001)
    out = torch.empty(n, dtype=torch.float32, device=device)

    def fill(s, c):
        u1 = 1.0 - _unit_f64(splitmix64(ka, s, c, device))   # (0, 1]
        u2 = _unit_f64(splitmix64(kb, s, c, device))
        return (torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)).to(torch.float32)
    return _chunked(n, out, fill)


def loguniform_lengths(count: int, seed: int, max_len: int = 1 << 20, stream: int = 7,
                       device="cpu") -> torch.Tensor:
    key = stream_key(seed, stream)
    u = _unit_f64(splitmix64(key, 0, count, device))
    L = torch.floor(torch.exp(u * math.log(max_len + 1.0))).to(torch.int64)
    return L.clamp_(1, max_len)


def offsets_from_lengths(lengths: torch.Tensor) -> torch.Tensor:
    """CSR offsets [S+1] (int64) of back-to-back segments."""
    off = torch.zeros(lengths.numel() + 1, dtype=torch.int64, device=lengths.device)
    off[1:] = torch.cumsum(lengths.to(torch.int64), 0)
    return off


def mlp_init(F: int, H: int, seed: int) -> torch.Tensor:
    """Initial cost-model parameters (FP32, flat [W1, b1, W2, b2, w3, b3]):
    uniform weights scaled by sqrt(6 / fan_in), zero biases."""
    key = stream_key(seed, 99)
    n_w = [H * F, H * H, H]
    fan = [F, H, H]
    u = [(_unit_f64(splitmix64(key, sum(n_w[:i]), n_w[i])) * 2.0 - 1.0) * math.sqrt(6.0 / fan[i])
         for i in range(3)]
    z = torch.zeros(H, dtype=torch.float64)
    return torch.cat([u[0], z, u[1], z, u[2], torch.zeros(1, dtype=torch.float64)]).to(torch.float32)


def tune_problems(count: int, seed: int) -> list:
    """Seeded shapes for schedule tuning, drawn from the benchmark families:
    reduce (full or per-group, log2 n in [10, 27]), scan (log2 n in [10, 27]),
    transpose (rows, cols powers of two, 2^10 <= rows * cols <= 2^26),
    segmented (10..5000 segments, log-uniform lengths up to 2^8..2^16),
    matmul (M, N, K each 2^8..2^12, FP32 operands; n = M, aux = N, k = K).
    Each item: dict(op, dtype, n, aux, lengths, k) with op 0..4 as in desc_op."""
    u = _unit_f64(splitmix64(stream_key(seed, 1234), 0, 8 * count)).reshape(count, 8).tolist()
    out = []
    for i in range(count):
        a = u[i]
        op = min(int(a[0] * 5), 4)
        if op == 4:
            M, N, K = (1 << (8 + int(a[j] * 5)) for j in (2, 3, 4))
            out.append(dict(op=4, dtype=1, n=M, aux=N, lengths=None, k=K))
            continue
        dtype = 0 if a[1] < 0.5 else 1
        if op == 0:
            ln = 10 + int(a[2] * 18)
            n = 1 << ln
            aux = 0 if a[3] < 0.5 else 1 << int(a[4] * min(ln - 2, 14))
            out.append(dict(op=0, dtype=dtype, n=n, aux=aux, lengths=None))
        elif op == 1:
            n = int(2 ** (10 + a[2] * 17.0))
            out.append(dict(op=1, dtype=dtype, n=n, aux=0, lengths=None))
        elif op == 2:
            lr = 5 + int(a[2] * 10)
            lc = 5 + int(a[3] * 10)
            while lr + lc > 26:
                lr, lc = lr - 1, lc - 1
            while lr + lc < 10:
                lr, lc = lr + 1, lc + 1
            out.append(dict(op=2, dtype=1, n=(1 << lr) * (1 << lc), aux=1 << lr, lengths=None))
        else:
            nseg = 10 + int(a[2] * 4990)
            mx = 1 << (8 + int(a[3] * 9))
            L = loguniform_lengths(nseg, seed=seed * 100003 + i, max_len=mx)
            out.append(dict(op=3, dtype=dtype, n=int(L.sum()), aux=nseg, lengths=L))
    return out
