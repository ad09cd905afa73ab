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


def _key_log2(n: int) -> int:
    return max(int(n), 1).bit_length() - 1


def tune_problems(count: int, seed: int, part: str = "all") -> list:
    """Seeded shapes for schedule tuning, drawn from the benchmark families:
      reduce     log2 n in [10, 27]: the whole array, per-group outputs
                 (group(k)[[block]]), the hierarchical view
                 group(1024)[[block]].group(32)[[warp]][[thread]] reduced per
                 grid or per block, a reversed array per group, or the columns
                 of a row-major matrix (transpose view, one output per column)
      scan       log2 n in [10, 27]: the whole array, per-group segments
                 (group(k)[[block]]), a reversed array, or a split-off tail
      transpose  rows, cols powers of two, 2^10 <= rows * cols <= 2^26
      segmented  10..5000 segments, log-uniform lengths up to 2^8..2^16
      matmul     M, N, K multiples of 128 in [256, 4096], log-uniform
    Sizes are drawn continuously (not only powers of two).  part "even" keeps
    the problems whose floor(log2 n) is even (n: the points reduced or
    scanned, the matrix elements, the segmented elements, or M), "odd" the
    others, so that the two parts share no size bucket; "all" keeps all.
    Each item: dict(op, dtype, n, aux, lengths, k, view, grid, block, level)
    with op 0..4 as in desc_op; view = (base_shape, ops) or None."""
    key = stream_key(seed, 1234)
    out = []
    i = 0
    GRID_, BLOCK_, WARP_, THREAD_ = 0, 1, 2, 3
    while len(out) < count:
        a = _unit_f64(splitmix64(key, 8 * i, 8)).tolist()
        i += 1
        op = min(int(a[0] * 5), 4)
        pr = dict(op=op, dtype=1, n=0, aux=0, lengths=None, k=0, view=None, grid=None, block=None, level=GRID_)
        if op == 4:
            M, N, K = (128 * max(2, int(2 ** (8 + a[j] * 4.0) / 128)) for j in (2, 3, 4))
            pr.update(n=M, aux=N, k=K)
            kn = M
        elif op == 2:
            dtype = 1
            lr = 5 + int(a[2] * 10)
            lc = 5 + int(a[3] * 10)
            while lr + lc > 26:
                lr, lc = lr - 1, lc - 1
            while lr + lc < 10:
                lr, lc = lr + 1, lc + 1
            pr.update(n=(1 << lr) * (1 << lc), aux=1 << lr)
            kn = pr["n"]
        elif op == 3:
            pr["dtype"] = 0 if a[1] < 0.5 else 1
            nseg = 10 + int(a[2] * 4990)
            mx = 1 << (8 + int(a[3] * 9))
            L = loguniform_lengths(nseg, seed=seed * 100003 + i, max_len=mx)
            pr.update(n=int(L.sum()), aux=nseg, lengths=L)
            kn = pr["n"]
        elif op == 0:
            pr["dtype"] = 0 if a[1] < 0.5 else 1
            n = 1024 * max(1, int(2 ** (a[2] * 17.0)))        # 2^10 .. 2^27, a multiple of 1024
            fam = min(int(a[3] * 5), 4)
            kn = n
            if fam == 0:
                pr.update(n=n)
            elif fam == 1:
                g = 1 << int(a[4] * min(_key_log2(n) - 2, 14))
                while n % g:
                    g //= 2
                pr.update(n=n, aux=g if g > 1 else 0)
            elif fam == 2:
                lvl = GRID_ if a[4] < 0.5 else BLOCK_
                ops = [("group", 1024, 0), ("select", BLOCK_, 0), ("group", 32, 0), ("select", WARP_, 0),
                       ("select", THREAD_, 0)]
                pr.update(n=n, view=([n], ops), grid=(n // 1024, 1, 1), block=(1024, 1, 1), level=lvl)
            elif fam == 3:
                k = 1 << (4 + int(a[4] * 10))
                while n % k:
                    k //= 2
                ops = [("reverse", 0), ("group", k, 0), ("select", BLOCK_, 0)]
                pr.update(n=n, view=([n], ops), grid=(n // k, 1, 1), block=(1, 1, 1), level=BLOCK_)
            else:
                C = 1 << (4 + int(a[4] * 8))
                while n % C:
                    C //= 2
                R = n // C
                ops = [("transpose", 0), ("select", BLOCK_, 0)]
                pr.update(n=n, view=([R, C], ops), grid=(C, 1, 1), block=(1, 1, 1), level=BLOCK_)
        else:
            pr["dtype"] = 0 if a[1] < 0.5 else 1
            n = 1024 * max(1, int(2 ** (a[2] * 17.0)))        # 2^10 .. 2^27
            fam = min(int(a[3] * 4), 3)
            kn = n
            if fam == 0:
                pr.update(n=n)
            elif fam == 1:
                k = 1 << (10 + int(a[4] * 8))
                while n % k:
                    k //= 2
                ops = [("group", k, 0), ("select", BLOCK_, 0)]
                pr.update(n=n, view=([n], ops), grid=(n // k, 1, 1), block=(1, 1, 1), level=BLOCK_)
            elif fam == 2:
                pr.update(n=n, view=([n], [("reverse", 0)]))
            else:
                s0 = 1 + int(a[4] * (n // 2))
                pr.update(n=n, view=([n], [("split_snd", s0, 0)]))
                kn = n - s0
        if part == "even" and _key_log2(kn) % 2 != 0:
            continue
        if part == "odd" and _key_log2(kn) % 2 != 1:
            continue
        out.append(pr)
    return out
