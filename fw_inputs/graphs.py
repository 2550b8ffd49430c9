"""Deterministic graph and query generators (input recipe only).

Graphs are returned as CSR with rows sorted ascending, no self loops and no
duplicate entries:

* ``row_ptr`` int64[n+1], ``col`` int32[m]
* ``w_f32`` float32[m] and ``w_u32`` int32[m] (uint32 bit pattern): the same
  edge weight as a float and as an integer.  For the [1, 5) real weights of the
  paper's workloads (Section 6.1, "Datasets and Workloads") the float sits on a
  2^-14 grid, w = 1 + k * 2^-14 with k in [0, 65536), so it is exact in FP32 and
  its integer companion is w * 2^14 in [16384, 81920).  Integer weights in
  {1..5} are stored unscaled in both arrays.
* ``etype`` int8[m] or None: edge labels uniform in {0..4} (same section).

An undirected edge {u, v} gets one weight and one label, used in both
directions (a hash of (min, max, seed)).

Randomness: ``mix32`` is a 32-bit avalanche permutation (xor-shift /
multiply rounds); every draw is mix32 applied to a (seed, counter) tuple.  All
arithmetic is done on non-negative int64 tensors holding 32-bit values, with
multiplications split so no intermediate exceeds 2^48, so CPU and CUDA agree
bit for bit.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Optional

import torch

MASK32 = 0xFFFFFFFF


def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2^32 for x in [0, 2^32) held in int64, without overflow."""
    c_hi, c_lo = (c >> 16) & 0xFFFF, c & 0xFFFF
    return ((((x * c_hi) & 0xFFFF) << 16) + x * c_lo) & MASK32


def mix32(x: torch.Tensor) -> torch.Tensor:
    """Bijective 32-bit mixer (xor-shift-multiply), elementwise on int64."""
    x = x & MASK32
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    x = x ^ (x >> 16)
    return x


def _mix_const(v: int) -> int:
    return int(mix32(torch.tensor([v & MASK32], dtype=torch.int64))[0])


def _hash2(seed: int, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """32-bit hash of (seed, a, b) with a, b in [0, 2^32)."""
    s = _mix_const(seed * 0x9E3779B9 + 0x632BE5AB)
    return mix32(mix32(a ^ s) ^ b)


@dataclasses.dataclass
class Graph:
    n: int
    m: int
    row_ptr: torch.Tensor          # int64 [n+1]
    col: torch.Tensor              # int32 [m]
    w_f32: torch.Tensor            # float32 [m]
    w_u32: torch.Tensor            # int32 [m], uint32 bit pattern
    etype: Optional[torch.Tensor]  # int8 [m] or None
    name: str = ""

    def to(self, device) -> "Graph":
        return Graph(self.n, self.m, self.row_ptr.to(device), self.col.to(device),
                     self.w_f32.to(device), self.w_u32.to(device),
                     None if self.etype is None else self.etype.to(device), self.name)

    def degrees(self) -> torch.Tensor:
        return self.row_ptr[1:] - self.row_ptr[:-1]

    def manifest(self) -> dict:
        d = self.degrees().to(torch.float64)
        m = max(self.m, 1)
        idx = torch.arange(self.m, device=self.col.device, dtype=torch.int64)
        fp = int(((self.col.to(torch.int64) * ((idx % 1009) + 1)) % 1000000007).sum().item())
        return {
            "name": self.name, "n": self.n, "m": self.m,
            "d_max": int(d.max().item()) if self.n else 0,
            "isolated": int((d == 0).sum().item()),
            "sum_d2_over_sum_d": float((d * d).sum().item() / m),
            "col_fingerprint": fp,
            "w_u32_sum": int(self.w_u32.to(torch.int64).sum().item()),
        }


def _csr_from_sorted_keys(keys: torch.Tensor, n: int):
    """keys = src * n + dst, sorted and unique -> (row_ptr, src, dst)."""
    src = torch.div(keys, n, rounding_mode="floor")
    dst = keys - src * n
    counts = torch.bincount(src, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=keys.device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr, src, dst


def _attributes(src, dst, seed: int, weights: str, types_seed: Optional[int]):
    lo = torch.minimum(src, dst)
    hi = torch.maximum(src, dst)
    h = _hash2(seed * 2 + 1, lo, hi)
    if weights == "int5":
        wu = 1 + h % 5
        w_u32 = wu.to(torch.int32)
        w_f32 = wu.to(torch.float32)
    elif weights == "grid14":
        k = h & 0xFFFF
        wu = 16384 + k
        w_u32 = wu.to(torch.int32)
        w_f32 = (wu.to(torch.float64) / 16384.0).to(torch.float32)
    elif weights.startswith("lognormal"):
        # log-normal weights, mean 0 and standard deviation sigma of the log
        # (Appendix C.1's sweep, sigma = 1..3): Z by Box-Muller from two
        # hashed uniforms, the integer weight round(e^(sigma Z) * 2^14) >= 1,
        # the float that integer times 2^-14 (to FP32 rounding).  float64
        # exp/log/cos may differ in the last bit between CPU and GPU, so this
        # recipe is reproducible per device only.
        sigma = float(weights[len("lognormal"):])
        h2 = _hash2(seed * 2 + 3, lo, hi)
        u1 = (h.to(torch.float64) + 0.5) / 4294967296.0
        u2 = (h2.to(torch.float64) + 0.5) / 4294967296.0
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
        wu = torch.clamp(torch.round(torch.exp(sigma * z) * 16384.0), 1.0, 2147483647.0).to(torch.int64)
        w_u32 = wu.to(torch.int32)
        w_f32 = (wu.to(torch.float64) / 16384.0).to(torch.float32)
    else:
        raise ValueError(f"unknown weights recipe {weights!r}")
    etype = None
    if types_seed is not None:
        etype = (_hash2(types_seed * 2 + 2, lo, hi) % 5).to(torch.int8)
    return w_f32, w_u32, etype


def chung_lu(n: int = 1000, sum_theta: float = 2.0e4, gamma: float = 2.1, seed: int = 1,
             weights: str = "int5", types_seed: Optional[int] = None, device="cpu") -> Graph:
    """Chung-Lu power-law graph.

    Expected degree theta_i proportional to (i+1)^(-1/(gamma-1)), scaled so that
    sum(theta) = sum_theta; undirected edge {i, j}, i < j, present with
    probability min(1, theta_i * theta_j / sum_theta).
    """
    i = torch.arange(n, dtype=torch.float64, device=device)
    theta = (i + 1.0) ** (-1.0 / (gamma - 1.0))
    theta = theta * (sum_theta / theta.sum())
    keys = []
    rows_per_chunk = max(1, (1 << 22) // max(n, 1))
    for r0 in range(0, n, rows_per_chunk):
        r1 = min(n, r0 + rows_per_chunk)
        a = torch.arange(r0, r1, dtype=torch.int64, device=device)[:, None].expand(r1 - r0, n)
        b = torch.arange(n, dtype=torch.int64, device=device)[None, :].expand(r1 - r0, n)
        mask = b > a
        a, b = a[mask], b[mask]
        p = torch.clamp(theta[a] * theta[b] / sum_theta, max=1.0)
        u = _hash2(seed * 2, a, b).to(torch.float64) * (1.0 / 4294967296.0)
        keep = u < p
        a, b = a[keep], b[keep]
        keys.append(a * n + b)
        keys.append(b * n + a)
    keys = torch.unique(torch.cat(keys)) if keys else torch.zeros(0, dtype=torch.int64, device=device)
    row_ptr, src, dst = _csr_from_sorted_keys(keys, n)
    w_f32, w_u32, etype = _attributes(src, dst, seed, weights, types_seed)
    return Graph(n, int(keys.numel()), row_ptr, dst.to(torch.int32), w_f32, w_u32, etype,
                 name=f"chunglu_n{n}_s{seed}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, weights: str = "grid14", types_seed: Optional[int] = None,
         device="cpu", chunk: int = 1 << 24) -> Graph:
    """R-MAT graph (Chakrabarti et al.), symmetrised, self loops and duplicates removed.

    Edge e in [0, edge_factor * 2^scale) descends ``scale`` levels; at each level
    one hash draw picks quadrant (0,0) with prob a, (0,1) with b, (1,0) with c,
    (1,1) with 1-a-b-c, most significant bit first.  Vertex ids are not
    permuted, so the hubs sit at small ids.
    """
    n = 1 << scale
    M = edge_factor * n
    tA = int(math.floor(a * 4294967296.0))
    tAB = int(math.floor((a + b) * 4294967296.0))
    tABC = int(math.floor((a + b + c) * 4294967296.0))
    lvl_const = [_mix_const((seed * 0x85EBCA6B + lv * 0x9E3779B9 + 0x27D4EB2F) & MASK32)
                 for lv in range(scale)]
    keys = []
    for e0 in range(0, M, chunk):
        e1 = min(M, e0 + chunk)
        e = torch.arange(e0, e1, dtype=torch.int64, device=device)
        base = _hash2(seed * 2, e & MASK32, e >> 32)
        src = torch.zeros_like(e)
        dst = torch.zeros_like(e)
        for lv in range(scale):
            u = mix32(base ^ lvl_const[lv])
            sbit = (u >= tAB).to(torch.int64)
            dbit = (((u >= tA) & (u < tAB)) | (u >= tABC)).to(torch.int64)
            src = src * 2 + sbit
            dst = dst * 2 + dbit
            del u
        keep = src != dst
        src, dst = src[keep], dst[keep]
        keys.append(src * n + dst)
        keys.append(dst * n + src)
        del e, base, src, dst, keep
    keys = torch.unique(torch.cat(keys))
    row_ptr, src, dst = _csr_from_sorted_keys(keys, n)
    del keys
    w_f32, w_u32, etype = _attributes(src, dst, seed, weights, types_seed)
    col = dst.to(torch.int32)
    del src, dst
    return Graph(n, int(col.numel()), row_ptr, col, w_f32, w_u32, etype,
                 name=f"rmat{scale}_ef{edge_factor}_s{seed}")


def one_per_vertex(n: int, device="cpu") -> torch.Tensor:
    """Start vertices 0..n-1 (one query per vertex, as in the paper's workloads)."""
    return torch.arange(n, dtype=torch.int32, device=device)


def random_starts(n: int, count: int, seed: int, device="cpu") -> torch.Tensor:
    """``count`` start vertices drawn uniformly from [0, n) by hash."""
    q = torch.arange(count, dtype=torch.int64, device=device)
    h = _hash2(seed * 2 + 7, q & MASK32, q >> 32)
    return (h % n).to(torch.int32)


def uniform_lengths(count: int, lo: int, hi: int, seed: int, device="cpu") -> torch.Tensor:
    """Per-query walk lengths uniform in [lo, hi] by hash."""
    q = torch.arange(count, dtype=torch.int64, device=device)
    h = _hash2(seed * 2 + 9, q & MASK32, q >> 32)
    return (lo + h % (hi - lo + 1)).to(torch.int32)
