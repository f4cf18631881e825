"""Seeded synthetic inputs for the merge, batched-merge, merge-sort and
learned-search workloads.

This module only draws random numbers, sorts inputs that the workloads
require to be sorted, and tags payloads.  It holds none of the merge's
arithmetic, so the tests can hand the same arrays to the GPU library and to
the CPU oracle.  Tensors are made on the requested device (CPU for the small
CPU tests, CUDA for the large GPU runs); a fixed seed and device always give
the same arrays.

Key storage: u32 keys are kept in int32 tensors holding the same 32-bit
pattern (all generated u32 keys are below 2**31, so the values agree too);
u64 keys in int64 tensors (all below 2**63); i32 in int32; f32 in float32.
Payloads are 32-bit words kept in int32 tensors.

Payload tag used for stability checks: (source << 31) | index, source 0 for A
and 1 for B, index the element's position in its (sorted) input array.
"""
from __future__ import annotations

import math

import torch

SEED_BASE = 0x5EED

KEY_DTYPES = {"u32": torch.int32, "i32": torch.int32, "u64": torch.int64, "f32": torch.float32}

DIST_NAMES = ("uniform_full", "uniform_1024", "all_equal", "zipf")


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def payload(src: int, count: int, device, start: int = 0) -> torch.Tensor:
    """(src << 31) | (start + index) as 32-bit words in an int32 tensor."""
    idx = torch.arange(start, start + count, dtype=torch.int64, device=device)
    word = idx | (int(src) << 31)
    word = torch.where(word >= (1 << 31), word - (1 << 32), word)   # same 32 bits, signed
    return word.to(torch.int32)


def widen_payload(word32: torch.Tensor) -> torch.Tensor:
    """64-bit payload words (int64 tensor) from 32-bit ones: the 32-bit word
    in the high half and a multiplicative hash of it (by 0x9E3779B1, mod
    2**32) in the low half, so that every bit of the wider word carries
    information and each 64-bit word names its 32-bit source uniquely."""
    t = word32.to(torch.int64) & 0xFFFFFFFF
    low = (t * 0x9E3779B1) & 0xFFFFFFFF                # wraps mod 2**64; the low 32 bits are exact
    return (t << 32) | low


def sorted_uniform_int(count: int, lo: int, hi: int, dtype, g, device) -> torch.Tensor:
    """Sorted sample of `count` i.i.d. integers uniform in [lo, hi)."""
    if count == 0:
        return torch.empty(0, dtype=dtype, device=device)
    x = torch.randint(lo, hi, (count,), generator=g, device=device, dtype=torch.int64)
    return torch.sort(x).values.to(dtype)


def sorted_zipf(count: int, values: int, s: float, dtype, g, device) -> torch.Tensor:
    """Sorted sample with P(v) proportional to (v + 1)**(-s), v in [0, values)."""
    if count == 0:
        return torch.empty(0, dtype=dtype, device=device)
    w = torch.arange(1, values + 1, dtype=torch.float64, device=device).pow(-s)
    cdf = torch.cumsum(w, 0)
    cdf = cdf / cdf[-1]
    u = torch.rand(count, generator=g, device=device, dtype=torch.float64)
    v = torch.searchsorted(cdf, u, right=True).clamp_(max=values - 1)
    return torch.sort(v).values.to(dtype)


def sorted_lognormal_mixture(count: int, g, device, mus=(0.0, 2.0, 5.0),
                             sigma: float = 0.5) -> torch.Tensor:
    """Sorted float32 sample of an equal-weight mixture of lognormals."""
    if count == 0:
        return torch.empty(0, dtype=torch.float32, device=device)
    comp = torch.randint(0, len(mus), (count,), generator=g, device=device)
    mu = torch.tensor(mus, dtype=torch.float64, device=device)[comp]
    z = torch.randn(count, generator=g, device=device, dtype=torch.float64)
    x = torch.exp(mu + sigma * z).to(torch.float32)
    return torch.sort(x).values


def keys_for_dist(dist: str, count: int, g, device) -> torch.Tensor:
    """int32 sorted keys of one of the four large-merge distributions."""
    if dist == "uniform_full":
        return sorted_uniform_int(count, -(1 << 31), 1 << 31, torch.int32, g, device)
    if dist == "uniform_1024":
        return sorted_uniform_int(count, 0, 1024, torch.int32, g, device)
    if dist == "all_equal":
        return torch.zeros(count, dtype=torch.int32, device=device)
    if dist == "zipf":
        return sorted_zipf(count, 1 << 20, 1.2, torch.int32, g, device)
    raise ValueError(f"unknown distribution {dist!r}")


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def small_merge(n: int, m: int, kt: str, seed: int, device="cpu", alphabet: int | None = None):
    """Sorted A (n) and B (m) of key type kt with tagged payloads.  `alphabet`
    limits keys to [0, alphabet) (heavy ties); None uses the type's range."""
    g = _gen(seed, device)
    if kt == "f32":
        if alphabet is None:
            A = sorted_lognormal_mixture(n, g, device)
            B = sorted_lognormal_mixture(m, g, device)
        else:
            A = sorted_uniform_int(n, 0, alphabet, torch.int64, g, device).to(torch.float32) * 0.5
            B = sorted_uniform_int(m, 0, alphabet, torch.int64, g, device).to(torch.float32) * 0.5
    else:
        if alphabet is not None:
            lo, hi = 0, alphabet
        elif kt == "i32":
            lo, hi = -(1 << 31), 1 << 31
        elif kt == "u32":
            lo, hi = 0, 1 << 31
        else:
            lo, hi = 0, 1 << 62
        A = sorted_uniform_int(n, lo, hi, KEY_DTYPES[kt], g, device)
        B = sorted_uniform_int(m, lo, hi, KEY_DTYPES[kt], g, device)
    return A, payload(0, n, device), B, payload(1, m, device)


def single_merge_1m(device="cpu"):
    """A n=2**20, B m=2**19 u32 keys uniform in [0, 2**16), sorted; tagged
    payloads; the merge is run with p = 1024 blocks per input."""
    g = _gen(SEED_BASE + 1, device)
    n, m = 1 << 20, 1 << 19
    A = sorted_uniform_int(n, 0, 1 << 16, torch.int32, g, device)
    B = sorted_uniform_int(m, 0, 1 << 16, torch.int32, g, device)
    return A, payload(0, n, device), B, payload(1, m, device)


def large_merge(dist: str, skewed: bool = False, device="cpu", log2n: int = 28,
                log2m_skewed: int = 18):
    """n = m = 2**28 int32 keys (or n = 2**28, m = 2**18 when skewed) of one
    distribution, sorted, with tagged int32 payloads.  Sizes can be reduced
    through log2n for small tests."""
    di = DIST_NAMES.index(dist)
    g = _gen(SEED_BASE + 2 + 16 * di + (8 if skewed else 0), device)
    n = 1 << log2n
    m = (1 << log2m_skewed) if skewed else n
    A = keys_for_dist(dist, n, g, device)
    B = keys_for_dist(dist, m, g, device)
    return A, payload(0, n, device), B, payload(1, m, device)


def batched_pairs(device="cpu", pairs: int = 65536, log2_max: int = 16, key_bits: int = 20,
                  seed: int = SEED_BASE + 3):
    """`pairs` independent merges.  Lengths n_k, m_k = floor(2**(log2_max*U))
    in [1, 2**log2_max - 1], independent per side (log-uniform); u64 keys
    uniform in [0, 2**key_bits), sorted within each array; CSR offsets start
    at 0.  Payload (source << 31) | global index within its CSR array."""
    g = _gen(seed, device)
    u = torch.rand(2, pairs, generator=g, device=device, dtype=torch.float64)
    lens = torch.floor(torch.pow(2.0, log2_max * u)).to(torch.int64).clamp_(1, 1 << log2_max)
    out = []
    for side in range(2):
        ln = lens[side]
        off = torch.zeros(pairs + 1, dtype=torch.int64, device=device)
        off[1:] = torch.cumsum(ln, 0)
        total = int(off[-1].item())
        seg = torch.repeat_interleave(torch.arange(pairs, device=device), ln)
        x = torch.randint(0, 1 << key_bits, (total,), generator=g, device=device, dtype=torch.int64)
        x = torch.sort(x + (seg << key_bits)).values - (seg << key_bits)
        del seg
        out.append((off, x, payload(side, total, device)))
    (a_off, A, Av), (b_off, B, Bv) = out
    return a_off, A, Av, b_off, B, Bv


def sort_input(device="cpu", n: int = 1 << 28, key_bits: int = 24, seed: int = SEED_BASE + 4):
    """n u64 keys uniform in [0, 2**key_bits) (unsorted), payload = index."""
    g = _gen(seed, device)
    keys = torch.randint(0, 1 << key_bits, (n,), generator=g, device=device, dtype=torch.int64)
    vals = torch.arange(n, dtype=torch.int64, device=device).to(torch.int32)
    return keys, vals


def lsm_base(device="cpu", n: int = 1 << 28, seed: int = SEED_BASE + 5):
    """Sorted float32 base of the mixture 1/3 LogN(0, .5) + 1/3 LogN(2, .5) +
    1/3 LogN(5, .5); payload = insertion sequence number 0..n-1."""
    g = _gen(seed, device)
    X = sorted_lognormal_mixture(n, g, device)
    return X, torch.arange(n, dtype=torch.int64, device=device).to(torch.int32)


def lsm_batch(k: int, device="cpu", size: int = 1 << 20, base_n: int = 1 << 28,
              seed: int = SEED_BASE + 5):
    """The k-th incoming sorted batch of the same mixture; payloads continue
    the insertion sequence after the base and the earlier batches."""
    g = _gen(seed * 7919 + 1000003 * (k + 1), device)
    Y = sorted_lognormal_mixture(size, g, device)
    start = base_n + k * size
    return Y, torch.arange(start, start + size, dtype=torch.int64, device=device).to(torch.int32)


def lsm_label_keys(device="cpu", count: int = 1 << 16, seed: int = SEED_BASE + 6):
    """Sorted training query keys drawn from the same mixture."""
    g = _gen(seed, device)
    return sorted_lognormal_mixture(count, g, device)


def cdf_init(hidden: int = 64, seed: int = SEED_BASE + 7):
    """Initial MLP parameters (float64 CPU tensors): W1 (hidden, 2), b1, w2, b2."""
    g = _gen(seed, "cpu")
    W1 = (torch.rand(hidden, 2, generator=g, dtype=torch.float64) * 2 - 1) * math.sqrt(3.0 / 2.0)
    b1 = (torch.rand(hidden, generator=g, dtype=torch.float64) * 2 - 1) * 0.5
    w2 = (torch.rand(hidden, generator=g, dtype=torch.float64) * 2 - 1) * 0.01
    b2 = torch.zeros((), dtype=torch.float64)
    return {"W1": W1, "b1": b1, "w2": w2, "b2": b2}
