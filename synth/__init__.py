"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module only *makes inputs*: random generator matrices, textbook codes built from
their definitions, the matrix-product codes printed in the paper (§6), and the batch /
request mixes.  It holds none of the method's arithmetic (no elimination, no
information sets, no enumeration, no weights), so neither side of a parity test can
borrow its logic from here.

Bit layout (the layout the library's C-ABI takes): an R x n bit matrix is an
``uint64`` array of shape (R, W), W >= ceil(n/64); bit i of row r is bit (i & 63) of
word (i >> 6) (LSB first).  Bits at positions >= n are zero.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): a Weyl sequence with gamma
    0x9E3779B97F4A7C15 followed by the variant-13 finaliser of MurmurHash3."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + self.GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform_int(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive), by rejection (no modulo bias)."""
        span = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % span)
        while True:
            v = self.next()
            if v < limit:
                return lo + (v % span)

    def uniform01(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


def words_per_row(n: int) -> int:
    return (n + 63) // 64


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """(R, n) array of 0/1 -> (R, ceil(n/64)) uint64, LSB-first."""
    bits = np.asarray(bits, dtype=np.uint8) & 1
    if bits.ndim == 1:
        bits = bits[None, :]
    r, n = bits.shape
    w = words_per_row(n)
    padded = np.zeros((r, 64 * w), dtype=np.uint8)
    padded[:, :n] = bits
    by = np.packbits(padded, axis=1, bitorder="little")
    return np.ascontiguousarray(by).view("<u8").reshape(r, w).astype(np.uint64)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """(R, W) uint64 -> (R, n) uint8 of 0/1."""
    words = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    if words.ndim == 1:
        words = words[None, :]
    by = words.view(np.uint8).reshape(words.shape[0], -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :n].copy()


# ----------------------------------------------------------------------------------
# Random codes: G = [I_k | R], R iid Bernoulli(1/2) from a SplitMix64 stream
# ----------------------------------------------------------------------------------

def random_redundancy(n: int, k: int, seed: int) -> np.ndarray:
    """k x (n-k) bit matrix R: row r takes ceil((n-k)/64) consecutive draws of the
    stream seeded with `seed`; bit t of the row is bit (t & 63) of draw (t >> 6)."""
    rng = SplitMix64(seed)
    nr = n - k
    nw = words_per_row(nr) if nr > 0 else 0
    out = np.zeros((k, nr), dtype=np.uint8)
    for r in range(k):
        draws = np.array([rng.next() for _ in range(nw)], dtype=np.uint64)
        if nw:
            out[r, :] = unpack_bits(draws[None, :], nr)[0]
    return out


def random_systematic(n: int, k: int, seed: int) -> np.ndarray:
    """Packed G = [I_k | R] (k x n) for a random binary [n, k] code."""
    if not (0 < k < n):
        raise ValueError("need 0 < k < n")
    bits = np.zeros((k, n), dtype=np.uint8)
    bits[:, :k] = np.eye(k, dtype=np.uint8)
    bits[:, k:] = random_redundancy(n, k, seed)
    return pack_bits(bits)


def accept_seed(n: int, k: int, want_ranks, rank_fn, seed0: int, max_tries: int = 4096):
    """First seed s >= seed0 whose code's information-set ranks (as computed by the
    caller's `rank_fn(G, n, k)`) equal `want_ranks`.  Returns (seed, G)."""
    want = list(want_ranks)
    for s in range(seed0, seed0 + max_tries):
        g = random_systematic(n, k, s)
        if list(rank_fn(g, n, k)) == want:
            return s, g
    raise RuntimeError(f"no seed in [{seed0}, {seed0 + max_tries}) gives ranks {want}")


# ----------------------------------------------------------------------------------
# Textbook codes, each built from its definition
# ----------------------------------------------------------------------------------

def poly_from_exponents(exps) -> int:
    v = 0
    for e in exps:
        v ^= 1 << e
    return v


def poly_mul(a: int, b: int) -> int:
    """Product in F2[x] (polynomials as int bit masks)."""
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def poly_mod_cyclic(a: int, m: int) -> int:
    """a mod (x^m - 1): fold exponent e onto e mod m."""
    r = 0
    e = 0
    while a:
        if a & 1:
            r ^= 1 << (e % m)
        a >>= 1
        e += 1
    return r


def poly_divmod(a: int, b: int):
    """Quotient and remainder in F2[x]."""
    if b == 0:
        raise ZeroDivisionError
    q = 0
    db = b.bit_length() - 1
    while a and a.bit_length() - 1 >= db:
        s = a.bit_length() - 1 - db
        q ^= 1 << s
        a ^= b << s
    return q, a


def cyclic_generator_rows(gpoly: int, m: int) -> np.ndarray:
    """Rows x^i g(x), i = 0..m-deg(g)-1, as length-m bit vectors (a basis of the cyclic
    code (g) when g divides x^m - 1)."""
    deg = gpoly.bit_length() - 1
    rows = []
    for i in range(m - deg):
        v = poly_mod_cyclic(gpoly << i, m)
        rows.append([(v >> t) & 1 for t in range(m)])
    return np.array(rows, dtype=np.uint8)


def hamming_7_4() -> np.ndarray:
    """Hamming [7,4,3] as the cyclic code generated by 1 + x + x^3 (a primitive
    polynomial of degree 3)."""
    return pack_bits(cyclic_generator_rows(poly_from_exponents([0, 1, 3]), 7))


def golay_24_12() -> np.ndarray:
    """Extended binary Golay [24,12,8]: the cyclic [23,12,7] code generated by
    x^11 + x^10 + x^6 + x^5 + x^4 + x^2 + 1 (a factor of x^23 - 1), plus an overall
    parity bit."""
    g23 = cyclic_generator_rows(poly_from_exponents([11, 10, 6, 5, 4, 2, 0]), 23)
    par = g23.sum(axis=1, keepdims=True) % 2
    return pack_bits(np.concatenate([g23, par], axis=1))


def reed_muller_1_5() -> np.ndarray:
    """First-order Reed-Muller RM(1,5) [32,6,16]: evaluations of the affine functions
    1, x1..x5 at the 32 points of F2^5 (point p has coordinates the bits of p)."""
    pts = np.arange(32)
    rows = [np.ones(32, dtype=np.uint8)]
    for i in range(5):
        rows.append(((pts >> i) & 1).astype(np.uint8))
    return pack_bits(np.array(rows))


def repetition(n: int) -> np.ndarray:
    """[n,1,n] repetition code."""
    return pack_bits(np.ones((1, n), dtype=np.uint8))


def even_weight(n: int) -> np.ndarray:
    """[n, n-1, 2] even-weight code: rows e_i + e_{n-1}."""
    bits = np.zeros((n - 1, n), dtype=np.uint8)
    for i in range(n - 1):
        bits[i, i] = 1
        bits[i, n - 1] = 1
    return pack_bits(bits)


# ----------------------------------------------------------------------------------
# Matrix-product codes of the paper (§6): C = [C1 C2] . [[1, p], [0, 1]]
# ----------------------------------------------------------------------------------

def matrix_product_code(f1: int, f2: int, p: int, m: int) -> np.ndarray:
    """Codewords (c1, c1*p + c2), c1 in (f1), c2 in (f2), cyclic codes of length m,
    products taken in F2[x]/(x^m - 1).  Returns the packed 2m-column generator matrix
    with rows (x^i f1, x^i f1 p) and (0, x^i f2)."""
    p = poly_mod_cyclic(p, m)
    rows = []
    d1 = f1.bit_length() - 1
    for i in range(m - d1):
        a = poly_mod_cyclic(f1 << i, m)
        b = poly_mod_cyclic(poly_mul(a, p), m)
        rows.append([(a >> t) & 1 for t in range(m)] + [(b >> t) & 1 for t in range(m)])
    d2 = f2.bit_length() - 1
    for i in range(m - d2):
        b = poly_mod_cyclic(f2 << i, m)
        rows.append([0] * m + [(b >> t) & 1 for t in range(m)])
    return pack_bits(np.array(rows, dtype=np.uint8))


def extend_code(G: np.ndarray, n: int) -> np.ndarray:
    """Append an overall parity bit to every generator row ([n,k,d] -> [n+1,k,d'])."""
    bits = unpack_bits(G, n)
    par = bits.sum(axis=1, keepdims=True) % 2
    return pack_bits(np.concatenate([bits, par], axis=1))


def puncture_code(G: np.ndarray, n: int, positions) -> np.ndarray:
    """Delete the given 0-based coordinates from every generator row."""
    bits = unpack_bits(G, n)
    keep = [i for i in range(n) if i not in set(positions)]
    return pack_bits(bits[:, keep])


# ----------------------------------------------------------------------------------
# Multi-code workloads (batched launch, request stream)
# ----------------------------------------------------------------------------------

@dataclass
class CodeSpec:
    n: int
    k: int
    seed: int


def batch_specs(count: int, k_lo: int, k_hi: int, nmul_lo: int, nmul_hi: int,
                seed: int, seed_base: int) -> list[CodeSpec]:
    """`count` codes: k uniform in [k_lo, k_hi], n uniform in [nmul_lo*k, nmul_hi*k],
    drawn from one SplitMix64 stream; code i's R uses seed `seed_base + i`."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        k = rng.uniform_int(k_lo, k_hi)
        n = rng.uniform_int(nmul_lo * k, nmul_hi * k)
        out.append(CodeSpec(n=n, k=k, seed=seed_base + i))
    return out


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative sums of Exp(rate) gaps drawn
    by inversion from the SplitMix64 stream."""
    rng = SplitMix64(seed)
    t = 0.0
    out = np.empty(count, dtype=np.float64)
    for i in range(count):
        u = rng.uniform01()
        t += -math.log1p(-u) / rate_per_s
        out[i] = t
    return out
