"""Seeded synthetic ELSR instances (input generator only).

This module holds none of the method's arithmetic: it only draws the problem
data of Section 2 (demand D, returns R, setup costs kM/kR, holding costs
hM/hR).  The paper's benchmark set of [SK2016] (K=300 products, T=52 periods)
is not available, so seeded instances with the value distributions of the
workloads stand in for it.

Recipe (integer throughout):

* stream per (seed, id): ``state = mix(mix(seed) ^ id)``; the i-th draw
  (i = 0, 1, ...) is ``fin(state + (i + 1) * GOLDEN)`` -- the splitmix64
  generator of Steele, Lea & Flood (2014), with ``fin`` its output mix and
  ``mix(x) = fin(x + GOLDEN)``.
* ``U{a..b} = a + draw mod (b - a + 1)``.
* draw order: (variable-size instances only) K then T; for each product k:
  kM ~ U{200..500}, kR ~ U{100..400}, hM ~ U{2..6}, hR ~ U{1..hM-1}; then for
  each (k, t) in row-major order: D ~ U{0..100}, p ~ U{200..600} and
  R = floor(D * p / 1000), the integer reading of "R = D * U[0.2, 0.6]".
  Hence 0 <= R <= D.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def _fin_np(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        return z ^ (z >> np.uint64(31))


def _mix_int(x: int) -> int:
    z = (x + GOLDEN) & _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


class Stream:
    """Counter-based splitmix64 stream keyed by (seed, id)."""

    def __init__(self, seed: int, ident: int):
        self.state = _mix_int(_mix_int(seed & _MASK) ^ (ident & _MASK))
        self.pos = 0

    def draws(self, n: int) -> np.ndarray:
        i = np.arange(self.pos + 1, self.pos + n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + i * np.uint64(GOLDEN)
        self.pos += n
        return _fin_np(z)

    def uniform(self, lo, hi, n: int) -> np.ndarray:
        """n draws of U{lo..hi} (lo/hi scalars or arrays of length n)."""
        span = (np.asarray(hi, np.int64) - np.asarray(lo, np.int64) + 1).astype(np.uint64)
        return np.asarray(lo, np.int64) + (self.draws(n) % span).astype(np.int64)


@dataclass
class ElsrInstance:
    """Problem data of Section 2 (int32 arrays, row-major D/R [K][T]); pM, pR:
    optional unit production costs [K] (None: none)."""
    D: np.ndarray
    R: np.ndarray
    kM: np.ndarray
    kR: np.ndarray
    hM: np.ndarray
    hR: np.ndarray
    pM: np.ndarray | None = None
    pR: np.ndarray | None = None

    @property
    def K(self) -> int:
        return int(self.D.shape[0])

    @property
    def T(self) -> int:
        return int(self.D.shape[1])


def make_instance(seed: int, ident: int = 0, K: int | None = None,
                  T: int | None = None, K_range=(5, 100), T_range=(12, 52)) -> ElsrInstance:
    """One instance from stream (seed, ident).  With K and T given the sizes
    are fixed; otherwise K ~ U{K_range}, T ~ U{T_range} are drawn first."""
    s = Stream(seed, ident)
    if K is None or T is None:
        K = int(s.uniform(K_range[0], K_range[1], 1)[0])
        T = int(s.uniform(T_range[0], T_range[1], 1)[0])
    c = s.draws(4 * K).reshape(K, 4)
    kM = 200 + (c[:, 0] % np.uint64(301)).astype(np.int64)
    kR = 100 + (c[:, 1] % np.uint64(301)).astype(np.int64)
    hM = 2 + (c[:, 2] % np.uint64(5)).astype(np.int64)
    hR = 1 + (c[:, 3] % (hM - 1).astype(np.uint64)).astype(np.int64)
    v = s.draws(2 * K * T).reshape(K, T, 2)
    D = (v[:, :, 0] % np.uint64(101)).astype(np.int64)
    p = 200 + (v[:, :, 1] % np.uint64(401)).astype(np.int64)
    R = (D * p) // 1000
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    return ElsrInstance(i32(D), i32(R), i32(kM), i32(kR), i32(hM), i32(hR))


# Workload shapes (sizes from the paper's experiments and the synthetic
# stand-ins for its missing benchmark set).

def plain_small() -> ElsrInstance:
    """Plain VNS case: K=5 products, T=12 periods, seed 0."""
    return make_instance(0, 0, K=5, T=12)


def plain_medium() -> ElsrInstance:
    """Plain VNS case: K=50 products, T=52 periods, seed 1."""
    return make_instance(1, 0, K=50, T=52)


def paper_shaped() -> ElsrInstance:
    """The paper's benchmark shape (Section 4): K=300 products, T=52 periods."""
    return make_instance(3, 0, K=300, T=52)


def batch_uneven(n: int = 1024, seed: int = 0):
    """n independent instances, K ~ U{5..100}, T ~ U{12..52}, keyed by id."""
    return [make_instance(seed, i, K_range=(5, 100), T_range=(12, 52)) for i in range(n)]


def multistart_large() -> ElsrInstance:
    """Multi-start case: one instance K=100, T=104 (seed 0, id 0)."""
    return make_instance(0, 0, K=100, T=104)


def serving_request(r: int, seed: int = 5) -> ElsrInstance:
    """Serving request r: K ~ U{5..200}, T ~ U{12..104}, keyed by request id."""
    return make_instance(seed, r, K_range=(5, 200), T_range=(12, 104))


def with_production_costs(g: ElsrInstance, seed: int, ident: int = 0,
                          pM_range=(10, 40), pR_range=(0, 60)) -> ElsrInstance:
    """The instance g with unit production costs pM ~ U{pM_range},
    pR ~ U{pR_range} per product, drawn (pM then pR for each product) from
    the stream (seed, ident).  The paper names p_M, p_R in Algorithm 1's
    signature without values; the default ranges make remanufacturing
    cheaper for some products and dearer for others, so pR - pM takes both
    signs and can outweigh the holding saving hR*(T-t)."""
    s = Stream(seed, ident)
    K = g.D.shape[0]
    v = s.draws(2 * K).reshape(K, 2)
    pM = pM_range[0] + (v[:, 0] % np.uint64(pM_range[1] - pM_range[0] + 1)).astype(np.int64)
    pR = pR_range[0] + (v[:, 1] % np.uint64(pR_range[1] - pR_range[0] + 1)).astype(np.int64)
    return ElsrInstance(g.D, g.R, g.kM, g.kR, g.hM, g.hR,
                        np.ascontiguousarray(pM, dtype=np.int32),
                        np.ascontiguousarray(pR, dtype=np.int32))
