"""Seeded synthetic embeddings shaped like the paper's retrieval workloads.

The paper evaluates on Market-1501 (3,368 queries, 19,732 gallery images,
1,501 identities), VeRi-776, Oxford-5k, Paris-6k and University-1652 with
CNN features of dimension 1536 / 2048 / 512 (Sec. 4.1, "Datasets and
Settings" and "Implementation Details").  None of those images or features
exist here, so this module draws stand-ins with the same shapes: clustered
Gaussian embeddings (one cluster per identity), optional uniform-on-sphere
distractors, every row L2-normalised.

This module is shared input plumbing: it holds none of the re-ranking
arithmetic (no similarity, no neighbour selection, no propagation) and both
the FP64 oracle and the CUDA path consume the arrays it returns.

Portability.  Every draw is bit-identical on x86-64 and AArch64: the random
bits come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator, and the Box-Muller transform uses the logarithm, sine and cosine
below, which are written with IEEE +, -, *, / only (series after an exact
range reduction), so they do not depend on the platform's libm.  Square
roots are IEEE correctly rounded; row norms are summed strictly left to right
(``np.cumsum``) so no SIMD reassociation can change a bit.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
from typing import Optional

import numpy as np

__all__ = [
    "WorkloadSpec", "Workload", "TINY", "MARKET_SCALE", "LARGE_50K", "SERVING_GALLERY",
    "make_workload", "batched_specs", "serving_requests", "array_digest", "SplitMix64",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)
_LN2 = 0.6931471805599453
_HALF_PI = 1.5707963267948966
_TWO_POW_M32 = 2.0 ** -32


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter-based SplitMix64 stream: output(i) = mix(key + (i + 1) * gamma).

    ``key`` is derived from (seed, stream name) so that independent purposes
    (cluster centres, noise, permutations, ...) never share random bits.
    """

    def __init__(self, seed: int, stream: str):
        h = int.from_bytes(hashlib.sha256(f"{seed}:{stream}".encode()).digest()[:8], "little")
        self.key = np.uint64(h)
        self.pos = 0

    def next_u64(self, n: int) -> np.ndarray:
        ctr = np.arange(self.pos, self.pos + n, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            z = self.key + (ctr + np.uint64(1)) * _GAMMA
        return _mix64(z)

    def uniform_pair(self, n: int) -> tuple[np.ndarray, np.ndarray]:
        """Two arrays of n uniforms in (0, 1) from the high and low 32 bits."""
        z = self.next_u64(n)
        hi = (z >> np.uint64(32)).astype(np.float64)
        lo = (z & np.uint64(0xFFFFFFFF)).astype(np.float64)
        return (hi + 0.5) * _TWO_POW_M32, (lo + 0.5) * _TWO_POW_M32

    def uniform(self, n: int) -> np.ndarray:
        return self.uniform_pair(n)[0]

    def below(self, n: int, bound: int) -> np.ndarray:
        """n integers uniform in [0, bound) (multiply-shift on 32 bits)."""
        z = self.next_u64(n) >> np.uint64(32)
        return ((z * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        """n standard normal draws by the Box-Muller transform."""
        m = (n + 1) // 2
        u1, u2 = self.uniform_pair(m)
        r = np.sqrt(-2.0 * _ln(u1))
        c, s = _cos_sin_turns(u2)
        out = np.empty(2 * m, dtype=np.float64)
        out[0::2] = r * c
        out[1::2] = r * s
        return out[:n]

    def permutation(self, n: int) -> np.ndarray:
        keys = self.next_u64(n)
        return np.argsort(keys, kind="stable")


def _ln(u: np.ndarray) -> np.ndarray:
    """Natural log for u > 0: exact frexp reduction, then the atanh series."""
    m, e = np.frexp(u)
    small = m < 0.7071067811865476
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    p = np.full_like(t, 1.0 / 23.0)
    for k in range(10, -1, -1):
        p = p * t2 + 1.0 / (2 * k + 1)
    return e * _LN2 + 2.0 * t * p


def _cos_sin_small(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Taylor series of cos and sin for |x| <= pi/4 (terms to x^21)."""
    x2 = x * x
    c = np.ones_like(x)
    s = np.ones_like(x)
    for k in range(10, 0, -1):
        c = 1.0 - x2 * c / ((2 * k - 1) * (2 * k))
        s = 1.0 - x2 * s / ((2 * k) * (2 * k + 1))
    return c, x * s


def _cos_sin_turns(v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """cos(2*pi*v), sin(2*pi*v) for v in [0, 1) via an exact quadrant split."""
    w = v * 4.0
    q = np.floor(w)
    r = w - q
    hi = r > 0.5
    x = np.where(hi, 1.0 - r, r) * _HALF_PI
    cx, sx = _cos_sin_small(x)
    c = np.where(hi, sx, cx)
    s = np.where(hi, cx, sx)
    qi = q.astype(np.int64) & 3
    cos_t = np.select([qi == 0, qi == 1, qi == 2], [c, -s, -c], s)
    sin_t = np.select([qi == 0, qi == 1, qi == 2], [s, c, -s], -c)
    return cos_t, sin_t


def _unit_rows(x: np.ndarray) -> np.ndarray:
    """Scale each FP64 row to unit length (left-to-right sum of squares)."""
    nrm = np.sqrt(np.cumsum(x * x, axis=1)[:, -1])
    return x / nrm[:, None]


@dataclasses.dataclass(frozen=True)
class WorkloadSpec:
    """One synthetic retrieval instance.

    Clustered samples: ``n_query + n_gallery - n_distractors`` of them, spread
    over ``n_clusters`` clusters.  With ``size_range`` set, sizes are
    ``clamp(lo + round(Exp(mean)), lo, hi)`` with ``mean = total/C - lo``,
    then adjusted by +-1 in a seeded order until they sum to the total;
    without it, sizes are as equal as possible.
    """
    name: str
    n_query: int
    n_gallery: int
    dim: int
    n_clusters: int
    sigma: float
    n_distractors: int = 0
    size_range: Optional[tuple[int, int]] = None
    seed: int = 0

    @property
    def n(self) -> int:
        return self.n_query + self.n_gallery


# 100 queries + 900 gallery, d = 128, 50 clusters of 20, noise norm 0.3.
TINY = WorkloadSpec("tiny", 100, 900, 128, 50, 0.3, 0, None, seed=0)
# Market-1501 shape (Sec. 4.1): 3,368 + 19,732, 1,501 identities, plus 2,000
# distractors; d = 2048 as the VeRi / Oxford / Paris features.
MARKET_SCALE = WorkloadSpec("market_23k_d2048", 3368, 19732, 2048, 1501, 0.35, 2000, (8, 30), seed=1)
# A 50,000-vertex instance with 512-d features (University-1652's dimension).
LARGE_50K = WorkloadSpec("large_50k_d512", 5000, 45000, 512, 3000, 0.35, 0, (8, 30), seed=2)
# The Market-1501 shape with 128-d features and noise of norm 1.6: the initial
# cosine ranking is far from perfect (mAP about 0.75), so the accuracy sweeps
# over layers and (k1, k2) have room to show the re-ranking's effect.
MARKET_HARD = WorkloadSpec("market_hard_d128", 3368, 19732, 128, 1501, 1.6, 2000, (8, 30), seed=5)
# Resident gallery for the serving loop: 40,000 vectors, 2,500 clusters of 16.
SERVING_GALLERY = WorkloadSpec("serving_gallery_40k", 0, 40000, 2048, 2500, 0.35, 0, None, seed=4)


@dataclasses.dataclass
class Workload:
    spec: WorkloadSpec
    xq: np.ndarray  # (n_query, dim) float32, unit rows
    xg: np.ndarray  # (n_gallery, dim) float32, unit rows
    yq: np.ndarray  # (n_query,) int32 cluster label
    yg: np.ndarray  # (n_gallery,) int32 cluster label, -1 for distractors
    centres: np.ndarray  # (n_clusters, dim) float64 unit rows


def _cluster_sizes(spec: WorkloadSpec, total: int) -> np.ndarray:
    c = spec.n_clusters
    if spec.size_range is None:
        base = np.full(c, total // c, dtype=np.int64)
        base[: total % c] += 1
        return base
    lo, hi = spec.size_range
    if not (lo * c <= total <= hi * c):
        raise ValueError("cluster size range cannot reach the requested total")
    rng = SplitMix64(spec.seed, "cluster_sizes")
    mean = total / c - lo
    sizes = np.clip(lo + np.rint(-mean * _ln(rng.uniform(c))), lo, hi).astype(np.int64)
    order = SplitMix64(spec.seed, "cluster_fixup").permutation(c)
    diff = total - int(sizes.sum())
    while diff != 0:
        step = 1 if diff > 0 else -1
        for k in order:
            if diff == 0:
                break
            if lo <= sizes[k] + step <= hi:
                sizes[k] += step
                diff -= step
    return sizes


def _noisy_samples(centres: np.ndarray, labels: np.ndarray, sigma: float, seed: int,
                   stream: str, chunk: int = 2048) -> np.ndarray:
    """centre + N(0, (sigma^2/d) I) per sample, then unit-normalised, FP32."""
    n, d = len(labels), centres.shape[1]
    out = np.empty((n, d), dtype=np.float32)
    rng = SplitMix64(seed, stream)
    scale = sigma / math.sqrt(d)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        eps = rng.normal((b - a) * d).reshape(b - a, d)
        out[a:b] = _unit_rows(centres[labels[a:b]] + scale * eps).astype(np.float32)
    return out


def _sphere(n: int, d: int, seed: int, stream: str, chunk: int = 2048) -> np.ndarray:
    out = np.empty((n, d), dtype=np.float64)
    rng = SplitMix64(seed, stream)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = _unit_rows(rng.normal((b - a) * d).reshape(b - a, d))
    return out


def make_workload(spec: WorkloadSpec) -> Workload:
    """Draw the query and gallery sets of ``spec`` (deterministic in its seed)."""
    n_clustered = spec.n - spec.n_distractors
    centres = _sphere(spec.n_clusters, spec.dim, spec.seed, "centres")
    sizes = _cluster_sizes(spec, n_clustered)
    labels = np.repeat(np.arange(spec.n_clusters, dtype=np.int32), sizes)
    x = _noisy_samples(centres, labels, spec.sigma, spec.seed, "noise")

    # Queries: walk the clustered samples in a seeded order and take one as a
    # query only while its cluster keeps at least one gallery member.
    remaining = sizes.copy()
    is_query = np.zeros(n_clustered, dtype=bool)
    taken = 0
    for s in SplitMix64(spec.seed, "query_pick").permutation(n_clustered):
        if taken == spec.n_query:
            break
        if remaining[labels[s]] >= 2:
            remaining[labels[s]] -= 1
            is_query[s] = True
            taken += 1
    if taken != spec.n_query:
        raise ValueError("not enough clustered samples to draw the queries")

    xq, yq = x[is_query], labels[is_query]
    xg, yg = x[~is_query], labels[~is_query]
    if spec.n_distractors:
        xd = _sphere(spec.n_distractors, spec.dim, spec.seed, "distractors").astype(np.float32)
        xg = np.concatenate([xg, xd])
        yg = np.concatenate([yg, np.full(spec.n_distractors, -1, dtype=np.int32)])
    pq = SplitMix64(spec.seed, "perm_query").permutation(len(yq))
    pg = SplitMix64(spec.seed, "perm_gallery").permutation(len(yg))
    return Workload(spec, np.ascontiguousarray(xq[pq]), np.ascontiguousarray(xg[pg]),
                    yq[pq].astype(np.int32), yg[pg].astype(np.int32), centres)


def _log_uniform_int(rng: SplitMix64, n: int, lo: int, hi: int) -> np.ndarray:
    u = rng.uniform(n)
    # exp(u * ln(hi/lo)) by its Taylor series (all IEEE arithmetic).
    a = u * (_ln(np.array([hi / lo]))[0])
    e = np.ones_like(a)
    term = np.ones_like(a)
    for k in range(1, 40):
        term = term * a / k
        e = e + term
    return np.clip(np.rint(lo * e), lo, hi).astype(np.int64)


def batched_specs(n_instances: int = 64, base_seed: int = 3) -> list[dict]:
    """Independent instances: N log-uniform on [500, 8000], d in {256, 512, 2048},
    Q = round(0.146 N) (Market's query share), clusters of 8-30 (C = round(N/14.06)),
    noise 0.35, k1 ~ U{20..30}, k2 ~ U{5..7}, layers ~ U{1..3}."""
    rng = SplitMix64(base_seed, "batched")
    ns = _log_uniform_int(rng, n_instances, 500, 8000)
    dims = np.array([256, 512, 2048])[rng.below(n_instances, 3)]
    k1s = 20 + rng.below(n_instances, 11)
    k2s = 5 + rng.below(n_instances, 3)
    ls = 1 + rng.below(n_instances, 3)
    out = []
    for i in range(n_instances):
        n = int(ns[i])
        q = int(round(0.146 * n))
        c = max(1, int(round(n / 14.06)))
        c = min(max(c, -(-n // 30)), n // 8)
        spec = WorkloadSpec(f"batched_{i}", q, n - q, int(dims[i]), c, 0.35, 0, (8, 30), seed=base_seed + i)
        out.append(dict(spec=spec, k1=int(k1s[i]), k2=int(k2s[i]), layers=int(ls[i])))
    return out


def serving_requests(gallery: Workload, rate_hz: float = 200.0, duration_s: float = 60.0,
                     q_lo: int = 1, q_hi: int = 512, seed: int = 4) -> list[dict]:
    """Poisson arrivals; each request brings log-uniform [q_lo, q_hi] new queries
    drawn around the resident gallery's cluster centres (noise as the gallery)."""
    rng = SplitMix64(seed, "arrivals")
    t, out, r = 0.0, [], 0
    while True:
        t += -_ln(rng.uniform(1))[0] / rate_hz
        if t >= duration_s:
            break
        nq = int(_log_uniform_int(rng, 1, q_lo, q_hi)[0])
        out.append(dict(t_arrival=t, n_query=nq, request_id=r))
        r += 1
    return out


def request_queries(gallery: Workload, request_id: int, n_query: int, seed: int = 4) -> np.ndarray:
    """The query rows of one serving request (float32, unit rows)."""
    rng = SplitMix64(seed, f"request_{request_id}")
    labels = rng.below(n_query, gallery.spec.n_clusters).astype(np.int32)
    return _noisy_samples(gallery.centres, labels, gallery.spec.sigma, seed, f"request_noise_{request_id}")


def array_digest(*arrays: np.ndarray) -> str:
    """SHA-256 over the raw bytes of the arrays (for portability pins)."""
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()
