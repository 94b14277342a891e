"""Counter-based random numbers for the oracle, written from their published definitions.

The paper does not say how its normals and Gamma variates are generated; both sides of the
parity tests implement the same published generator independently so that a GPU draw and
an oracle draw can be compared value by value (the draws themselves are what Algorithm 2
and the Gamma full conditionals of Appendix A consume).

* Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3"
  (SC'11). Round: (hi0, lo0) = M0*c0, (hi1, lo1) = M1*c2 (32x32->64 products),
  c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the Weyl constants
  between rounds; 10 rounds.
* Uniforms: 53 bits from two words, u_open = (m + 1) 2^-53 in (0, 1], u = m 2^-53 in [0, 1).
* Normals: Box-Muller (1958) in float64, two normals per Philox call.
* Gamma: Marsaglia & Tsang (2000), "A simple method for generating gamma variables",
  exact log acceptance test only, a fixed budget of 8 attempts, each from its own counter;
  shapes below 1 use the u^(1/c) boost from the same paper.

Counter layout (one 128-bit counter per call, key = seed split into two 32-bit words):
  c0 = site      (lattice-linear voxel index * 4 + slot; slot 0..2 = edge in +x/+y/+z,
                  slot 3 = the voxel itself; for hyperparameters the site is the index k/p)
  c1 = sub       (pair index j for normals 2j, 2j+1; attempt number for Gamma draws)
  c2 = counter   (draw counter, e.g. the Gibbs sweep number)
  c3 = tag << 24 | stream  (purpose tag, 24-bit stream id = chain / sample / probe)
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

# purpose tags
TAG_W = 1        # perturbation of the W right-hand side
TAG_A = 2        # perturbation of the A right-hand side
TAG_LAMBDA = 3   # lambda Gamma draws
TAG_ALPHA = 4    # alpha Gamma draws
TAG_BETA = 5     # beta Gamma draws
TAG_PROBE = 6    # Rademacher probes for traces / log-determinants
TAG_ALPHA_PROP = 7   # anisotropic prior: proposal normals (sub 0, 1) and acceptance uniform (sub 2)
TAG_ALPHA_AUX = 8    # anisotropic prior: edge normals of the exchange step's auxiliary draw


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10; inputs are broadcastable integer arrays (< 2^32)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK32 for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def key_of(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def c3_of(tag, stream):
    return (int(tag) << 24) | (int(stream) & 0xFFFFFF)


def uniform_open(seed, sites, sub, counter, tag, stream):
    """u in (0, 1] per site from words 0 and 1 of the call (site, sub, counter, tag/stream)."""
    k0, k1 = key_of(seed)
    w = philox4x32_10(np.asarray(sites, dtype=np.uint64), sub, counter, c3_of(tag, stream), k0, k1)
    return (u53(w[0], w[1]) + 1.0) * 2.0 ** -53


def u53(a, b):
    """m = 53 bits from words a (27 high bits) and b (26 bits), as a float64 integer."""
    return (a >> np.uint64(5)).astype(np.float64) * 67108864.0 + (b >> np.uint64(6)).astype(np.float64)


def normal_pair(words):
    w0, w1, w2, w3 = words
    u1 = (u53(w0, w1) + 1.0) * 2.0 ** -53     # (0, 1]
    u2 = u53(w2, w3) * 2.0 ** -53             # [0, 1)
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def normals(seed, sites, width, counter, tag, stream):
    """Standard normals z[s, k] for each site s and lane k < width: lane k comes from the
    Philox call with sub = k // 2, output (k % 2) of its Box-Muller pair."""
    k0, k1 = key_of(seed)
    sites = np.asarray(sites, dtype=np.uint64)
    out = np.empty((len(sites), width))
    for j in range((width + 1) // 2):
        z0, z1 = normal_pair(philox4x32_10(sites, j, counter, c3_of(tag, stream), k0, k1))
        out[:, 2 * j] = z0
        if 2 * j + 1 < width:
            out[:, 2 * j + 1] = z1
    return out


def rademacher(seed, sites, width, counter, tag, stream):
    """Rademacher signs r[s, k]: lane k uses word (k % 4) of the call with sub = k // 4;
    the sign is - when the word's top bit is set."""
    k0, k1 = key_of(seed)
    sites = np.asarray(sites, dtype=np.uint64)
    out = np.empty((len(sites), width))
    for j in range((width + 3) // 4):
        w = philox4x32_10(sites, j, counter, c3_of(tag, stream), k0, k1)
        for i in range(4):
            k = 4 * j + i
            if k < width:
                out[:, k] = np.where((w[i] >> np.uint64(31)) != 0, -1.0, 1.0)
    return out


GAMMA_ATTEMPTS = 8


def gamma(seed, sites, shape, scale, counter, tag, stream):
    """Gamma(shape c, scale b) draws (density x^(c-1) e^(-x/b), mean b c; the paper's Ga(b, c)
    of Appendix A). Marsaglia-Tsang: d = c' - 1/3, cc = 1/sqrt(9 d); attempt a uses the Philox
    calls with sub = 2a (normal x = first Box-Muller output) and sub = 2a + 1 (uniform u in
    (0, 1] from words 0, 1); accept d v with v = (1 + cc x)^3 when v > 0 and
    log u < x^2/2 + d - d v + d log v. If all 8 attempts reject, d itself is returned and the
    event is counted. For c < 1 the draw for c' = c + 1 is multiplied by u^(1/c), u from
    sub = 2 * 8. Returns (draws, n_exhausted)."""
    k0, k1 = key_of(seed)
    sites = np.asarray(sites, dtype=np.uint64)
    shape = np.broadcast_to(np.asarray(shape, dtype=np.float64), sites.shape)
    scale = np.broadcast_to(np.asarray(scale, dtype=np.float64), sites.shape)
    c3 = c3_of(tag, stream)
    boost = shape < 1.0
    cp = np.where(boost, shape + 1.0, shape)
    d = cp - 1.0 / 3.0
    cc = 1.0 / np.sqrt(9.0 * d)
    result = np.full(sites.shape, np.nan)
    done = np.zeros(sites.shape, dtype=bool)
    for a in range(GAMMA_ATTEMPTS):
        x, _ = normal_pair(philox4x32_10(sites, 2 * a, counter, c3, k0, k1))
        w = philox4x32_10(sites, 2 * a + 1, counter, c3, k0, k1)
        u = (u53(w[0], w[1]) + 1.0) * 2.0 ** -53
        v = 1.0 + cc * x
        pos = v > 0.0
        v3 = np.where(pos, v * v * v, 1.0)
        with np.errstate(invalid="ignore", divide="ignore"):
            acc = pos & (np.log(u) < 0.5 * x * x + d - d * v3 + d * np.log(v3))
        take = acc & ~done
        result[take] = d[take] * v3[take]
        done |= acc
    n_exhausted = int((~done).sum())
    result[~done] = d[~done]
    if boost.any():
        w = philox4x32_10(sites, 2 * GAMMA_ATTEMPTS, counter, c3, k0, k1)
        u = (u53(w[0], w[1]) + 1.0) * 2.0 ** -53
        result = np.where(boost, result * u ** (1.0 / np.where(boost, shape, 1.0)), result)
    return result * scale, n_exhausted
