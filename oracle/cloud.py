"""Oracle cloud sampler (test infrastructure).

Section 3 of the paper draws bubble centres uniformly and radii from a
log-normal law clipped to [r_min, r_max]; it does not fix a random-number
generator.  Reading: SplitMix64 (Steele, Lea & Flood 2014) seeded with
seed XOR (sample_id * 0x9E3779B97F4A7C15); a uniform double is the top 53
bits times 2^-53.  Per bubble, centres are drawn by rejection from the cube
[-R, R]^3 until inside the ball of radius R (x, then y, then z per try);
then the radius: uniform r_min + u (r_max - r_min), or log-normal by
Box-Muller (n = sqrt(-2 ln(1-u1)) cos(2 pi u2), r = exp(mu + sigma n)),
redrawn until inside [r_min, r_max].  Centres are offset by L/2.

Written independently of the library's C sampler; a test asserts that the
two give identical bits.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    def __init__(self, seed: int, sample_id: int):
        self.state = (seed ^ ((sample_id * _GOLDEN) & _M64)) & _M64

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def sample_cloud(cp, seed: int, sample_id: int) -> np.ndarray:
    """(n_bubbles, 4) array of (x, y, z, r) in metres."""
    rng = SplitMix64(seed, sample_id)
    R = cp.cloud_radius
    c = 0.5 * cp.domain_L
    out = np.zeros((cp.n_bubbles, 4))
    for b in range(cp.n_bubbles):
        while True:
            x = (2.0 * rng.uniform() - 1.0) * R
            y = (2.0 * rng.uniform() - 1.0) * R
            z = (2.0 * rng.uniform() - 1.0) * R
            if x * x + y * y + z * z <= R * R:
                break
        if cp.radius_law == 0:
            r = cp.r_min + rng.uniform() * (cp.r_max - cp.r_min)
        else:
            while True:
                u1 = rng.uniform()
                u2 = rng.uniform()
                n = math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)
                r = math.exp(cp.ln_mu + cp.ln_sigma * n)
                if cp.r_min <= r <= cp.r_max:
                    break
        out[b] = (c + x, c + y, c + z, r)
    return out
