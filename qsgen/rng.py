"""Seeded pseudo-random numbers for the synthetic workloads.

SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): a 64-bit Weyl sequence with step
0x9E3779B97F4A7C15 passed through a fixed mixing function.  Uniform doubles
take the top 53 bits; normal deviates use the Box-Muller transform.

Everything here is plain Python integer arithmetic so that the streams are
identical on every host (x86_64 and aarch64) and for every numpy version.
"""

import math

_MASK = (1 << 64) - 1


class SplitMix64:
    """The SplitMix64 generator; ``next_u64`` returns the next 64-bit output."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1): the top 53 bits times 2^-53."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def randint(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("randint needs n > 0")
        bits = max(1, (n - 1).bit_length())
        while True:
            v = self.next_u64() >> (64 - bits)
            if v < n:
                return v

    def normal(self) -> float:
        """Standard normal deviate by the Box-Muller transform (one of the pair)."""
        u1 = 1.0 - self.uniform()  # in (0, 1]: the logarithm stays finite
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
