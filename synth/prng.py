"""Seeded pseudo-random numbers for the synthetic scene generators.

Two published generators, written from their definitions:

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) expands a user seed into well-mixed 64-bit words.
* PCG32, the XSH-RR output function over a 64-bit LCG (O'Neill, "PCG: A family
  of simple fast space-efficient statistically good algorithms for random
  number generation", 2014), draws the stream.

Doubles in [0, 1) take 53 bits from two 32-bit outputs (27 high + 26 low
bits).  Normal deviates use the Box-Muller transform (Box and Muller, 1958),
keeping only the cosine branch so that every draw consumes exactly two
uniforms.  Nothing here knows about visibility; the module only makes numbers.
"""

import math

_M64 = (1 << 64) - 1
_PCG_MULT = 6364136223846793005


def splitmix64(state):
    """One SplitMix64 step: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


class PCG32:
    """PCG32 (XSH-RR) seeded through SplitMix64."""

    def __init__(self, seed, stream=0):
        s = int(seed) & _M64
        s, init_state = splitmix64(s ^ (int(stream) * 0xD1B54A32D192ED03 & _M64))
        s, init_seq = splitmix64(s)
        self.inc = ((init_seq << 1) | 1) & _M64
        self.state = 0
        self.next_u32()
        self.state = (self.state + init_state) & _M64
        self.next_u32()

    def next_u32(self):
        old = self.state
        self.state = (old * _PCG_MULT + self.inc) & _M64
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self, lo=0.0, hi=1.0):
        a = self.next_u32() >> 5
        b = self.next_u32() >> 6
        u = (a * 67108864 + b) / 9007199254740992.0
        return lo + (hi - lo) * u

    def randint(self, lo, hi):
        """Integer uniform on [lo, hi] (inclusive) by rejection, no modulo bias."""
        span = hi - lo + 1
        if span <= 0:
            raise ValueError("empty range")
        limit = (1 << 32) - ((1 << 32) % span)
        while True:
            x = self.next_u32()
            if x < limit:
                return lo + x % span

    def normal(self, mean=0.0, sigma=1.0):
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return mean + sigma * math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def exponential(self, rate):
        return -math.log(1.0 - self.uniform()) / rate
