"""Counter-free SplitMix64 generator used by every seeded input draw.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the state advances by the golden-ratio increment
0x9E3779B97F4A7C15 and each output is the state passed through the
variant-13 finaliser (xor-shift 30/27/31 with two odd multipliers).
Uniform doubles take the top 53 bits.  The module holds no arithmetic of the
divergence-distance method; it only draws numbers.
"""

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


class SplitMix64:
    """Deterministic 64-bit generator; identical streams on every platform."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in the closed range [lo, hi] (rejection, no modulo bias)."""
        span = hi - lo + 1
        if span <= 0:
            raise ValueError("empty range")
        limit = ((1 << 64) // span) * span
        while True:
            v = self.next_u64()
            if v < limit:
                return lo + v % span

    def choice(self, n: int) -> int:
        """Uniform index in [0, n)."""
        return self.randint(0, n - 1)
