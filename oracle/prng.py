"""Random choices of the blocking stage, written from their published definitions.

The paper draws RAC anchors at random (Alg. 3) and reorders the blocks at
random (Alg. 1, Step 2) without naming a generator.  Reading adopted: one
SplitMix64 stream (Steele, Lea & Flood, OOPSLA 2014) seeded by the caller,
bounded integers by Lemire's multiply-and-reject method (ACM TOMS 2019), and
Fisher-Yates shuffles.  Python integers keep every step exact.
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


class SplitMix64:
    """state += gamma; output = mix(state) with the two published multipliers."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, s: int) -> int:
        """Uniform integer in [0, s): high word of x*s, rejecting low words below (2^64 - s) mod s."""
        assert 0 < s <= MASK64
        prod = self.next() * s
        low = prod & MASK64
        if low < s:
            t = ((1 << 64) - s) % s
            while low < t:
                prod = self.next() * s
                low = prod & MASK64
        return prod >> 64


def partial_shuffle_prefix(n: int, k: int, rng: SplitMix64) -> list[int]:
    """First k entries of a Fisher-Yates shuffle of [0, n): step j swaps a[j] with a[j + U(n - j)]."""
    swapped: dict[int, int] = {}
    out = []
    for j in range(k):
        r = j + rng.below(n - j)
        aj = swapped.get(j, j)
        ar = swapped.get(r, r)
        swapped[j] = ar
        swapped[r] = aj
        out.append(ar)
    return out


def full_shuffle(n: int, rng: SplitMix64) -> list[int]:
    """Fisher-Yates shuffle of [0, n) with steps j = 0 .. n-2 (n-1 draws)."""
    a = list(range(n))
    for j in range(n - 1):
        r = j + rng.below(n - j)
        a[j], a[r] = a[r], a[j]
    return a
