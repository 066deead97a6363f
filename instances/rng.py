"""SplitMix64: the 64-bit counter-based generator of Steele, Lea and Flood (OOPSLA 2014).

Written from its published definition (golden-gamma increment, two xor-shift-multiply
rounds, final xor-shift).  Used so that instances are bit-identical on x86 and Arm hosts.
"""

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, k: int) -> int:
        """Integer in [0, k) by rejection (exactly uniform)."""
        if k <= 0:
            raise ValueError("k must be positive")
        limit = ((1 << 64) // k) * k
        while True:
            x = self.next_u64()
            if x < limit:
                return x % k
