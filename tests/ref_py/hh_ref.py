"""Second, independent transcription of HighwayHash (arXiv:1612.06257, Section 4).

Test infrastructure.  Written in pure Python integers and byte strings, without
looking at the C oracle's code, and deriving its tables differently:

* the constants come from pi computed with Machin's formula (Section 4.4);
* the ZipperMerge map is parsed from the string printed in Section 4.1;
* Permute follows the prose of Section 4.3 (swap the 128-bit halves of v0 and
  the 32-bit halves of each lane) rather than the printed index list;
* Update follows the second printing of the listing (Section 6.2).

The readings of unspecified details are the same ones the C oracle uses: the
64-bit add of (r << 32) + r, a left rotation of v1's 32-bit halves by r, and
the last r mod 4 bytes in packet bytes 28..30.
"""
from __future__ import annotations

from .pi_hex import pi_fraction_words

M64 = (1 << 64) - 1
M32 = (1 << 32) - 1

# Section 4.1, as printed (result byte 15 listed first).
ZIPPER_PRINTED = "7 8 6 9 D A 4 B 0 F 1 E 5 2 C 3"
# Section 4.3, as printed (indices of 32-bit parts).
PERMUTE_PRINTED = "2 3 0 1 6 7 4 5"


def zipper_offsets() -> list[int]:
    """P_i for i = 0..15 (the printed list reversed, since i = 15 is first)."""
    printed = [int(tok, 16) for tok in ZIPPER_PRINTED.split()]
    return printed[::-1]


_P = zipper_offsets()


def _constant(words: list[int]) -> list[int]:
    """Lanes 3, 2, 1 take the first three words; lane 0 the fourth, with every
    bit set that at most one of the other three lanes has."""
    a, b, c, d = words
    lanes = [0, c, b, a]
    for bit in range(64):
        others = ((a >> bit) & 1) + ((b >> bit) & 1) + ((c >> bit) & 1)
        if others <= 1:
            d |= 1 << bit
    lanes[0] = d
    return lanes


def constants() -> tuple[list[int], list[int]]:
    w = pi_fraction_words(8)
    return _constant(w[0:4]), _constant(w[4:8])


def zipper_merge(v: list[int]) -> list[int]:
    out = []
    for k in (0, 2):
        src = v[k].to_bytes(8, "little") + v[k + 1].to_bytes(8, "little")
        res = bytes(src[_P[i]] for i in range(16))
        out.append(int.from_bytes(res[:8], "little"))
        out.append(int.from_bytes(res[8:], "little"))
    return out


def rot32(x: int) -> int:
    return ((x << 32) | (x >> 32)) & M64


def permute(v0: list[int]) -> list[int]:
    """Swap the two 128-bit halves, and the 32-bit halves within each lane."""
    swapped = [v0[2], v0[3], v0[0], v0[1]]
    return [rot32(x) for x in swapped]


def mul_epu32(a: int, b: int) -> int:
    return (a & M32) * (b & M32)


class State:
    def __init__(self, key: list[int]):
        c0, c1 = constants()
        self.v0 = [(key[i] ^ c0[i]) & M64 for i in range(4)]
        self.v1 = [(rot32(key[i]) ^ c1[i]) & M64 for i in range(4)]
        self.mul0 = list(c0)
        self.mul1 = list(c1)

    def update(self, pkt: list[int]) -> None:
        v0, v1, mul0, mul1 = self.v0, self.v1, self.mul0, self.mul1
        for i in range(4):
            v1[i] = (v1[i] + pkt[i]) & M64
            v1[i] = (v1[i] + mul0[i]) & M64
            mul0[i] ^= mul_epu32(v1[i], v0[i] >> 32)
            v0[i] = (v0[i] + mul1[i]) & M64
            mul1[i] ^= mul_epu32(v0[i], v1[i] >> 32)
        z = zipper_merge(v1)
        for i in range(4):
            v0[i] = (v0[i] + z[i]) & M64
        z = zipper_merge(v0)
        for i in range(4):
            v1[i] = (v1[i] + z[i]) & M64

    def digest(self, words: int) -> list[int]:
        return [(self.v0[i] + self.v1[i] + self.mul0[i] + self.mul1[i]) & M64
                for i in range(words)]


def _rotl32(w: int, r: int) -> int:
    r %= 32
    return ((w << r) | (w >> (32 - r))) & M32 if r else w


def hash_words(key: list[int], msg: bytes, words: int = 1, rounds: int = 4) -> list[int]:
    st = State(key)
    full = len(msg) - len(msg) % 32
    for pos in range(0, full, 32):
        st.update([int.from_bytes(msg[pos + 8 * i: pos + 8 * i + 8], "little")
                   for i in range(4)])
    tail = msg[full:]
    r = len(tail)
    if r:
        inject = (r << 32) | r
        st.v0 = [(x + inject) & M64 for x in st.v0]
        st.v1 = [(_rotl32(x >> 32, r) << 32) | _rotl32(x & M32, r) for x in st.v1]
        q = r - r % 4
        pkt = tail[:q] + bytes(28 - q) + tail[q:] + bytes(4 - r % 4)
        assert len(pkt) == 32
        st.update([int.from_bytes(pkt[8 * i: 8 * i + 8], "little") for i in range(4)])
    for _ in range(rounds):
        st.update(permute(st.v0))
    return st.digest(words)


def hash64(key, msg: bytes) -> int:
    return hash_words(key, msg, 1)[0]
