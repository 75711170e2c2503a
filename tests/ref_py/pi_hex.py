"""Hexadecimal digits of pi from Machin's formula, in exact integer arithmetic.

pi = 16 atan(1/5) - 4 atan(1/239).  Used to pin the initialisation constants
of Section 4.4 (openly derived numbers taken from pi's hex digits)
without trusting any stored digit table.
"""


def _atan_inv(x: int, one: int) -> int:
    """atan(1/x) scaled by `one`, by its alternating Taylor series."""
    total = 0
    power = one // x          # one / x^(2k+1)
    x2 = x * x
    k = 0
    while power:
        term = power // (2 * k + 1)
        total += -term if k & 1 else term
        power //= x2
        k += 1
    return total


def pi_fraction_words(count: int) -> list[int]:
    """The first `count` 64-bit words of the fractional part of pi."""
    bits = 64 * count
    guard = 64
    one = 1 << (bits + guard)
    pi = 16 * _atan_inv(5, one) - 4 * _atan_inv(239, one)
    frac = (pi - 3 * one) >> guard          # fractional part, `bits` bits
    return [(frac >> (bits - 64 * (i + 1))) & ((1 << 64) - 1) for i in range(count)]
