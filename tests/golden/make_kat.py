"""Write kat_paper_reading_v1.txt from the CPU oracle alone.

The paper prints no test vectors, so this file is a regression guard for the
oracle's reading of the paper, not a set of official HighwayHash vectors.
Message bytes are msg[j] = (7 * j + 3) mod 256; keys are fixed word patterns.
Run from the repository root:  python tests/golden/make_kat.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

KEYS = [
    [0, 0, 0, 0],
    [0x0706050403020100, 0x0F0E0D0C0B0A0908, 0x1716151413121110, 0x1F1E1D1C1B1A1918],
    [0xFFFFFFFFFFFFFFFF] * 4,
]
LENGTHS = list(range(0, 100)) + [127, 128, 129, 255, 256, 257, 1000, 1023, 1024, 1025, 4096, 65536]


def message(length: int) -> bytes:
    return bytes((7 * j + 3) & 0xFF for j in range(length))


def main(path=os.path.join(HERE, "kat_paper_reading_v1.txt")):
    lines = ["# HighwayHash known answers, paper reading v1 (arXiv:1612.06257 Section 4).",
             "# Written by tests/golden/make_kat.py from the CPU oracle; NOT official vectors.",
             "# msg[j] = (7*j + 3) mod 256.  Columns: key_index length h0 h1 h2 h3 (hex,",
             "# h0 = 64-bit hash, h0 h1 = 128-bit hash, h0..h3 = 256-bit hash)."]
    for ki, key in enumerate(KEYS):
        for length in LENGTHS:
            h = oracle.hash256(key, message(length))
            lines.append("%d %d %s" % (ki, length, " ".join("%016x" % x for x in h)))
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
