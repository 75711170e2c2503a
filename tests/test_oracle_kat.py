"""The oracle still reproduces its stored known answers (regression guard).

The file was written by tests/golden/make_kat.py, which calls only the
oracle; the paper prints no vectors of its own.
"""
import os

from tests.golden.make_kat import KEYS, message

KAT = os.path.join(os.path.dirname(__file__), "golden", "kat_paper_reading_v1.txt")


def load_kat():
    rows = []
    for line in open(KAT):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        rows.append((int(parts[0]), int(parts[1]), [int(x, 16) for x in parts[2:6]]))
    return rows


def test_oracle_reproduces_kat(oracle):
    rows = load_kat()
    assert len(rows) == len(KEYS) * 112
    for ki, length, h in rows:
        assert oracle.hash256(KEYS[ki], message(length)) == h, (ki, length)
