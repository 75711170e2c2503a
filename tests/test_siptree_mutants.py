"""The SipTreeHash pins catch plausible slips in its oracle (no GPU).

Each case copies oracle/sipo.c to a temporary directory, plants one plausible
mistake, builds the copy with gcc and runs every pin of
tests/test_siptree_oracle.py against it.  At least one pin must fail for every
mutant.  The committed oracle source is never modified.
"""
import inspect
import os
import shutil

import pytest

from oracle import siptree
from tests import test_siptree_oracle as pins

MUTANTS = {
    "rotation 13 read as 12": ("rotl64(s->v1, 13)", "rotl64(s->v1, 12)"),
    "rotation 21 read as 12": ("rotl64(s->v3, 21)", "rotl64(s->v3, 12)"),
    "missing v2 rotation": ("  s->v2 = rotl64(s->v2, 32);\n", ""),
    "finalisation marker on v3": ("s.v2 ^= 0xff;", "s.v3 ^= 0xff;"),
    "length byte one place low": ("(uint64_t)(len & 0xff) << 56", "(uint64_t)(len & 0xff) << 48"),
    "no v0 ^= m after the rounds": ("  s->v0 ^= m;\n", ""),
    "key words swapped in v0": ("s.v0 = k0 ^ ascii_constant(0);", "s.v0 = k1 ^ ascii_constant(0);"),
    "constants little-endian": ("x = (x << 8) | (uint8_t)kText[8 * which + i];",
                                "x |= (uint64_t)(uint8_t)kText[8 * which + i] << (8 * i);"),
    "words dealt in blocks, not interleaved": ("padded + 8 * (4 * i + j)",
                                               "padded + 8 * (j * vectors + i)"),
    "fold without the length": ("store_le64(fold + 32, (uint64_t)len);", "store_le64(fold + 32, 0);"),
    "fold lanes in reverse order": ("store_le64(fold + 8 * j, lanes[j]);",
                                    "store_le64(fold + 8 * j, lanes[3 - j]);"),
    "lanes keyed with words 2 and 3": ("sipo_siphash(key[0], key[1], lane_bytes",
                                       "sipo_siphash(key[2], key[3], lane_bytes"),
    "fold with c and d swapped": ("return sipo_siphash(key[0], key[1], fold, sizeof(fold), c, d);",
                                  "return sipo_siphash(key[0], key[1], fold, sizeof(fold), d, c);"),
    "padding to 16-byte vectors": ("(len + 31) / 32", "(len + 15) / 16"),
}


def _pin_functions():
    out = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        params = list(inspect.signature(fn).parameters)
        cases = [dict(zip(params, cd)) for cd in pins.ROUNDS] if params == ["c", "d"] else [{}]
        for kw in cases:
            out.append((name, fn, kw))
    return out


def _detectors(lib):
    saved = siptree._lib
    siptree._lib = lib
    failures = []
    try:
        for name, fn, kw in _pin_functions():
            try:
                fn(**kw)
            except AssertionError:
                failures.append(name)
    finally:
        siptree._lib = saved
    return failures


def test_unmutated_oracle_passes_every_pin():
    assert _detectors(siptree.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(siptree.SRC).read()
    assert text.count(old) == 1, "mutation site not found: " + name
    shutil.copy(siptree.HDR, tmp_path / "sipo.h")
    src = tmp_path / "sipo_mutant.c"
    src.write_text(text.replace(old, new))
    path = siptree.build(force=True, src=str(src), out=str(tmp_path / "libmutant.so"))
    caught = _detectors(siptree.SipOracle(path))
    assert caught, "no pin caught the mutant: " + name
