"""The pins catch plausible slips in the oracle (no GPU).

Each case copies oracle/hho.c to a temporary directory, plants one plausible
mistake by text substitution, builds that copy with gcc and runs the pin
checks against it.  At least one check must fail for every mutant.  The
committed oracle source is never modified.
"""
import os
import random

import pytest

import oracle as oracle_pkg
from tests import test_oracle_pins as pins
from tests.ref_py import hh_ref

SRC = os.path.join(os.path.dirname(oracle_pkg.__file__), "hho.c")

MUTANTS = {
    "drop v1 += mul0": (
        "for (i = 0; i < 4; ++i) s->v1[i] += s->mul0[i];", ""),
    "multiply without >> 32": (
        "mul_lo32(s->v1[i], s->v0[i] >> 32)", "mul_lo32(s->v1[i], s->v0[i])"),
    "second ZipperMerge from old v0": (
        "  hho_zipper_merge(s->v0, zm);\n  for (i = 0; i < 4; ++i) s->v1[i] += zm[i];",
        "  for (i = 0; i < 4; ++i) s->v1[i] += zm[i];"),
    "swap the two ZipperMerge targets": (
        "for (i = 0; i < 4; ++i) s->v0[i] += zm[i];", "for (i = 0; i < 4; ++i) s->v1[i] += zm[i];"),
    "ZipperMerge map read i = 0 first": (
        "res[i] = src[kZipperPrinted[15 - i]]", "res[i] = src[kZipperPrinted[i]]"),
    "ZipperMerge map one entry off": (
        "0x5, 0x2, 0xC, 0x3}", "0x2, 0x5, 0xC, 0x3}"),
    "Permute indices read part 0 first": (
        "res[j] = part[kPermutePrinted[7 - j]]", "res[j] = part[kPermutePrinted[j]]"),
    "constant lanes in listing order": (
        "  c[3] = w[0];\n  c[2] = w[1];\n  c[1] = w[2];\n  c[0] = w[3] | ~majority(w[0], w[1], w[2]);",
        "  c[0] = w[0];\n  c[1] = w[1];\n  c[2] = w[2];\n  c[3] = w[3] | ~majority(w[0], w[1], w[2]);"),
    "fix with AND instead of OR": (
        "w[3] | ~majority", "w[3] & ~majority"),
    "second constant from the same pi words": (
        "make_constant(&kPiWords[4], c1);", "make_constant(&kPiWords[0], c1);"),
    "v1 init without rotation": (
        "s->v1[i] = rot32(key[i]) ^ c1[i];", "s->v1[i] = key[i] ^ c1[i];"),
    "size injected into v1": (
        "s->v0[i] += ((uint64_t)r << 32) + (uint64_t)r;",
        "s->v1[i] += ((uint64_t)r << 32) + (uint64_t)r;"),
    "last bytes at packet start": (
        "pkt[28 + k] = tail[q + k];", "pkt[q + k] = tail[q + k];"),
    "last bytes dropped": (
        "for (k = 0; k < (r & 3); ++k) pkt[28 + k] = tail[q + k];", ""),
    "big-endian packet words": (
        "for (i = 7; i >= 0; --i) x = (x << 8) | p[i];",
        "for (i = 0; i < 8; ++i) x = (x << 8) | p[i];"),
    "three finalisation rounds": (
        "hho_hash_rounds(key, msg, len, 64, 4, out);", "hho_hash_rounds(key, msg, len, 64, 3, out);"),
    "output xor instead of add": (
        "h[i] = s->v0[i] + s->v1[i] + s->mul0[i] + s->mul1[i];",
        "h[i] = s->v0[i] ^ s->v1[i] ^ s->mul0[i] ^ s->mul1[i];"),
    "remainder update for whole packets": (
        "  if (r == 0) return;\n", ""),
    "last packet treated as remainder": (
        "size_t pos, full = len & ~(size_t)31;", "size_t pos, full = len ? (len - 1) & ~(size_t)31 : 0;"),
}

PIN_CHECKS = [
    pins.test_constants_from_pi,
    pins.test_init_state,
    pins.test_zipper_merge_matches_printed_map,
    pins.test_zipper_merge_random_vs_byte_definition,
    pins.test_permute_matches_printed_indices,
    pins.test_permute_matches_prose,
    pins.test_update_inverse_round_trip,
    pins.test_update_multiply_is_32x32,
    pins.test_multiple_of_32_needs_no_padding,
    pins.test_zero_messages_of_every_length_differ,
    pins.test_trailing_zeros_change_the_hash,
    pins.test_remainder_uses_every_tail_byte,
    pins.test_remainder_structure_via_inverse,
    pins.test_output_widths_share_lanes,
]


def _transcription_agrees(lib):
    r = random.Random(30)
    key = [r.getrandbits(64) for _ in range(4)]
    data = bytes(r.getrandbits(8) for _ in range(160))
    for length in range(0, 161):
        assert lib.hash256(key, data[:length]) == hh_ref.hash_words(key, data[:length], 4)


def _detectors(lib):
    failures = []
    for check in PIN_CHECKS + [_transcription_agrees]:
        try:
            check(lib)
        except AssertionError:
            failures.append(check.__name__)
    return failures


def test_unmutated_oracle_passes_every_detector(oracle):
    assert _detectors(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, "mutation site not found: " + name
    src = tmp_path / "hho_mutant.c"
    src.write_text(text.replace(old, new))
    path = oracle_pkg.build(force=True, src=str(src), out=str(tmp_path / "libmutant.so"))
    lib = oracle_pkg.OracleLib(path)
    caught = _detectors(lib)
    assert caught, "no pin caught the mutant: " + name
    # The pins alone (without the second transcription) catch every mutant
    # except those in details only the transcription fixes.
    pin_only = [c for c in caught if c != "_transcription_agrees"]
    if name not in ("three finalisation rounds",):
        assert pin_only, "only the transcription caught: " + name
