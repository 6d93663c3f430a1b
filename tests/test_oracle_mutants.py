"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (on the CPU, in a
temporary directory), builds it, and checks that at least one pin from
test_oracle.py fails against the mutant.
"""
from __future__ import annotations

import os
import subprocess

import pytest

import oracle
import test_oracle as pins
from conftest import load_golden

MUTANTS = {
    "letter_range_Z": ("b <= 'Z'", "b < 'Z'"),
    "letter_range_a": ("b >= 'a'", "b > 'a'"),
    "signed_compare": ("std::memcmp(a, c, L) > 0",
                       "(int8_t)a[0] != (int8_t)c[0] ? (int8_t)a[0] > (int8_t)c[0] : std::memcmp(a, c, L) > 0"),
    "non_strict_swap": ("std::memcmp(a, c, L) > 0", "std::memcmp(a, c, L) >= 0"),
    "short_inner_loop": ("j + 1 < m - pass", "j + 2 < m - pass"),
    "early_exit_first_pass": ("if (!swapped) break;", "break;"),
    "off_shifted": ("off[L] = r;", "off[L] = r + 1;"),
    "longer_first": ("for (uint32_t L = 1; L <= W; ++L) {\n    off[L] = r;",
                     "for (uint32_t L = W; L >= 1; --L) {\n    off[L] = r;"),
    "compare_short": ("std::memcmp(a, c, L) > 0", "std::memcmp(a, c, L - 1) > 0"),
    "stable_by_len_only": ("return std::memcmp(rec + (uint64_t)a * W, rec + (uint64_t)b * W, len[a]) < 0;",
                           "return false;"),
    "whole_non_strict_swap": ("return std::lexicographical_compare(c, c + len[y], a, a + len[x]);",
                              "return !std::lexicographical_compare(a, a + len[x], c, c + len[y]);"),
    "whole_prefix_equal": ("return std::lexicographical_compare(c, c + len[y], a, a + len[x]);",
                           "return std::memcmp(a, c, std::min(len[x], len[y])) > 0;"),
    "whole_stable_descending": ("return std::lexicographical_compare(a, a + len[x], c, c + len[y]);",
                                "return std::lexicographical_compare(c, c + len[y], a, a + len[x]);"),
}


def _run_pins(orc_mod):
    """Returns True when every pin passes against the current oracle build."""
    try:
        for case in load_golden():
            for m in ("bubble", "stable"):
                pins.test_golden(orc_mod, case, m)
        for args in [(0, 300, 8, b"ab", False), (3, 600, 8, None, True),
                     (6, 700, 24, b"aA", False)]:
            pins.test_sort_matches_python_sort(orc_mod, *args)
        for seed in range(12):
            pins.test_brute_force_tiny(orc_mod, seed)
        for seed in range(3):
            pins.test_tokenize_matches_regex(orc_mod, seed)
        pins.test_tokenize_letter_boundaries(orc_mod)
        pins.test_reverse_sorted_swaps(orc_mod)
        pins.test_identical_and_sorted_are_identity(orc_mod)
        pins.test_whole_hand_worked(orc_mod)
        for args in [(10, 300, 8, b"ab", False), (13, 600, 8, None, True)]:
            pins.test_whole_matches_python_sort(orc_mod, *args)
        for seed in range(8):
            pins.test_whole_brute_force_tiny(orc_mod, seed)
        pins.test_whole_reverse_sorted_swaps_and_differs_from_bucketed(orc_mod)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, monkeypatch, name):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert old in src, f"mutation anchor missing: {old!r}"
    mutated = src.replace(old, new, 1)
    cpp = tmp_path / "m.cpp"
    cpp.write_text(mutated)
    so = tmp_path / "libm.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so),
                           str(cpp)])
    monkeypatch.setattr(oracle, "_lib", oracle.bind(str(so)))
    assert not _run_pins(oracle), f"mutant {name} passed every pin"


def test_unmutated_passes(orc):
    assert _run_pins(orc)
