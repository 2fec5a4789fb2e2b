"""Planted mistakes: do the oracle's pins catch a wrong oracle?

Each mutant is a copy of ``oracle/bshuffle_oracle.c`` with one plausible
error planted by text replacement -- a dropped term, swapped operands, a
wrong index or shift, an off-by-one comparison, a mistyped constant, a scan
taken in the wrong order.  It is built with gcc into a temporary library,
and the CPU pin modules run against it in a child process (the oracle loads
the library named by BSHUFFLE_ORACLE_LIB).  Every mutant must make a pin
fail on an assertion (or trip the oracle's own check that Algorithm 1 keeps
exactly n indices); the unmodified source, built the same way, must pass.
This tests the pins, not the oracle: nothing here changes oracle/."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bshuffle_oracle.c")

# The pin modules, fastest first (the child stops at its first failure).
PINS = ["tests/test_oracle_bijection.py", "tests/test_oracle_shuffle.py", "tests/test_oracle_shapley.py",
        "tests/test_oracle_statistics.py"]

# name -> (text of the correct source, its planted replacement); each text
# occurs exactly once in the source.
MUTANTS = {
    # Listing 1 / Sec. 3.2, forward round
    "round key dropped from F": (
        "state0 = (uint32_t)(((uint64_t)(hi ^ keys[r]) ^ state1) & left_mask);",
        "state0 = (uint32_t)(((uint64_t)hi ^ state1) & left_mask);"),
    "high and low product words swapped": (
        "uint32_t hi = (uint32_t)(product >> 32);\n        uint32_t lo = (uint32_t)product;",
        "uint32_t hi = (uint32_t)product;\n        uint32_t lo = (uint32_t)(product >> 32);"),
    "odd bit taken from the bottom of the right half": (
        "| (uint32_t)(state1 >> left_bits);",
        "| (uint32_t)(state1 & 1u);"),
    "halves joined with the wrong shift": (
        "    return ((uint64_t)state0 << right_bits) | (uint64_t)state1;\n}\n\n/* Multiplicative",
        "    return ((uint64_t)state0 << left_bits) | (uint64_t)state1;\n}\n\n/* Multiplicative"),
    # Sec. 3.2, inversion steps
    "inverse puts the odd bit above the right half": (
        "uint64_t right = right_low | (b << left_bits);",
        "uint64_t right = right_low | (b << right_bits);"),
    "M0 inverse with too few Newton steps": (
        "for (it = 0; it < 5; it++)",
        "for (it = 0; it < 3; it++)"),
    # key schedule and domain readings
    "SplitMix64 multiplier mistyped": (
        "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;",
        "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B8ULL;"),
    "smallest domain exponent 3": (
        "static const uint32_t ORACLE_K_MIN = 4;",
        "static const uint32_t ORACLE_K_MIN = 3;"),
    # Algorithm 1 (Sec. 4)
    "filter keeps the image equal to n": (
        "int flag = (b < n) ? 1 : 0;",
        "int flag = (b <= n) ? 1 : 0;"),
    "threaded scan of the range counts in reverse order": (
        "for (t = 0; t < threads; t++) {   /* exclusive scan of the range counts */",
        "for (t = threads; t-- > 0;) {   /* exclusive scan of the range counts */"),
    "inverse shuffle gathers instead of scattering": (
        "memcpy(y + b * elem_bytes, x + j * elem_bytes, elem_bytes);",
        "memcpy(y + j * elem_bytes, x + b * elem_bytes, elem_bytes);"),
    # Sec. 3.1 LCG, the permutation test statistic, Shapley pivots
    "LCG multiplier not forced odd": (
        "*a = (oracle_splitmix64_next(&state) | 1) & mask;",
        "*a = oracle_splitmix64_next(&state) & mask;"),
    "group-mean difference taken the other way": (
        "T[b] = sum1 / (double)n1 - sum2 / (double)(n - n1);",
        "T[b] = sum2 / (double)(n - n1) - sum1 / (double)n1;"),
    "first group one slot too long": (
        "if (slot < n1)",
        "if (slot <= n1)"),
    "pivot needs the quota strictly exceeded": (
        "if (before < quota && before + w[player] >= quota) {",
        "if (before < quota && before + w[player] > quota) {"),
}


def _build(source: str, tmp_path) -> str:
    c = tmp_path / "oracle_variant.c"
    c.write_text(source)
    so = tmp_path / "liboracle_variant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-pthread", "-shared", "-fPIC", "-o", str(so), str(c)])
    return str(so)


def _run_pins(lib: str) -> subprocess.CompletedProcess:
    env = dict(os.environ, BSHUFFLE_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                           *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_unmodified_source_passes_the_pins(tmp_path):
    with open(SRC) as fh:
        src = fh.read()
    r = _run_pins(_build(src, tmp_path))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    with open(SRC) as fh:
        src = fh.read()
    good, bad = MUTANTS[name]
    assert src.count(good) == 1, name
    r = _run_pins(_build(src.replace(good, bad), tmp_path))
    # 1: tests ran and one failed (not a crash, a collection error or a usage error)
    assert r.returncode == 1, (name, r.returncode, r.stdout[-3000:], r.stderr[-2000:])
    # the failure is an assertion of a pin, or the oracle's own invariant
    # check (oracle/__init__.py raises ValueError when Algorithm 1 keeps a
    # number of indices other than n), not an exception from the harness;
    # pytest ends each traceback with "<file>.py:<line>: <exception>"
    ends = re.findall(r"^(\S+\.py):\d+: (\w+)$", r.stdout, flags=re.M)
    assert ends, (name, r.stdout[-3000:])
    for path, exc in ends:
        assert exc == "AssertionError" or (exc == "ValueError" and path == "oracle/__init__.py"), \
            (name, path, exc, r.stdout[-3000:])
