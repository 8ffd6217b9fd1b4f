"""The score c / L (§3.2) as a correctly rounded binary64 quotient computed with integer
arithmetic only (the routine the flags kernel runs), checked on the host against Python's
correctly rounded true division of the two integers."""
import os
import random
import shutil
import struct
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1706_06664_gb300", "csrc")


def _bits(v: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", v))[0]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("exact_div") / "exact_div_check")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "exact_div_check.cpp"),
                           "-o", out])

    def run(pairs):
        text = "".join(f"{c} {L}\n" for c, L in pairs)
        res = subprocess.run([out], input=text, capture_output=True, text=True, check=True).stdout.split()
        return [int(r, 16) for r in res]
    return run


def _divisors():
    ds = set(range(1, 600))
    for k in range(17):
        for v in (2 ** k - 1, 2 ** k, 2 ** k + 1, 3 * 2 ** k, 5 * 2 ** k):
            if 1 <= v <= 65536:
                ds.add(v)
    ds.update({20, 50, 64, 750, 1000, 4096, 65521, 65519, 65535, 65536, 32767, 43691, 21845})
    return sorted(ds)


def _numerators(L, rng):
    cs = {0, 1, 2, 3, L - 1, L, L + 1, 2 * L - 1, 2 * L + 1, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, 2 ** 32 - 1,
          2 ** 32 - 2, (2 ** 32 - 1) // L * L, (2 ** 32 - 1) // L * L - 1}
    for k in range(33):
        for v in (2 ** k - 1, 2 ** k, 2 ** k + 1, (2 ** k) * L, (2 ** k) * L - 1, (2 ** k) * L + 1):
            cs.add(v)
    for _ in range(40):
        cs.add(rng.getrandbits(32))
        cs.add(rng.randrange(0, 1 << rng.randrange(1, 33)))
    return sorted(c for c in cs if 0 <= c < 2 ** 32)


def test_quotient_matches_correct_rounding(checker):
    rng = random.Random(1706)
    pairs = [(c, L) for L in _divisors() for c in _numerators(L, rng)]
    got = checker(pairs)
    assert len(got) == len(pairs)
    bad = [(c, L, hex(g), hex(_bits(c / L))) for (c, L), g in zip(pairs, got) if g != _bits(c / L)]
    assert not bad, bad[:10]


def test_quotient_random_numerators(checker):
    # many random 32-bit numerators for divisors with large odd parts (the long-quotient case)
    rng = random.Random(7)
    pairs = [(rng.getrandbits(32), L) for L in (3, 7, 25, 50, 641, 2047, 65535, 65521) for _ in range(3000)]
    got = checker(pairs)
    bad = [(c, L) for (c, L), g in zip(pairs, got) if g != _bits(c / L)]
    assert not bad, bad[:10]


def test_checker_detects_truncation(checker):
    # the reference really distinguishes rounding from truncation on these inputs
    assert _bits(2 / 3) != _bits(2 / 3) - 1
    assert checker([(2, 3)]) == [_bits(2 / 3)]
    assert checker([(1, 3)]) == [_bits(1 / 3)]
