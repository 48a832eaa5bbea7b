"""The oracle's pins catch plausible mistakes: each case compiles the oracle
with one deliberate mistake (-DORC_PLANT=n, test builds only), runs the pins
that should notice it in a child process against that build, and requires
them to fail.  The unplanted oracle passes the same pins in the rest of the
CPU suite.  Mistakes: a wrong sign in the chord formula, a missing doubling
case, a reconstruction prefix sum that skips its first term, a wrong sign
in the closed form, a wrong sign in a Strassen quadrant combination, a comb
window built from the wrong power of two, the ladder's two registers
swapped, a wrong tracking pointer in the un-sort step, a skipped difference
in the compression, k-tuple entries missing a column, and decryption's
giant step of the wrong sign."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "p256_oracle.c")

PLANTS = {
    1: ("chord x3 = lambda^2 - x1 + x2", "tests/test_oracle_curve.py"),
    2: ("P + P returns infinity instead of 2P", "tests/test_oracle_curve.py"),
    3: ("reconstruction prefix sums skip the first term", "tests/test_oracle_pcmm.py"),
    4: ("closed form uses r x - b", "tests/test_oracle_elgamal.py tests/test_oracle_pcmm.py"),
    5: ("Strassen C22 = M1 - M2 + M3 - M6", "tests/test_oracle_strassen.py"),
    6: ("comb window 5 built from 2^41 G", "tests/test_oracle_curve.py"),
    7: ("ladder registers swapped", "tests/test_oracle_pcmm.py"),
    8: ("un-sort takes the wrong entry for the first row", "tests/test_oracle_pcmm.py"),
    9: ("compression skips the first difference", "tests/test_oracle_pcmm.py"),
    10: ("k-tuple entries drop their last column", "tests/test_oracle_pcmm.py"),
    11: ("decryption's giant step adds instead of subtracting", "tests/test_oracle_elgamal.py"),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_mistake_fails_a_pin(plant, tmp_path):
    what, targets = PLANTS[plant]
    lib = str(tmp_path / f"liboracle_plant{plant}.so")
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", f"-DORC_PLANT={plant}",
                    "-o", lib, SRC], check=True)
    env = dict(os.environ, ORACLE_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
                       + targets.split(), cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"plant {plant} ({what}) was not caught:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout
