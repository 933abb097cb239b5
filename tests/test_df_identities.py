"""Host tier for the exact FP32 identities of the double-float generator (no GPU): the
rewrites that drop conversions and instructions from the device code are only valid if these
hold bit for bit.  tests/native/df_identities.c checks, in IEEE single precision with round to
nearest and no contraction (the device's arithmetic):
* the stored values' FP64 high word from an arithmetic shift, a mask and one addition equals the
  masked rebias, for all 2^32 FP32 bit patterns (f32_to_f64_bits_fast);
* 1 - cos(theta) and cos(theta) (times 2^31) from the converted parts a, b of x + 1/2 by exact
  subtractions equal the integer conversions, for all 2^32 draws (df_direction);
* each mass gap from the neighbouring draws' parts gives FastTwoSum's pair of the converted
  integer difference, summing to it exactly (all low-byte pairs on 2048 high parts, 2^26 random
  pairs)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_exact_identities(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "df_identities")
    subprocess.check_call([cc, "-std=c11", "-O2", "-ffp-contract=off", "-o", exe,
                           os.path.join(ROOT, "tests", "native", "df_identities.c")])
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.strip() == "high word 0, direction parts 0, gaps 0", run.stdout
