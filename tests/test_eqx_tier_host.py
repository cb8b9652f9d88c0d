"""The short index-tier comparison of triples that each lie on one x-value
(time_cmp_eqx in the device predicates) against the general index tier
(time_cmp_index), compiled for the host from the same header: identical signs
on seeded random pairs with shared points, both orientations, and coordinates
spread over the full range or packed into a few values (so that the second,
dy, coefficient decides too).  A wrong sign on either coefficient shows up as
thousands of mismatches."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_equal_x_short_form_matches_the_general_index_tier(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "eqx_tier_check"
    subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "host", "eqx_tier_check.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe), "200000"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    checked, mismatches = (int(t) for t in out.stdout.split()[-3::2])
    assert checked > 100000 and mismatches == 0
