"""The algorithmic flop counts that bench.py uses for the roofline are the
census of the element code itself: the device arithmetic is compiled as host
code with a counting scalar (tests/flopcount/count.cpp) and its operation
counts must equal bench.py's constants."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def bench_constants():
    src = open(os.path.join(ROOT, "bench.py")).read()
    pat = r'\{"fwd": (\d+), "vjp": (\d+), "rhs_vjp": (\d+)\}'
    plain = re.search(r'FLOPS_PER_TET = ' + pat, src)
    vrem = re.search(r'FLOPS_PER_TET_VREMAN = ' + pat, src)
    return tuple(map(int, plain.groups())), tuple(map(int, vrem.groups()))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_flop_census_matches_bench(tmp_path):
    d = os.path.join(HERE, "flopcount")
    exe = str(tmp_path / "count")
    subprocess.check_call(["g++", "-std=c++17", "-O0", "-I" + d, "-o", exe,
                           os.path.join(d, "count.cpp")])
    out = subprocess.check_output([exe], text=True)
    got = {}
    for line in out.splitlines():
        m = re.match(r"(\w+) fwd (\d+) sfu \d+ vjp (\d+) sfu \d+", line)
        if m:
            got[m.group(1)] = (int(m.group(2)), int(m.group(3)))
        m = re.match(r"(\w+) rhs\+vjp (\d+) sfu", line)
        if m:
            got[m.group(1)] += (int(m.group(2)),)
    plain, vrem = bench_constants()
    assert got["plain"] == plain
    assert got["vreman"] == vrem
