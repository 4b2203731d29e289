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


def oracle_element_source() -> str:
    """The oracle's parameter struct, constants and element routine, with its
    double type replaced by the recording scalar GT of method_count.cpp (and
    its real-part helpers left to the harness)."""
    src = open(os.path.join(ROOT, "oracle", "nsrhs_oracle.cpp")).read()
    start = src.index("struct Params")
    end = src.index("template <class T>\nvoid gather")
    body = src[start:end]
    body = "\n".join(ln for ln in body.splitlines() if not ln.startswith("inline double re("))
    return re.sub(r"\bdouble\b", "GT", body)


def method_census(tmp_path):
    d = os.path.join(HERE, "flopcount")
    (tmp_path / "oracle_element.inc").write_text(oracle_element_source())
    exe = str(tmp_path / "method_count")
    subprocess.check_call(["g++", "-std=c++17", "-O0", "-I" + str(tmp_path), "-o", exe,
                           os.path.join(d, "method_count.cpp")])
    out = subprocess.check_output([exe], text=True)
    got = {}
    for line in out.splitlines():
        m = re.match(r"(\w+) method fwd_total (\d+) geometry (\d+) per_call (\d+) "
                     r"vjp_per_call (\d+)", line)
        if m:
            got[m.group(1)] = tuple(int(x) for x in m.groups()[1:])
    return got


def bench_method_constants():
    src = open(os.path.join(ROOT, "bench.py")).read()
    pat = r'\{"fwd": (\d+), "vjp": (\d+), "geometry": (\d+)\}'
    plain = re.search(r'FLOPS_PER_TET_METHOD = ' + pat, src)
    vrem = re.search(r'FLOPS_PER_TET_METHOD_VREMAN = ' + pat, src)
    return tuple(map(int, plain.groups())), tuple(map(int, vrem.groups()))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_method_census_matches_bench(tmp_path):
    """The method's own operation count (the oracle's definition recorded as
    an expression DAG, plus a reverse-mode sweep for the adjoint) equals
    bench.py's constants, and is at least the kernels' restructured count
    (the restructuring may only remove work)."""
    got = method_census(tmp_path)
    plain, vrem = bench_method_constants()
    for name, (fwd, vjp, geo) in (("plain", plain), ("vreman", vrem)):
        total, geometry, per_call, vjp_per_call = got[name]
        assert (per_call, vjp_per_call, geometry) == (fwd, vjp, geo), (name, got[name])
        assert total == per_call + geometry
    kernel_plain, kernel_vrem = bench_constants()
    assert plain[0] >= kernel_plain[0] and vrem[0] >= kernel_vrem[0]
