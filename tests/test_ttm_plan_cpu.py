"""CPU checks of the split-K launch planning (csrc/ttm_plan.h): the partial
sums and group sums of a K-split TTM always fit the scratch they are given,
the Multi-TTM that runs from the fixed array of cpals_multi_ttm_static
never writes past it, and the row kernels' register width covers the rank
with as few unused columns as the instantiated widths allow.  The planning header is plain C++; it is compiled
here with g++ and driven over many shapes, without a GPU."""
import os
import subprocess

import numpy as np
import pytest

from paper_2112_10855_gb300 import _build

HERE = os.path.dirname(os.path.abspath(__file__))
CAPACITY = 1 << 21          # doubles in the static array (16 MiB)
SMS = 152


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("plan") / "ttm_plan_driver")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", _build.CSRC, os.path.join(HERE, "ttm_plan_driver.cpp"),
                           "-o", exe])

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [list(map(int, ln.split())) for ln in out.stdout.strip().splitlines()]
    return run


def group_sums(ks, outn):
    return (ks + (ks + 15) // 16 if ks > 16 else ks) * outn if ks > 1 else 0


def test_split_count_respects_the_scratch(driver):
    rng = np.random.default_rng(7)
    cmds, args = [], []
    for _ in range(20000):
        ctas = int(rng.integers(1, 400))
        tpb = int(rng.choice([64, 96, 128, 256]))
        K = int(rng.integers(1, 200000))
        outn = int(rng.integers(1, 50000))
        part = int(rng.integers(0, 4 * outn * 64))
        cmds.append(f"k {ctas} {tpb} {K} {SMS} {outn} {part}")
        args.append((ctas, tpb, K, outn, part))
    for (ctas, tpb, K, outn, part), (ks, need) in zip(args, driver(cmds)):
        assert ks >= 1
        assert need == group_sums(ks, outn)
        assert need <= part, (ctas, tpb, K, outn, part, ks, need)
        # the count is already the one equal chunks of K give
        kchunk = -(-K // ks)
        assert -(-K // kchunk) == ks
        if ks > 1:
            assert K // ks >= 8 - 1   # at least ~8 indices per split


@pytest.mark.parametrize("dims,R,n", [
    ((2275, 2343, 74), 10, 2),      # split counts above 16 with the partials near the end of the array
    ((378, 1568, 1488), 3, 1),
])
def test_static_plan_of_shapes_that_used_to_overflow(driver, dims, R, n):
    ok, s0, s1, part, peak, splits = driver([f"s {len(dims)} {' '.join(map(str, dims))} {R} {n} {SMS} {CAPACITY}"])[0]
    assert s0 + s1 <= CAPACITY
    assert ok == 1 and peak <= CAPACITY
    assert splits > 1


def test_static_plan_never_exceeds_the_array(driver):
    rng = np.random.default_rng(11)
    cmds, cases = [], []
    for _ in range(6000):
        N = int(rng.integers(2, 6))
        R = int(rng.integers(1, 17))
        # log-uniform dims so that some modes are long and the rest short
        dims = [max(R, int(np.exp(rng.uniform(np.log(R), np.log(60000 if N == 2 else 4000))))) for _ in range(N)]
        n = int(rng.integers(0, N))
        cmds.append(f"s {N} {' '.join(map(str, dims))} {R} {n} {SMS} {CAPACITY}")
        cases.append((dims, R, n))
    fitted = 0
    for (dims, R, n), (ok, s0, s1, part, peak, splits) in zip(cases, driver(cmds)):
        if s0 + s1 <= CAPACITY:
            fitted += 1
            assert ok == 1 and peak <= CAPACITY, (dims, R, n, s0, s1, peak)
        else:
            assert ok == 0
    assert fitted > 1000


def test_static_plan_rejects_overflowing_products(driver):
    # prod(dims) wraps around in 64 bits
    dims = [1 << 20] * 4
    ok = driver([f"s 4 {' '.join(map(str, dims))} 2 0 {SMS} {CAPACITY}"])[0][0]
    assert ok == 0


def test_near_capacity_case_of_the_gpu_test(driver):
    # the shape test_zz_no_alloc runs: a long first mode, split more than 16
    # ways, with the partials filling most of the array
    ok, s0, s1, part, peak, splits = driver([f"s 3 40000 10 10 10 1 {SMS} {CAPACITY}"])[0]
    assert ok == 1 and splits > 16 and peak <= CAPACITY and peak > 0.9 * CAPACITY


def test_register_width_covers_the_rank(driver):
    widths = {R: w for R, (w,) in zip(range(1, 65), driver([f"w {R}" for R in range(1, 65)]))}
    allowed = set(range(1, 17)) | {20, 24, 32}
    for R, w in widths.items():
        gy = -(-R // w)
        assert w in allowed and gy * w >= R, (R, w)
        if R <= 32:
            assert gy == 1 and w == min(x for x in allowed if x >= R), (R, w)
        else:
            # the column blocks of the 32-wide tiling, each cut to the next
            # instantiated width above its share (R = 40 as 2 x 20, not 2 x 32)
            assert gy == -(-R // 32) and w == min(x for x in (20, 24, 32) if x >= -(-R // gy)), (R, w)
    assert (widths[10], widths[17], widths[33], widths[40], widths[48], widths[64]) == (10, 20, 20, 20, 24, 32)

