"""The lane-group combine's shared-memory layout is free of bank conflicts.

The combine of deep stacks (more than 64 frames) stages each CTA's samples
in shared memory pixel-major, with a pad word after every J samples and an
odd pixel stride, so that (1) the staging stores of one frame for the CTA's
32 pixels and (2) the lanes' loads of their lane-major blocks in the sort
each touch 32 distinct banks.  The index expressions are read from the CUDA
sources, so a change of the layout is checked here, on the CPU, for every
group size G the kernel instantiates.
"""
import os
import re

import pytest

from paper_2008_11486_gb300 import build as irp_build

BANKS = 32


def _src(name):
    with open(os.path.join(irp_build.CSRC, name)) as f:
        return f.read()


def _expr(pattern, text):
    m = re.search(pattern, text)
    assert m, f"layout expression not found: {pattern}"
    # C integer division on non-negative ints
    return m.group(1).replace("/", "//")


WIDE = _src("wide.cuh")
KERNEL = _src("k_wide.cu")
PIX_STRIDE = _expr(r"kPixStride = ([^;]+);", WIDE)
AT = _expr(r"at\(int p, int e\) \{ return ([^;]+); \}", WIDE)
PIX_PER_WARP = _expr(r"constexpr int P = ([^;]+);", KERNEL)
PIXEL_OF_GROUP = _expr(r"const int p = ([^;]+);", KERNEL)
LOAD = _expr(r"col\[(tg \* \(J \+ 1\) \+ i)\]", KERNEL)
GROUPS = [int(g) for g in re.findall(r"case (\d+): return combine_wide_j<\1, 32", KERNEL)]


def _at(G, J, p, e):
    return eval(AT, {}, {"p": p, "e": e, "J": J, "kPixStride": eval(PIX_STRIDE, {}, {"G": G, "J": J})})


@pytest.mark.parametrize("G", [4, 8, 16, 32])
def test_staging_stores_hit_distinct_banks(G):
    assert G in GROUPS or G == 32  # 32 is the switch's default case
    J = 32
    for k in range(G * J):  # one frame, the CTA's 32 pixels (lane = pixel)
        banks = {_at(G, J, lane, k) % BANKS for lane in range(32)}
        assert len(banks) == 32, (G, k)


@pytest.mark.parametrize("G", [4, 8, 16, 32])
def test_sort_loads_hit_distinct_banks(G):
    J = 32
    P = eval(PIX_PER_WARP, {}, {"G": G})
    for q in range(32 // P):
        for i in range(J):
            addrs = []
            for lane in range(32):
                g, tg = lane // G, lane % G
                p = eval(PIXEL_OF_GROUP, {}, {"q": q, "g": g, "P": P})
                assert 0 <= p < 32
                addrs.append(_at(G, J, p, 0) + eval(LOAD, {}, {"tg": tg, "J": J, "i": i}))
            assert len({a % BANKS for a in addrs}) == 32, (G, q, i)


def test_sample_positions_match_the_load_index():
    # the sort reads sample e = tg J + i of pixel p at col[tg (J + 1) + i]
    for G in (4, 8, 16, 32):
        J = 32
        for tg in range(G):
            for i in range(J):
                e = tg * J + i
                assert _at(G, J, 3, e) == _at(G, J, 3, 0) + eval(LOAD, {}, {"tg": tg, "J": J,
                                                                             "i": i})
