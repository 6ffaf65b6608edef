"""The diagnostics reduction's work split (csrc/lbmhd_diag_plan.h), checked
on the host: the header is plain C++, compiled here with g++ into a small
driver that prints the plan for a list of (nx, ny, resident warps, SMs).

Properties: the strips and segments cover the lattice exactly once; the
grid never exceeds the 1024 partial rows; the launched warps are a whole
number of waves of the resident warps (unless the lattice has fewer
units), at least 48 per SM when the cap allows; and the split follows the
device it is planned for -- two SM counts give different plans for the
same lattice."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

DRIVER = r"""
#include <cstdio>
#include "lbmhd_diag_plan.h"
int main() {
    long long nx, ny, warps; int nsm;
    while (std::scanf("%lld %lld %lld %d", &nx, &ny, &warps, &nsm) == 4) {
        const lbmhd::DiagPlan d = lbmhd::diag_plan((int)nx, (int)ny, warps, nsm);
        std::printf("%d %d %d %d %lld\n", d.nstrips, d.nseg, d.seglen, d.nblocks, d.nunits);
    }
    return 0;
}
"""

CASES = [(8192, 8192, 3 * 8 * 152, 152), (8192, 8192, 3 * 8 * 132, 132),
         (8192, 8192, 1 * 8 * 152, 152), (2048, 2048, 3 * 8 * 152, 152),
         (2048, 2048, 2 * 8 * 76, 76), (30007, 53, 3 * 8 * 152, 152), (1, 1, 24 * 152, 152),
         (123, 77, 3 * 8 * 152, 152), (32768, 32768, 3 * 8 * 152, 152),
         (1 << 24, 4, 3 * 8 * 152, 152), (4, 1 << 24, 3 * 8 * 152, 152)]


@pytest.fixture(scope="module")
def plans(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("plan")
    src, exe = d / "plan.cpp", d / "plan"
    src.write_text(DRIVER)
    inc = os.path.join(ROOT, "paper_1607_08675_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)], check=True)
    inp = "".join(f"{a} {b} {c} {e}\n" for a, b, c, e in CASES)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True)
    return {c: tuple(int(v) for v in line.split())
            for c, line in zip(CASES, out.stdout.strip().splitlines())}


def wave_target(warps, nsm):
    """Warps the split aims at: whole waves of the resident warps, at least
    48 per SM, at most the 8192 partial rows."""
    cap = 1024 * 8
    if warps >= cap:
        return cap
    waves = -(-48 * nsm // warps)
    if waves * warps > cap:
        waves = cap // warps
    return max(8, waves * warps)


@pytest.mark.parametrize("case", CASES)
def test_plan_covers_the_lattice_in_whole_waves(plans, case):
    nx, ny, warps, nsm = case
    nstrips, nseg, seglen, nblocks, nunits = plans[case]
    assert nstrips * 30 >= nx > (nstrips - 1) * 30
    assert nseg * seglen >= ny > (nseg - 1) * seglen
    assert nunits == nstrips * nseg
    assert 1 <= nblocks <= 1024
    target = wave_target(warps, nsm)
    assert target % warps == 0 or target == 1024 * 8
    launched = min(nunits, target)
    assert nblocks == -(-launched // 8)
    nseg0 = target // nstrips
    if 1 <= nseg0 <= ny:
        # rows are not the bound: as many segments as fit the target, then
        # even lengths (never more units than the target)
        assert seglen == -(-ny // nseg0) and nunits <= target


def test_plan_follows_the_device(plans):
    """The same lattice on a 152-SM and a 132-SM device: each split is cut
    to its own device's waves."""
    a = plans[(8192, 8192, 3 * 8 * 152, 152)]
    b = plans[(8192, 8192, 3 * 8 * 132, 132)]
    assert a != b
    assert a[4] <= wave_target(3 * 8 * 152, 152) and b[4] <= wave_target(3 * 8 * 132, 132)
    assert a[4] > wave_target(3 * 8 * 132, 132)
