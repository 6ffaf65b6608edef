// lbmhd_diag_plan.h -- the work split of the diagnostics reduction (plain
// host C++, no CUDA types, so that it can be checked on its own).
//
// A warp sweeps a strip of kOwn columns down a segment of rows; the work is
// cut into units of one warp each, a whole number of waves of the kernel's
// resident warps and at least kDiagMinWarps warps per SM (the fastest split
// at 8192^2 for every ring depth and residency tried: fewer warps leave the
// memory system short of requests, a part-filled last wave leaves SMs
// idle), and never more than kDiagBlocks blocks of kDiagWarps warps (the
// partial rows a call may write).
#pragma once

namespace lbmhd {

constexpr int kOwn = 30, kDiagWarps = 8, kDiagBlocks = 1024;
constexpr int kDiagMinWarps = 48;

struct DiagPlan {
    int nstrips, nseg, seglen, nblocks;
    long long nunits;
};

// nx, ny: the lattice; resident_warps: warps of the reduction kernel the
// device holds at once; nsm: its SM count.
inline DiagPlan diag_plan(int nx, int ny, long long resident_warps, int nsm) {
    DiagPlan d;
    d.nstrips = (nx + kOwn - 1) / kOwn;
    const long long want = (long long)kDiagMinWarps * nsm;
    const long long cap = (long long)kDiagBlocks * kDiagWarps;  // partial rows
    long long target = cap;
    if (resident_warps < cap) {
        long long waves = (want + resident_warps - 1) / resident_warps;
        if (waves * resident_warps > cap) waves = cap / resident_warps;  // whole waves only
        target = waves * resident_warps;
    }
    if (target < kDiagWarps) target = kDiagWarps;
    long long nseg = target / d.nstrips;
    if (nseg > ny) nseg = ny;
    if (nseg < 1) nseg = 1;
    d.seglen = (int)((ny + nseg - 1) / nseg);
    d.nseg = (int)((ny + d.seglen - 1) / d.seglen);
    d.nunits = (long long)d.nstrips * d.nseg;
    const long long warps = d.nunits < target ? d.nunits : target;
    d.nblocks = (int)((warps + kDiagWarps - 1) / kDiagWarps);
    return d;
}

}  // namespace lbmhd
