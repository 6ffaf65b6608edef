// lbmhd_batch_run.cuh -- one run of an ensemble as the device sees it
// (shared by the ensemble step kernel and the ensemble kinetic kernels).
#pragma once

#include "lbmhd_device.cuh"

namespace lbmhd {

template <class R>
struct RunDev {
    long long off;   // element offset of the run's 19 planes in each state buffer
    long long moff;  // element offset of its 5 moment planes (les 2, 3)
    long long ps;    // plane stride (elements)
    int nx, ny;
    unsigned total;  // live threads of the run (nx / V * ny)
    unsigned unit0;  // first work unit of the run
    int kstrips;     // fused kinetic kernel: column strips of the run
    int kseglen;     // ... and rows per segment (units = strips x segments)
    Coll<R> c;
};

}  // namespace lbmhd
