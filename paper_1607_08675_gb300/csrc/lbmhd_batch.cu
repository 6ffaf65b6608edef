// lbmhd_batch.cu -- an ensemble of independent lattices (uneven sizes,
// own C_S and relaxation times) advanced together by one persistent kernel.
//
// All runs live in one pair of buffers (each run a 19-plane block).  The
// work of one step is cut into units of `block` threads; a unit belongs to
// exactly one run (each run's thread range is padded to a whole number of
// units), and unit_run[] maps units to runs.  A persistent grid of
// co-resident CTAs walks the units of step s, meets at a grid barrier, and
// goes on with step s + 1 -- `steps_per_launch` steps per launch; the host
// replays a captured CUDA graph of such launches.  A launch of a single step
// needs no barrier and covers the units with one CTA each instead.  Per thread the work is
// step_body, the same code as the single-lattice kernel, so every run
// evolves bit-identically to its own lbmhd_t.
//
// The grid barrier spins with a bounded wait (%globaltimer, about one
// second): on expiry the CTA records LBMHD_ETIMEOUT in the status word and
// returns, so a missing arrival can never hang the GPU.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbmhd_batch_run.cuh"
#include "lbmhd_internal.h"
#include "lbmhd_step_body.cuh"

namespace lbmhd {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier over co-resident CTAs (sense by generation counter).
// Returns false when this CTA gave up waiting (status bit 2 set).
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned* gen, unsigned nblocks,
                                          int* status) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = *(volatile unsigned*)gen;
        __threadfence();  // this CTA's stores before its arrival
        if (atomicAdd(count, 1u) == nblocks - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*(volatile unsigned*)gen == g) {
                if (global_ns() - t0 > 1000000000ull) {  // ~1 s
                    atomicOr(status, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();  // the other CTAs' stores before this CTA reads
    }
    __syncthreads();
    return ok != 0;
}

template <int P, int V>
__global__ void __launch_bounds__(256) batch_kernel(const RunDev<typename Fmt<P>::R>* __restrict__ runs,
                                                    const int* __restrict__ unit_run,
                                                    unsigned nunits, typename Fmt<P>::S* bufA,
                                                    typename Fmt<P>::S* bufB, int nsteps,
                                                    int start_parity, unsigned* bar, int* status,
                                                    int drop_arrival, float scale,
                                                    float inv_scale) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    // fault injection for tests: CTA 0 leaves before the first barrier
    const bool leave = drop_arrival && blockIdx.x == 0;
    for (int s = 0; s < nsteps; ++s) {
        const bool odd = ((start_parity + s) & 1) != 0;
        const S* src = odd ? bufB : bufA;
        S* dst = odd ? bufA : bufB;
        // the unit -> run lookup of the next unit is issued one unit ahead,
        // and the run descriptor stays in registers while the run repeats
        unsigned u = blockIdx.x;
        int r_next = u < nunits ? __ldg(unit_run + u) : 0;
        int r_cur = -1;
        RunDev<R> rd;
        for (; u < nunits; u += gridDim.x) {
            const int r = r_next;
            const unsigned un = u + gridDim.x;
            r_next = un < nunits ? __ldg(unit_run + un) : 0;
            if (r != r_cur) {
                rd = runs[r];
                r_cur = r;
            }
            const unsigned t = (u - rd.unit0) * blockDim.x + threadIdx.x;
            step_body<P, V>(src + rd.off, dst + rd.off, rd.nx, rd.ny, rd.ps, t, rd.total, rd.c,
                            scale, inv_scale);
        }
        if (s + 1 < nsteps) {
            if (leave) return;
            if (!grid_sync(bar, bar + 1, gridDim.x, status)) return;
        }
    }
}

}  // namespace lbmhd

using namespace lbmhd;

struct lbmhd_batch_t {
    int nruns;
    std::vector<int> nx, ny;
    std::vector<double> tau_nu, tau_eta, cs;
    std::vector<long long> off, ps;
    lbmhd_params p;
    int device;
    cudaStream_t stream;
    bool own_stream, capturable;
    void* buf[2];
    void* d_runs;
    int* d_unit_run;
    void* d_mom;  // les 2, 3: every run's five moment planes
    unsigned nunits;
    unsigned* d_bar;
    int* d_flag;
    int vec, block, spl, grid;
    int cur;
    int64_t steps, launches;
    std::vector<char> run_init;
    cudaGraphExec_t graph;
    int graph_cur, graph_len;
    bool failed;
    int drop_arrival;
};

namespace {

constexpr int kGraphLaunches = 8;

int bfail(int code, const std::string& m) {
    set_error(m);
    return code;
}

int bcuda(lbmhd_batch_t* b, cudaError_t e, const char* where) {
    if (b) b->failed = true;
    cudaGetLastError();
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return LBMHD_ECUDA;
}

#define LBMHD_BCK(b, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call);  \
    } while (0)

HostColl run_coll(const lbmhd_batch_t* b, int r) {
    lbmhd_params q = b->p;
    q.tau_nu = b->tau_nu[r];
    q.tau_eta = b->tau_eta[r];
    q.C_S = b->cs[r];
    HostColl c;
    c.tn = q.tau_nu;
    c.te = q.tau_eta;
    const double cd2 = q.C_S * q.delta * q.delta;
    c.k18 = 18.0 * cd2;
    c.k36 = 36.0 * cd2;
    c.s5 = q.s5 > 0.0 ? q.s5 : 1.0 / q.tau_nu;
    c.s6 = q.s6 > 0.0 ? q.s6 : 1.0 / q.tau_nu;
    c.tie5 = q.s5 > 0.0 ? 0 : 1;
    c.tie6 = q.s6 > 0.0 ? 0 : 1;
    c.s7 = q.s7 > 0.0 ? q.s7 : 0.0;
    c.s8 = q.s8 > 0.0 ? q.s8 : 0.0;
    c.les = q.les == 1 ? 1 : 0;
    c.kin = q.les >= 2 ? q.les : 0;
    c.d2 = q.delta * q.delta;
    c.scale = (float)q.fp16_scale;
    c.inv_scale = (float)(1.0 / q.fp16_scale);
    return c;
}

Geom run_geom(const lbmhd_batch_t* b, int r) {
    Geom g;
    g.nx = b->nx[r];
    g.ny = b->ny[r];
    g.ps = b->ps[r];
    return g;
}

void* run_ptr(const lbmhd_batch_t* b, int which, int r) {
    return (char*)b->buf[which] + b->off[r] * (long long)storage_bytes(b->p.precision);
}

template <int P, int V>
const void* kernel_ptr() {
    return (const void*)batch_kernel<P, V>;
}

const void* pick_kernel(int prec, int vec) {
#define LBMHD_K(P)                                 \
    case P:                                        \
        if (vec == 1) return kernel_ptr<P, 1>();   \
        if (vec == 2) return kernel_ptr<P, 2>();   \
        if (vec == 4) return kernel_ptr<P, 4>();   \
        break;
    switch (prec) {
        LBMHD_K(P_FP64)
        LBMHD_K(P_FP32)
        LBMHD_K(P_FP32_DEV)
        LBMHD_K(P_FP16_DEV)
        LBMHD_K(P_FF)
    }
#undef LBMHD_K
    return nullptr;
}

// Rows per segment of the fused kinetic ensemble kernel: segments of at
// most 128 rows, of even length within a run (each segment forms two moment
// rows again, 1.6% extra pulls at 128).
int kin_seglen(int ny) {
    const int nseg = (ny + 127) / 128;
    return (ny + nseg - 1) / nseg;
}

template <class R>
int upload_runs_t(lbmhd_batch_t* b) {
    std::vector<RunDev<R>> rd(b->nruns);
    std::vector<int> map;
    unsigned unit = 0;
    long long moff = 0;
    const bool kin = b->p.les >= 2;
    const int ksw = kinetic_fused_strip(b->p.precision);
    for (int r = 0; r < b->nruns; ++r) {
        const HostColl hc = run_coll(b, r);
        rd[r].off = b->off[r];
        rd[r].moff = moff;
        moff += 5 * b->ps[r];
        rd[r].ps = b->ps[r];
        rd[r].nx = b->nx[r];
        rd[r].ny = b->ny[r];
        // kinetic closures: one node per thread (vec 0 selects the two-pass kernels)
        const int v = kin ? 1 : b->vec;
        rd[r].total = (unsigned)((long long)b->nx[r] / v * b->ny[r]);
        rd[r].unit0 = unit;
        rd[r].kstrips = (b->nx[r] + ksw - 1) / ksw;
        rd[r].kseglen = kin_seglen(b->ny[r]);
        rd[r].c = coll_for_prec<R>(hc, b->p.precision);
        const unsigned units =
            kin && b->vec == 1
                ? (unsigned)rd[r].kstrips * (unsigned)((b->ny[r] + rd[r].kseglen - 1) / rd[r].kseglen)
                : (rd[r].total + b->block - 1) / b->block;
        for (unsigned u = 0; u < units; ++u) map.push_back(r);
        unit += units;
    }
    b->nunits = unit;
    if (b->d_runs) cudaFree(b->d_runs);
    if (b->d_unit_run) cudaFree(b->d_unit_run);
    b->d_runs = nullptr;
    b->d_unit_run = nullptr;
    LBMHD_BCK(b, cudaMalloc(&b->d_runs, rd.size() * sizeof(RunDev<R>)));
    LBMHD_BCK(b, cudaMalloc((void**)&b->d_unit_run, map.size() * sizeof(int)));
    LBMHD_BCK(b, cudaMemcpy(b->d_runs, rd.data(), rd.size() * sizeof(RunDev<R>),
                            cudaMemcpyHostToDevice));
    LBMHD_BCK(b, cudaMemcpy(b->d_unit_run, map.data(), map.size() * sizeof(int),
                            cudaMemcpyHostToDevice));
    return LBMHD_OK;
}

// (Re)build the unit map and the co-resident grid for the current shape.
int configure(lbmhd_batch_t* b) {
    int rc = b->p.precision == LBMHD_FP64 ? upload_runs_t<double>(b)
             : b->p.precision == LBMHD_FF ? upload_runs_t<ff>(b)
                                          : upload_runs_t<float>(b);
    if (rc) return rc;
    if (b->p.les >= 2) {  // one CTA per unit, no persistent grid
        b->grid = 1;
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        return LBMHD_OK;
    }
    const void* k = pick_kernel(b->p.precision, b->vec);
    if (!k) return bfail(LBMHD_EINVAL, "no batched kernel for this precision / vector width");
    int per_sm = 0, sms = 0;
    LBMHD_BCK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, b->block, 0));
    LBMHD_BCK(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    if (per_sm < 1) return bfail(LBMHD_EINVAL, "batched kernel cannot be resident at this shape");
    long long grid = (long long)per_sm * sms;
    if (grid > (long long)b->nunits) grid = b->nunits;
    b->grid = (int)std::max<long long>(1, grid);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    return LBMHD_OK;
}

cudaError_t launch_batch(lbmhd_batch_t* b, int nsteps, int parity) {
    if (b->p.les >= 2) {  // kinetic closures: the fused kernel, or moments pass + step
        const HostColl hc = run_coll(b, 0);
        for (int s = 0; s < nsteps; ++s) {
            const bool odd = ((parity + s) & 1) != 0;
            const cudaError_t e = launch_batch_kinetic(
                b->p.precision, hc.kin, b->vec == 1, b->d_runs, b->d_unit_run, b->nunits,
                b->block, odd ? b->buf[1] : b->buf[0], odd ? b->buf[0] : b->buf[1], b->d_mom,
                hc.inv_scale, b->stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const void* k = pick_kernel(b->p.precision, b->vec);
    const HostColl hc = run_coll(b, 0);
    void* bufA = b->buf[0];
    void* bufB = b->buf[1];
    int drop = b->drop_arrival;
    float scale = hc.scale, inv_scale = hc.inv_scale;
    void* args[] = {&b->d_runs, &b->d_unit_run, &b->nunits, &bufA, &bufB, &nsteps,
                    &parity, &b->d_bar, &b->d_flag, &drop, &scale, &inv_scale};
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3((unsigned)b->block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident (grid barrier)
    attr[0].val.cooperative = 1;
    if (nsteps > 1) {
        cfg.gridDim = dim3((unsigned)b->grid);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    } else {
        // one step, no barrier: one CTA per work unit, scheduled by the hardware
        cfg.gridDim = dim3(b->nunits);
        cfg.attrs = nullptr;
        cfg.numAttrs = 0;
    }
    return cudaLaunchKernelExC(&cfg, k, args);
}

// Capture kGraphLaunches persistent launches (spl steps each) starting at
// the current buffer parity.  False (with the error cleared) when the
// driver refuses to capture them.
bool capture_graph(lbmhd_batch_t* b) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int parity = b->cur;
    bool ok = true;
    for (int l = 0; l < kGraphLaunches && ok; ++l) {
        ok = launch_batch(b, b->spl, parity) == cudaSuccess;
        parity = (parity + b->spl) & 1;
    }
    const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    ok = ok && ee == cudaSuccess && g;
    if (ok) ok = cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        b->graph = nullptr;
        return false;
    }
    b->graph_cur = b->cur;
    b->graph_len = b->spl * kGraphLaunches;
    return true;
}

int check_batch(lbmhd_batch_t* b) {
    if (!b) return bfail(LBMHD_EINVAL, "batch is NULL");
    if (b->failed) return bfail(LBMHD_ECUDA, "batch is unusable after a CUDA error");
    return LBMHD_OK;
}

int read_batch_flag(lbmhd_batch_t* b) {
    int flag = 0;
    LBMHD_BCK(b, cudaMemcpyAsync(&flag, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    LBMHD_BCK(b, cudaStreamSynchronize(b->stream));
    if (flag & 2) {
        // a barrier wait expired: the ensemble state is undefined until
        // re-initialised; clear the barrier and the report
        cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->stream);
        cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream);
        cudaStreamSynchronize(b->stream);
        std::fill(b->run_init.begin(), b->run_init.end(), 0);
        return bfail(LBMHD_ETIMEOUT, "a grid-barrier wait expired in the batched kernel");
    }
    if (flag & 1) return bfail(LBMHD_ENONFINITE, "non-finite density detected");
    return LBMHD_OK;
}

// ---- autotuner cache: a flat JSON object {"key": [vec, block, spl, mlups]} ----
std::mutex g_tune_mu;

std::map<std::string, std::vector<double>> load_cache(const std::string& path) {
    std::map<std::string, std::vector<double>> m;
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) return m;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, n);
    std::fclose(f);
    size_t i = 0;
    while ((i = s.find('"', i)) != std::string::npos) {
        const size_t j = s.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string key = s.substr(i + 1, j - i - 1);
        const size_t a = s.find('[', j), e = s.find(']', j);
        if (a == std::string::npos || e == std::string::npos || e < a) break;
        std::vector<double> v;
        const char* q = s.c_str() + a + 1;
        while (q < s.c_str() + e) {
            char* end = nullptr;
            const double x = std::strtod(q, &end);
            if (end == q) {
                ++q;
                continue;
            }
            v.push_back(x);
            q = end;
        }
        if (v.size() == 4) m[key] = v;
        i = e + 1;
    }
    return m;
}

void save_cache(const std::string& path, const std::map<std::string, std::vector<double>>& m) {
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    std::fprintf(f, "{\n");
    size_t k = 0;
    for (const auto& kv : m) {
        std::fprintf(f, "  \"%s\": [%d, %d, %d, %.1f]%s\n", kv.first.c_str(), (int)kv.second[0],
                     (int)kv.second[1], (int)kv.second[2], kv.second[3],
                     ++k < m.size() ? "," : "");
    }
    std::fprintf(f, "}\n");
    std::fclose(f);
    std::rename(tmp.c_str(), path.c_str());
}

std::string tune_key(const lbmhd_batch_t* b) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, b->device) == cudaSuccess) name = prop.name;
    for (char& ch : name)
        if (ch == '"' || ch == '\\') ch = '_';
    // the size mix: a histogram of lattice shapes
    std::map<std::pair<int, int>, int> hist;
    for (int r = 0; r < b->nruns; ++r) ++hist[{b->nx[r], b->ny[r]}];
    std::string key = name + "|p" + std::to_string(b->p.precision);
    for (const auto& kv : hist)
        key += "|" + std::to_string(kv.first.first) + "x" + std::to_string(kv.first.second) +
               ":" + std::to_string(kv.second);
    return key;
}

}  // namespace

extern "C" {

int lbmhd_batch_create(int nruns, const int* nx, const int* ny, const double* tau_nu,
                       const double* tau_eta, const double* C_S, const lbmhd_params* common,
                       lbmhd_batch_t** out) {
    if (!out || !nx || !ny || !tau_nu || !tau_eta || !C_S || !common)
        return bfail(LBMHD_EINVAL, "NULL argument");
    if (nruns < 1) return bfail(LBMHD_EINVAL, "nruns must be >= 1");
    // every run must pass the single-lattice validation
    long long total_cells = 0;
    for (int r = 0; r < nruns; ++r) {
        lbmhd_params q = *common;
        q.tau_nu = tau_nu[r];
        q.tau_eta = tau_eta[r];
        q.C_S = C_S[r];
        const int rc = validate_params(nx[r], ny[r], &q);
        if (rc) return rc;
        total_cells += (long long)nx[r] * ny[r];
    }
    if (total_cells > (1LL << 31)) return bfail(LBMHD_EINVAL, "ensemble exceeds 2^31 nodes");

    lbmhd_batch_t* b = new (std::nothrow) lbmhd_batch_t();
    if (!b) return bfail(LBMHD_ENOMEM, "host allocation failed");
    b->nruns = nruns;
    b->nx.assign(nx, nx + nruns);
    b->ny.assign(ny, ny + nruns);
    b->tau_nu.assign(tau_nu, tau_nu + nruns);
    b->tau_eta.assign(tau_eta, tau_eta + nruns);
    b->cs.assign(C_S, C_S + nruns);
    b->p = *common;
    b->run_init.assign(nruns, 0);
    long long off = 0;
    for (int r = 0; r < nruns; ++r) {
        const long long ps = plane_stride(nx[r], ny[r]);
        b->off.push_back(off);
        b->ps.push_back(ps);
        off += kNumPlanes * ps;
    }
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
        delete b;
        return bcuda(nullptr, e, "cudaGetDevice");
    }
    if (common->stream) {
        b->stream = (cudaStream_t)common->stream;
        b->own_stream = false;
        b->capturable = common->stream != (void*)cudaStreamLegacy &&
                        common->stream != (void*)cudaStreamPerThread;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return bcuda(nullptr, e, "cudaStreamCreateWithFlags");
        }
        b->own_stream = true;
        b->capturable = true;
    }
    const size_t bytes = (size_t)off * storage_bytes(common->precision);
    void* mem[4] = {nullptr, nullptr, nullptr, nullptr};
    const size_t sizes[4] = {bytes, bytes, 2 * sizeof(unsigned), sizeof(int)};
    for (int i = 0; i < 4; ++i) {
        e = cudaMalloc(&mem[i], sizes[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaFree(mem[j]);
            if (b->own_stream) cudaStreamDestroy(b->stream);
            delete b;
            cudaGetLastError();
            return bfail(e == cudaErrorMemoryAllocation ? LBMHD_ENOMEM : LBMHD_ECUDA,
                         std::string("device allocation failed: ") + cudaGetErrorString(e));
        }
    }
    b->buf[0] = mem[0];
    b->buf[1] = mem[1];
    b->d_bar = (unsigned*)mem[2];
    b->d_flag = (int*)mem[3];
    if (common->les >= 2) {
        long long mplanes = 0;
        for (int r = 0; r < nruns; ++r) mplanes += 5 * b->ps[r];
        const size_t rb =
            common->precision == LBMHD_FP64 || common->precision == LBMHD_FF ? 8 : 4;
        e = cudaMalloc(&b->d_mom, (size_t)mplanes * rb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            lbmhd_batch_destroy(b);
            return bfail(LBMHD_ENOMEM, "device allocation failed (ensemble moment planes)");
        }
    }
    cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned));
    cudaMemset(b->d_flag, 0, sizeof(int));
    // default shape: the widest vector dividing every run's nx, 64 threads
    int v = 4;
    if (common->precision == LBMHD_FP64 || common->precision == LBMHD_FF) v = 2;
    for (; v > 1; v >>= 1) {
        bool ok = true;
        for (int r = 0; r < nruns; ++r) ok = ok && nx[r] % v == 0;
        if (ok) break;
    }
    b->vec = v;
    b->block = v == 4 ? 64 : 128;
    b->spl = 8;
    if (common->les >= 2) {
        // kinetic closures, one step per launch: the fused kernel (vec 1)
        // where the single lattice takes it, else the two-pass kernels (vec 0,
        // 128 nodes per unit) -- FP64, and FF with the filtered equilibria
        b->vec = common->precision == LBMHD_FP64 ||
                         (common->precision == LBMHD_FF && common->les == 2)
                     ? 0
                     : 1;
        b->block = 128;
        b->spl = 1;
    }
    int rc = configure(b);
    if (rc) {
        lbmhd_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBMHD_OK;
}

int lbmhd_batch_set_launch(lbmhd_batch_t* b, int vec, int block, int steps_per_launch) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (b->p.les >= 2) {
        if ((vec != 0 && vec != 1) || steps_per_launch != 1)
            return bfail(LBMHD_EINVAL,
                         "les 2, 3 ensembles: vec 1 (fused kernel) or 0 (two-pass kernels), "
                         "one step per launch");
    } else {
        if (vec != 1 && vec != 2 && vec != 4) return bfail(LBMHD_EINVAL, "vec must be 1, 2 or 4");
        for (int r = 0; r < b->nruns; ++r)
            if (b->nx[r] % vec) return bfail(LBMHD_EINVAL, "vec must divide every run's nx");
    }
    if (block < 32 || block > 256 || block % 32)
        return bfail(LBMHD_EINVAL, "block must be a multiple of 32 in [32, 256]");
    if (steps_per_launch < 1 || steps_per_launch > 4096)
        return bfail(LBMHD_EINVAL, "steps_per_launch must be in [1, 4096]");
    LBMHD_BCK(b, cudaStreamSynchronize(b->stream));
    b->vec = vec;
    b->block = block;
    b->spl = steps_per_launch;
    return configure(b);
}

int lbmhd_batch_get_launch(const lbmhd_batch_t* b, int* vec, int* block, int* steps_per_launch) {
    if (!b || !vec || !block || !steps_per_launch) return bfail(LBMHD_EINVAL, "NULL argument");
    *vec = b->vec;
    *block = b->block;
    *steps_per_launch = b->spl;
    return LBMHD_OK;
}

int lbmhd_batch_init(lbmhd_batch_t* b, int run, const double* rho, const double* ux,
                     const double* uy, const double* bx, const double* by) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (run < 0 || run >= b->nruns) return bfail(LBMHD_EINVAL, "run index out of range");
    if (!rho || !ux || !uy || !bx || !by) return bfail(LBMHD_EINVAL, "NULL field");
    const long long n = (long long)b->nx[run] * b->ny[run];
    for (long long c = 0; c < n; ++c)
        if (!(rho[c] > 0.0) || !std::isfinite(rho[c]))
            return bfail(LBMHD_EINVAL, "rho must be positive and finite");
    double* tmp = nullptr;
    LBMHD_BCK(b, cudaMallocAsync((void**)&tmp, 5 * n * sizeof(double), b->stream));
    const double* src[5] = {rho, ux, uy, bx, by};
    for (int i = 0; i < 5; ++i)
        LBMHD_BCK(b, cudaMemcpyAsync(tmp + i * n, src[i], n * sizeof(double),
                                     cudaMemcpyHostToDevice, b->stream));
    LBMHD_BCK(b, launch_init(b->p.precision, tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, tmp + 4 * n,
                             run_ptr(b, b->cur, run), run_geom(b, run), run_coll(b, run),
                             b->stream));
    LBMHD_BCK(b, cudaFreeAsync(tmp, b->stream));
    LBMHD_BCK(b, cudaStreamSynchronize(b->stream));
    b->run_init[run] = 1;
    b->steps = 0;
    return LBMHD_OK;
}

int lbmhd_batch_step(lbmhd_batch_t* b, int n) {
    TraceRange trace_("lbmhd_batch_step");
    int rc = check_batch(b);
    if (rc) return rc;
    if (n < 0) return bfail(LBMHD_EINVAL, "n must be >= 0");
    for (int r = 0; r < b->nruns; ++r)
        if (!b->run_init[r]) return bfail(LBMHD_ESTATE, "every run must be initialised first");
    int done = 0;
    const int chunk = b->spl * kGraphLaunches;
    while (done < n) {
        if (n - done >= chunk && b->capturable && !b->drop_arrival) {
            if (!b->graph || b->graph_cur != b->cur) {
                if (b->graph) cudaGraphExecDestroy(b->graph);
                b->graph = nullptr;
                if (!capture_graph(b)) {
                    // capture of the cooperative launch is not available:
                    // keep issuing launches directly
                    b->capturable = false;
                    continue;
                }
            }
            LBMHD_BCK(b, cudaGraphLaunch(b->graph, b->stream));
            b->cur = (b->cur + chunk) & 1;
            b->launches += kGraphLaunches;
            b->steps += chunk;
            done += chunk;
            continue;
        }
        const int k = std::min(b->spl, n - done);
        LBMHD_BCK(b, launch_batch(b, k, b->cur));
        b->cur = (b->cur + k) & 1;
        ++b->launches;
        b->steps += k;
        done += k;
    }
    return LBMHD_OK;
}

int lbmhd_batch_moments(lbmhd_batch_t* b, int run, double* rho, double* ux, double* uy,
                        double* bx, double* by) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (run < 0 || run >= b->nruns) return bfail(LBMHD_EINVAL, "run index out of range");
    if (!rho || !ux || !uy || !bx || !by) return bfail(LBMHD_EINVAL, "NULL field");
    if (!b->run_init[run]) return bfail(LBMHD_ESTATE, "run not initialised");
    const long long n = (long long)b->nx[run] * b->ny[run];
    double* tmp = nullptr;
    LBMHD_BCK(b, cudaMallocAsync((void**)&tmp, 5 * n * sizeof(double), b->stream));
    LBMHD_BCK(b, launch_moments(b->p.precision, run_ptr(b, b->cur, run), tmp, tmp + n, tmp + 2 * n,
                                tmp + 3 * n, tmp + 4 * n, run_geom(b, run), run_coll(b, run),
                                b->stream));
    double* dst[5] = {rho, ux, uy, bx, by};
    for (int i = 0; i < 5; ++i)
        LBMHD_BCK(b, cudaMemcpyAsync(dst[i], tmp + i * n, n * sizeof(double),
                                     cudaMemcpyDeviceToHost, b->stream));
    LBMHD_BCK(b, cudaFreeAsync(tmp, b->stream));
    return read_batch_flag(b);
}

int lbmhd_batch_get_state(lbmhd_batch_t* b, int run, double* state) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (run < 0 || run >= b->nruns) return bfail(LBMHD_EINVAL, "run index out of range");
    if (!state) return bfail(LBMHD_EINVAL, "state is NULL");
    if (!b->run_init[run]) return bfail(LBMHD_ESTATE, "run not initialised");
    const long long n = (long long)b->nx[run] * b->ny[run];
    double* tmp = nullptr;
    LBMHD_BCK(b, cudaMallocAsync((void**)&tmp, kNumPlanes * n * sizeof(double), b->stream));
    LBMHD_BCK(b, launch_get_state(b->p.precision, run_ptr(b, b->cur, run), tmp, run_geom(b, run),
                                  run_coll(b, run), b->stream));
    LBMHD_BCK(b, cudaMemcpyAsync(state, tmp, kNumPlanes * n * sizeof(double),
                                 cudaMemcpyDeviceToHost, b->stream));
    LBMHD_BCK(b, cudaFreeAsync(tmp, b->stream));
    return read_batch_flag(b);
}

int lbmhd_batch_sync(lbmhd_batch_t* b) {
    int rc = check_batch(b);
    if (rc) return rc;
    return read_batch_flag(b);
}

int64_t lbmhd_batch_step_count(const lbmhd_batch_t* b) { return b ? b->steps : 0; }

int64_t lbmhd_batch_launch_count(const lbmhd_batch_t* b) { return b ? b->launches : 0; }

int lbmhd_batch_debug(lbmhd_batch_t* b, int flags) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (flags & ~LBMHD_DEBUG_DROP_BARRIER_ARRIVAL) return bfail(LBMHD_EINVAL, "unknown debug flag");
    b->drop_arrival = (flags & LBMHD_DEBUG_DROP_BARRIER_ARRIVAL) ? 1 : 0;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    return LBMHD_OK;
}

int lbmhd_batch_autotune(lbmhd_batch_t* b, const char* cache_path, int trial_steps,
                         double* best_mlups) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (trial_steps < 2) return bfail(LBMHD_EINVAL, "trial_steps must be >= 2");
    for (int r = 0; r < b->nruns; ++r)
        if (b->run_init[r]) return bfail(LBMHD_ESTATE, "autotune runs before lbmhd_batch_init");
    const std::string key = tune_key(b);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::map<std::string, std::vector<double>> cache;
    if (cache_path && *cache_path) {
        cache = load_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end()) {
            rc = lbmhd_batch_set_launch(b, (int)it->second[0], (int)it->second[1],
                                        (int)it->second[2]);
            if (rc == LBMHD_OK) {
                if (best_mlups) *best_mlups = it->second[3];
                return LBMHD_OK;
            }
        }
    }
    // timing state: every run at rest (rho = 1, u = B = 0), built on device
    long long maxn = 0, cells = 0;
    for (int r = 0; r < b->nruns; ++r) {
        maxn = std::max(maxn, (long long)b->nx[r] * b->ny[r]);
        cells += (long long)b->nx[r] * b->ny[r];
    }
    double* f = nullptr;
    LBMHD_BCK(b, cudaMallocAsync((void**)&f, 5 * maxn * sizeof(double), b->stream));
    LBMHD_BCK(b, cudaMemsetAsync(f, 0, 5 * maxn * sizeof(double), b->stream));
    {
        std::vector<double> ones(maxn, 1.0);
        LBMHD_BCK(b, cudaMemcpyAsync(f, ones.data(), maxn * sizeof(double), cudaMemcpyHostToDevice,
                                     b->stream));
        LBMHD_BCK(b, cudaStreamSynchronize(b->stream));
    }
    for (int r = 0; r < b->nruns; ++r)
        LBMHD_BCK(b, launch_init(b->p.precision, f, f + maxn, f + 2 * maxn, f + 3 * maxn,
                                 f + 4 * maxn, run_ptr(b, b->cur, r), run_geom(b, r),
                                 run_coll(b, r), b->stream));
    LBMHD_BCK(b, cudaFreeAsync(f, b->stream));
    cudaEvent_t e0, e1;
    LBMHD_BCK(b, cudaEventCreate(&e0));
    LBMHD_BCK(b, cudaEventCreate(&e1));
    double best = -1.0;
    int bv = b->vec, bb = b->block, bs = b->spl;
    const int vecs[4] = {4, 2, 1, 0};
    const int blocks[3] = {64, 128, 256};
    const int spls[3] = {1, 8, 64};
    for (int v : vecs)
        for (int bl : blocks)
            for (int s : spls) {
                if (lbmhd_batch_set_launch(b, v, bl, s) != LBMHD_OK) continue;
                const int warm = std::min(s, trial_steps);
                LBMHD_BCK(b, launch_batch(b, warm, b->cur));
                b->cur = (b->cur + warm) & 1;
                LBMHD_BCK(b, cudaEventRecord(e0, b->stream));
                int done = 0;
                while (done < trial_steps) {
                    const int k = std::min(s, trial_steps - done);
                    LBMHD_BCK(b, launch_batch(b, k, b->cur));
                    b->cur = (b->cur + k) & 1;
                    done += k;
                }
                LBMHD_BCK(b, cudaEventRecord(e1, b->stream));
                LBMHD_BCK(b, cudaEventSynchronize(e1));
                float ms = 0.f;
                LBMHD_BCK(b, cudaEventElapsedTime(&ms, e0, e1));
                const double mlups = (double)cells * trial_steps / (ms * 1e-3) / 1e6;
                if (mlups > best) {
                    best = mlups;
                    bv = v;
                    bb = bl;
                    bs = s;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    rc = read_batch_flag(b);
    if (rc) return rc;
    rc = lbmhd_batch_set_launch(b, bv, bb, bs);
    if (rc) return rc;
    if (best_mlups) *best_mlups = best;
    if (cache_path && *cache_path) {
        cache[key] = {(double)bv, (double)bb, (double)bs, best};
        save_cache(cache_path, cache);
    }
    b->steps = 0;
    return LBMHD_OK;
}

void lbmhd_batch_destroy(lbmhd_batch_t* b) {
    if (!b) return;
    if (!b->failed) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->buf[0]);
    cudaFree(b->buf[1]);
    cudaFree(b->d_runs);
    cudaFree(b->d_unit_run);
    cudaFree(b->d_mom);
    cudaFree(b->d_bar);
    cudaFree(b->d_flag);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
