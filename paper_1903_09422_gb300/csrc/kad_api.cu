// Host runtime and C ABI of libkad (see include/kad.h).
//
// kad_run = Algorithm 1 of arXiv 1903.09422 (Section 2.1) with KADABRA's
// sample() and stopping condition (Section 2.3, Appendix B):
//   1. omega from the graph's vertex-diameter bound (host, a few flops);
//   2. calibration: tau0 samples (phase 1 of the Philox stream) counted per
//      vertex on the device, then the histogram of those counts, then on the
//      host the bisection for tau* and the table L[c] = log(1/delta_v);
//   3. adaptive sampling: one persistent launch of the sampling kernel that
//      also folds and checks epochs in index order until the stop rule holds
//      (another launch only if the epoch ring fills first);
//   4. b~(v) = c(v)/tau on the device.
// The host never touches per-vertex data except to return it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kad_internal.cuh"

namespace {

const int kDefaultEpoch = 1000;   // N = 1000 (Appendix C.2)
const int kDefaultCalibDiv = 100; // tau0 ~ omega / 100
const int kDefaultMcap = 256;
const int kDefaultPairCost = KAD_DEFAULT_PAIR_COST;
const int kMaxPairCost = 1 << 20;
const int kMext = 3840; // meeting-set members per slot recorded beyond the first mcap
const int32_t kTuneMinVertices = 16384;   // smaller graphs keep the default variant
const uint32_t kTuneEpochs = 4;           // epochs of the truncated query timed per candidate
const uint64_t kTuneSeed = 0x6b61646162726174ull;

struct Workspace {
    int slots = 0;            // sampling slots the scratch was last zeroed for
    size_t scratch_elems = 0; // allocated entries (slots x n) of the label records, sigma2 and list
    size_t bits_words = 0;    // allocated words of the bitmap
    size_t n_cap = 0;         // allocated entries of cnt / c0
    size_t path_elems = 0;    // allocated entries of the epoch ring's path rows
    uint32_t *label = nullptr; // 16-byte records per vertex and slot: label, -, sigma
    unsigned long long *sigma2 = nullptr;
    int32_t *list = nullptr;
    uint32_t *bits = nullptr; // labelled-vertex bitmap, nw words per slot
    size_t mext_rows = 0;     // slots the meeting-set extension holds (kMext entries each)
    int32_t *mext_id = nullptr;
    unsigned long long *mext_w = nullptr;
    // epoch ring (or record buffer)
    size_t rows = 0;
    int32_t cap = 0;
    int32_t *paths = nullptr;
    int32_t *plen = nullptr;
    uint8_t *pflag = nullptr;
    unsigned long long *pidx = nullptr; // completion order: the sample index at each fold position
    size_t pidx_cap = 0;
    int32_t *stage = nullptr;           // completion order: one staging path row per slot
    size_t stage_elems = 0;
    // the last run on this workspace, for kad_run_order
    bool last_fast = false;
    uint64_t last_positions = 0;
    // per-vertex state
    uint32_t *cnt = nullptr, *c0 = nullptr;
    double *bc = nullptr;         // bc output staged here before a copy to host memory
    // per-class state
    size_t nclass_cap = 0;
    int32_t *classmax = nullptr;
    double *ltab = nullptr;
    uint32_t *hist = nullptr;
    // control
    KadCtl *ctl = nullptr;
    uint32_t *epoch_done = nullptr;
    size_t ring_cap = 0;
    unsigned long long *work = nullptr; // [KAD_WORK_WORDS]
    bool dirty = false;                 // scratch must be re-zeroed
    // calibration hand-off: mapped pinned page (histogram + flag), pinned L table
    // and class presence for the upload, a side stream and two events
    KadHostPage *hpage = nullptr;
    KadHostPage *dpage = nullptr; // device-visible address of hpage
    size_t hpage_cap = 0;         // nclass the page and buffers hold
    double *h_ltab = nullptr;
    int32_t *h_cmax = nullptr;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_launch = nullptr, ev_aux = nullptr;
    cudaEvent_t tev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr}; // timing events
    bool tev_ok = false;
};

} // namespace

struct kad_graph {
    int device = 0;
    KadGraphDev gd{};
    int32_t vd = 0, ncomp = 0;
    int32_t max_deg = 0; // largest degree
    bool poisoned = false;
    Workspace ws;
    int tuned_threads = 0, tuned_per_sm = 0; // sampling-kernel variant chosen for this graph (0 = not yet)
    int tuned_pair_cost = 0;                 // pairwise-test cost factor chosen for it (0 = not yet)
};

namespace {

void ws_free_slots(Workspace &w) {
    cudaFree(w.label);
    cudaFree(w.sigma2);
    cudaFree(w.list);
    cudaFree(w.bits);
    cudaFree(w.mext_id);
    cudaFree(w.mext_w);
    w.label = nullptr;
    w.sigma2 = nullptr;
    w.list = nullptr;
    w.bits = nullptr;
    w.mext_id = nullptr;
    w.mext_w = nullptr;
    w.mext_rows = 0;
    w.slots = 0;
    w.scratch_elems = 0;
    w.bits_words = 0;
}

void ws_free_all(Workspace &w) {
    ws_free_slots(w);
    cudaFree(w.paths);
    cudaFree(w.plen);
    cudaFree(w.pflag);
    cudaFree(w.pidx);
    cudaFree(w.stage);
    cudaFree(w.cnt);
    cudaFree(w.c0);
    cudaFree(w.bc);
    cudaFree(w.classmax);
    cudaFree(w.ltab);
    cudaFree(w.hist);
    cudaFree(w.ctl);
    cudaFree(w.epoch_done);
    cudaFree(w.work);
    if (w.hpage) cudaFreeHost(w.hpage);
    if (w.h_ltab) cudaFreeHost(w.h_ltab);
    if (w.h_cmax) cudaFreeHost(w.h_cmax);
    if (w.aux) cudaStreamDestroy(w.aux);
    if (w.ev_launch) cudaEventDestroy(w.ev_launch);
    if (w.ev_aux) cudaEventDestroy(w.ev_aux);
    for (auto &x : w.tev)
        if (x) cudaEventDestroy(x);
    w = Workspace();
}

// A freed graph's workspace is kept for the next graph on the same device (one
// per device), so that creating, running and freeing graphs in a loop reuses
// the slot scratch instead of allocating and clearing gigabytes every time.
// kad_trim releases what is kept.
std::mutex g_ws_cache_mu;
Workspace g_ws_cache[64];
bool g_ws_cached[64];

// Graph arrays and the graph set-up's scratch come from a memory pool of the
// library's own (one per device) whose release threshold is unlimited: memory a
// freed graph returns stays mapped, so creating and freeing graphs in a loop
// maps nothing after the first round (rmat20: cudaMalloc + cudaFree of the CSR
// and the set-up scratch took 0.8 ms of a 2.9 ms create).  kad_trim unmaps it.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
bool g_pool_made[64];

cudaMemPool_t graph_pool(int dev) {
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_made[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
        g_pool_made[dev] = true;
    }
    return g_pool[dev];
}

} // namespace

cudaError_t kad_pool_alloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool = graph_pool(dev);
    if (!pool) return cudaMallocAsync(p, bytes ? bytes : 1, st);
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, st);
}

namespace {

template <typename T> cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

// Workspace buffers grow in stream order (cudaMallocAsync / cudaFreeAsync on the
// run's stream): unlike cudaMalloc / cudaFree these never synchronise the whole
// device, so one run growing its workspace does not stall runs on other streams.
template <typename T> cudaError_t dalloc_s(T **p, size_t count, cudaStream_t st) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMallocAsync((void **)p, count * sizeof(T), st);
}

template <typename T> void dfree_s(T *&p, cudaStream_t st) {
    if (p) cudaFreeAsync((void *)p, st);
    p = nullptr;
}

// geometric growth, so that a workspace meeting ever larger queries reallocates rarely
size_t grow(size_t need, size_t have) { return (need > have + have / 2) ? need : have + have / 2; }

// bytes of sampling scratch per slot and vertex: label record 16 (label, -,
// sigma), sigma2 8, list 4 (plus one bit of the labelled-vertex bitmap)
const size_t kSlotBytesPerVertex = 29;

size_t nwords(int32_t n) { return ((size_t)n + 31) / 32; }

kad_status map_err(cudaError_t e) {
    if (e == cudaSuccess) return KAD_OK;
    if (e == cudaErrorMemoryAllocation) return KAD_ERR_OOM;
    return KAD_ERR_CUDA;
}

kad_status fail(kad_graph *g, cudaError_t e) {
    kad_status s = map_err(e);
    if (s == KAD_ERR_OOM) {
        cudaGetLastError(); // allocation failures are not sticky
        return s;
    }
    if (g) g->poisoned = true;
    return s;
}

// Slot scratch for `slots` samples of a graph with n vertices.  The scratch is
// all zero between samples (each sample clears what it labelled), so a
// workspace moves between graphs without re-zeroing; only new or dirty
// (error-interrupted) scratch is cleared.
kad_status ensure_slots(kad_graph *g, Workspace &w, int slots, cudaStream_t st) {
    const size_t n = (size_t)g->gd.n;
    const size_t need = (size_t)slots * n, need_bits = (size_t)slots * nwords(g->gd.n);
    bool clear = w.dirty;
    if (need > w.scratch_elems || need_bits > w.bits_words) {
        const size_t ne = grow(need, w.scratch_elems), nb = grow(need_bits, w.bits_words);
        dfree_s(w.label, st);
        dfree_s(w.sigma2, st);
        dfree_s(w.list, st);
        dfree_s(w.bits, st);
        w.scratch_elems = w.bits_words = 0;
        if (dalloc_s(&w.label, 4 * ne, st) != cudaSuccess || dalloc_s(&w.sigma2, ne, st) != cudaSuccess ||
            dalloc_s(&w.list, ne, st) != cudaSuccess || dalloc_s(&w.bits, nb, st) != cudaSuccess) {
            cudaGetLastError();
            dfree_s(w.label, st);
            dfree_s(w.sigma2, st);
            dfree_s(w.list, st);
            dfree_s(w.bits, st);
            return KAD_ERR_OOM;
        }
        w.scratch_elems = ne;
        w.bits_words = nb;
        clear = true;
    }
    if ((size_t)slots > w.mext_rows) {
        // written before it is read by every sample: never cleared
        const size_t nr = grow((size_t)slots, w.mext_rows);
        dfree_s(w.mext_id, st);
        dfree_s(w.mext_w, st);
        w.mext_rows = 0;
        if (dalloc_s(&w.mext_id, nr * kMext, st) != cudaSuccess || dalloc_s(&w.mext_w, nr * kMext, st) != cudaSuccess) {
            cudaGetLastError();
            dfree_s(w.mext_id, st);
            dfree_s(w.mext_w, st);
            return KAD_ERR_OOM;
        }
        w.mext_rows = nr;
    }
    w.slots = slots;
    if (clear) {
        cudaError_t e;
        if ((e = cudaMemsetAsync(w.label, 0, w.scratch_elems * 16, st)) != cudaSuccess) return fail(g, e);
        if ((e = cudaMemsetAsync(w.sigma2, 0, w.scratch_elems * 8, st)) != cudaSuccess) return fail(g, e);
        if ((e = cudaMemsetAsync(w.bits, 0, w.bits_words * 4, st)) != cudaSuccess) return fail(g, e);
        w.dirty = false;
    }
    return KAD_OK;
}

kad_status ensure_rows(Workspace &w, size_t rows, int32_t cap, cudaStream_t st) {
    if (w.rows >= rows && w.path_elems >= rows * (size_t)cap) return KAD_OK;
    const size_t nr = grow(rows, w.rows), ne = grow(rows * (size_t)cap, w.path_elems);
    dfree_s(w.paths, st);
    dfree_s(w.plen, st);
    dfree_s(w.pflag, st);
    w.rows = 0;
    w.path_elems = 0;
    if (dalloc_s(&w.paths, ne, st) != cudaSuccess || dalloc_s(&w.plen, nr, st) != cudaSuccess ||
        dalloc_s(&w.pflag, nr, st) != cudaSuccess) {
        cudaGetLastError();
        dfree_s(w.paths, st);
        dfree_s(w.plen, st);
        dfree_s(w.pflag, st);
        return KAD_ERR_OOM;
    }
    w.rows = nr;
    w.cap = cap;
    w.path_elems = ne;
    return KAD_OK;
}

// Completion order: a path row per slot for the trace-back before the sample
// takes its fold position, and the sample index of every fold position a run
// can hand out (at most max_epochs * N).
kad_status ensure_order(Workspace &w, size_t stage_elems, size_t positions, cudaStream_t st) {
    if (w.stage_elems < stage_elems) {
        const size_t ne = grow(stage_elems, w.stage_elems);
        dfree_s(w.stage, st);
        w.stage_elems = 0;
        if (dalloc_s(&w.stage, ne, st) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
        w.stage_elems = ne;
    }
    if (w.pidx_cap < positions) {
        const size_t np = grow(positions, w.pidx_cap);
        dfree_s(w.pidx, st);
        w.pidx_cap = 0;
        if (dalloc_s(&w.pidx, np, st) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
        w.pidx_cap = np;
    }
    return KAD_OK;
}

kad_status ensure_fixed(kad_graph *g, Workspace &w, size_t nclass, size_t ring, cudaStream_t st) {
    const size_t n = (size_t)g->gd.n;
    if (!w.ctl) {
        if (dalloc(&w.ctl, 1) != cudaSuccess || dalloc(&w.work, KAD_WORK_WORDS) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
    }
    if (w.n_cap < n) {
        const size_t nn = grow(n, w.n_cap);
        dfree_s(w.cnt, st);
        dfree_s(w.c0, st);
        dfree_s(w.bc, st);
        w.n_cap = 0;
        if (dalloc_s(&w.cnt, nn, st) != cudaSuccess || dalloc_s(&w.c0, nn, st) != cudaSuccess ||
            dalloc_s(&w.bc, nn, st) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
        w.n_cap = nn;
    }
    if (w.nclass_cap < nclass) {
        const size_t nc = grow(nclass < 4096 ? 4096 : nclass, w.nclass_cap);
        dfree_s(w.classmax, st);
        dfree_s(w.ltab, st);
        dfree_s(w.hist, st);
        w.nclass_cap = 0;
        if (dalloc_s(&w.classmax, nc, st) != cudaSuccess || dalloc_s(&w.ltab, nc, st) != cudaSuccess ||
            dalloc_s(&w.hist, nc, st) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
        w.nclass_cap = nc;
    }
    if (!w.aux) {
        if (cudaStreamCreateWithFlags(&w.aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&w.ev_launch, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&w.ev_aux, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_CUDA;
        }
    }
    if (w.hpage_cap < nclass) {
        nclass = w.nclass_cap; // size the pinned pages like the device arrays (grown geometrically)
        if (w.hpage) cudaFreeHost(w.hpage);
        if (w.h_ltab) cudaFreeHost(w.h_ltab);
        if (w.h_cmax) cudaFreeHost(w.h_cmax);
        w.hpage = w.dpage = nullptr;
        w.h_ltab = nullptr;
        w.h_cmax = nullptr;
        w.hpage_cap = 0;
        void *dp = nullptr;
        if (cudaHostAlloc((void **)&w.hpage, sizeof(KadHostPage) + nclass * 4, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer(&dp, w.hpage, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&w.h_ltab, nclass * 8, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&w.h_cmax, nclass * 4, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
        w.dpage = (KadHostPage *)dp;
        w.hpage_cap = nclass;
    }
    if (w.ring_cap < ring) {
        ring = grow(ring, w.ring_cap);
        dfree_s(w.epoch_done, st);
        w.ring_cap = 0;
        if (dalloc_s(&w.epoch_done, ring, st) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
        w.ring_cap = ring;
    }
    return KAD_OK;
}

// ------------------------------------------------ host arithmetic of the run
// (same readings as the oracle, written independently; built with
// -ffp-contract=off so that no fused multiply-add changes a rounding)

int floor_log2(uint64_t x) {
    int r = -1;
    for (; x; x >>= 1) r++;
    return r;
}

// omega = ceil((0.5/eps^2)(floor(log2(max(VD-2,1))) + 1 + ln(2/delta)))
uint64_t run_omega(int32_t vd, double eps, double delta) {
    const int64_t a = ((int64_t)vd - 2 < 1) ? 1 : (int64_t)vd - 2;
    const double c = 0.5 / (eps * eps);
    const double inner = ((double)floor_log2((uint64_t)a) + 1.0) + log(2.0 / delta);
    return (uint64_t)ceil(c * inner);
}

uint64_t run_calib(uint64_t omega, uint32_t N, uint32_t div) {
    uint64_t a = (omega + div - 1) / div;
    if (a < 1) a = 1;
    return ((a + N - 1) / N) * N;
}

// L(b0, tau*) = tau* eps^2 / (2 b0 omega / tau* + 2 eps (1/3 + omega/tau*)): the
// log(1/delta_v) at which g(b0, delta_v, omega, tau*) = eps.
double run_L(double b0, double ts, double eps, uint64_t omega) {
    const double W = (double)omega;
    const double num = ts * (eps * eps);
    const double den = ((2.0 * b0) * W) / ts + (2.0 * eps) * ((1.0 / 3.0) + W / ts);
    return num / den;
}

double run_mass(const uint32_t *hist, uint64_t tau0, double ts, double eps, uint64_t omega) {
    double acc = 0.0;
    for (uint64_t c = 0; c <= tau0; c++) {
        if (hist[c] == 0) continue;
        const double L = run_L((double)c / (double)tau0, ts, eps, omega);
        acc += (double)hist[c] * (2.0 * exp(-L));
    }
    return acc;
}

// tau* with sum_c hist[c] 2 exp(-L) <= delta/2: hi from omega doubling, then
// exactly 100 bisection steps on [1, hi]; the result is the final hi.
double run_tau_star(const uint32_t *hist, uint64_t tau0, double eps, double delta, uint64_t omega) {
    const double target = 0.5 * delta;
    double hi = (double)omega, lo = 1.0;
    for (int i = 0; i < 4096 && run_mass(hist, tau0, hi, eps, omega) > target; i++) hi = hi * 2.0;
    for (int i = 0; i < 100; i++) {
        const double mid = 0.5 * (lo + hi);
        if (run_mass(hist, tau0, mid, eps, omega) <= target)
            hi = mid;
        else
            lo = mid;
    }
    return hi;
}

// Timing events of a run: five events owned by the workspace, created on the
// first timed run and kept (creating and destroying events on every query of a
// serving process takes driver locks that the other workers' calls wait on).
struct Events {
    cudaEvent_t *e = nullptr;
    bool on = false;
    Events(Workspace &w, bool want) {
        if (!want) return;
        if (!w.tev_ok) {
            for (auto &x : w.tev)
                if (!x && cudaEventCreate(&x) != cudaSuccess) {
                    cudaGetLastError();
                    return;
                }
            w.tev_ok = true;
        }
        e = w.tev;
        on = true;
    }
    void record(int i, cudaStream_t st) {
        if (on) cudaEventRecord(e[i], st);
    }
    double ms(int a, int b) {
        float t = 0;
        if (!on || cudaEventElapsedTime(&t, e[a], e[b]) != cudaSuccess) return 0.0;
        return (double)t;
    }
};

// Device facts that do not change while the process runs, cached (a serving
// process asks for them on every query).
int device_sms(int dev) {
    static std::mutex mu;
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[dev]) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = sms > 0 ? sms : 1;
    }
    return cache[dev];
}

int blocks_per_sm_cached(int dev, int threads, int per_sm, size_t dyn_smem) {
    static std::mutex mu;
    static std::unordered_map<unsigned long long, int> cache;
    const unsigned long long key = ((unsigned long long)(dev & 0xff) << 56) | ((unsigned long long)threads << 40) |
                                   ((unsigned long long)per_sm << 32) | (unsigned long long)(dyn_smem & 0xffffffffu);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int b = kad_sample_max_blocks_per_sm(threads, per_sm, dyn_smem);
    cache[key] = b;
    return b;
}

struct LaunchCfg {
    int threads;
    int per_sm;      // resident blocks per SM the kernel variant is compiled for
    size_t dyn_smem; // bytes of dynamic shared memory (the slot bitmap) or 0
    int warp = 0;    // 1: the warp-per-sample kernel (1024 threads, one block per SM)
    int nctx = 0;    // its sampling contexts (owner warps) per block
    int pair_cost = kDefaultPairCost; // the pairwise test's cost factor
};

bool pair_cost_ok(const kad_options &o) { return o.pair_cost >= 0 && o.pair_cost <= kMaxPairCost; }

// Threads per block and blocks per SM.  Unknown combinations fall back to the
// variant with the same block size and the default occupancy.
LaunchCfg resolve_cfg(const kad_options &o) {
    LaunchCfg c;
    if (o.pair_cost > 0) c.pair_cost = o.pair_cost;
    if (o.samples_per_block > 0) {
        c.threads = 1024;
        c.per_sm = 1;
        c.dyn_smem = 0;
        c.warp = 1;
        c.nctx = o.samples_per_block < 32 ? o.samples_per_block : 32;
        return c;
    }
    c.threads = (o.block_threads == 128 || o.block_threads == 256 || o.block_threads == 1024) ? o.block_threads : 512;
    const int def = (c.threads == 128) ? 4 : (c.threads == 256) ? 2 : (c.threads == 512) ? 2 : 1;
    c.per_sm = (o.blocks_per_sm > 0 && kad_sample_variant_exists(c.threads, o.blocks_per_sm)) ? o.blocks_per_sm : def;
    c.dyn_smem = 0;
    return c;
}

// The kernel variant when the caller names none: 256 threads x 4 blocks per SM
// on graphs of average degree up to 8 (more samples in flight pay off when rows
// are short and searches deep: the 2048^2 grid 69 ms against 105 ms), else
// 512 x 2 (hub rows want wide blocks: R-MAT scale 20 2.8 ms against 4.1 ms, the
// 4M-vertex hyperbolic graph 24.9 against 26.2 ms).
LaunchCfg default_cfg(const kad_graph *g, const kad_options &o) {
    if (o.block_threads != 0 || o.blocks_per_sm != 0 || o.samples_per_block > 0) return resolve_cfg(o);
    const bool sparse = g->gd.m <= 8 * (int64_t)g->gd.n;
    kad_options d = o;
    d.block_threads = sparse ? 256 : 512;
    d.blocks_per_sm = sparse ? 4 : 2;
    return resolve_cfg(d);
}

// The slot bitmap goes to shared memory when per_sm blocks of the variant,
// each with the bitmap, still fit an SM's shared memory.
void choose_bitmap_home(LaunchCfg &c, int32_t n, int dev) {
    int per_sm_max = 0, per_block_max = 0;
    cudaDeviceGetAttribute(&per_sm_max, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&per_block_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t stat = kad_sample_static_smem(c.threads, c.per_sm);
    const size_t dyn = ((((size_t)n + 31) / 32) * 4 + 127) & ~(size_t)127;
    const size_t reserve = 1024; // per-block system use
    if (stat + dyn <= (size_t)per_block_max && (size_t)c.per_sm * (stat + dyn + reserve) <= (size_t)per_sm_max)
        c.dyn_smem = dyn;
}

// Number of sampling slots: all resident blocks, capped by a share of free memory.
int resolve_slots(kad_graph *g, const Workspace &w, const kad_options &o, const LaunchCfg &cfg) {
    int slots = o.slots;
    if (slots <= 0 && cfg.warp) slots = device_sms(g->device) * cfg.nctx;
    if (slots <= 0) {
        const int per_sm = blocks_per_sm_cached(g->device, cfg.threads, cfg.per_sm, cfg.dyn_smem);
        slots = device_sms(g->device) * (per_sm > 0 ? per_sm : 1);
    }
    // the free-memory cap matters only when the scratch would have to grow
    const bool fits = (size_t)slots * (size_t)g->gd.n <= w.scratch_elems &&
                      (size_t)slots * nwords(g->gd.n) <= w.bits_words;
    size_t fr = 0, tot = 0;
    if (!fits && cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
        const size_t per = kSlotBytesPerVertex * (size_t)g->gd.n;
        size_t budget = fr / 3 + w.scratch_elems * (kSlotBytesPerVertex - 1) + w.bits_words * 4; // held counts too
        const size_t maxb = (size_t)96 << 30;
        if (budget > maxb) budget = maxb;
        const size_t cap = per ? budget / per : (size_t)slots;
        if ((size_t)slots > cap) slots = (int)(cap > 0 ? cap : 1);
    }
    return slots < 1 ? 1 : slots;
}

void fill_defaults(kad_options *o) {
    memset(o, 0, sizeof(*o));
    o->epoch_size = kDefaultEpoch;
    o->calib_div = kDefaultCalibDiv;
    o->ring_epochs = 0;
    o->slots = 0;
    o->mcap = -1;
    o->block_threads = 0;
    o->blocks_per_sm = 0;
    o->flags = 0;
    o->samples_per_block = 0;
}

__global__ void k_set_ctl(KadCtl *c, unsigned long long next) { c->next = next; }

__global__ void k_hist_init(uint32_t *hist, uint32_t n) {
    if (threadIdx.x == 0) hist[0] = n;
}

const double kCalibWaitMs = 600000.0; // a run's calibration never takes this long

double now_ms() {
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec * 1e3 + (double)t.tv_nsec * 1e-6;
}

// The warp-per-sample kernel's shape for `slots` sampling slots: K contexts in
// each of nb blocks (at most one per SM), nb * K <= slots; fewer contexts per
// block rather than fewer blocks when slots are scarce.
void warp_geometry(const kad_graph *g, const LaunchCfg &cfg, int slots, int *K_out, int *nb_out) {
    const int sms = device_sms(g->device);
    int K = cfg.nctx > 0 ? cfg.nctx : 1;
    if (K > slots / sms) K = slots / sms > 0 ? slots / sms : 1;
    int nb = slots / K;
    if (nb > sms) nb = sms;
    if (nb < 1) nb = 1;
    *K_out = K;
    *nb_out = nb;
}

kad_status launch_phase(kad_graph *g, Workspace &w, const SampleArgs &a, int blocks, const LaunchCfg &cfg,
                        unsigned long long next0, cudaStream_t st) {
    k_set_ctl<<<1, 1, 0, st>>>(a.ctl, next0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(g, e);
    SampleArgs b = a;
    b.bits_smem = cfg.dyn_smem ? 1 : 0;
    // The labelled-vertex bitmap filters label reads: it pays when most scanned
    // arcs lead to unlabelled vertices (average degree above 8: C4 36.5 ms with,
    // 45.0 without), and costs a round trip per pass when few rows are long and
    // many neighbours are already labelled (the grid: 67.9 ms without, 91.0 with).
    b.no_bits = (g->gd.m <= 8 * (int64_t)g->gd.n) ? 1 : 0;
    if (a.debug & KAD_DEBUG_NO_BITMAP) b.no_bits = 1;
    if (a.debug & KAD_DEBUG_BITMAP) b.no_bits = 0;
    // One bit per group of 2^shift vertices, coarse enough that the slots'
    // bitmaps take at most 32 MB of L2 (a sample labels a tiny fraction of the
    // vertices, so a set group bit rarely hides an unlabelled vertex).
    b.bits_shift = 0;
    while (b.bits_shift < 5 && (size_t)blocks * nwords(g->gd.n >> b.bits_shift) * 4 > ((size_t)32 << 20)) b.bits_shift++;
    if (a.debug & KAD_DEBUG_COARSE_BITMAP) b.bits_shift = 3;
    if (b.bits_smem) b.bits_shift = 0;
    // meeting sets of up to mcap + kMext members are recorded during the search
    const bool ext = !(a.debug & KAD_DEBUG_NO_MEXT) && w.mext_id && (size_t)blocks <= w.mext_rows;
    b.mext_id = ext ? w.mext_id : nullptr;
    b.mext_w = ext ? w.mext_w : nullptr;
    b.mext = ext ? kMext : 0;
    if (cfg.warp) {
        // `blocks` is the number of sampling slots: nctx contexts in each of up to
        // one block per SM (fewer contexts per block when slots are scarce)
        int K = 0, nb = 0;
        warp_geometry(g, cfg, blocks, &K, &nb);
        b.nctx = K;
        // every context's bitmap of labelled vertices in shared memory, one bit
        // per 2^shift consecutive vertices, as fine as the space allows
        int per_block_max = 0;
        cudaDeviceGetAttribute(&per_block_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
        const size_t stat = kad_wsample_static_smem();
        const size_t avail = (size_t)per_block_max > stat + 1024 ? (size_t)per_block_max - stat - 1024 : 0;
        const size_t per_ctx = avail / 4 / (size_t)K;
        const int n = g->gd.n;
        int shift = 0;
        while (shift < 30 && (size_t)((((n - 1) >> shift) >> 5) + 1) > per_ctx) shift++;
        b.bits_shift = shift;
        b.nw = (int32_t)((((n - 1) >> shift) >> 5) + 1);
        if ((a.debug & KAD_DEBUG_COARSE_BITMAP) && shift < 3) {
            b.bits_shift = 3;
            b.nw = (int32_t)((((n - 1) >> 3) >> 5) + 1);
        }
        b.bits_smem = 1;
        const size_t dyn = b.no_bits ? 0 : (size_t)K * (size_t)b.nw * 4;
        if ((size_t)nb * K > (size_t)blocks) return KAD_ERR_INTERNAL; // cannot happen
        e = kad_launch_wsample(b, nb, dyn, st);
    } else {
        e = kad_launch_sample(b, blocks, cfg.threads, cfg.per_sm, cfg.dyn_smem, st);
    }
    if (e == cudaSuccess && w.ev_launch) e = cudaEventRecord(w.ev_launch, st);
    if (e != cudaSuccess) return fail(g, e);
    return KAD_OK;
}

SampleArgs base_args(kad_graph *g, const Workspace &w, uint64_t seed) {
    SampleArgs a;
    memset(&a, 0, sizeof(a));
    a.rows[0] = g->gd.rp;
    a.cols[0] = g->gd.col;
    a.rows[1] = g->gd.rpT;
    a.cols[1] = g->gd.colT;
    a.comp = g->gd.comp;
    a.n = g->gd.n;
    a.label = w.label;
    a.sigma2 = w.sigma2;
    a.list = w.list;
    a.bits = w.bits;
    a.nw = (int32_t)nwords(g->gd.n);
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.ctl = w.ctl;
    a.work = w.work;
    a.mcap = kDefaultMcap;
    a.pair_cost = kDefaultPairCost;
    return a;
}

int32_t path_cap(const kad_graph *g) { return (g->vd - 2 > 1) ? g->vd - 2 : 1; }

kad_status read_ctl(kad_graph *g, Workspace &w, KadCtl *h, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h, w.ctl, sizeof(KadCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(g, e);
    if (h->err) {
        w.dirty = true;
        return (h->err == KAD_DERR_WAIT) ? KAD_ERR_TIMEOUT : KAD_ERR_INTERNAL;
    }
    return KAD_OK;
}

kad_status run_impl(kad_graph *g, Workspace &w, double eps, double delta, uint64_t seed, cudaStream_t st,
                    const kad_options *opt_in, double *d_bc, uint32_t *d_counts, kad_result *out, bool host_out);

// The autotuner: the first run on a graph that leaves the kernel variant to the
// library runs the same query, truncated after kTuneEpochs epochs, twice under
// each candidate variant and keeps the fastest for the graph; when the caller
// leaves the pairwise test's cost factor open too, the chosen variant is timed
// the same way under each candidate factor.  Every variant and factor computes
// the same samples, so the choice changes speed only.
kad_status autotune(kad_graph *g, Workspace &w, double eps, double delta, const kad_options &o, cudaStream_t st,
                    LaunchCfg &best) {
    best = default_cfg(g, o);
    // the faster of two truncated runs: the first launch of a variant also pays
    // for loading its code and for growing the workspace
    auto time_opts = [&](kad_options o2, double *ms) -> kad_status {
        o2.max_epochs = kTuneEpochs;
        o2.flags = (o2.flags | KAD_RUN_TIMING) & ~KAD_RUN_AUTOTUNE;
        for (int rep = 0; rep < 2; rep++) {
            kad_result r;
            memset(&r, 0, sizeof(r));
            const kad_status s = run_impl(g, w, eps, delta, kTuneSeed, st, &o2, nullptr, nullptr, &r, false);
            if (s != KAD_OK) return s;
            if (rep == 0 || r.t_total_ms < *ms) *ms = r.t_total_ms;
        }
        return KAD_OK;
    };
    const bool small = g->gd.n < kTuneMinVertices; // too small to matter
    if (!g->tuned_threads && small) {
        g->tuned_threads = best.threads;
        g->tuned_per_sm = best.per_sm;
    }
    double best_ms = -1.0; // the chosen variant's time at the default factor, if measured here
    if (!g->tuned_threads) {
        // block per sample (threads, blocks per SM), then warp per sample
        // (0, samples per block): one block of 1024 threads per SM
        static const int cand[7][2] = {{512, 2}, {256, 4}, {256, 2}, {1024, 1}, {128, 8}, {0, 8}, {0, 24}};
        for (int c = 0; c < 7; c++) {
            kad_options o2 = o;
            o2.block_threads = cand[c][0];
            o2.blocks_per_sm = cand[c][0] ? cand[c][1] : 0;
            o2.samples_per_block = cand[c][0] ? 0 : cand[c][1];
            double ms = 0.0;
            const kad_status s = time_opts(o2, &ms);
            if (s != KAD_OK) return s;
            if (c == 0 || ms < best_ms) {
                best_ms = ms;
                g->tuned_threads = cand[c][0] ? cand[c][0] : -1; // -1: warp per sample
                g->tuned_per_sm = cand[c][1];
            }
        }
        if (o.pair_cost != 0) best_ms = -1.0; // measured at the caller's factor
    }
    kad_options o3 = o;
    o3.block_threads = g->tuned_threads > 0 ? g->tuned_threads : 0;
    o3.blocks_per_sm = g->tuned_threads > 0 ? g->tuned_per_sm : 0;
    o3.samples_per_block = g->tuned_threads > 0 ? 0 : g->tuned_per_sm;
    if (o.pair_cost == 0) {
        if (!g->tuned_pair_cost && small) g->tuned_pair_cost = kDefaultPairCost;
        if (!g->tuned_pair_cost) {
            static const int pcand[3] = {kDefaultPairCost, 4, 16};
            double pbest = 0.0;
            for (int c = 0; c < 3; c++) {
                double ms = best_ms;
                if (c > 0 || ms < 0.0) {
                    kad_options o4 = o3;
                    o4.pair_cost = pcand[c];
                    const kad_status s = time_opts(o4, &ms);
                    if (s != KAD_OK) return s;
                }
                if (c == 0 || ms < pbest) {
                    pbest = ms;
                    g->tuned_pair_cost = pcand[c];
                }
            }
        }
        o3.pair_cost = g->tuned_pair_cost;
    }
    best = resolve_cfg(o3);
    return KAD_OK;
}

// A graph without a workspace of its own takes the one kept from a freed graph.
void ws_adopt(kad_graph *g) {
    if (g->ws.ctl || g->device < 0 || g->device >= 64) return;
    std::lock_guard<std::mutex> lk(g_ws_cache_mu);
    if (g_ws_cached[g->device]) {
        g->ws = g_ws_cache[g->device];
        g_ws_cache[g->device] = Workspace();
        g_ws_cached[g->device] = false;
        g->ws.last_fast = false; // its last run was on another graph
    }
}

kad_status run_impl(kad_graph *g, Workspace &w, double eps, double delta, uint64_t seed, cudaStream_t st,
                    const kad_options *opt_in, double *d_bc, uint32_t *d_counts, kad_result *out, bool host_out) {
    if (!g || !out) return KAD_ERR_INVALID_ARG;
    const double t_entry = now_ms();
    if (g->poisoned) return KAD_ERR_CUDA;
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) return KAD_ERR_INVALID_ARG;
    kad_options o;
    if (opt_in)
        o = *opt_in;
    else
        fill_defaults(&o);
    if (o.epoch_size == 0 || o.calib_div == 0 || !pair_cost_ok(o)) return KAD_ERR_INVALID_ARG;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(g, cudaGetLastError());

    const int32_t n = g->gd.n;
    const uint32_t N = o.epoch_size;
    const uint64_t omega = run_omega(g->vd, eps, delta);
    const uint64_t tau0 = run_calib(omega, N, o.calib_div);
    uint64_t max_epochs = (omega + N - 1) / N; // the stop rule holds at tau >= omega
    if (o.max_epochs && o.max_epochs < max_epochs) max_epochs = o.max_epochs;
    const size_t nclass = (size_t)tau0 + 1;
    if (nclass > (size_t)0x7fffffff || omega > ((uint64_t)1 << 40)) return KAD_ERR_INVALID_ARG;
    kad_status s;
    LaunchCfg cfg = default_cfg(g, o);
    if (o.block_threads == 0 && o.blocks_per_sm == 0 && o.samples_per_block == 0 && (o.flags & KAD_RUN_AUTOTUNE))
        if ((s = autotune(g, w, eps, delta, o, st, cfg)) != KAD_OK) return s;
    if (o.debug & KAD_DEBUG_SMEM_BITMAP) choose_bitmap_home(cfg, g->gd.n, g->device);
    const int slots = resolve_slots(g, w, o, cfg);
    const int32_t cap = path_cap(g);
    // Epoch ring: enough to hold the whole run when it fits in about 1 GiB of
    // path rows, else as many epochs as fit (at least 2).
    size_t ring = o.ring_epochs ? o.ring_epochs : (size_t)max_epochs;
    const size_t row_bytes = (size_t)cap * 4 + 5;
    const size_t max_ring = ((size_t)1 << 30) / ((size_t)N * row_bytes);
    if (!o.ring_epochs && ring > max_ring) ring = max_ring;
    if (ring < 2) ring = 2;
    if (ring > max_epochs && max_epochs >= 2 && !o.ring_epochs) ring = max_epochs;

    if ((s = ensure_fixed(g, w, nclass, ring, st)) != KAD_OK) return s;
    if ((s = ensure_slots(g, w, slots, st)) != KAD_OK) return s;
    if ((s = ensure_rows(w, ring * N, cap, st)) != KAD_OK) return s;
    const bool fast = (o.flags & KAD_RUN_COMPLETION_ORDER) != 0;
    if (fast && (s = ensure_order(w, (size_t)slots * cap, (size_t)max_epochs * N, st)) != KAD_OK) return s;
    w.last_fast = false;

    Events ev(w, (o.flags & KAD_RUN_TIMING) != 0);
    cudaError_t e;
    ev.record(0, st);
    const double t_setup = now_ms() - t_entry;

    // ---- one launch: calibration samples (phase 1), then adaptive samples (phase 0)
    if ((e = cudaMemsetAsync(w.c0, 0, (size_t)n * 4, st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.cnt, 0, (size_t)n * 4, st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.hist, 0, nclass * 4, st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.ctl, 0, sizeof(KadCtl), st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.epoch_done, 0, ring * 4, st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.work, 0, KAD_WORK_WORDS * sizeof(unsigned long long), st)) != cudaSuccess)
        return fail(g, e);
    k_hist_init<<<1, 32, 0, st>>>(w.hist, (uint32_t)n); // every vertex starts with count 0
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(g, e);
    *(volatile int *)&w.hpage->calib_flag = 0;
    w.hpage->one = 1;

    SampleArgs a = base_args(g, w, seed);
    a.mcap = (o.mcap < 0) ? kDefaultMcap : o.mcap;
    a.pair_cost = cfg.pair_cost;
    a.debug = o.debug;
    a.mode = KAD_MODE_RING;
    a.calib_n = tau0;
    a.c0w = w.c0;
    a.hist = w.hist;
    a.hpage = w.dpage;
    a.epoch = N;
    a.ring = (uint32_t)ring;
    a.paths = w.paths;
    a.cap = cap;
    a.plen = w.plen;
    a.pflag = w.pflag;
    a.fast = fast ? 1 : 0;
    a.stage = fast ? w.stage : nullptr;
    a.pidx = fast ? w.pidx : nullptr;
    a.pidx_cap = fast ? (unsigned long long)max_epochs * N : 0ull;
    a.epoch_done = w.epoch_done;
    a.cnt = w.cnt;
    a.c0 = w.c0;
    a.classmax = w.classmax;
    a.ltab = w.ltab;
    a.nclass = (int32_t)nclass;
    a.eps = eps;
    a.omega = omega;
    a.max_epochs = o.max_epochs;
    a.i0 = 0;
    a.i1 = (uint64_t)((ring < max_epochs) ? ring : max_epochs) * N;
    a.k_end = a.i1 / N;
    ev.record(2, st);
    if ((s = launch_phase(g, w, a, slots, cfg, 0, st)) != KAD_OK) return s;
    ev.record(3, st);
    uint32_t launches = 1;
    uint64_t issued = a.i1; // adaptive samples handed to launches so far

    // ---- host: wait for the calibration histogram (the kernel keeps sampling),
    // then tau* by bisection, the L table and class presence, uploaded on a side
    // stream; the kernel's closer starts once ltab_ready is set.
    // The flag lives in mapped host memory: poll it with plain reads, look at the
    // launch's event only every 64th time (or after 2 ms), and back off with short
    // sleeps, so that waiting threads do not crowd the driver.
    const double t_wait0 = now_ms();
    for (unsigned it = 0;; it++) {
        if (*(volatile int *)&w.hpage->calib_flag) break;
        const double waited = now_ms() - t_wait0;
        if (waited > 0.05) {
            struct timespec ts = {0, waited > 2.0 ? 50000 : 5000};
            nanosleep(&ts, nullptr);
        }
        if ((it & 63) != 63 && waited < 2.0) continue;
        const cudaError_t q = cudaEventQuery(w.ev_launch);
        if (q == cudaSuccess) { // the launch ended; the flag must be set by now
            if (*(volatile int *)&w.hpage->calib_flag) break;
            KadCtl hc0;
            kad_status s0 = read_ctl(g, w, &hc0, st);
            w.dirty = true;
            return (s0 != KAD_OK) ? s0 : KAD_ERR_INTERNAL;
        }
        if (q != cudaErrorNotReady) return fail(g, q);
        if (now_ms() - t_wait0 > kCalibWaitMs) {
            cudaStreamSynchronize(st);
            w.dirty = true;
            return KAD_ERR_TIMEOUT;
        }
    }
    __sync_synchronize();
    const double t_calib = now_ms() - t_wait0;
    const double ts = run_tau_star(w.hpage->hist, tau0, eps, delta, omega);
    for (size_t c = 0; c < nclass; c++) {
        w.h_ltab[c] = run_L((double)c / (double)tau0, ts, eps, omega);
        w.h_cmax[c] = w.hpage->hist[c] ? 0 : -1;
    }
    const double t_table = now_ms() - t_wait0 - t_calib;
    e = cudaMemcpyAsync(w.ltab, w.h_ltab, nclass * 8, cudaMemcpyHostToDevice, w.aux);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.classmax, w.h_cmax, nclass * 4, cudaMemcpyHostToDevice, w.aux);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&w.ctl->ltab_ready, &w.hpage->one, sizeof(int), cudaMemcpyHostToDevice, w.aux);
    if (e == cudaSuccess) e = cudaEventRecord(w.ev_aux, w.aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, w.ev_aux, 0); // later launches see the table
    if (e != cudaSuccess) return fail(g, e);

    // ---- further launches only if the ring filled up (or the table arrived
    // after the last sample): each continues the index space and first closes
    // what is pending
    KadCtl hc;
    for (;;) {
        if ((s = read_ctl(g, w, &hc, st)) != KAD_OK) return s;
        if (hc.stop) break;
        if (launches > 4 * max_epochs + 8) return KAD_ERR_INTERNAL; // cannot happen: tau >= omega stops
        const uint64_t closed = hc.closed;
        const uint64_t lim = closed + ring < max_epochs ? closed + ring : max_epochs;
        uint64_t i1 = lim * N;
        if (fast) // every issued sample takes one fold position, all inside the ring window
            i1 = issued + (lim * N > hc.qnext ? lim * N - hc.qnext : 0);
        if (i1 < issued) i1 = issued;
        a.calib_n = 0;
        a.i0 = issued;
        a.i1 = i1;
        a.k_end = lim;
        if ((s = launch_phase(g, w, a, slots, cfg, 0, st)) != KAD_OK) return s;
        launches++;
        issued = i1;
    }
    const uint64_t tau = hc.tau;
    w.last_fast = fast;
    w.last_positions = hc.qnext < (uint64_t)max_epochs * N ? hc.qnext : (uint64_t)max_epochs * N;
    unsigned long long work[KAD_WORK_WORDS];
    if ((e = cudaMemcpyAsync(work, w.work, sizeof(work), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(g, e);

    // ---- outputs
    double *bc_dst = (host_out && out->bc) ? w.bc : d_bc;
    if (bc_dst)
        if ((e = kad_launch_finalize(w.cnt, n, tau, bc_dst, st)) != cudaSuccess) return fail(g, e);
    if (!host_out && d_counts)
        if ((e = cudaMemcpyAsync(d_counts, w.cnt, (size_t)n * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return fail(g, e);
    if (host_out) {
        if (out->bc) e = cudaMemcpyAsync(out->bc, bc_dst, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->counts)
            e = cudaMemcpyAsync(out->counts, w.cnt, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->c0) e = cudaMemcpyAsync(out->c0, w.c0, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && out->ltab && out->ltab_cap >= (int64_t)nclass)
            e = cudaMemcpyAsync(out->ltab, w.ltab, nclass * 8, cudaMemcpyDeviceToHost, st);
    }
    ev.record(4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(g, e);

    out->tau = tau;
    out->omega = omega;
    out->calib_samples = tau0;
    out->samples_computed = work[6];
    out->overflow_samples = hc.overflow;
    out->epochs = (uint32_t)(tau / N);
    out->vd_bound = g->vd;
    out->sigma_overflow = hc.overflow ? 1 : 0;
    out->stopped_by_omega = hc.stopped_by_omega;
    out->tau_star = ts;
    for (int i = 0; i < 6; i++) out->work[i] = work[i];
    for (int i = 0; i < 6; i++) out->phase_cycles[i] = work[8 + i];
    out->bfs_split_cycles[0] = work[14];
    out->bfs_split_cycles[1] = work[15];
    out->ads_launches = launches;
    out->slots_used = slots;
    out->block_threads_used = cfg.threads;
    out->blocks_per_sm_used = cfg.per_sm;
    out->pair_cost_used = cfg.pair_cost;
    out->samples_per_block_used = 0;
    if (cfg.warp) {
        int K = 0, nb = 0;
        warp_geometry(g, cfg, slots, &K, &nb);
        out->samples_per_block_used = K;
        out->slots_used = K * nb;
    }
    // k_hist_init, then k_set_ctl + k_sample per launch, and k_finalize if b~ was wanted
    out->kernel_launches = 1u + 2u * launches + (bc_dst ? 1u : 0u);
    if (ev.on) {
        out->t_total_ms = ev.ms(0, 4);
        out->t_calib_ms = t_calib; // host wall time from launch to the histogram (sampling continues meanwhile)
        out->t_ads_ms = ev.ms(2, 4);
        out->t_ads_kernel_ms = ev.ms(2, 3);
        out->t_setup_ms = t_setup;
        out->t_table_ms = t_table;
        auto rel = [&](unsigned long long t) { return (t && hc.t_start && t >= hc.t_start) ? (double)(t - hc.t_start) * 1e-6 : 0.0; };
        out->t_dev_calib_ms = rel(hc.t_calib);
        out->t_dev_first_close_ms = rel(hc.t_first_close);
        out->t_dev_stop_ms = rel(hc.t_stop);
        out->t_dev_end_ms = rel(hc.t_end);
        out->issued_at_stop = hc.issued_at_stop;
        out->t_host_ms = now_ms() - t_entry;
    }
    return KAD_OK;
}

kad_status create_common(int32_t n, int64_t m, const int32_t *rp, const int32_t *col, bool from_host, uint32_t flags,
                         cudaStream_t st, kad_graph **out) {
    if (!out) return KAD_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 2 || !rp || (m > 0 && !col) || m < 0 || m >= ((int64_t)1 << 31)) return KAD_ERR_INVALID_ARG;
    kad_graph *g = new (std::nothrow) kad_graph();
    if (!g) return KAD_ERR_OOM;
    cudaGetDevice(&g->device);
    g->gd.n = n;
    g->gd.m = m;
    g->gd.directed = (flags & KAD_GRAPH_DIRECTED) != 0;
    cudaError_t e = cudaSuccess;
    kad_status s = KAD_OK;
    if (kad_pool_alloc((void **)&g->gd.rp, ((size_t)n + 1) * 4, st) != cudaSuccess ||
        kad_pool_alloc((void **)&g->gd.col, (size_t)m * 4, st) != cudaSuccess ||
        kad_pool_alloc((void **)&g->gd.comp, (size_t)n * 4, st) != cudaSuccess) {
        cudaGetLastError();
        kad_graph_free(g);
        return KAD_ERR_OOM;
    }
    const cudaMemcpyKind kind = from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    e = cudaMemcpyAsync(g->gd.rp, rp, ((size_t)n + 1) * 4, kind, st);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(g->gd.col, col, (size_t)m * 4, kind, st);
    if (e != cudaSuccess) {
        kad_graph_free(g);
        return map_err(e);
    }
    int32_t vd = 0, nc = 0, md = 0;
    s = kad_graph_setup(g->gd, flags, st, &vd, &nc, &md, &e);
    if (s != KAD_OK) {
        kad_graph_free(g);
        return s;
    }
    if (vd < 1 || vd >= (1 << 27)) {
        kad_graph_free(g);
        return KAD_ERR_INVALID_ARG;
    }
    if (!g->gd.directed) { // one symmetric CSR serves both sides
        g->gd.rpT = g->gd.rp;
        g->gd.colT = g->gd.col;
    }
    g->vd = vd;
    g->ncomp = nc;
    g->max_deg = md;
    *out = g;
    return KAD_OK;
}

} // namespace

// ================================================================ serving
namespace {

struct ServerQuery {
    uint64_t ticket = 0;
    int32_t gid = 0;
    double eps = 0, delta = 0;
    uint64_t seed = 0;
    double *bc_out = nullptr;
    size_t footprint = 0;
    uint64_t samples_max = 0; // omega + tau0: the most samples the query can use
    double est_ms = 0;        // expected service time when it was last looked at
    kad_result result;
    kad_status status = KAD_OK;
    bool done = false;
    double t_submit = 0, t_start = 0, t_end = 0;
};

} // namespace

struct kad_server {
    int device = 0;
    int workers = 4, slots_per_query = 0, threads = 512, per_sm = 2;
    int resident = 1; // sampling blocks the device holds at once
    size_t budget = 0, inflight = 0;
    std::vector<kad_graph *> graphs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerQuery *> pending;
    std::unordered_map<uint64_t, ServerQuery *> queries;
    uint64_t next_ticket = 1;
    int running = 0; // queries on workers
    bool stopping = false;
    int policy = 0;  // 0: highest response ratio next, 1: arrival order
    std::vector<double> ms_per_sample; // per graph: running mean of device time per used sample (0 = none yet)
    double ms_per_sample_all = 0;       // the same over every graph
    std::vector<std::thread> pool;
};

namespace {

// Device memory a query needs on top of its graph: slot scratch, the epoch ring
// and the per-vertex and per-class arrays (the same sizes run_impl allocates).
size_t query_footprint(const kad_graph *g, double eps, double delta, int slots) {
    const size_t n = (size_t)g->gd.n;
    const uint64_t omega = run_omega(g->vd, eps, delta);
    const uint64_t tau0 = run_calib(omega, kDefaultEpoch, kDefaultCalibDiv);
    const uint64_t epochs = (omega + kDefaultEpoch - 1) / kDefaultEpoch;
    const size_t cap = (size_t)path_cap(g);
    const size_t row_bytes = cap * 4 + 5;
    size_t ring = (size_t)epochs;
    const size_t max_ring = ((size_t)1 << 30) / ((size_t)kDefaultEpoch * row_bytes);
    if (ring > max_ring) ring = max_ring;
    if (ring < 2) ring = 2;
    return (size_t)slots * (n * kSlotBytesPerVertex + (size_t)kMext * 12) + ring * kDefaultEpoch * row_bytes + 8 * n +
           ((size_t)tau0 + 1) * 16;
}

// Expected service time of a query (caller holds the lock): the most samples it
// can use times the graph's mean device time per sample, or the mean over every
// graph before the graph has answered a query (1 us per sample before any).
double expected_ms(const kad_server *S, const ServerQuery *q) {
    double per = S->ms_per_sample[q->gid];
    if (per <= 0) per = S->ms_per_sample_all;
    if (per <= 0) per = 1e-3;
    const double e = per * (double)q->samples_max;
    return e > 1e-3 ? e : 1e-3;
}

void server_worker(kad_server *S) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    Workspace ws;
    for (;;) {
        ServerQuery *q = nullptr;
        int slots = 1;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stopping) break;
                // Slots: a fixed number per query, or (adaptive) the resident blocks
                // shared among the queries that will be in flight, so that a query
                // arriving at an idle server gets the whole device.
                int share = S->running + (int)S->pending.size();
                if (share > S->workers) share = S->workers;
                if (share < 1) share = 1;
                slots = S->slots_per_query > 0 ? S->slots_per_query : S->resident / share;
                if (slots < 1) slots = 1;
                // Among the queued queries whose footprint fits next to those in
                // flight (a query larger than the whole budget runs when nothing
                // else does): the first in arrival order, or the one with the
                // highest response ratio (waited + expected) / expected, which
                // serves short queries first without starving long ones.
                const double now = now_ms();
                auto pick = S->pending.end();
                double best = -1.0;
                for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
                    const size_t fp = query_footprint(S->graphs[(*it)->gid], (*it)->eps, (*it)->delta, slots);
                    if (!(S->inflight + fp <= S->budget || S->running == 0)) continue;
                    (*it)->footprint = fp;
                    if (S->policy == 1) {
                        pick = it;
                        break;
                    }
                    const double est = expected_ms(S, *it);
                    const double ratio = (now - (*it)->t_submit + est) / est;
                    if (ratio > best) {
                        best = ratio;
                        pick = it;
                    }
                }
                if (pick != S->pending.end()) {
                    q = *pick;
                    S->pending.erase(pick);
                    break;
                }
                S->cv_work.wait(lk);
            }
            if (!q) break;
            S->inflight += q->footprint;
            S->running++;
        }
        q->t_start = now_ms();
        kad_graph *g = S->graphs[q->gid];
        kad_options o;
        fill_defaults(&o);
        o.block_threads = S->threads;
        o.blocks_per_sm = S->per_sm;
        o.slots = slots;
        o.flags |= KAD_RUN_TIMING;
        kad_result r;
        memset(&r, 0, sizeof(r));
        r.bc = q->bc_out;
        const kad_status status =
            have_stream ? run_impl(g, ws, q->eps, q->delta, q->seed, st, &o, nullptr, nullptr, &r, true) : KAD_ERR_CUDA;
        const double t_end = now_ms();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (status == KAD_OK && r.t_total_ms > 0 && r.tau + r.calib_samples > 0) {
                const double per = r.t_total_ms / (double)(r.tau + r.calib_samples);
                double &g_per = S->ms_per_sample[q->gid];
                g_per = (g_per > 0) ? 0.75 * g_per + 0.25 * per : per;
                S->ms_per_sample_all = (S->ms_per_sample_all > 0) ? 0.9 * S->ms_per_sample_all + 0.1 * per : per;
            }
            q->t_end = t_end;
            q->result = r;
            q->status = status;
            q->done = true;
            S->inflight -= q->footprint;
            S->running--;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    ws_free_all(ws);
    if (have_stream) cudaStreamDestroy(st);
}

} // namespace

// ================================================================ C ABI

extern "C" {

void kad_options_default(kad_options *opt) {
    if (opt) fill_defaults(opt);
}

kad_status kad_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col, uint32_t flags, kad_stream_t stream,
                            kad_graph **out) {
    if (!row_ptr) return KAD_ERR_INVALID_ARG;
    if (n < 2) return KAD_ERR_INVALID_ARG;
    const int64_t m = row_ptr[n];
    if (row_ptr[0] != 0 || m < 0) return KAD_ERR_BAD_CSR;
    return create_common(n, m, row_ptr, col, true, flags, (cudaStream_t)stream, out);
}

kad_status kad_graph_create_device(int32_t n, int64_t m, const int32_t *d_row_ptr, const int32_t *d_col, uint32_t flags,
                                   kad_stream_t stream, kad_graph **out) {
    return create_common(n, m, d_row_ptr, d_col, false, flags, (cudaStream_t)stream, out);
}

void kad_graph_free(kad_graph *g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    if (!g->poisoned && g->ws.ctl && g->device >= 0 && g->device < 64) {
        std::lock_guard<std::mutex> lk(g_ws_cache_mu);
        if (!g_ws_cached[g->device]) {
            g_ws_cache[g->device] = g->ws;
            g_ws_cached[g->device] = true;
            g->ws = Workspace();
        }
    }
    ws_free_all(g->ws);
    // the graph's arrays go back to the pool once the device is idle (as
    // cudaFree would wait for it)
    cudaDeviceSynchronize();
    if (g->gd.rp) cudaFreeAsync(g->gd.rp, 0);
    if (g->gd.col) cudaFreeAsync(g->gd.col, 0);
    if (g->gd.comp) cudaFreeAsync(g->gd.comp, 0);
    if (g->gd.directed && g->gd.rpT) cudaFreeAsync(g->gd.rpT, 0);
    if (g->gd.directed && g->gd.colT) cudaFreeAsync(g->gd.colT, 0);
    cudaSetDevice(cur);
    delete g;
}

kad_status kad_graph_info(const kad_graph *g, int32_t *n, int64_t *m, int32_t *vd_bound, int32_t *components) {
    if (!g) return KAD_ERR_INVALID_ARG;
    if (n) *n = g->gd.n;
    if (m) *m = g->gd.m;
    if (vd_bound) *vd_bound = g->vd;
    if (components) *components = g->ncomp;
    return KAD_OK;
}

kad_status kad_run(kad_graph *g, double eps, double delta, uint64_t seed, kad_stream_t stream, const kad_options *opt,
                   kad_result *out) {
    if (!g) return KAD_ERR_INVALID_ARG;
    ws_adopt(g);
    return run_impl(g, g->ws, eps, delta, seed, (cudaStream_t)stream, opt, nullptr, nullptr, out, true);
}

kad_status kad_run_device(kad_graph *g, double eps, double delta, uint64_t seed, kad_stream_t stream,
                          const kad_options *opt, double *d_bc, uint32_t *d_counts, kad_result *out) {
    if (!g) return KAD_ERR_INVALID_ARG;
    ws_adopt(g);
    return run_impl(g, g->ws, eps, delta, seed, (cudaStream_t)stream, opt, d_bc, d_counts, out, false);
}

void kad_shard_range(int64_t count, int32_t rank, int32_t world, int64_t *lo, int64_t *hi) {
    if (!lo || !hi) return;
    if (count < 0 || world < 1 || rank < 0 || rank >= world) {
        *lo = *hi = 0;
        return;
    }
    // contiguous chunks whose sizes differ by at most one, in rank order
    *lo = (int64_t)(((__int128)count * rank) / world);
    *hi = (int64_t)(((__int128)count * (rank + 1)) / world);
}

kad_status kad_run_sharded(kad_graph *g, double eps, double delta, uint64_t seed, int32_t rank, int32_t world,
                           kad_allgather_fn allgather, void *user, kad_stream_t stream, const kad_options *opt_in,
                           kad_result *out) {
    if (!g || !out || !allgather || world < 1 || rank < 0 || rank >= world) return KAD_ERR_INVALID_ARG;
    if (g->poisoned) return KAD_ERR_CUDA;
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) return KAD_ERR_INVALID_ARG;
    const double t_entry = now_ms();
    kad_options o;
    if (opt_in)
        o = *opt_in;
    else
        fill_defaults(&o);
    if (o.epoch_size == 0 || o.calib_div == 0 || (o.flags & KAD_RUN_COMPLETION_ORDER) || !pair_cost_ok(o))
        return KAD_ERR_INVALID_ARG;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(g, cudaGetLastError());
    ws_adopt(g);
    Workspace &w = g->ws;
    const cudaStream_t st = (cudaStream_t)stream;
    const int32_t n = g->gd.n;
    const uint32_t N = o.epoch_size;
    const uint64_t omega = run_omega(g->vd, eps, delta);
    const uint64_t tau0 = run_calib(omega, N, o.calib_div);
    uint64_t max_epochs = (omega + N - 1) / N;
    if (o.max_epochs && o.max_epochs < max_epochs) max_epochs = o.max_epochs;
    const size_t nclass = (size_t)tau0 + 1;
    if (nclass > (size_t)0x7fffffff || omega > ((uint64_t)1 << 40)) return KAD_ERR_INVALID_ARG;
    const int32_t cap = path_cap(g);
    // every rank pads its chunk to maxc rows: the largest chunk of either phase
    const int64_t maxc = (int64_t)(((tau0 > N ? tau0 : N) + (uint64_t)world - 1) / (uint64_t)world);
    const size_t blk_ints = (size_t)maxc * (size_t)(2 + cap);
    if ((double)blk_ints * (double)world * 4.0 > (double)((size_t)1 << 34)) return KAD_ERR_INVALID_ARG;
    LaunchCfg cfg = default_cfg(g, o);
    int slots = resolve_slots(g, w, o, cfg);
    kad_status s;
    if ((s = ensure_fixed(g, w, nclass, 2, st)) != KAD_OK) return s;
    if ((s = ensure_slots(g, w, slots, st)) != KAD_OK) return s;
    if ((s = ensure_rows(w, (size_t)maxc, cap, st)) != KAD_OK) return s;

    int32_t *d_blocks = nullptr, *d_s = nullptr, *d_t = nullptr, *d_D = nullptr;
    unsigned long long *d_sst = nullptr, *d_ovf = nullptr;
    int *d_fail = nullptr;
    int32_t *h_send = nullptr, *h_recv = nullptr;
    uint8_t *h_flag = nullptr;
    uint32_t *h_hist = nullptr;
    cudaError_t e = cudaSuccess;
    uint64_t tau = 0, epochs = 0, ovf = 0;
    int stopped_by = 0;
    double ts = 0.0;
    unsigned long long work[KAD_WORK_WORDS];
    if (dalloc(&d_blocks, blk_ints * (size_t)world) != cudaSuccess || dalloc(&d_s, (size_t)maxc) != cudaSuccess ||
        dalloc(&d_t, (size_t)maxc) != cudaSuccess || dalloc(&d_D, (size_t)maxc) != cudaSuccess ||
        dalloc(&d_sst, (size_t)maxc) != cudaSuccess || dalloc(&d_ovf, 1) != cudaSuccess ||
        dalloc(&d_fail, 1) != cudaSuccess) {
        cudaGetLastError();
        s = KAD_ERR_OOM;
        goto done;
    }
    h_send = (int32_t *)malloc(blk_ints * 4);
    h_recv = (int32_t *)malloc(blk_ints * 4 * (size_t)world);
    h_flag = (uint8_t *)malloc((size_t)maxc);
    h_hist = (uint32_t *)malloc(nclass * 4);
    if (!h_send || !h_recv || !h_flag || !h_hist) {
        s = KAD_ERR_OOM;
        goto done;
    }
    if ((e = cudaMemsetAsync(w.c0, 0, (size_t)n * 4, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.cnt, 0, (size_t)n * 4, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.hist, 0, nclass * 4, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.ctl, 0, sizeof(KadCtl), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_ovf, 0, 8, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.work, 0, KAD_WORK_WORDS * sizeof(unsigned long long), st)) != cudaSuccess) {
        s = fail(g, e);
        goto done;
    }
    k_hist_init<<<1, 32, 0, st>>>(w.hist, (uint32_t)n);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        s = fail(g, e);
        goto done;
    }
    // phase 0: calibration (domain 1, indices [0, tau0)); phase k >= 1: adaptive
    // epoch k-1 (domain 0, indices [(k-1)N, kN))
    for (uint64_t ph = 0; ph <= max_epochs; ph++) {
        const bool calib = ph == 0;
        const uint64_t base = calib ? 0 : (ph - 1) * (uint64_t)N;
        const int64_t count = calib ? (int64_t)tau0 : (int64_t)N;
        int64_t lo = 0, hi = 0;
        kad_shard_range(count, rank, world, &lo, &hi);
        const int64_t c = hi - lo;
        // this rank's chunk, in record mode: one path row per sample
        if (c > 0) {
            SampleArgs a = base_args(g, w, seed);
            a.mcap = (o.mcap < 0) ? kDefaultMcap : o.mcap;
            a.pair_cost = cfg.pair_cost;
            a.debug = o.debug;
            a.domain = calib ? 1 : 0;
            a.i0 = base + (uint64_t)lo;
            a.i1 = base + (uint64_t)hi;
            a.mode = KAD_MODE_RECORD;
            a.paths = w.paths;
            a.cap = cap;
            a.plen = w.plen;
            a.pflag = w.pflag;
            a.rec_s = d_s;
            a.rec_t = d_t;
            a.rec_D = d_D;
            a.rec_sst = d_sst;
            a.epoch = 1;
            a.ring = 1;
            if ((s = launch_phase(g, w, a, (int)(c < slots ? c : slots), cfg, a.i0, st)) != KAD_OK) goto done;
        }
        // pack [lengths][flags][paths] of maxc rows; absent rows have length -1
        for (int64_t j = 0; j < maxc; j++) h_send[j] = -1;
        if (c > 0) {
            e = cudaMemcpyAsync(h_send, w.plen, (size_t)c * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_flag, w.pflag, (size_t)c, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_send + 2 * maxc, w.paths, (size_t)c * (size_t)cap * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                s = fail(g, e);
                goto done;
            }
            KadCtl hc;
            if ((s = read_ctl(g, w, &hc, st)) != KAD_OK) goto done;
        }
        for (int64_t j = 0; j < maxc; j++) h_send[maxc + j] = (j < c) ? (int32_t)h_flag[j] : 0;
        if (allgather(user, h_send, blk_ints * 4, h_recv) != 0) {
            s = KAD_ERR_CANCELLED;
            goto done;
        }
        if ((e = cudaMemcpyAsync(d_blocks, h_recv, blk_ints * 4 * (size_t)world, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = kad_launch_fold_rows(d_blocks, world, (int)maxc, cap, calib ? 1 : 0, w.c0, w.hist, w.cnt, w.classmax,
                                      w.c0, d_ovf, st)) != cudaSuccess) {
            s = fail(g, e);
            goto done;
        }
        if (calib) {
            // every rank now holds the same c0: the histogram, tau* and the L
            // table on the host, as in kad_run
            if ((e = cudaMemcpyAsync(h_hist, w.hist, nclass * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                s = fail(g, e);
                goto done;
            }
            ts = run_tau_star(h_hist, tau0, eps, delta, omega);
            for (size_t q = 0; q < nclass; q++) {
                w.h_ltab[q] = run_L((double)q / (double)tau0, ts, eps, omega);
                w.h_cmax[q] = h_hist[q] ? 0 : -1;
            }
            if ((e = cudaMemcpyAsync(w.ltab, w.h_ltab, nclass * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(w.classmax, w.h_cmax, nclass * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                s = fail(g, e);
                goto done;
            }
            continue;
        }
        // the stop rule on the state after epochs 0..ph-1 (Appendix B)
        tau = ph * (uint64_t)N;
        epochs = ph;
        if (tau >= omega) {
            stopped_by = 1;
            break;
        }
        int failed = 1;
        if ((e = cudaMemsetAsync(d_fail, 0, sizeof(int), st)) != cudaSuccess ||
            (e = kad_launch_check_classes(w.classmax, w.ltab, (int)nclass, tau, omega, eps, d_fail, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&failed, d_fail, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            s = fail(g, e);
            goto done;
        }
        if (!failed) {
            stopped_by = 0;
            break;
        }
        if (o.max_epochs && ph >= o.max_epochs) {
            stopped_by = 2;
            break;
        }
    }
    if (epochs == 0) { // cannot happen: the loop runs at least one adaptive epoch
        s = KAD_ERR_INTERNAL;
        goto done;
    }
    // outputs, as kad_run's host outputs
    e = cudaMemcpyAsync(work, w.work, sizeof(work), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ovf, d_ovf, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && out->bc) {
        e = kad_launch_finalize(w.cnt, n, tau, w.bc, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out->bc, w.bc, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess && out->counts) e = cudaMemcpyAsync(out->counts, w.cnt, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && out->c0) e = cudaMemcpyAsync(out->c0, w.c0, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && out->ltab && out->ltab_cap >= (int64_t)nclass)
        e = cudaMemcpyAsync(out->ltab, w.ltab, nclass * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        s = fail(g, e);
        goto done;
    }
    out->tau = tau;
    out->omega = omega;
    out->calib_samples = tau0;
    out->samples_computed = work[6];
    out->overflow_samples = ovf;
    out->epochs = (uint32_t)epochs;
    out->vd_bound = g->vd;
    out->sigma_overflow = ovf ? 1 : 0;
    out->stopped_by_omega = stopped_by;
    out->tau_star = ts;
    for (int i = 0; i < 6; i++) out->work[i] = work[i];
    for (int i = 0; i < 6; i++) out->phase_cycles[i] = work[8 + i];
    out->slots_used = slots;
    out->block_threads_used = cfg.threads;
    out->blocks_per_sm_used = cfg.per_sm;
    out->samples_per_block_used = cfg.warp ? cfg.nctx : 0;
    out->pair_cost_used = cfg.pair_cost;
    out->t_host_ms = now_ms() - t_entry;
    out->t_total_ms = out->t_host_ms;
    s = KAD_OK;
done:
    cudaFree(d_blocks);
    cudaFree(d_s);
    cudaFree(d_t);
    cudaFree(d_D);
    cudaFree(d_sst);
    cudaFree(d_ovf);
    cudaFree(d_fail);
    free(h_send);
    free(h_recv);
    free(h_flag);
    free(h_hist);
    return s;
}

kad_status kad_run_order(kad_graph *g, uint64_t *idx_out, uint64_t count) {
    if (!g || (count && !idx_out)) return KAD_ERR_INVALID_ARG;
    const Workspace &w = g->ws;
    if (!w.last_fast || count > w.last_positions) return KAD_ERR_INVALID_ARG;
    if (count == 0) return KAD_OK;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(g, cudaGetLastError());
    const cudaError_t e = cudaMemcpy(idx_out, w.pidx, count * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(g, e);
    return KAD_OK;
}

kad_status kad_sample_records(kad_graph *g, uint64_t seed, uint32_t domain, uint64_t i0, int64_t count,
                              kad_stream_t stream, const kad_options *opt, int32_t *s_out, int32_t *t_out,
                              int32_t *D_out, uint64_t *sst_out, int32_t *ovf_out, int32_t *paths, int32_t cap,
                              uint64_t *work_out) {
    if (!g || count < 0 || domain > 1 || !s_out || !t_out || !D_out || !sst_out || !ovf_out || !paths)
        return KAD_ERR_INVALID_ARG;
    if (g->poisoned) return KAD_ERR_CUDA;
    if (cap < path_cap(g)) return KAD_ERR_INVALID_ARG;
    if (count == 0) return KAD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(g, cudaGetLastError());
    ws_adopt(g);
    kad_options o;
    if (opt)
        o = *opt;
    else
        fill_defaults(&o);
    if (!pair_cost_ok(o)) return KAD_ERR_INVALID_ARG;
    LaunchCfg cfg = default_cfg(g, o);
    if (o.debug & KAD_DEBUG_SMEM_BITMAP) choose_bitmap_home(cfg, g->gd.n, g->device);
    Workspace &w = g->ws;
    int slots = resolve_slots(g, w, o, cfg);
    if ((int64_t)slots > count) slots = (int)count;
    kad_status s;
    if ((s = ensure_fixed(g, w, 1, 2, st)) != KAD_OK) return s;
    if ((s = ensure_slots(g, w, slots, st)) != KAD_OK) return s;
    int32_t *d_paths = nullptr, *d_plen = nullptr, *d_s = nullptr, *d_t = nullptr, *d_D = nullptr;
    uint8_t *d_flag = nullptr;
    unsigned long long *d_sst = nullptr;
    const size_t c = (size_t)count;
    cudaError_t e;
    if (dalloc(&d_paths, c * (size_t)cap) != cudaSuccess || dalloc(&d_plen, c) != cudaSuccess ||
        dalloc(&d_flag, c) != cudaSuccess || dalloc(&d_s, c) != cudaSuccess || dalloc(&d_t, c) != cudaSuccess ||
        dalloc(&d_D, c) != cudaSuccess || dalloc(&d_sst, c) != cudaSuccess) {
        cudaGetLastError();
        s = KAD_ERR_OOM;
        goto out;
    }
    {
        SampleArgs a = base_args(g, w, seed);
        a.mcap = (o.mcap < 0) ? kDefaultMcap : o.mcap;
        a.pair_cost = cfg.pair_cost;
        a.debug = o.debug;
        a.domain = domain;
        a.i0 = i0;
        a.i1 = i0 + c;
        a.mode = KAD_MODE_RECORD;
        a.paths = d_paths;
        a.cap = cap;
        a.plen = d_plen;
        a.pflag = d_flag;
        a.rec_s = d_s;
        a.rec_t = d_t;
        a.rec_D = d_D;
        a.rec_sst = d_sst;
        a.epoch = 1;
        a.ring = 1;
        if ((e = cudaMemsetAsync(d_paths, 0xff, c * (size_t)cap * 4, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(w.ctl, 0, sizeof(KadCtl), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(w.work, 0, KAD_WORK_WORDS * 8, st)) != cudaSuccess) {
            s = fail(g, e);
            goto out;
        }
        if ((s = launch_phase(g, w, a, slots, cfg, i0, st)) != KAD_OK) goto out;
        uint8_t *hflag = (uint8_t *)malloc(c);
        unsigned long long hw[KAD_WORK_WORDS];
        if (!hflag) {
            s = KAD_ERR_OOM;
            goto out;
        }
        e = cudaMemcpyAsync(paths, d_paths, c * (size_t)cap * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s_out, d_s, c * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(t_out, d_t, c * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(D_out, d_D, c * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sst_out, d_sst, c * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hflag, d_flag, c, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hw, w.work, sizeof(hw), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            free(hflag);
            s = fail(g, e);
            goto out;
        }
        for (size_t i = 0; i < c; i++) ovf_out[i] = hflag[i];
        free(hflag);
        if (work_out)
            for (int i = 0; i < 6; i++) work_out[i] = hw[i];
        KadCtl hc;
        s = read_ctl(g, w, &hc, st);
    }
out:
    cudaFree(d_paths);
    cudaFree(d_plen);
    cudaFree(d_flag);
    cudaFree(d_s);
    cudaFree(d_t);
    cudaFree(d_D);
    cudaFree(d_sst);
    return s;
}

kad_status kad_eval_fg(int32_t n, const uint32_t *counts, const uint32_t *c0, const double *ltab, int32_t nclass,
                       uint64_t tau, uint64_t omega, double *f, double *g) {
    if (n < 1 || !counts || !c0 || !ltab || nclass < 1 || !f || !g || tau == 0) return KAD_ERR_INVALID_ARG;
    for (int32_t v = 0; v < n; v++)
        if (c0[v] >= (uint32_t)nclass) return KAD_ERR_INVALID_ARG;
    uint32_t *dc = nullptr, *d0 = nullptr;
    double *dl = nullptr, *df = nullptr, *dg = nullptr;
    kad_status s = KAD_OK;
    cudaError_t e;
    if (dalloc(&dc, n) != cudaSuccess || dalloc(&d0, n) != cudaSuccess || dalloc(&dl, nclass) != cudaSuccess ||
        dalloc(&df, n) != cudaSuccess || dalloc(&dg, n) != cudaSuccess) {
        cudaGetLastError();
        s = KAD_ERR_OOM;
    } else {
        e = cudaMemcpy(dc, counts, (size_t)n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d0, c0, (size_t)n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dl, ltab, (size_t)nclass * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = kad_launch_fg(dc, d0, dl, n, tau, omega, df, dg, 0);
        if (e == cudaSuccess) e = cudaMemcpy(f, df, (size_t)n * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(g, dg, (size_t)n * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) s = map_err(e);
    }
    cudaFree(dc);
    cudaFree(d0);
    cudaFree(dl);
    cudaFree(df);
    cudaFree(dg);
    return s;
}

kad_status kad_server_create(const kad_server_options *opt, kad_server **out) {
    if (!out) return KAD_ERR_INVALID_ARG;
    *out = nullptr;
    kad_server *S = new (std::nothrow) kad_server();
    if (!S) return KAD_ERR_OOM;
    cudaGetDevice(&S->device);
    if (opt && opt->workers > 0) S->workers = opt->workers;
    if (S->workers > 64) S->workers = 64;
    if (opt && opt->block_threads > 0) S->threads = opt->block_threads;
    if (opt && opt->blocks_per_sm > 0) S->per_sm = opt->blocks_per_sm;
    if (opt && opt->policy == 1) S->policy = 1;
    kad_options o;
    fill_defaults(&o);
    o.block_threads = S->threads;
    o.blocks_per_sm = S->per_sm;
    const LaunchCfg cfg = resolve_cfg(o);
    S->threads = cfg.threads;
    S->per_sm = cfg.per_sm;
    const int resident = device_sms(S->device) * (kad_sample_max_blocks_per_sm(cfg.threads, cfg.per_sm, 0) > 0
                                                      ? kad_sample_max_blocks_per_sm(cfg.threads, cfg.per_sm, 0)
                                                      : 1);
    S->resident = resident > 0 ? resident : 1;
    S->slots_per_query = (opt && opt->slots_per_query > 0) ? opt->slots_per_query : 0; // 0 = adaptive
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    S->budget = (opt && opt->hbm_budget > 0) ? (size_t)opt->hbm_budget : fr / 2;
    for (int i = 0; i < S->workers; i++) S->pool.emplace_back(server_worker, S);
    *out = S;
    return KAD_OK;
}

kad_status kad_server_add_graph(kad_server *S, int32_t n, const int32_t *row_ptr, const int32_t *col, uint32_t flags,
                                int32_t *gid) {
    if (!S || !gid) return KAD_ERR_INVALID_ARG;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(S->device);
    kad_graph *g = nullptr;
    const kad_status st = kad_graph_create(n, row_ptr, col, flags, nullptr, &g);
    cudaSetDevice(cur);
    if (st != KAD_OK) return st;
    std::lock_guard<std::mutex> lk(S->mu);
    S->graphs.push_back(g);
    S->ms_per_sample.push_back(0.0);
    *gid = (int32_t)S->graphs.size() - 1;
    return KAD_OK;
}

kad_status kad_submit(kad_server *S, int32_t gid, double eps, double delta, uint64_t seed, double *bc_out,
                      uint64_t *ticket) {
    if (!S || !ticket) return KAD_ERR_INVALID_ARG;
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) return KAD_ERR_INVALID_ARG;
    ServerQuery *q = new (std::nothrow) ServerQuery();
    if (!q) return KAD_ERR_OOM;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (gid < 0 || gid >= (int32_t)S->graphs.size() || S->stopping) {
            delete q;
            return KAD_ERR_INVALID_ARG;
        }
        q->ticket = S->next_ticket++;
        q->gid = gid;
        q->eps = eps;
        q->delta = delta;
        q->seed = seed;
        q->bc_out = bc_out;
        {
            const kad_graph *g = S->graphs[gid];
            const uint64_t om = run_omega(g->vd, eps, delta);
            q->samples_max = om + run_calib(om, kDefaultEpoch, kDefaultCalibDiv);
        }
        memset(&q->result, 0, sizeof(q->result));
        q->t_submit = now_ms();
        S->queries[q->ticket] = q;
        S->pending.push_back(q);
        *ticket = q->ticket;
    }
    S->cv_work.notify_one();
    return KAD_OK;
}

kad_status kad_poll(kad_server *S, uint64_t ticket, int *done) {
    if (!S || !done) return KAD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->queries.find(ticket);
    if (it == S->queries.end()) return KAD_ERR_INVALID_ARG;
    *done = it->second->done ? 1 : 0;
    return KAD_OK;
}

kad_status kad_wait(kad_server *S, uint64_t ticket, int64_t timeout_ns, kad_result *out, double *queue_ms,
                    double *latency_ms) {
    if (!S) return KAD_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->queries.find(ticket);
    if (it == S->queries.end()) return KAD_ERR_INVALID_ARG;
    ServerQuery *q = it->second;
    if (timeout_ns < 0) {
        S->cv_done.wait(lk, [q] { return q->done; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [q] { return q->done; })) {
        return KAD_ERR_TIMEOUT;
    }
    if (out) {
        double *keep_bc = out->bc;
        *out = q->result;
        out->bc = keep_bc;
    }
    if (queue_ms) *queue_ms = q->t_start - q->t_submit;
    if (latency_ms) *latency_ms = q->t_end - q->t_submit;
    const kad_status st = q->status;
    S->queries.erase(it);
    delete q;
    return st;
}

void kad_server_free(kad_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (ServerQuery *q : S->pending) {
            q->status = KAD_ERR_CANCELLED;
            q->done = true;
        }
        S->pending.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    for (auto &t : S->pool) t.join();
    for (auto &kv : S->queries) delete kv.second;
    for (kad_graph *g : S->graphs) kad_graph_free(g);
    delete S;
}

const char *kad_status_string(kad_status s) {
    switch (s) {
    case KAD_OK:
        return "ok";
    case KAD_ERR_INVALID_ARG:
        return "invalid argument";
    case KAD_ERR_BAD_CSR:
        return "CSR is not a symmetric, sorted, loop-free, duplicate-free graph";
    case KAD_ERR_OOM:
        return "out of memory";
    case KAD_ERR_CUDA:
        return "CUDA error (graph handle poisoned)";
    case KAD_ERR_TIMEOUT:
        return "device-side wait timed out";
    case KAD_ERR_CANCELLED:
        return "cancelled";
    case KAD_ERR_INTERNAL:
        return "device-side consistency check failed";
    }
    return "unknown status";
}

void kad_trim(void) {
    int cur = 0;
    cudaGetDevice(&cur);
    std::lock_guard<std::mutex> lk(g_ws_cache_mu);
    for (int d = 0; d < 64; d++) {
        if (!g_ws_cached[d]) continue;
        cudaSetDevice(d);
        ws_free_all(g_ws_cache[d]);
        g_ws_cached[d] = false;
    }
    {
        std::lock_guard<std::mutex> lp(g_pool_mu);
        for (int d = 0; d < 64; d++) {
            if (!g_pool_made[d]) continue;
            cudaSetDevice(d);
            cudaDeviceSynchronize();
            cudaMemPoolTrimTo(g_pool[d], 0);
        }
    }
    cudaSetDevice(cur);
}

uint32_t kad_version(void) { return (0u << 16) | 1u; }

} // extern "C"
