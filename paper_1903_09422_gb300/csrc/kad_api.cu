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

#include <new>

#include "kad_internal.cuh"

namespace {

const int kDefaultEpoch = 1000;   // N = 1000 (Appendix C.2)
const int kDefaultCalibDiv = 100; // tau0 ~ omega / 100
const int kDefaultMcap = 256;

struct Workspace {
    int slots = 0; // sampling slots allocated
    uint32_t *label = nullptr;
    unsigned long long *sigma = nullptr, *sigma2 = nullptr;
    int32_t *list = nullptr;
    uint32_t *bits = nullptr; // labelled-vertex bitmap, nw words per slot
    // epoch ring (or record buffer)
    size_t rows = 0;
    int32_t cap = 0;
    int32_t *paths = nullptr;
    int32_t *plen = nullptr;
    uint8_t *pflag = nullptr;
    // per-vertex state
    uint32_t *cnt = nullptr, *c0 = nullptr;
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
};

} // namespace

struct kad_graph {
    int device = 0;
    KadGraphDev gd{};
    int32_t vd = 0, ncomp = 0;
    bool poisoned = false;
    Workspace ws;
};

namespace {

void ws_free_slots(Workspace &w) {
    cudaFree(w.label);
    cudaFree(w.sigma);
    cudaFree(w.sigma2);
    cudaFree(w.list);
    cudaFree(w.bits);
    w.label = nullptr;
    w.sigma = w.sigma2 = nullptr;
    w.list = nullptr;
    w.bits = nullptr;
    w.slots = 0;
}

void ws_free_all(Workspace &w) {
    ws_free_slots(w);
    cudaFree(w.paths);
    cudaFree(w.plen);
    cudaFree(w.pflag);
    cudaFree(w.cnt);
    cudaFree(w.c0);
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
    w = Workspace();
}

template <typename T> cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

// bytes of sampling scratch per slot and vertex: label 4, sigma 8, sigma2 8, list 4
// (plus one bit of the labelled-vertex bitmap)
const size_t kSlotBytesPerVertex = 25;

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

kad_status ensure_slots(kad_graph *g, int slots, cudaStream_t st) {
    Workspace &w = g->ws;
    const size_t n = (size_t)g->gd.n;
    if (w.slots >= slots && !w.dirty) return KAD_OK;
    if (w.slots < slots) {
        ws_free_slots(w);
        const size_t cnt = (size_t)slots * n;
        if (dalloc(&w.label, cnt) != cudaSuccess || dalloc(&w.sigma, cnt) != cudaSuccess ||
            dalloc(&w.sigma2, cnt) != cudaSuccess || dalloc(&w.list, cnt) != cudaSuccess ||
            dalloc(&w.bits, (size_t)slots * nwords(g->gd.n)) != cudaSuccess) {
            cudaGetLastError();
            ws_free_slots(w);
            return KAD_ERR_OOM;
        }
        w.slots = slots;
    }
    const size_t cnt = (size_t)w.slots * n;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.label, 0, cnt * 4, st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.sigma, 0, cnt * 8, st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.sigma2, 0, cnt * 8, st)) != cudaSuccess) return fail(g, e);
    if ((e = cudaMemsetAsync(w.bits, 0, (size_t)w.slots * nwords(g->gd.n) * 4, st)) != cudaSuccess) return fail(g, e);
    w.dirty = false;
    return KAD_OK;
}

kad_status ensure_rows(kad_graph *g, size_t rows, int32_t cap) {
    Workspace &w = g->ws;
    if (w.rows >= rows && w.cap == cap) return KAD_OK;
    cudaFree(w.paths);
    cudaFree(w.plen);
    cudaFree(w.pflag);
    w.paths = nullptr;
    w.plen = nullptr;
    w.pflag = nullptr;
    w.rows = 0;
    if (dalloc(&w.paths, rows * (size_t)cap) != cudaSuccess || dalloc(&w.plen, rows) != cudaSuccess ||
        dalloc(&w.pflag, rows) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(w.paths);
        cudaFree(w.plen);
        cudaFree(w.pflag);
        w.paths = nullptr;
        w.plen = nullptr;
        w.pflag = nullptr;
        return KAD_ERR_OOM;
    }
    w.rows = rows;
    w.cap = cap;
    return KAD_OK;
}

kad_status ensure_fixed(kad_graph *g, size_t nclass, size_t ring) {
    Workspace &w = g->ws;
    const size_t n = (size_t)g->gd.n;
    if (!w.cnt) {
        if (dalloc(&w.cnt, n) != cudaSuccess || dalloc(&w.c0, n) != cudaSuccess || dalloc(&w.ctl, 1) != cudaSuccess ||
            dalloc(&w.work, KAD_WORK_WORDS) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
    }
    if (w.nclass_cap < nclass) {
        cudaFree(w.classmax);
        cudaFree(w.ltab);
        cudaFree(w.hist);
        w.classmax = nullptr;
        w.ltab = nullptr;
        w.hist = nullptr;
        w.nclass_cap = 0;
        if (dalloc(&w.classmax, nclass) != cudaSuccess || dalloc(&w.ltab, nclass) != cudaSuccess ||
            dalloc(&w.hist, nclass) != cudaSuccess) {
            cudaGetLastError();
            return KAD_ERR_OOM;
        }
        w.nclass_cap = nclass;
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
        cudaFree(w.epoch_done);
        w.epoch_done = nullptr;
        w.ring_cap = 0;
        if (dalloc(&w.epoch_done, ring) != cudaSuccess) {
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

struct Events {
    cudaEvent_t e[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool on = false;
    void create(bool want) {
        on = want;
        if (on)
            for (auto &x : e)
                if (cudaEventCreate(&x) != cudaSuccess) on = false;
    }
    void record(int i, cudaStream_t st) {
        if (on) cudaEventRecord(e[i], st);
    }
    double ms(int a, int b) {
        float t = 0;
        if (!on || cudaEventElapsedTime(&t, e[a], e[b]) != cudaSuccess) return 0.0;
        return (double)t;
    }
    ~Events() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
};

int device_sms(int dev) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

struct LaunchCfg {
    int threads;
    int per_sm;      // resident blocks per SM the kernel variant is compiled for
    size_t dyn_smem; // bytes of dynamic shared memory (the slot bitmap) or 0
};

// Threads per block and blocks per SM.  Unknown combinations fall back to the
// variant with the same block size and the default occupancy.
LaunchCfg resolve_cfg(const kad_options &o) {
    LaunchCfg c;
    c.threads = (o.block_threads == 128 || o.block_threads == 256 || o.block_threads == 1024) ? o.block_threads : 512;
    const int def = (c.threads == 128) ? 4 : (c.threads == 256) ? 2 : (c.threads == 512) ? 2 : 1;
    c.per_sm = (o.blocks_per_sm > 0 && kad_sample_variant_exists(c.threads, o.blocks_per_sm)) ? o.blocks_per_sm : def;
    c.dyn_smem = 0;
    return c;
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
int resolve_slots(kad_graph *g, const kad_options &o, const LaunchCfg &cfg) {
    int slots = o.slots;
    if (slots <= 0) {
        const int per_sm = kad_sample_max_blocks_per_sm(cfg.threads, cfg.per_sm, cfg.dyn_smem);
        slots = device_sms(g->device) * (per_sm > 0 ? per_sm : 1);
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
        const size_t per = kSlotBytesPerVertex * (size_t)g->gd.n;
        size_t budget = fr / 3 + (size_t)g->ws.slots * per; // what we already hold counts too
        const size_t maxb = (size_t)64 << 30;
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

kad_status launch_phase(kad_graph *g, const SampleArgs &a, int blocks, const LaunchCfg &cfg,
                        unsigned long long next0, cudaStream_t st) {
    k_set_ctl<<<1, 1, 0, st>>>(a.ctl, next0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(g, e);
    SampleArgs b = a;
    b.bits_smem = cfg.dyn_smem ? 1 : 0;
    e = kad_launch_sample(b, blocks, cfg.threads, cfg.per_sm, cfg.dyn_smem, st);
    if (e == cudaSuccess) e = cudaEventRecord(g->ws.ev_launch, st);
    if (e != cudaSuccess) return fail(g, e);
    return KAD_OK;
}

SampleArgs base_args(kad_graph *g, uint64_t seed) {
    SampleArgs a;
    memset(&a, 0, sizeof(a));
    a.rp = g->gd.rp;
    a.col = g->gd.col;
    a.comp = g->gd.comp;
    a.n = g->gd.n;
    a.label = g->ws.label;
    a.sigma = g->ws.sigma;
    a.sigma2 = g->ws.sigma2;
    a.list = g->ws.list;
    a.bits = g->ws.bits;
    a.nw = (int32_t)nwords(g->gd.n);
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.ctl = g->ws.ctl;
    a.work = g->ws.work;
    a.mcap = kDefaultMcap;
    return a;
}

int32_t path_cap(const kad_graph *g) { return (g->vd - 2 > 1) ? g->vd - 2 : 1; }

kad_status read_ctl(kad_graph *g, KadCtl *h, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h, g->ws.ctl, sizeof(KadCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(g, e);
    if (h->err) {
        g->ws.dirty = true;
        return KAD_ERR_INTERNAL;
    }
    return KAD_OK;
}

kad_status run_impl(kad_graph *g, double eps, double delta, uint64_t seed, cudaStream_t st, const kad_options *opt_in,
                    double *d_bc, uint32_t *d_counts, kad_result *out, bool host_out) {
    if (!g || !out) return KAD_ERR_INVALID_ARG;
    if (g->poisoned) return KAD_ERR_CUDA;
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) return KAD_ERR_INVALID_ARG;
    kad_options o;
    if (opt_in)
        o = *opt_in;
    else
        fill_defaults(&o);
    if (o.epoch_size == 0 || o.calib_div == 0) return KAD_ERR_INVALID_ARG;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(g, cudaGetLastError());

    const int32_t n = g->gd.n;
    const uint32_t N = o.epoch_size;
    const uint64_t omega = run_omega(g->vd, eps, delta);
    const uint64_t tau0 = run_calib(omega, N, o.calib_div);
    uint64_t max_epochs = (omega + N - 1) / N; // the stop rule holds at tau >= omega
    if (o.max_epochs && o.max_epochs < max_epochs) max_epochs = o.max_epochs;
    const size_t nclass = (size_t)tau0 + 1;
    if (nclass > (size_t)0x7fffffff || omega > ((uint64_t)1 << 40)) return KAD_ERR_INVALID_ARG;
    LaunchCfg cfg = resolve_cfg(o);
    if (o.debug & KAD_DEBUG_SMEM_BITMAP) choose_bitmap_home(cfg, g->gd.n, g->device);
    const int slots = resolve_slots(g, o, cfg);
    const int32_t cap = path_cap(g);
    // Epoch ring: enough to hold the whole run when it fits in about 1 GiB of
    // path rows, else as many epochs as fit (at least 2).
    size_t ring = o.ring_epochs ? o.ring_epochs : (size_t)max_epochs;
    const size_t row_bytes = (size_t)cap * 4 + 5;
    const size_t max_ring = ((size_t)1 << 30) / ((size_t)N * row_bytes);
    if (!o.ring_epochs && ring > max_ring) ring = max_ring;
    if (ring < 2) ring = 2;
    if (ring > max_epochs && max_epochs >= 2 && !o.ring_epochs) ring = max_epochs;

    kad_status s;
    if ((s = ensure_fixed(g, nclass, ring)) != KAD_OK) return s;
    if ((s = ensure_slots(g, slots, st)) != KAD_OK) return s;
    if ((s = ensure_rows(g, ring * N, cap)) != KAD_OK) return s;
    Workspace &w = g->ws;

    Events ev;
    ev.create((o.flags & KAD_RUN_TIMING) != 0);
    cudaError_t e;
    ev.record(0, st);

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

    SampleArgs a = base_args(g, seed);
    a.mcap = (o.mcap < 0) ? kDefaultMcap : o.mcap;
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
    if ((s = launch_phase(g, a, slots, cfg, 0, st)) != KAD_OK) return s;
    ev.record(3, st);
    uint32_t launches = 1;
    uint64_t issued = a.i1; // adaptive samples handed to launches so far

    // ---- host: wait for the calibration histogram (the kernel keeps sampling),
    // then tau* by bisection, the L table and class presence, uploaded on a side
    // stream; the kernel's closer starts once ltab_ready is set.
    const double t_wait0 = now_ms();
    for (;;) {
        if (*(volatile int *)&w.hpage->calib_flag) break;
        const cudaError_t q = cudaEventQuery(w.ev_launch);
        if (q == cudaSuccess) { // the launch ended; the flag must be set by now
            if (*(volatile int *)&w.hpage->calib_flag) break;
            KadCtl hc0;
            kad_status s0 = read_ctl(g, &hc0, st);
            g->ws.dirty = true;
            return (s0 != KAD_OK) ? s0 : KAD_ERR_INTERNAL;
        }
        if (q != cudaErrorNotReady) return fail(g, q);
        if (now_ms() - t_wait0 > kCalibWaitMs) {
            cudaStreamSynchronize(st);
            g->ws.dirty = true;
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
        if ((s = read_ctl(g, &hc, st)) != KAD_OK) return s;
        if (hc.stop) break;
        if (launches > 4 * max_epochs + 8) return KAD_ERR_INTERNAL; // cannot happen: tau >= omega stops
        const uint64_t closed = hc.closed;
        uint64_t i1 = (closed + ring < max_epochs ? closed + ring : max_epochs) * N;
        if (i1 < issued) i1 = issued;
        a.calib_n = 0;
        a.i0 = issued;
        a.i1 = i1;
        a.k_end = i1 / N;
        if ((s = launch_phase(g, a, slots, cfg, 0, st)) != KAD_OK) return s;
        launches++;
        issued = i1;
    }
    const uint64_t tau = hc.tau;
    unsigned long long work[KAD_WORK_WORDS];
    if ((e = cudaMemcpyAsync(work, w.work, sizeof(work), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return fail(g, e);

    // ---- outputs
    double *bc_dst = d_bc;
    if (host_out && out->bc) {
        if ((e = cudaMalloc(&bc_dst, (size_t)n * 8)) != cudaSuccess) return fail(g, e);
    }
    if (bc_dst) {
        if ((e = kad_launch_finalize(w.cnt, n, tau, bc_dst, st)) != cudaSuccess) {
            if (host_out) cudaFree(bc_dst);
            return fail(g, e);
        }
    }
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
    if (host_out && out->bc) cudaFree(bc_dst);
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
    out->ads_launches = launches;
    out->slots_used = slots;
    // k_hist_init, then k_set_ctl + k_sample per launch, and k_finalize if b~ was wanted
    out->kernel_launches = 1u + 2u * launches + (bc_dst ? 1u : 0u);
    if (ev.on) {
        out->t_total_ms = ev.ms(0, 4);
        out->t_calib_ms = t_calib; // host wall time from launch to the histogram (sampling continues meanwhile)
        out->t_ads_ms = ev.ms(2, 4);
        out->t_ads_kernel_ms = ev.ms(2, 3);
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
    cudaError_t e = cudaSuccess;
    kad_status s = KAD_OK;
    if (dalloc(&g->gd.rp, (size_t)n + 1) != cudaSuccess || dalloc(&g->gd.col, (size_t)m) != cudaSuccess ||
        dalloc(&g->gd.comp, (size_t)n) != cudaSuccess) {
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
    int32_t vd = 0, nc = 0;
    s = kad_graph_setup(g->gd, flags, st, &vd, &nc, &e);
    if (s != KAD_OK) {
        kad_graph_free(g);
        return s;
    }
    if (vd < 1 || vd >= (1 << 27)) {
        kad_graph_free(g);
        return KAD_ERR_INVALID_ARG;
    }
    g->vd = vd;
    g->ncomp = nc;
    *out = g;
    return KAD_OK;
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
    ws_free_all(g->ws);
    cudaFree(g->gd.rp);
    cudaFree(g->gd.col);
    cudaFree(g->gd.comp);
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
    return run_impl(g, eps, delta, seed, (cudaStream_t)stream, opt, nullptr, nullptr, out, true);
}

kad_status kad_run_device(kad_graph *g, double eps, double delta, uint64_t seed, kad_stream_t stream,
                          const kad_options *opt, double *d_bc, uint32_t *d_counts, kad_result *out) {
    return run_impl(g, eps, delta, seed, (cudaStream_t)stream, opt, d_bc, d_counts, out, false);
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
    kad_options o;
    if (opt)
        o = *opt;
    else
        fill_defaults(&o);
    LaunchCfg cfg = resolve_cfg(o);
    if (o.debug & KAD_DEBUG_SMEM_BITMAP) choose_bitmap_home(cfg, g->gd.n, g->device);
    int slots = resolve_slots(g, o, cfg);
    if ((int64_t)slots > count) slots = (int)count;
    kad_status s;
    if ((s = ensure_fixed(g, 1, 2)) != KAD_OK) return s;
    if ((s = ensure_slots(g, slots, st)) != KAD_OK) return s;
    Workspace &w = g->ws;
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
        SampleArgs a = base_args(g, seed);
        a.mcap = (o.mcap < 0) ? kDefaultMcap : o.mcap;
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
        if ((s = launch_phase(g, a, slots, cfg, i0, st)) != KAD_OK) goto out;
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
        s = read_ctl(g, &hc, st);
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

uint32_t kad_version(void) { return (0u << 16) | 1u; }

} // extern "C"
