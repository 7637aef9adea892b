// kad_sample_records_noalloc: the per-sample records of kad_sample_records for
// callers that cannot allocate device memory.
//
// Who needs it: a process whose device memory is owned by someone else's pool --
// a framework's caching allocator, a serving process with a fixed memory budget --
// may not let a library call cudaMalloc/cudaFree: those calls can synchronise the
// device, stall the caller's other streams, and take memory outside the pool's
// accounting.  Such a caller allocates the inputs and outputs itself and passes
// them in; the sampling kernel's scratch (per-slot labels, path counts, labelled
// lists, control block, work counters) comes from one file-scope device array of
// fixed size that every GPU loading this library holds until the process exits.
//
// There is no counterpart in the paper; the kernel is the same sampling kernel
// (record mode) that kad_sample_records launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "kad_internal.cuh"

namespace {

// ---- the static scratch and its layout
constexpr size_t kNoallocBytes = (size_t)48 << 20;   // 48 MiB per device
constexpr size_t kHeadBytes = 4096;                  // control block at 0, work counters at 512
constexpr int64_t kMaxRecords = (int64_t)1 << 20;    // samples per call
constexpr size_t kPlenBytes = (size_t)kMaxRecords * 4;
constexpr size_t kSlotAreaOffset = kHeadBytes + kPlenBytes;
constexpr size_t kSlotArea = kNoallocBytes - kSlotAreaOffset;
constexpr int kMaxSlots = 64;
constexpr int kThreads = 512;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes the slot area needs for n vertices and `slots` sampling slots: a zero
// component array (used when the caller passes none), then a 16-byte record
// (label, unused word, sigma), sigma2 (8 B) and list (4 B) per vertex and slot,
// and a bitmap of labelled vertices (1 bit per vertex and slot).
size_t nwords(int64_t n) { return ((size_t)n + 31) / 32; }

size_t slot_area_bytes(int64_t n, int64_t slots) {
    return align256((size_t)n * 4) + align256((size_t)(slots * n) * 16) + align256((size_t)(slots * n) * 8) +
           align256((size_t)(slots * n) * 4) + align256((size_t)slots * nwords(n) * 4);
}

// The array's device address on the current device.  In host code the name
// g_noalloc_scratch is only a host stand-in, never a device address, so every
// call looks the address up (a host-side query with no stream work) rather than
// keeping it: a cached address could outlive the context it belongs to.
kad_status scratch_for_device(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return KAD_ERR_CUDA;
    }
    *out = (unsigned char *)p;
    return KAD_OK;
}

__global__ void k_noalloc_reset(KadCtl *ctl, unsigned long long *work, unsigned long long next) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctl->next = next;
        ctl->closed = 0;
        ctl->tau = 0;
        ctl->overflow = 0;
        ctl->computed = 0;
        ctl->stop = 0;
        ctl->closer = 0;
        ctl->err = 0;
        ctl->stopped_by_omega = 0;
        for (int i = 0; i < KAD_WORK_WORDS; i++) work[i] = 0;
    }
}

} // namespace

extern "C" kad_status kad_sample_records_noalloc(int32_t n, const int32_t *d_row_ptr, const int32_t *d_col,
                                                 const int32_t *d_comp, uint64_t seed, uint32_t domain, uint64_t i0,
                                                 int64_t count, kad_stream_t stream, int32_t *d_s, int32_t *d_t,
                                                 int32_t *d_D, uint64_t *d_sigma_st, uint8_t *d_overflow,
                                                 int32_t *d_paths, int32_t cap) {
    if (n < 2 || !d_row_ptr || !d_col || domain > 1 || count < 0 || cap < 1 || !d_s || !d_t || !d_D ||
        !d_sigma_st || !d_overflow || !d_paths)
        return KAD_ERR_INVALID_ARG;
    if (count > kMaxRecords) return KAD_ERR_INVALID_ARG;               // more samples than one call holds
    if (slot_area_bytes(n, 1) > kSlotArea) return KAD_ERR_INVALID_ARG; // graph too large for the scratch
    if (count == 0) return KAD_OK;
    if ((uint64_t)count * (uint64_t)cap > (uint64_t)1 << 40) return KAD_ERR_INVALID_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    kad_status s = scratch_for_device(&base);
    if (s != KAD_OK) return s;

    int64_t slots = kMaxSlots;
    while (slots > 1 && slot_area_bytes(n, slots) > kSlotArea) slots--;
    if (slots > count) slots = count;
    const size_t sn = (size_t)slots * (size_t)n;

    KadCtl *ctl = (KadCtl *)base;
    unsigned long long *work = (unsigned long long *)(base + 512);
    int32_t *plen = (int32_t *)(base + kHeadBytes);
    unsigned char *p = base + kSlotAreaOffset;
    int32_t *zero_comp = (int32_t *)p;
    p += align256((size_t)n * 4);
    uint32_t *label = (uint32_t *)p; // 16-byte records: label, -, sigma
    p += align256(sn * 16);
    unsigned long long *sigma2 = (unsigned long long *)p;
    p += align256(sn * 8);
    int32_t *list = (int32_t *)p;
    p += align256(sn * 4);
    uint32_t *bits = (uint32_t *)p;
    const size_t bw = (size_t)slots * nwords(n);

    // The array keeps the previous call's contents.  Labels and path counts must
    // start at zero (the kernel restores zeros after every sample it finishes,
    // but a call that ended on an error may not have); the component array is
    // all zeros when the caller has none (pairs in different components are then
    // found disconnected by the search itself).
    cudaError_t e = cudaSuccess;
    if (!d_comp) e = cudaMemsetAsync(zero_comp, 0, (size_t)n * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(label, 0, sn * 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sigma2, 0, sn * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bits, 0, bw * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_paths, 0xff, (size_t)count * (size_t)cap * 4, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KAD_ERR_CUDA;
    }
    k_noalloc_reset<<<1, 32, 0, st>>>(ctl, work, (unsigned long long)i0);

    SampleArgs a;
    memset(&a, 0, sizeof(a));
    a.rows[0] = a.rows[1] = d_row_ptr; // an undirected graph: in-arc rows = out-arc rows
    a.cols[0] = a.cols[1] = d_col;
    a.comp = d_comp ? d_comp : zero_comp;
    a.n = n;
    a.label = label;
    a.sigma2 = sigma2;
    a.list = list;
    a.bits = bits;
    a.nw = (int32_t)nwords(n);
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.pair_cost = KAD_DEFAULT_PAIR_COST;
    a.domain = domain;
    a.i0 = i0;
    a.i1 = i0 + (uint64_t)count;
    a.mode = KAD_MODE_RECORD;
    a.mcap = 256;
    a.paths = d_paths;
    a.cap = cap;
    a.plen = plen;
    a.pflag = d_overflow;
    a.epoch = 1;
    a.ring = 1;
    a.rec_s = d_s;
    a.rec_t = d_t;
    a.rec_D = d_D;
    a.rec_sst = (unsigned long long *)d_sigma_st;
    a.ctl = ctl;
    a.work = work;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = kad_launch_sample(a, (int)slots, kThreads, 1, 0, st);
    int derr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&derr, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return KAD_ERR_CUDA;
    }
    if (derr == KAD_DERR_CAP) return KAD_ERR_INVALID_ARG; // a path longer than cap
    if (derr) return KAD_ERR_INTERNAL;
    return KAD_OK;
}
