// Device helpers shared by the sampling kernels (block per sample and warp per
// sample): the random stream, the per-vertex records of a sampling slot, warp
// scans, and the output of a sample's interior vertices.  Every definition is
// internal to the translation unit that includes this header.
// (Nothing here is shared with the CPU oracle.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kad_internal.cuh"

#define FULL_MASK 0xffffffffu
#define KAD_MAXLV 62    // levels whose list ranges are kept for the trace-back

namespace {

// atomic add with release semantics at GPU scope: every write of this thread
// before it is visible to whoever observes the new value
__device__ __forceinline__ unsigned int atom_add_release(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.release.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011).
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Block `blk` of sample `idx` in phase `dom`: two 64-bit words, low word first.
// Out of line, so that every draw site shares one copy of the ten rounds.
__device__ __noinline__ ulonglong2 philox_block(uint32_t k0, uint32_t k1, unsigned long long idx, uint32_t blk,
                                                uint32_t dom) {
    uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), blk, dom};
    philox10(c, k0, k1);
    return make_ulonglong2((unsigned long long)c[0] | ((unsigned long long)c[1] << 32),
                           (unsigned long long)c[2] | ((unsigned long long)c[3] << 32));
}

// Lemire's rejection threshold (2^64 - m) mod m, out of line: it is needed
// only when the low half of a product falls below m.
__device__ __noinline__ unsigned long long lemire_threshold(unsigned long long m) { return (0ull - m) % m; }

// The random stream of one sample; used by a single thread.
struct Stream {
    uint32_t k0, k1, dom, blk;
    unsigned long long idx, w0, w1;
    int pos;

    __device__ void init(uint32_t key0, uint32_t key1, unsigned long long index, uint32_t domain) {
        k0 = key0;
        k1 = key1;
        idx = index;
        dom = domain;
        blk = 0;
        pos = 2;
    }
    __device__ unsigned long long next() {
        if (pos == 2) {
            const ulonglong2 b = philox_block(k0, k1, idx, blk, dom);
            w0 = b.x;
            w1 = b.y;
            blk++;
            pos = 0;
        }
        return (pos++ == 0) ? w0 : w1;
    }
    // Uniform in [0, m), m >= 1: Lemire's multiply-and-reject.  The rejection
    // loop is bounded; 64 rejections in a row have probability below 2^-64.
    __device__ __noinline__ unsigned long long uniform(unsigned long long m, KadCtl *ctl) {
        unsigned long long x = next();
        unsigned long long lo = x * m, hi = __umul64hi(x, m);
        if (lo < m) {
            const unsigned long long th = lemire_threshold(m);
            int guard = 0;
            while (lo < th) {
                if (++guard > 64) {
                    kad_set_err(ctl, KAD_DERR_REJECT);
                    break;
                }
                x = next();
                lo = x * m;
                hi = __umul64hi(x, m);
            }
        }
        return hi;
    }
};

__device__ __forceinline__ unsigned long long warp_incl_sat_scan(unsigned long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x = kad_sat_add(y, x);
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    return x;
}

// Per vertex and slot one 16-byte record: the label (word 0), an unused word,
// and the path count sigma (words 2-3), so that a label and its count come in
// one load and one 32-byte sector.
__device__ __forceinline__ uint32_t *lab_at(uint32_t *vs, int v) { return vs + 4 * (size_t)v; }
__device__ __forceinline__ const uint32_t *lab_at(const uint32_t *vs, int v) { return vs + 4 * (size_t)v; }
__device__ __forceinline__ unsigned long long *sig_at(uint32_t *vs, int v) {
    return (unsigned long long *)(vs + 4 * (size_t)v + 2);
}
__device__ __forceinline__ const unsigned long long *sig_at(const uint32_t *vs, int v) {
    return (const unsigned long long *)(vs + 4 * (size_t)v + 2);
}
// label and sigma of v, read through L2 in one 16-byte load
__device__ __forceinline__ void ld_vs(const uint32_t *vs, int v, uint32_t &lab, unsigned long long &sig) {
    const uint4 x = __ldcg((const uint4 *)(vs + 4 * (size_t)v));
    lab = x.x;
    sig = (unsigned long long)x.z | ((unsigned long long)x.w << 32);
}
// the path count to use: saturated when the label says it wrapped
__device__ __forceinline__ unsigned long long sig_val(uint32_t lab, unsigned long long sig) {
    return (lab & KAD_OVF) ? KAD_U64MAX : sig;
}

// Physical list position of the j-th vertex labelled on side z: the s side
// fills the slot's list from the front, the t side from the back.
__device__ __forceinline__ int phys(int z, int j, int n) { return z ? (n - 1 - j) : j; }

// Write one interior vertex (at distance j from s, 1 <= j <= D-1).  A null row
// means a calibration sample: count v and move it one histogram bin up.
__device__ __forceinline__ void emit(const SampleArgs &a, int32_t *row, int D, int j, int v) {
    if (j < 1 || j > D - 1) return;
    if (!row) {
        const unsigned int c = atomicAdd(a.c0w + v, 1u);
        atomicSub(a.hist + c, 1u);
        atomicAdd(a.hist + c + 1, 1u);
    } else {
        if (j - 1 < a.cap)
            row[j - 1] = v;
        else
            kad_set_err(a.ctl, KAD_DERR_CAP);
    }
}

// Epoch k can be closed once all its samples are written, no stop has been
// decided, and the host has uploaded the L table (calibration's result).
__device__ __forceinline__ bool epoch_ready(const SampleArgs &a, unsigned long long k) {
    return k < a.k_end && *(volatile int *)&a.ctl->stop == 0 && *(volatile int *)&a.ctl->ltab_ready != 0 &&
           *(volatile uint32_t *)&a.epoch_done[k % a.ring] == a.epoch;
}

} // namespace
