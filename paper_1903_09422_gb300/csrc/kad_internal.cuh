// Internal definitions shared by the CUDA translation units of libkad.
// (Nothing here is shared with the CPU oracle.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kad.h"

// ----------------------------------------------------------------- labels
// One 32-bit word per vertex and sampling slot:
//   bit 31      side (0 = s side, 1 = t side)
//   bit 30      OVF : sigma[v] wrapped (its true value is >= 2^64 -> saturate)
//   bit 29      INM : v is in the meeting set M
//   bit 28      OVF2: sigma2[v] (the expanding side's count at a meeting vertex) wrapped
//   bits 0..27  level + 1  (0 in the whole word = unlabelled)
#define KAD_SIDE 0x80000000u
#define KAD_OVF 0x40000000u
#define KAD_INM 0x20000000u
#define KAD_OVF2 0x10000000u
#define KAD_LVL 0x0FFFFFFFu
#define KAD_KEY (KAD_SIDE | KAD_LVL)
#define KAD_MAX_LEVEL (KAD_LVL - 2)

#define KAD_U64MAX 0xffffffffffffffffull
#define KAD_WORK_WORDS 16
#define KAD_DEFAULT_PAIR_COST 8 // one pairwise adjacency test counted as 8 arc reads

// sample-kernel output modes
#define KAD_MODE_RING 1   // a KADABRA run: calibration samples first (counted into c0 and
                          // its histogram), then adaptive samples whose paths go into the
                          // epoch ring, folded and checked in order by the closer
#define KAD_MODE_RECORD 2 // full per-sample records (parity tests)

// device error codes (KadCtl.err)
#define KAD_DERR_CAP 1       // path longer than the buffer row (VD bound violated)
#define KAD_DERR_REJECT 2    // bounded-draw rejection limit
#define KAD_DERR_TRACE 3     // trace-back found no predecessor
#define KAD_DERR_SELECT 4    // meeting draw found no vertex
#define KAD_DERR_LEVEL 5     // level overflow
#define KAD_DERR_FRONTIER 6  // list overflow
#define KAD_DERR_WAIT 7      // a bounded wait of the warp-per-sample kernel ran out

// Control block of one adaptive run (device memory).
struct KadCtl {
    unsigned long long next;     // next sample index of the current launch
    unsigned long long closed;   // epochs folded and checked so far
    unsigned long long tau;      // samples used when stopped
    unsigned long long overflow; // overflowed samples among the folded epochs
    unsigned long long computed; // samples computed (all launches)
    unsigned long long calib_done; // calibration samples finished
    int stop;                    // 1 once the stop rule held
    int closer;                  // closer role taken (0/1)
    int err;                     // KAD_DERR_*, first error wins
    int stopped_by_omega;
    int ltab_ready;              // 1 once the host has uploaded the L table and class presence
    // timeline of the run (device global timer, ns): first sample started,
    // calibration histogram published, first epoch closed, stop decided, last
    // block finished; and the sample indices handed out when the stop was decided
    unsigned long long t_start, t_calib, t_first_close, t_stop, t_end;
    unsigned long long issued_at_stop;
    unsigned long long qnext; // completion order: fold positions taken so far
};

// Host-mapped page of a run (pinned host memory the kernel writes through).
struct KadHostPage {
    int calib_flag;  // set to 1 by the kernel once the histogram below is final
    int one;         // constant 1, copied into KadCtl.ltab_ready by the host
    int pad[2];
    uint32_t hist[1]; // nclass entries: hist[c] = |{v : c0[v] = c}|
};

// Arguments of the sampling kernel.
struct SampleArgs {
    // rows[0]/cols[0]: the out-arc rows (the s side expands along them, the t
    // side traces back over them); rows[1]/cols[1]: the in-arc rows (the t side
    // expands, the s side traces back); the same arrays for an undirected graph.
    // Indexed by side, so a kernel reads the pointer it needs from the
    // parameter space at the point of use.
    const int32_t *rows[2];
    const int32_t *cols[2];
    const int32_t *comp;
    int32_t n;
    // per-slot scratch, slot-major: slot k uses [k*n, (k+1)*n) of each array; the
    // label array holds one 16-byte record per vertex (label, unused word, sigma)
    uint32_t *label;
    // per-slot bitmap of labelled vertices, slot k uses words [k*nw, (k+1)*nw);
    // small enough to stay in L2, it spares most label reads
    uint32_t *bits;
    int32_t nw;
    int bits_smem; // 1: the bitmap is in dynamic shared memory (nw words), bits unused
    int no_bits;   // 1: no bitmap at all (labels read directly)
    int bits_shift; // one bitmap bit per 2^bits_shift consecutive vertices
    unsigned long long *sigma2;
    int32_t *list;
    // meeting-set members beyond the first mcap (kept in shared memory): mext
    // ids and weights per slot, slot k uses [k*mext, (k+1)*mext); mext = 0: none
    int32_t *mext_id;
    unsigned long long *mext_w;
    int mext;
    // random stream
    uint32_t key0, key1, domain;
    // index space of this launch: [0, calib_n) are calibration samples 0..calib_n-1
    // (phase 1), then adaptive samples i0..i1-1 (phase 0); RECORD mode: [i0, i1)
    // of phase `domain`
    unsigned long long calib_n;
    unsigned long long i0, i1;
    int mode;
    int mcap;
    int pair_cost; // the meeting round's pairwise test runs when |F_X| |F_Y| pair_cost < arcs of F_X
    int nctx; // warp-per-sample kernel: sampling contexts (owner warps) per block
    uint32_t debug; // KAD_DEBUG_*
    // outputs (RING, RECORD)
    int32_t *paths;
    int32_t cap;
    // completion order (RING): 1 = an adaptive sample takes the next fold
    // position when its path is complete; its path is traced into the slot's
    // staging row (cap entries per slot) and then copied to the position's ring
    // row; pidx[position] = its sample index (positions < pidx_cap)
    int fast;
    int32_t *stage;
    unsigned long long *pidx;
    unsigned long long pidx_cap;
    int32_t *plen;
    uint8_t *pflag;
    uint32_t epoch; // N
    uint32_t ring;  // R
    // calibration (RING): counts, their histogram, and where to publish it
    uint32_t *c0w;
    uint32_t *hist;
    KadHostPage *hpage; // device-visible pointer to the mapped host page
    // RECORD extras
    int32_t *rec_s, *rec_t, *rec_D;
    unsigned long long *rec_sst;
    // closer (RING)
    KadCtl *ctl;
    uint32_t *epoch_done; // [R]
    uint32_t *cnt;        // [n]
    const uint32_t *c0;   // [n] (written by this launch's calibration samples: read through L2)
    int32_t *classmax;    // [nclass]
    const double *ltab;   // [nclass]
    int32_t nclass;
    double eps;
    unsigned long long omega;
    unsigned long long k_end; // epochs of this launch end before k_end
    unsigned long long max_epochs; // forced stop after this many epochs (truncated runs); 0 = none
    // work counters [0..5], samples [6], SM cycles per phase [8..13], and of the BFS
    // phase: expansion passes [14] and round closes [15] (KAD_WORK_WORDS)
    unsigned long long *work;
};

// Rows of side z (0: s, 1: t) in the direction it expands, and in the direction
// its trace-back walks toward its root (the other side's expansion rows).  The
// sampling kernels are compiled twice: with KAD_DIRECTED 1 (kad_*_dir.cu) the
// sides read their own rows; the undirected build reads rows[0] for both, so
// its code is that of a one-CSR kernel.
#ifndef KAD_DIRECTED
#define KAD_DIRECTED 0
#endif
static __device__ __forceinline__ const int32_t *xrp(const SampleArgs &a, int z) {
    return KAD_DIRECTED ? a.rows[z] : a.rows[0];
}
static __device__ __forceinline__ const int32_t *xcol(const SampleArgs &a, int z) {
    return KAD_DIRECTED ? a.cols[z] : a.cols[0];
}
static __device__ __forceinline__ const int32_t *trp(const SampleArgs &a, int z) {
    return KAD_DIRECTED ? a.rows[z ^ 1] : a.rows[0];
}
static __device__ __forceinline__ const int32_t *tcol(const SampleArgs &a, int z) {
    return KAD_DIRECTED ? a.cols[z ^ 1] : a.cols[0];
}

// ----------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned long long kad_sat_add(unsigned long long a, unsigned long long b) {
    unsigned long long s = a + b;
    return (s < a) ? KAD_U64MAX : s;
}

__device__ __forceinline__ unsigned long long kad_sat_mul(unsigned long long a, unsigned long long b) {
    return __umul64hi(a, b) ? KAD_U64MAX : a * b;
}

__device__ __forceinline__ uint32_t kad_ld_u32(const uint32_t *p) { return __ldcg(p); }
__device__ __forceinline__ unsigned long long kad_ld_u64(const unsigned long long *p) { return __ldcg(p); }

__device__ __forceinline__ void kad_fence_sc() { asm volatile("fence.sc.gpu;" ::: "memory"); }

__device__ __forceinline__ void kad_set_err(KadCtl *ctl, int code) {
    if (ctl) atomicCAS(&ctl->err, 0, code);
}

// f and g of Appendix B with a fixed operation order and correctly rounded
// operations only (no contraction), so that host and device agree bit for bit
// (out of line: one copy of its divisions and square root per kernel):
//   T = tau, W = omega, b = c/T, q = W/T, a = 1/3 -+ q, x = ((2b) W)/L,
//   f|g = (L/T) (a + sqrt(a*a + x)).
static __device__ __noinline__ double kad_fg_dev(unsigned long long c, double L, unsigned long long tau,
                                             unsigned long long omega, bool upper) {
    double T = (double)tau, W = (double)omega;
    double b = __ddiv_rn((double)c, T);
    double q = __ddiv_rn(W, T);
    double third = 1.0 / 3.0;
    double a = upper ? __dadd_rn(third, q) : __dsub_rn(third, q);
    double x = __ddiv_rn(__dmul_rn(__dmul_rn(2.0, b), W), L);
    return __dmul_rn(__ddiv_rn(L, T), __dadd_rn(a, __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), x))));
}

// Host-side launchers (defined in the .cu files).
cudaError_t kad_launch_sample(const SampleArgs &a, int blocks, int threads, int per_sm, size_t dyn_smem,
                              cudaStream_t st);
bool kad_sample_variant_exists(int threads, int per_sm);
size_t kad_sample_static_smem(int threads, int per_sm);
int kad_sample_max_blocks_per_sm(int threads, int per_sm, size_t dyn_smem);
// the warp-per-sample kernel (kad_wsample.cu): 1024 threads, one block per SM,
// a.nctx contexts per block, dyn_smem = a.nctx x a.nw words of bitmap
cudaError_t kad_launch_wsample(const SampleArgs &a, int blocks, size_t dyn_smem, cudaStream_t st);
// the directed-graph builds (kad_sample_dir.cu, kad_wsample_dir.cu); the launchers
// above hand a directed graph (rows[1] != rows[0]) to them
cudaError_t kad_launch_sample_directed(const SampleArgs &a, int blocks, int threads, int per_sm, size_t dyn_smem,
                                       cudaStream_t st);
cudaError_t kad_launch_wsample_directed(const SampleArgs &a, int blocks, size_t dyn_smem, cudaStream_t st);
size_t kad_wsample_static_smem();
int kad_wsample_max_blocks_per_sm(size_t dyn_smem);
// the sharded run's fold of all ranks' path rows and its stop check (kad_shard.cu)
cudaError_t kad_launch_fold_rows(const int32_t *blocks, int world, int maxc, int cap, int calib, uint32_t *c0w,
                                 uint32_t *hist, uint32_t *cnt, int32_t *classmax, const uint32_t *c0,
                                 unsigned long long *ovf, cudaStream_t st);
cudaError_t kad_launch_check_classes(const int32_t *classmax, const double *ltab, int nclass, unsigned long long tau,
                                     unsigned long long omega, double eps, int *fail, cudaStream_t st);
cudaError_t kad_launch_finalize(const uint32_t *cnt, int32_t n, unsigned long long tau, double *bc, cudaStream_t st);
cudaError_t kad_launch_fg(const uint32_t *counts, const uint32_t *c0, const double *ltab, int32_t n,
                          unsigned long long tau, unsigned long long omega, double *f, double *g, cudaStream_t st);

// graph set-up (kad_graph.cu)
// rp/col: the out-arc rows (the s side expands along them); rpT/colT: the
// in-arc rows (the t side's), the same arrays when the graph is undirected.
struct KadGraphDev {
    int32_t n;
    int64_t m;
    int32_t *rp;
    int32_t *col;
    int32_t *comp;
    int32_t *rpT;
    int32_t *colT;
    bool directed;
};
kad_status kad_graph_setup(KadGraphDev &gd, uint32_t flags, cudaStream_t st, int32_t *vd, int32_t *ncomp, int32_t *maxdeg,
                           cudaError_t *cerr);

// Stream-ordered allocation from the library's graph pool on the current device
// (freed memory stays mapped for the next graph until kad_trim); free with
// cudaFreeAsync.
cudaError_t kad_pool_alloc(void **p, size_t bytes, cudaStream_t st);
