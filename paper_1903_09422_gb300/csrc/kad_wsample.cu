// The warp-per-sample KADABRA sampling kernel (sm_103a).
//
// One persistent block of 1024 threads per SM.  Warp c < nctx owns sampling
// context c (a sampling slot: its own labels, path counts and labelled list in
// global scratch, its own bitmap of labelled vertices in shared memory) and
// computes samples one after another, every step of a sample with its own 32
// lanes: the pair draw, the rounds of the balanced bidirectional search, the
// meeting draw, the trace-back, the output and the reset (Section 2.3
// sample(), Appendix C.1).  The steps are those of the block-per-sample kernel
// (kad_sample.cu) and of the oracle; a sample's result depends only on its index.
//
// A round whose work exceeds what one warp should do alone -- a chunk of the
// expanding side's frontier with many arcs (a hub's row), a frontier of more
// than 32 vertices, or many pairwise adjacency tests -- is posted on the block's
// job board in shared memory.  Any warp that is waiting (for its own job to
// finish) or has no sample of its own claims pieces of posted jobs and expands
// them for the posting context.  Expansion commutes (claims, saturating path
// count pushes, meeting-set marks are order-independent), so the result is the
// same whoever expands which arcs.  No warp waits at a block barrier; a warp
// waits only for the pieces of its own jobs, and helps others meanwhile.
//
// Job protocol (one per warp for arc jobs, one per context for frontier and
// pairwise jobs): the poster writes the job's data, then its claim counter,
// then sets its bit in the board's mask.  A helper increments the job's
// in-flight count, re-reads the mask bit (after a sequentially consistent fence),
// and leaves if it is clear; else it claims pieces with atomicAdd until none is
// left, and decrements the in-flight count when done.  The poster, once its own
// claims run out, clears the bit (fence), then waits until the in-flight count
// is zero: every claimed piece has then been expanded.  The in-flight count is
// never reset, so a late helper is counted for whichever job it meets.
//
// Epochs, the closer, calibration hand-off and completion order are those of
// the block kernel, run by one warp.  Every wait is bounded (global timer); a
// wait that runs out sets KAD_DERR_WAIT and the warp leaves the kernel.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "kad_device.cuh"

#define W_THREADS 1024
#define W_WARPS 32
#define W_MC 32            // meeting-set members kept in shared memory per context
#define W_ITEMS 4          // arcs per lane and expansion pass (128 per warp pass)
#define W_SOLO_ARCS 512    // a chunk with at most this many arcs is expanded by its warp alone
#define W_PIECE_ARCS 256   // arcs per claimed piece of an arc job
#define W_PIECE_PAIRS 128  // pairs per claimed piece of a pairwise job
#define W_LCAP 64          // largest predecessor level tested for adjacency in a trace step
#define W_DEG_SCAN 128     // adjacency lists up to this length are always scanned in a trace step
#define W_PAIR_MIN_ARCS 1024
#define W_PROBE_MIN_ARCS 256 // rounds with more arcs are probed for the meeting before claiming
#define W_WAIT_NS 20000000000ull // a wait without progress gives up after 20 s

namespace {

// ---------------------------------------------------------------- shared state
// A warp's scratch: the frontier chunk it expands (or posts as an arc job), or
// the candidates of a trace step, or the bins of a digit-wise meeting draw.
struct WChunkData {
    int32_t uid[32];
    int32_t rs[32];
    int32_t re[32];
    int32_t off[32];
    unsigned long long sig[32];
};
struct WTraceData {
    int32_t p[W_LCAP];
    unsigned long long s[W_LCAP];
};
struct WBins {
    unsigned long long lo[16], hi[16];
};
struct WWarp {
    union {
        WChunkData ch;
        WTraceData tr;
        WBins bins;
    } u;
    int cnt;      // chunk entries
    int total;    // chunk arcs
    int ctx;      // context the chunk is expanded for
    int next;     // arc job: next arc offset to claim
    int inflight; // warps inside this warp's arc job (never reset)
    int pad[3];
};

// A sampling context: one sample in flight.
struct WCtx {
    unsigned long long idx;
    unsigned long long dsum[2];
    unsigned long long next_dsum; // next frontier's degree sum (atomic)
    unsigned long long pred;      // arcs into the next level / meeting set this round (atomic)
    unsigned long long st_w0, st_w1;
    unsigned long long acc[KAD_WORK_WORDS];
    long long tmark;
    uint32_t st_blk, dom;
    int st_pos;
    int calib, s, t, D, X, mid, watch, abort;
    int fb[2], fe[2], lev[2], tail[2], root_rs[2];
    int met;    // the round reached the other side's frontier
    int probe;  // this scan of the round only looks for the other side's frontier (no claims)
    int probe_score, probe_rounds; // probe-first policy (as the block kernel's)
    int mcount; // meeting-set members recorded (atomic)
    int predm;  // pred counts arcs into M (1) or into the next level (0)
    uint32_t sideX, keyNext;
    int tailY;
    // context job: frontier entries [jnext, jend) of side X (kind 1), or
    // pairwise tests [jnext, jend) (kind 2); in-flight count never reset
    int jkind, jnext, jend, inflight;
    int pfx, pyb; // pairwise job: |F_X| (its data in the owner warp's chunk), start of F_Y
    int lvs[2][KAD_MAXLV + 2];
    int32_t m_id[W_MC];
    unsigned long long m_w[W_MC];
};

struct WShared {
    unsigned arcmask;   // bit w: warp w's chunk is an open arc job
    unsigned ctxmask;   // bit c: context c has an open frontier or pairwise job
    int active;         // owner warps still sampling
    int pad;
    WWarp w[W_WARPS];
    WCtx c[W_WARPS];
};

extern __shared__ uint32_t w_bits_dyn[]; // nctx per-context bitmaps of labelled vertices

__device__ __forceinline__ void fence_sc_cta() { asm volatile("fence.sc.cta;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T vload(const T &x) {
    return *(const volatile T *)&x;
}

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
    return __shfl_sync(FULL_MASK, v, src);
}

// Global scratch of a context (slot = block * nctx + context).
struct Slot {
    uint32_t *label; // 16-byte records: label, -, sigma
    unsigned long long *sigma2;
    int32_t *list;
    int32_t *mext_id;
    unsigned long long *mext_w;
    int32_t *stage;
    uint32_t *bits; // shared memory, a.nw words (one bit per 2^bits_shift vertices)
};

__device__ __forceinline__ Slot slot_of(const SampleArgs &a, int c) {
    const size_t slot = (size_t)blockIdx.x * (size_t)a.nctx + (size_t)c;
    const size_t soff = slot * (size_t)a.n;
    Slot s;
    s.label = a.label + 4 * soff;
    s.sigma2 = a.sigma2 + soff;
    s.list = a.list + soff;
    const int mext = a.mext_id ? a.mext : 0;
    s.mext_id = mext ? a.mext_id + slot * (size_t)mext : nullptr;
    s.mext_w = mext ? a.mext_w + slot * (size_t)mext : nullptr;
    s.stage = a.stage ? a.stage + slot * (size_t)a.cap : nullptr;
    s.bits = w_bits_dyn + (size_t)c * (size_t)a.nw;
    return s;
}

// Bounded wait bookkeeping: a deadline that moves whenever progress is seen.
__device__ __forceinline__ bool wait_expired(unsigned long long &deadline, const SampleArgs &a) {
    if (*(volatile int *)&a.ctl->err) return true; // another warp failed: stop waiting
    const unsigned long long now = global_ns();
    if (deadline == 0) deadline = now + W_WAIT_NS;
    if (now > deadline) {
        kad_set_err(a.ctl, KAD_DERR_WAIT);
        return true;
    }
    return false;
}

// ---------------------------------------------------------------- expansion
// One warp pass over arcs [base, base + 128) (below `end`) of chunk `cw` for
// context c: lane l takes arcs base + l + 32k, k < W_ITEMS.  All neighbour ids
// are loaded before any bitmap word, those before any label or atomic.  The
// claim of an unlabelled vertex and its path-count push commute with every
// other arc's (only side X labels this round, and a vertex it labels gets the
// level keyNext), so any warp may expand any arcs in any order.  The arc that
// first marks a vertex of the other side's frontier records it in M.  Returns
// true (for the whole warp) when the run has stopped and the sample may give up.
__device__ __noinline__ bool w_expand_pass(const SampleArgs &a, WShared &S, int c, int cw, int base, int end) {
    WCtx &C = S.c[c];
    const WWarp &W = S.w[cw];
    const Slot sl = slot_of(a, c);
    const int lane = threadIdx.x & 31;
    const bool nobits = a.no_bits != 0;
    const int gs = a.bits_shift;
    int stop_now = 0;
    if (lane == 0 && vload(C.watch)) stop_now = *(volatile int *)&a.ctl->stop;
    const int met_before = vload(C.met);
    const bool probe = vload(C.probe) != 0;
    const int cnt = W.cnt;
    const uint32_t sideX = C.sideX, keyNext = C.keyNext;
    const int X = C.X; // side X's rows (its direction) are a.rows[X], a.cols[X]
    int vv[W_ITEMS], ix[W_ITEMS];
    uint32_t ll[W_ITEMS];
#pragma unroll
    for (int k = 0; k < W_ITEMS; k++) {
        const int e = base + lane + 32 * k;
        vv[k] = -1;
        ix[k] = 0;
        if (e < end) {
            int lo = 0, hi = cnt - 1; // last j with off[j] <= e
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (W.u.ch.off[mid] <= e)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            vv[k] = __ldg(xcol(a, X) + W.u.ch.rs[lo] + (e - W.u.ch.off[lo]));
            ix[k] = lo;
        }
    }
    bool fresh[W_ITEMS];
    if (nobits) {
#pragma unroll
        for (int k = 0; k < W_ITEMS; k++) ll[k] = (vv[k] >= 0) ? kad_ld_u32(lab_at(sl.label, vv[k])) : 0u;
    } else {
#pragma unroll
        for (int k = 0; k < W_ITEMS; k++) {
            bool set = false;
            if (vv[k] >= 0) {
                const int b = vv[k] >> gs;
                set = (sl.bits[b >> 5] >> (b & 31)) & 1u;
            }
            ll[k] = set ? kad_ld_u32(lab_at(sl.label, vv[k])) : 0u;
        }
    }
#pragma unroll
    for (int k = 0; k < W_ITEMS; k++) fresh[k] = vv[k] >= 0 && ll[k] == 0u;
    int reaches_y = 0;
#pragma unroll
    for (int k = 0; k < W_ITEMS; k++)
        if (ll[k] != 0u && (ll[k] & KAD_SIDE) != sideX) reaches_y = 1;
    const bool warp_meets = __any_sync(FULL_MASK, reaches_y) != 0;
    if (__shfl_sync(FULL_MASK, stop_now, 0)) return true;
    if (warp_meets && lane == 0) C.met = 1;
    const bool meeting_seen = warp_meets || met_before != 0;
    uint32_t old[W_ITEMS];
    unsigned long long prev[W_ITEMS], add[W_ITEMS];
    int kind[W_ITEMS]; // 0 none, 1 next level of X, 2 other side's frontier
#pragma unroll
    for (int k = 0; k < W_ITEMS; k++) {
        old[k] = 0u;
        kind[k] = 0;
        prev[k] = 0;
        add[k] = W.u.ch.sig[ix[k]];
        const int v = vv[k];
        if (fresh[k]) {
            if (meeting_seen || probe) continue;
            old[k] = atomicCAS(lab_at(sl.label, v), 0u, keyNext);
            kind[k] = 1;
            prev[k] = atomicAdd(sig_at(sl.label, v), add[k]);
        } else if (ll[k] != 0u) {
            const uint32_t lv = ll[k];
            if ((lv & KAD_KEY) == keyNext) {
                kind[k] = 1;
                prev[k] = atomicAdd(sig_at(sl.label, v), add[k]);
            } else if ((lv & KAD_SIDE) != sideX) {
                kind[k] = 2;
                if (!(lv & KAD_INM) && !(atomicOr(lab_at(sl.label, v), KAD_INM) & KAD_INM)) {
                    const int slot = atomicAdd(&C.mcount, 1);
                    const int mc = (a.mcap < W_MC) ? a.mcap : W_MC;
                    if (slot < mc)
                        C.m_id[slot] = v;
                    else if (sl.mext_id && slot - mc < a.mext)
                        sl.mext_id[slot - mc] = v;
                }
                prev[k] = atomicAdd(sl.sigma2 + v, add[k]);
            }
        }
    }
    int rs0[W_ITEMS], rs1[W_ITEMS];
#pragma unroll
    for (int k = 0; k < W_ITEMS; k++) {
        rs0[k] = rs1[k] = 0;
        if (fresh[k] && kind[k] == 1) {
            rs0[k] = __ldg(xrp(a, X) + vv[k]);
            rs1[k] = __ldg(xrp(a, X) + vv[k] + 1);
        }
    }
    bool claimed[W_ITEMS];
    bool any_m = false;
    unsigned long long pn = 0, pm = 0;
#pragma unroll
    for (int k = 0; k < W_ITEMS; k++) {
        claimed[k] = fresh[k] && kind[k] == 1 && old[k] == 0u;
        if (fresh[k] && kind[k] == 1 && old[k] != 0u && old[k] != keyNext) kad_set_err(a.ctl, KAD_DERR_LEVEL);
        if (claimed[k] && !nobits) {
            const int b = vv[k] >> gs;
            atomicOr(sl.bits + (b >> 5), 1u << (b & 31));
        }
        if (kind[k] == 1) {
            pn++;
            if (prev[k] + add[k] < prev[k]) atomicOr(lab_at(sl.label, vv[k]), KAD_OVF);
        } else if (kind[k] == 2) {
            pm++;
            any_m = true;
            if (prev[k] + add[k] < prev[k]) atomicOr(lab_at(sl.label, vv[k]), KAD_OVF2);
        }
    }
    if (any_m) C.met = 1;
    // arcs into the next level and into M: kept apart, the round keeps one
    pn = warp_sum_u64(pn);
    pm = warp_sum_u64(pm);
    if (lane == 0 && (pn | pm)) atomicAdd(&C.pred, pn | (pm << 40));
    unsigned mask[W_ITEMS];
    int nclaim = 0;
    unsigned long long mydeg = 0;
#pragma unroll
    for (int k = 0; k < W_ITEMS; k++) {
        mask[k] = __ballot_sync(FULL_MASK, claimed[k]);
        nclaim += __popc(mask[k]);
        if (claimed[k]) mydeg += (unsigned long long)(rs1[k] - rs0[k]);
    }
    if (nclaim) {
        const int tailY = C.tailY, n = a.n;
        int pos0 = 0;
        if (lane == 0) pos0 = atomicAdd(&C.tail[X], nclaim);
        pos0 = __shfl_sync(FULL_MASK, pos0, 0);
#pragma unroll
        for (int k = 0; k < W_ITEMS; k++) {
            if (claimed[k]) {
                const int pos = pos0 + __popc(mask[k] & lanemask_lt());
                if (pos + tailY < n)
                    sl.list[phys(X, pos, n)] = vv[k];
                else
                    kad_set_err(a.ctl, KAD_DERR_FRONTIER);
            }
            pos0 += __popc(mask[k]);
        }
        const unsigned long long ds = warp_sum_u64(mydeg);
        if (lane == 0) atomicAdd(&C.next_dsum, ds);
    }
    return false;
}

// Expand arcs [b0, b1) of chunk cw for context c, pass by pass; an abandoned
// sample (the run stopped) skips the rest.
__device__ __forceinline__ void w_expand_range(const SampleArgs &a, WShared &S, int c, int cw, int b0, int b1) {
    for (int b = b0; b < b1; b += 32 * W_ITEMS) {
        if (vload(S.c[c].abort)) return;
        if (w_expand_pass(a, S, c, cw, b, b1)) {
            if ((threadIdx.x & 31) == 0) S.c[c].abort = 1;
            return;
        }
    }
}

// Pairwise tests [p0, p1) of context c's round: pair p tests u = F_X[p % fx]
// (row bounds and path count in the owner warp's chunk) against
// w = F_Y[p / fx] with binary searches in the shorter row, four pairs per lane
// interleaved.  An adjacent pair is an arc from X's frontier into Y's: w joins
// M and receives sigma_X(u).
__device__ __noinline__ void w_pair_range(const SampleArgs &a, WShared &S, int c, int p0, int p1) {
    WCtx &C = S.c[c];
    const WWarp &F = S.w[c]; // F_X lives in the owner warp's chunk
    const Slot sl = slot_of(a, c);
    const int lane = threadIdx.x & 31;
    const int fx = C.pfx, yb = C.pyb, Y = 1 - C.X, n = a.n;
    const int mcap = (a.mcap < W_MC) ? a.mcap : W_MC;
    // u in F_X has an arc toward w in F_Y when w is in u's row (X's direction)
    // or u in w's row (Y's direction)
    unsigned long long pm = 0;
    for (int q0 = p0; q0 < p1; q0 += 128) {
        if (vload(C.abort)) break;
        int pi[4], pw[4], lo[4], hi[4], key[4];
        bool hit[4], inU[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int p = q0 + lane + 32 * k;
            pi[k] = -1;
            pw[k] = -1;
            hit[k] = false;
            inU[k] = false;
            lo[k] = hi[k] = key[k] = 0;
            if (p < p1) {
                pi[k] = p % fx;
                pw[k] = __ldcg(sl.list + phys(Y, yb + p / fx, n));
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (pw[k] < 0) continue;
            const int rsW = __ldg(xrp(a, Y) + pw[k]), reW = __ldg(xrp(a, Y) + pw[k] + 1);
            const int rsU = F.u.ch.rs[pi[k]], reU = F.u.ch.re[pi[k]];
            if (reU - rsU <= reW - rsW) {
                lo[k] = rsU;
                hi[k] = reU;
                key[k] = pw[k];
                inU[k] = true;
            } else {
                lo[k] = rsW;
                hi[k] = reW;
                key[k] = F.u.ch.uid[pi[k]];
            }
        }
        for (int step = 0; step < 32; step++) {
            bool any = false;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (hit[k] || lo[k] >= hi[k]) continue;
                any = true;
                const int mid = (lo[k] + hi[k]) >> 1;
                const int v = __ldg(xcol(a, inU[k] ? 1 - Y : Y) + mid);
                if (v < key[k])
                    lo[k] = mid + 1;
                else if (v > key[k])
                    hi[k] = mid;
                else
                    hit[k] = true;
            }
            if (!any) break;
        }
        unsigned long long prev[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            prev[k] = 0;
            if (!hit[k]) continue;
            if (!(atomicOr(lab_at(sl.label, pw[k]), KAD_INM) & KAD_INM)) {
                const int slot = atomicAdd(&C.mcount, 1);
                if (slot < mcap)
                    C.m_id[slot] = pw[k];
                else if (sl.mext_id && slot - mcap < a.mext)
                    sl.mext_id[slot - mcap] = pw[k];
            }
            prev[k] = atomicAdd(sl.sigma2 + pw[k], F.u.ch.sig[pi[k]]);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (!hit[k]) continue;
            pm++;
            C.met = 1;
            if (prev[k] + F.u.ch.sig[pi[k]] < prev[k]) atomicOr(lab_at(sl.label, pw[k]), KAD_OVF2);
        }
    }
    pm = warp_sum_u64(pm);
    if (lane == 0 && pm) atomicAdd(&C.pred, pm << 40);
}

// Load frontier entries [j0, j1) (at most 32) of context c's expanding side
// into warp `me`'s chunk: row bounds, path counts, exclusive arc offsets.
__device__ __forceinline__ void w_build_chunk(const SampleArgs &a, WShared &S, int c, int me, int j0, int j1) {
    WCtx &C = S.c[c];
    WWarp &W = S.w[me];
    const Slot sl = slot_of(a, c);
    const int lane = threadIdx.x & 31;
    const int X = C.X, cnt = j1 - j0;
    int d = 0;
    if (C.lev[X] == 0) { // the root alone: its row is known and sigma = 1
        if (lane == 0) {
            W.u.ch.rs[0] = C.root_rs[X];
            W.u.ch.sig[0] = 1ull;
            d = (int)C.dsum[X];
        }
    } else if (lane < cnt) {
        const int u = __ldcg(sl.list + phys(X, j0 + lane, a.n));
        const int rs = __ldg(xrp(a, X) + u), re = __ldg(xrp(a, X) + u + 1);
        uint32_t lu;
        unsigned long long su;
        ld_vs(sl.label, u, lu, su);
        W.u.ch.rs[lane] = rs;
        W.u.ch.sig[lane] = sig_val(lu, su);
        d = re - rs;
    }
    int x = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane < cnt) W.u.ch.off[lane] = x - d;
    const int total = __shfl_sync(FULL_MASK, x, 31);
    if (lane == 0) {
        W.cnt = cnt;
        W.total = total;
        W.ctx = c;
    }
    __syncwarp();
}

// ---------------------------------------------------------------- jobs
// Helping: enter warp w's arc job, expand claimed pieces until none is left.
__device__ __noinline__ bool w_help_arc(const SampleArgs &a, WShared &S, int me) {
    const int lane = threadIdx.x & 31;
    unsigned m = vload(S.arcmask) & ~(1u << me);
    if (!m) return false;
    const unsigned rot = (m >> me) | (me ? (m << (32 - me)) : 0u); // start looking after my own id
    const int w = (__ffs(rot) - 1 + me) & 31;
    WWarp &W = S.w[w];
    int ok = 0;
    if (lane == 0) {
        atomicAdd(&W.inflight, 1);
        fence_sc_cta();
        ok = (vload(S.arcmask) >> w) & 1u;
        if (!ok) atomicSub(&W.inflight, 1);
    }
    ok = __shfl_sync(FULL_MASK, ok, 0);
    if (!ok) return false;
    for (;;) {
        int off = 0;
        if (lane == 0) off = atomicAdd(&W.next, W_PIECE_ARCS);
        off = __shfl_sync(FULL_MASK, off, 0);
        const int total = vload(W.total);
        if (off >= total) break;
        w_expand_range(a, S, vload(W.ctx), w, off, min(off + W_PIECE_ARCS, total));
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        atomicSub(&W.inflight, 1);
    }
    return true;
}

__device__ void w_run_chunk(const SampleArgs &a, WShared &S, int c, int me);

// Helping: an arc job if there is one, else a piece of a context job.  Uses
// warp `me`'s chunk (a frontier piece is loaded there): only for warps whose
// chunk is free.
__device__ __noinline__ bool w_help_any(const SampleArgs &a, WShared &S, int me) {
    if (w_help_arc(a, S, me)) return true;
    const int lane = threadIdx.x & 31;
    unsigned m = vload(S.ctxmask);
    if (!m) return false;
    const unsigned rot = (m >> me) | (me ? (m << (32 - me)) : 0u);
    const int c = (__ffs(rot) - 1 + me) & 31;
    WCtx &C = S.c[c];
    int ok = 0;
    if (lane == 0) {
        atomicAdd(&C.inflight, 1);
        fence_sc_cta();
        ok = (vload(S.ctxmask) >> c) & 1u;
        if (!ok) atomicSub(&C.inflight, 1);
    }
    ok = __shfl_sync(FULL_MASK, ok, 0);
    if (!ok) return false;
    const int kind = vload(C.jkind);
    const int piece = (kind == 1) ? 32 : W_PIECE_PAIRS;
    for (;;) {
        int j = 0;
        if (lane == 0) j = atomicAdd(&C.jnext, piece);
        j = __shfl_sync(FULL_MASK, j, 0);
        const int je = vload(C.jend);
        if (j >= je) break;
        if (vload(C.abort)) continue; // drain the claims quickly
        if (kind == 1) {
            w_build_chunk(a, S, c, me, j, min(j + 32, je));
            w_run_chunk(a, S, c, me);
        } else {
            w_pair_range(a, S, c, j, min(j + piece, je));
        }
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        atomicSub(&C.inflight, 1);
    }
    return true;
}

// Expand warp me's chunk (context c): alone when small, else as an arc job that
// other warps help with; returns when every arc is expanded.  While waiting it
// helps other arc jobs only (its chunk is in use).
__device__ void w_run_chunk(const SampleArgs &a, WShared &S, int c, int me) {
    WWarp &W = S.w[me];
    const int lane = threadIdx.x & 31;
    const int total = W.total;
    if (total <= W_SOLO_ARCS) {
        w_expand_range(a, S, c, me, 0, total);
        return;
    }
    if (lane == 0) {
        W.next = 0;
        __threadfence_block();
        atomicOr(&S.arcmask, 1u << me);
    }
    __syncwarp();
    for (;;) {
        int off = 0;
        if (lane == 0) off = atomicAdd(&W.next, W_PIECE_ARCS);
        off = __shfl_sync(FULL_MASK, off, 0);
        if (off >= total) break;
        w_expand_range(a, S, c, me, off, min(off + W_PIECE_ARCS, total));
    }
    if (lane == 0) {
        atomicAnd(&S.arcmask, ~(1u << me));
        fence_sc_cta();
    }
    unsigned long long deadline = 0;
    for (;;) {
        int busy = 0;
        if (lane == 0) busy = vload(W.inflight);
        busy = __shfl_sync(FULL_MASK, busy, 0);
        if (!busy) break;
        if (w_help_arc(a, S, me)) {
            deadline = 0;
            continue;
        }
        if (wait_expired(deadline, a)) break;
        __nanosleep(32);
    }
    __syncwarp();
    __threadfence_block();
}

// Post context c's frontier entries or pairwise tests [j0, j1) as a context job,
// work on it, and wait until every piece is done.  While waiting the owner helps
// others: anything for a frontier job; arc jobs only for a pairwise job, whose
// data sits in the owner's chunk.
__device__ void w_run_ctx_job(const SampleArgs &a, WShared &S, int c, int kind, int j0, int j1) {
    WCtx &C = S.c[c];
    const int lane = threadIdx.x & 31;
    const int piece = (kind == 1) ? 32 : W_PIECE_PAIRS;
    if (lane == 0) {
        C.jkind = kind;
        C.jend = j1;
        C.jnext = j0;
        __threadfence_block();
        atomicOr(&S.ctxmask, 1u << c);
    }
    __syncwarp();
    for (;;) {
        int j = 0;
        if (lane == 0) j = atomicAdd(&C.jnext, piece);
        j = __shfl_sync(FULL_MASK, j, 0);
        if (j >= j1) break;
        if (vload(C.abort)) continue;
        if (kind == 1) {
            w_build_chunk(a, S, c, c, j, min(j + 32, j1));
            w_run_chunk(a, S, c, c);
        } else {
            w_pair_range(a, S, c, j, min(j + piece, j1));
        }
    }
    if (lane == 0) {
        atomicAnd(&S.ctxmask, ~(1u << c));
        fence_sc_cta();
    }
    unsigned long long deadline = 0;
    for (;;) {
        int busy = 0;
        if (lane == 0) busy = vload(C.inflight);
        busy = __shfl_sync(FULL_MASK, busy, 0);
        if (!busy) break;
        const bool did = (kind == 1) ? w_help_any(a, S, c) : w_help_arc(a, S, c);
        if (did) {
            deadline = 0;
            continue;
        }
        if (wait_expired(deadline, a)) break;
        __nanosleep(32);
    }
    __syncwarp();
    __threadfence_block();
}

// ---------------------------------------------------------------- search
// The balanced bidirectional search of context c's sample (Section 2.3,
// Appendix C.1): each round expands the side whose frontier has the smaller
// degree sum (s on ties); the round that reaches the other side's frontier
// collects M and sigma_X on M.  Sets C.D (0: no path or abandoned).
__device__ __noinline__ void w_search(const SampleArgs &a, WShared &S, int c) {
    WCtx &C = S.c[c];
    const Slot sl = slot_of(a, c);
    const int lane = threadIdx.x & 31, n = a.n;
    for (;;) {
        __syncwarp();
        if (C.D >= 0) break;
        const int X = (C.dsum[0] <= C.dsum[1]) ? 0 : 1, Y = 1 - X;
        const int fb = C.fb[X], fe = C.fe[X], levX = C.lev[X];
        if (fb == fe || levX + 2 > (int)KAD_LVL) {
            if (lane == 0) {
                if (fb != fe) kad_set_err(a.ctl, KAD_DERR_LEVEL);
                C.D = 0;
            }
            continue;
        }
        const int yb = C.fb[Y], fx = fe - fb, fy = C.fe[Y] - yb;
        const unsigned long long dX = C.dsum[X];
        if (lane == 0) {
            C.X = X;
            C.sideX = X ? KAD_SIDE : 0u;
            C.keyNext = C.sideX | (uint32_t)(levX + 2);
            C.tailY = C.tail[Y];
            C.met = 0;
            C.next_dsum = 0;
            C.pred = 0;
            C.acc[0] += (unsigned long long)fx;
            C.acc[1] += dX;
        }
        __syncwarp();
        const bool pairs = !(a.debug & KAD_DEBUG_FULL_SCAN) && fx <= 32 && dX >= W_PAIR_MIN_ARCS &&
                           (unsigned long long)fx * (unsigned long long)fy * (unsigned)a.pair_cost < dX;
        if (pairs) {
            WWarp &W = S.w[c];
            if (lane < fx) {
                const int u = __ldcg(sl.list + phys(X, fb + lane, n));
                uint32_t lu;
                unsigned long long su;
                ld_vs(sl.label, u, lu, su);
                W.u.ch.uid[lane] = u;
                W.u.ch.rs[lane] = __ldg(xrp(a, X) + u);
                W.u.ch.re[lane] = __ldg(xrp(a, X) + u + 1);
                W.u.ch.sig[lane] = sig_val(lu, su);
            }
            if (lane == 0) {
                C.pfx = fx;
                C.pyb = yb;
            }
            __syncwarp();
            const int np = fx * fy;
            if (np <= W_PIECE_PAIRS)
                w_pair_range(a, S, c, 0, np);
            else
                w_run_ctx_job(a, S, c, 2, 0, np);
            __syncwarp();
        }
        // A large round is probed first: one scan that only looks for arcs into
        // the other side's frontier, and claims new vertices only if it found
        // none (the meeting round holds almost all of a sample's arcs).
        const bool large = dX > W_PROBE_MIN_ARCS;
        const bool probe_first = !(a.debug & KAD_DEBUG_NO_PROBE) && large &&
                                 (C.probe_score > 0 || (C.probe_rounds & 15) == 0);
        long long tp = 0;
        if (lane == 0) tp = clock64();
        for (int ph = probe_first ? 0 : 1; ph < 2; ph++) {
            __syncwarp();
            if (vload(C.met) || vload(C.abort)) break;
            if (lane == 0) C.probe = (ph == 0) ? 1 : 0;
            __syncwarp();
            if (fx <= 32) {
                w_build_chunk(a, S, c, c, fb, fe);
                w_run_chunk(a, S, c, c);
            } else {
                w_run_ctx_job(a, S, c, 1, fb, fe);
            }
        }
        __syncwarp();
        __threadfence_block();
        if (lane == 0) {
            const long long tc = clock64();
            C.acc[14] += (unsigned long long)(tc - tp);
            const int met = C.met;
            if (large) {
                C.probe_rounds++;
                if (probe_first) C.probe_score = met ? min(C.probe_score + 1, 8) : C.probe_score - 1;
            }
            const unsigned long long pr = C.pred;
            C.acc[3] += met ? (pr >> 40) : (pr & ((1ull << 40) - 1));
            if (C.abort) {
                C.D = 0; // the run stopped: this sample is never counted
            } else if (met) {
                C.D = C.lev[X] + 1 + C.lev[Y];
            } else {
                const int tl = min(C.tail[X], n - C.tailY);
                C.acc[2] += (unsigned long long)(tl - fe);
                C.fb[X] = fe;
                C.fe[X] = tl;
                C.lev[X] = levX + 1;
                if (levX + 2 <= KAD_MAXLV + 1) C.lvs[X][levX + 2] = tl;
                C.dsum[X] = C.next_dsum;
            }
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------- meeting draw
// w in M with probability sigma_X(w) sigma_Y(w) / sigma_st, M in ascending id
// (Section 2.3).  Lane 0 holds the stream.  Returns sigma_st; sets C.mid.
__device__ __noinline__ unsigned long long w_meeting(const SampleArgs &a, WShared &S, int c, Stream &st) {
    WCtx &C = S.c[c];
    WWarp &W = S.w[c];
    const Slot sl = slot_of(a, c);
    const int lane = threadIdx.x & 31, n = a.n;
    const int X = C.X, Y = 1 - X;
    const int yb = C.fb[Y], ye = C.fe[Y];
    const int mcap = (a.mcap < W_MC) ? a.mcap : W_MC;
    const int mext = sl.mext_id ? a.mext : 0;
    const int mc = C.mcount;
    const bool recorded = mc <= mcap + mext;
    unsigned long long part = 0;
    if (recorded) {
        for (int i = lane; i < mc; i += 32) {
            const int v = (i < mcap) ? C.m_id[i] : __ldcg(sl.mext_id + (i - mcap));
            uint32_t lv;
            unsigned long long s1;
            const unsigned long long s2 = kad_ld_u64(sl.sigma2 + v);
            ld_vs(sl.label, v, lv, s1);
            const unsigned long long w = kad_sat_mul((lv & KAD_OVF2) ? KAD_U64MAX : s2, sig_val(lv, s1));
            part = kad_sat_add(part, w);
            if (i < mcap)
                C.m_w[i] = w;
            else
                sl.mext_w[i - mcap] = w;
        }
    } else {
        for (int j = yb + lane; j < ye; j += 32) {
            const int v = __ldcg(sl.list + phys(Y, j, n));
            uint32_t lv;
            unsigned long long s1;
            ld_vs(sl.label, v, lv, s1);
            if (lv & KAD_INM) {
                const unsigned long long sx = (lv & KAD_OVF2) ? KAD_U64MAX : kad_ld_u64(sl.sigma2 + v);
                part = kad_sat_add(part, kad_sat_mul(sx, sig_val(lv, s1)));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part = kad_sat_add(part, __shfl_xor_sync(FULL_MASK, part, o));
    const unsigned long long sst = part;
    unsigned long long r = 0;
    if (lane == 0) r = st.uniform(sst ? sst : 1ull, a.ctl);
    r = shfl64(r, 0);
    __syncwarp();
    int mid = -1;
    if (recorded && mc <= 32) {
        // one member per lane: its exclusive prefix in id order is the sum of the
        // weights of the members with smaller ids
        int id = -1;
        unsigned long long w = 0;
        if (lane < mc) {
            id = (lane < mcap) ? C.m_id[lane] : __ldcg(sl.mext_id + (lane - mcap));
            w = (lane < mcap) ? C.m_w[lane] : __ldcg(sl.mext_w + (lane - mcap));
        }
        unsigned long long ex = 0;
        for (int q = 0; q < mc; q++) {
            const int iq = __shfl_sync(FULL_MASK, id, q);
            const unsigned long long wq = shfl64(w, q);
            if (iq < id) ex = kad_sat_add(ex, wq);
        }
        const unsigned hit = __ballot_sync(FULL_MASK, lane < mc && ex <= r && kad_sat_add(ex, w) > r);
        if (hit) mid = __shfl_sync(FULL_MASK, id, __ffs(hit) - 1);
    } else {
        // digit-wise selection, 4 bits per pass from the top, exact 128-bit bin
        // sums, over the recorded members, else over the other side's frontier
        const int nb = 32 - __clz(max(n - 1, 1));
        const int top = ((nb + 3) / 4) * 4;
        unsigned int prefix = 0;
        unsigned long long P = 0;
        for (int shift = top - 4; shift >= 0; shift -= 4) {
            if (lane < 16) {
                W.u.bins.lo[lane] = 0;
                W.u.bins.hi[lane] = 0;
            }
            __syncwarp();
            const unsigned long long want = (unsigned long long)prefix >> (shift + 4);
            if (recorded) {
                for (int i = lane; i < mc; i += 32) {
                    const int v = (i < mcap) ? C.m_id[i] : __ldcg(sl.mext_id + (i - mcap));
                    if (((unsigned long long)(unsigned)v >> (shift + 4)) != want) continue;
                    const unsigned long long w = (i < mcap) ? C.m_w[i] : __ldcg(sl.mext_w + (i - mcap));
                    const int b = ((unsigned)v >> shift) & 15;
                    const unsigned long long o = atomicAdd(&W.u.bins.lo[b], w);
                    if (o + w < o) atomicAdd(&W.u.bins.hi[b], 1ull);
                }
            } else {
                for (int j = yb + lane; j < ye; j += 32) {
                    const int v = __ldcg(sl.list + phys(Y, j, n));
                    if (((unsigned long long)(unsigned)v >> (shift + 4)) != want) continue;
                    uint32_t lv;
                    unsigned long long s1;
                    ld_vs(sl.label, v, lv, s1);
                    if (!(lv & KAD_INM)) continue;
                    const unsigned long long sx = (lv & KAD_OVF2) ? KAD_U64MAX : kad_ld_u64(sl.sigma2 + v);
                    const unsigned long long w = kad_sat_mul(sx, sig_val(lv, s1));
                    const int b = ((unsigned)v >> shift) & 15;
                    const unsigned long long o = atomicAdd(&W.u.bins.lo[b], w);
                    if (o + w < o) atomicAdd(&W.u.bins.hi[b], 1ull);
                }
            }
            __syncwarp();
            // lane b < 16: the running sum through bin b, saturating, in bin order
            unsigned long long bw = 0;
            if (lane < 16) bw = W.u.bins.hi[lane] ? KAD_U64MAX : W.u.bins.lo[lane];
            unsigned long long incl = bw;
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL_MASK, incl, o);
                if (lane >= o) incl = kad_sat_add(y, incl);
            }
            unsigned long long excl = __shfl_up_sync(FULL_MASK, incl, 1);
            if (lane == 0) excl = 0;
            const unsigned long long cum = kad_sat_add(P, incl);
            const unsigned hit = __ballot_sync(FULL_MASK, lane < 16 && cum > r);
            int chosen = hit ? __ffs(hit) - 1 : -1;
            if (chosen < 0) {
                if (lane == 0) kad_set_err(a.ctl, KAD_DERR_SELECT);
                chosen = 0;
            }
            // the running sum before the chosen bin (saturating addition is associative)
            P = shfl64(kad_sat_add(P, excl), chosen);
            prefix |= (unsigned)chosen << shift;
            __syncwarp();
        }
        mid = (int)prefix;
    }
    if (lane == 0) C.mid = mid;
    __syncwarp();
    return sst;
}

// ---------------------------------------------------------------- trace-back
// One trace step at cur (side z, distance d) when level d-1 has lcnt <= W_LCAP
// vertices: each is tested for adjacency to cur by G lanes together (a search
// in the shorter of the two sorted rows, G-1 probes per round when G > 1), and
// the adjacent ones are ranked by id: the same candidates, order and choice as
// scanning adj(cur).  Returns the chosen vertex and its path count to every lane.
__device__ __forceinline__ void w_from_level(const SampleArgs &a, WShared &S, int c, const Slot &sl, int z, int ls,
                                             int lcnt, int cur, int rsC, int reC, unsigned long long r, int &p_sel,
                                             unsigned long long &s_sel, unsigned long long &probes_out) {
    WWarp &W = S.w[c];
    const int lane = threadIdx.x & 31, n = a.n;
    int G = 1;
    while (G < 32 && 2 * G * lcnt <= 32) G *= 2;
    const int P = (G > 1) ? G - 1 : 1;
    const int lgP1 = (G > 1) ? __ffs(G) - 1 : 1; // P + 1 = 2^lgP1
    const int lgG = __ffs(G) - 1;
    const int per = 32 >> lgG, j_sub = lane >> lgG, sub = lane & (G - 1);
    unsigned long long probes = 0;
    for (int base = 0; base < lcnt; base += per) {
        const int j = base + j_sub;
        const bool mine = j < lcnt;
        // p precedes cur on side z when cur is in p's row in side z's
        // direction, equivalently p in cur's trace row [rsC, reC)
        int p = -1, lo = 0, hi = 0, key = 0;
        const int32_t *scol = tcol(a, z);
        if (mine) {
            p = __ldcg(sl.list + phys(z, ls + j, n));
            const int rsP = __ldg(xrp(a, z) + p), reP = __ldg(xrp(a, z) + p + 1);
            if (reP - rsP <= reC - rsC) {
                lo = rsP;
                hi = reP;
                key = cur;
                scol = xcol(a, z);
            } else {
                lo = rsC;
                hi = reC;
                key = p;
            }
        }
        bool done = !mine, found = false;
        while (__any_sync(FULL_MASK, !done)) {
            const int len = hi - lo;
            if (!done && len <= G) {
                found = sub < len && __ldg(scol + lo + sub) == key;
                probes += (sub < len) ? 1 : 0;
                done = true;
            }
            int v = 0, q = 0;
            const bool probe = !done && sub < P;
            if (probe) {
                q = lo + (int)(((long long)len * (sub + 1)) >> lgP1);
                v = __ldg(scol + q);
                probes++;
            }
            int nlo = (probe && v < key) ? q + 1 : -0x7fffffff;
            int nhi = (probe && v > key) ? q : 0x7fffffff;
            int eq = (probe && v == key) ? 1 : 0;
            for (int o = 1; o < G; o <<= 1) {
                nlo = max(nlo, __shfl_xor_sync(FULL_MASK, nlo, o));
                nhi = min(nhi, __shfl_xor_sync(FULL_MASK, nhi, o));
                eq |= __shfl_xor_sync(FULL_MASK, eq, o);
            }
            if (!done) {
                if (eq) {
                    found = true;
                    done = true;
                } else {
                    lo = max(lo, nlo);
                    hi = min(hi, nhi);
                    if (lo >= hi) done = true;
                }
            }
        }
        int f = found ? 1 : 0;
        for (int o = 1; o < G; o <<= 1) f |= __shfl_xor_sync(FULL_MASK, f, o);
        if (mine && sub == 0) {
            W.u.tr.p[j] = f ? p : -1;
            if (f) {
                uint32_t lp;
                unsigned long long sp;
                ld_vs(sl.label, p, lp, sp);
                W.u.tr.s[j] = sig_val(lp, sp);
            }
        }
    }
    __syncwarp();
    int pc[2];
    unsigned long long wc[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int jj = lane + 32 * k;
        pc[k] = (jj < lcnt) ? W.u.tr.p[jj] : -1;
        wc[k] = (pc[k] >= 0) ? W.u.tr.s[jj] : 0ull;
    }
    unsigned long long ex[2] = {0ull, 0ull};
#pragma unroll
    for (int slot = 0; slot < 2; slot++) {
        if (32 * slot >= lcnt) break;
#pragma unroll 4
        for (int q = 0; q < 32; q++) {
            const int pq = __shfl_sync(FULL_MASK, pc[slot], q);
            const unsigned long long wq = shfl64(wc[slot], q);
#pragma unroll
            for (int k = 0; k < 2; k++)
                if (pq >= 0 && pc[k] >= 0 && pq < pc[k]) ex[k] = kad_sat_add(ex[k], wq);
        }
    }
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const bool win = pc[k] >= 0 && ex[k] <= r && kad_sat_add(ex[k], wc[k]) > r;
        const unsigned hitm = __ballot_sync(FULL_MASK, win);
        if (hitm) {
            const int fl = __ffs(hitm) - 1;
            p_sel = __shfl_sync(FULL_MASK, pc[k], fl);
            s_sel = shfl64(wc[k], fl);
        }
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) probes += __shfl_xor_sync(FULL_MASK, probes, o);
    probes_out += probes;
}

// Scan adj(cur) 128 arcs per pass in CSR order: among the neighbours at level
// d-1 of side z, the first whose running sum of sigma exceeds r.
__device__ __forceinline__ void w_trace_scan(const SampleArgs &a, const Slot &sl, int z, int d, int rsC, int reC,
                                             unsigned long long r, int &p_sel, unsigned long long &s_sel,
                                             unsigned long long &w_trace) {
    const int lane = threadIdx.x & 31;
    const uint32_t key = (z ? KAD_SIDE : 0u) | (uint32_t)d; // level d-1
    const bool nobits = a.no_bits != 0;
    const int gs = a.bits_shift;
    const bool direct = nobits || reC - rsC <= 32;
    unsigned long long carry = 0;
    for (int base = rsC; base < reC; base += 128) {
        int pp[4];
        uint32_t lp[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int e = base + 32 * k + lane;
            pp[k] = (e < reC) ? __ldg(tcol(a, z) + e) : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            bool rd = pp[k] >= 0;
            if (rd && !direct) {
                const int b = pp[k] >> gs;
                rd = (sl.bits[b >> 5] >> (b & 31)) & 1u;
            }
            lp[k] = rd ? kad_ld_u32(lab_at(sl.label, pp[k])) : 0u;
        }
        unsigned long long wk[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            wk[k] = 0;
            if (pp[k] >= 0 && (lp[k] & KAD_KEY) == key)
                wk[k] = (lp[k] & KAD_OVF) ? KAD_U64MAX : kad_ld_u64(sig_at(sl.label, pp[k]));
        }
        // the running sums item by item (a loop, so that the scan exists once)
#pragma unroll 1
        for (int k = 0; k < 4; k++) {
            unsigned long long wkk = wk[0];
            int ppk = pp[0];
#pragma unroll
            for (int q = 1; q < 4; q++)
                if (k == q) {
                    wkk = wk[q];
                    ppk = pp[q];
                }
            const unsigned long long incl = warp_incl_sat_scan(wkk);
            const unsigned long long cum = kad_sat_add(carry, incl);
            const unsigned hit = __ballot_sync(FULL_MASK, ppk >= 0 && cum > r);
            if (hit) {
                const int fl = __ffs(hit) - 1;
                p_sel = __shfl_sync(FULL_MASK, ppk, fl);
                s_sel = shfl64(wkk, fl);
                if (lane == 0) w_trace += (unsigned long long)(base + 32 * k + fl - rsC + 1);
                return;
            }
            carry = kad_sat_add(carry, shfl64(incl, 31));
        }
    }
}

// Trace side z of context c's sample from the meeting vertex (distance d, path
// count sc) back to its root (Appendix C.1): per step lane 0 draws
// r = U(sigma(cur)), and the first neighbour at distance d-1 in ascending id
// (CSR) order whose running sum of sigma exceeds r is taken.  Each chosen
// interior vertex goes out at its distance from s.  Returns false on error.
__device__ __noinline__ bool w_trace_side(const SampleArgs &a, WShared &S, int c, const Slot &sl, Stream &st, int z, int d,
                             unsigned long long sc, int cur, int D, int32_t *out) {
    WCtx &C = S.c[c];
    const int lane = threadIdx.x & 31;
    // rows toward root z: in-arcs for s, out-arcs for t
    int rsC = __ldg(trp(a, z) + cur), reC = __ldg(trp(a, z) + cur + 1);
    unsigned long long wtr = 0;
    while (d >= 1) {
        unsigned long long r = 0;
        if (lane == 0) r = st.uniform(sc, a.ctl);
        r = shfl64(r, 0);
        int p_sel = -1;
        unsigned long long s_sel = 0;
        const int ls = (d <= KAD_MAXLV) ? C.lvs[z][d - 1] : 0;
        const int lcnt = (d <= KAD_MAXLV) ? C.lvs[z][d] - ls : W_LCAP + 1;
        if (d == 1) {
            p_sel = z ? C.t : C.s;
            s_sel = 1ull;
        } else if (!(a.debug & KAD_DEBUG_TRACE_SCAN) && reC - rsC > W_DEG_SCAN && lcnt <= W_LCAP) {
            w_from_level(a, S, c, sl, z, ls, lcnt, cur, rsC, reC, r, p_sel, s_sel, wtr);
        } else {
            w_trace_scan(a, sl, z, d, rsC, reC, r, p_sel, s_sel, wtr);
        }
        if (p_sel < 0) {
            if (lane == 0) kad_set_err(a.ctl, KAD_DERR_TRACE);
            return false;
        }
        d--;
        if (d >= 1 && lane == 0) emit(a, out, D, (z == 0) ? d : D - d, p_sel);
        cur = p_sel;
        sc = s_sel;
        rsC = __ldg(trp(a, z) + cur);
        reC = __ldg(trp(a, z) + cur + 1);
    }
    if (lane == 0) C.acc[4] += wtr;
    return true;
}

// ---------------------------------------------------------------- closer
__device__ __noinline__ void w_close_epoch(const SampleArgs &a, unsigned long long k) {
    const int lane = threadIdx.x & 31;
    const size_t rb = (size_t)(k % a.ring) * a.epoch;
    unsigned long long ovf = 0;
    for (uint32_t j = lane; j < a.epoch; j += 32) {
        const size_t row = rb + j;
        const int len = __ldcg(a.plen + row);
        if (__ldcg(a.pflag + row)) ovf++;
        const int32_t *pr = a.paths + row * (size_t)a.cap;
        int t = 0;
        for (; t + 4 <= len; t += 4) {
            int v[4];
            unsigned int cv[4];
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] = __ldcg(pr + t + q);
#pragma unroll
            for (int q = 0; q < 4; q++) cv[q] = atomicAdd(a.cnt + v[q], 1u) + 1u;
#pragma unroll
            for (int q = 0; q < 4; q++) atomicMax(a.classmax + __ldcg(a.c0 + v[q]), (int)cv[q]);
        }
        for (; t < len; t++) {
            const int v = __ldcg(pr + t);
            const unsigned int cv = atomicAdd(a.cnt + v, 1u) + 1u;
            atomicMax(a.classmax + __ldcg(a.c0 + v), (int)cv);
        }
    }
    ovf = warp_sum_u64(ovf);
    __threadfence();
    __syncwarp();
    const unsigned long long tau = (k + 1) * (unsigned long long)a.epoch;
    int pass = 1;
    if (tau < a.omega) {
        // Appendix B, per calibration class: f and g are non-decreasing in the
        // count for a fixed L, so the class's largest count decides for it
        for (int j = lane; j < a.nclass; j += 32) {
            const int cm = __ldcg(a.classmax + j);
            if (cm >= 0) {
                const double L = __ldcg(a.ltab + j);
                const double f = kad_fg_dev((unsigned long long)cm, L, tau, a.omega, false);
                const double g = kad_fg_dev((unsigned long long)cm, L, tau, a.omega, true);
                if (!(f <= a.eps && g <= a.eps)) pass = 0;
            }
        }
    }
    const int all = __all_sync(FULL_MASK, pass);
    if (lane == 0) {
        if (a.ctl->t_first_close == 0) a.ctl->t_first_close = global_ns();
        a.ctl->overflow += ovf;
        a.epoch_done[k % a.ring] = 0;
        const bool cut = a.max_epochs && k + 1 >= a.max_epochs;
        if (tau >= a.omega || all || cut) {
            a.ctl->tau = tau;
            a.ctl->stopped_by_omega = (tau >= a.omega) ? 1 : (all ? 0 : 2);
            a.ctl->t_stop = global_ns();
            a.ctl->issued_at_stop = *(volatile unsigned long long *)&a.ctl->next;
            __threadfence();
            *(volatile int *)&a.ctl->stop = 1;
        }
        __threadfence();
        *(volatile unsigned long long *)&a.ctl->closed = k + 1;
        __threadfence();
    }
    __syncwarp();
}

// The closer role, held by at most one warp (same protocol as the block kernel).
__device__ __noinline__ void w_run_closer(const SampleArgs &a) {
    const int lane = threadIdx.x & 31;
    bool holding = false;
    if (lane == 0) holding = (atomicCAS(&a.ctl->closer, 0, 1) == 0);
    for (;;) {
        int action = 0;
        unsigned long long k = 0;
        if (lane == 0) {
            for (int guard = 0; holding && guard < 4; guard++) {
                kad_fence_sc();
                k = *(volatile unsigned long long *)&a.ctl->closed;
                if (epoch_ready(a, k)) {
                    action = 1;
                    break;
                }
                atomicExch(&a.ctl->closer, 0);
                holding = false;
                kad_fence_sc();
                k = *(volatile unsigned long long *)&a.ctl->closed;
                if (epoch_ready(a, k) && atomicCAS(&a.ctl->closer, 0, 1) == 0) holding = true;
            }
            if (holding && action == 0) {
                atomicExch(&a.ctl->closer, 0);
                holding = false;
            }
        }
        action = __shfl_sync(FULL_MASK, action, 0);
        k = shfl64(k, 0);
        if (!action) break;
        w_close_epoch(a, k);
    }
}

// ---------------------------------------------------------------- one sample
// The owner warp of context c computes samples until none is left.
__device__ void w_owner(const SampleArgs &a, WShared &S, int c) {
    WCtx &C = S.c[c];
    const Slot sl = slot_of(a, c);
    const int lane = threadIdx.x & 31;
    const int32_t n = a.n;
    const bool nobits = a.no_bits != 0;
    const int gs = a.bits_shift;
    const int mcap = (a.mcap < W_MC) ? a.mcap : W_MC;
    const int mext = sl.mext_id ? a.mext : 0;
    for (;;) {
        // ------------------------------------------------ next sample index
        unsigned long long idx = ~0ull;
        int calib = 0;
        uint32_t dom = a.domain;
        if (lane == 0) {
            const bool stopped = (a.mode == KAD_MODE_RING) && (*(volatile int *)&a.ctl->stop != 0);
            const bool failed = *(volatile int *)&a.ctl->err != 0;
            if (!stopped && !failed) {
                const unsigned long long g = atomicAdd(&a.ctl->next, 1ull);
                if (a.mode == KAD_MODE_RECORD) {
                    if (g < a.i1) idx = g;
                } else if (g < a.calib_n) {
                    idx = g;
                    calib = 1;
                    dom = 1;
                } else if (a.i0 + (g - a.calib_n) < a.i1) {
                    idx = a.i0 + (g - a.calib_n);
                    dom = 0;
                }
            }
            C.tmark = clock64();
        }
        idx = shfl64(idx, 0);
        if (idx == ~0ull) break;
        calib = __shfl_sync(FULL_MASK, calib, 0);
        dom = __shfl_sync(FULL_MASK, dom, 0);

        // ------------------------------------------------ pair draw
        Stream st;
        if (lane == 0) {
            st.init(a.key0, a.key1, idx, dom);
            const int s = (int)st.uniform((unsigned long long)n, a.ctl);
            int t = (int)st.uniform((unsigned long long)(n - 1), a.ctl);
            if (t >= s) t++;
            C.idx = idx;
            C.calib = calib;
            C.dom = dom;
            C.watch = (!calib && a.mode == KAD_MODE_RING) ? 1 : 0;
            C.abort = 0;
            C.s = s;
            C.t = t;
            C.tail[0] = C.tail[1] = 0;
            C.D = 0;
            C.mcount = 0;
            C.st_w0 = st.w0;
            C.st_w1 = st.w1;
            C.st_blk = st.blk;
            C.st_pos = st.pos;
            if (__ldg(a.comp + s) == __ldg(a.comp + t)) {
                *(uint4 *)lab_at(sl.label, s) = make_uint4(1u, 0u, 1u, 0u);
                *(uint4 *)lab_at(sl.label, t) = make_uint4(KAD_SIDE | 1u, 0u, 1u, 0u);
                if (!nobits) {
                    atomicOr(sl.bits + ((s >> gs) >> 5), 1u << ((s >> gs) & 31));
                    atomicOr(sl.bits + ((t >> gs) >> 5), 1u << ((t >> gs) & 31));
                }
                sl.list[0] = s;
                sl.list[n - 1] = t;
                C.tail[0] = C.tail[1] = 1;
                C.fb[0] = C.fb[1] = 0;
                C.fe[0] = C.fe[1] = 1;
                C.lev[0] = C.lev[1] = 0;
                C.lvs[0][0] = C.lvs[1][0] = 0;
                C.lvs[0][1] = C.lvs[1][1] = 1;
                // each root's row in its side's direction: out-arcs of s, in-arcs of t
                C.root_rs[0] = __ldg(a.rows[0] + s);
                C.root_rs[1] = __ldg(a.rows[1] + t);
                C.dsum[0] = (unsigned long long)(__ldg(a.rows[0] + s + 1) - C.root_rs[0]);
                C.dsum[1] = (unsigned long long)(__ldg(a.rows[1] + t + 1) - C.root_rs[1]);
                C.D = -1; // searching
            }
            __threadfence_block();
            const long long now = clock64();
            C.acc[8] += (unsigned long long)(now - C.tmark);
            C.tmark = now;
        }
        __syncwarp();

        // ------------------------------------------------ search
        w_search(a, S, c);
        if (lane == 0) {
            const long long now = clock64();
            C.acc[9] += (unsigned long long)(now - C.tmark);
            C.tmark = now;
        }
        const int D = C.D;
        const int X = C.X;

        // ------------------------------------------------ meeting draw
        unsigned long long sst = 0;
        if (lane == 0) {
            st.init(a.key0, a.key1, idx, dom);
            st.w0 = C.st_w0;
            st.w1 = C.st_w1;
            st.blk = C.st_blk;
            st.pos = C.st_pos;
        }
        if (D > 0) sst = w_meeting(a, S, c, st);
        if (lane == 0) {
            const long long now = clock64();
            C.acc[10] += (unsigned long long)(now - C.tmark);
            C.tmark = now;
        }

        // ------------------------------------------------ trace-back + output
        const bool by_completion = a.mode == KAD_MODE_RING && a.fast && !calib;
        size_t row = 0;
        if (a.mode == KAD_MODE_RING)
            row = (size_t)((idx / a.epoch) % a.ring) * a.epoch + (size_t)(idx % a.epoch);
        else if (a.mode == KAD_MODE_RECORD)
            row = (size_t)(idx - a.i0);
        int32_t *const out = calib ? nullptr : (by_completion ? sl.stage : a.paths + row * (size_t)a.cap);
        const int mid = C.mid;
        const bool traced = D > 0 && mid >= 0 && mid < n;
        if (D > 0 && !traced && lane == 0) kad_set_err(a.ctl, KAD_DERR_SELECT);
        if (traced) {
            uint32_t lm;
            unsigned long long sm1;
            const unsigned long long sm2 = kad_ld_u64(sl.sigma2 + mid);
            ld_vs(sl.label, mid, lm, sm1);
            const int dX = C.lev[X] + 1, dY = C.lev[1 - X];
            const unsigned long long gX = (lm & KAD_OVF2) ? KAD_U64MAX : sm2;
            const unsigned long long gY = sig_val(lm, sm1);
            const int d0 = (X == 0) ? dX : dY, d1 = (X == 1) ? dX : dY;
            const unsigned long long g0 = (X == 0) ? gX : gY, g1 = (X == 1) ? gX : gY;
            if (lane == 0) emit(a, out, D, d0, mid);
            // the s side first, then the t side, from one stream (as the oracle)
            if (w_trace_side(a, S, c, sl, st, 0, d0, g0, mid, D, out))
                w_trace_side(a, S, c, sl, st, 1, d1, g1, mid, D, out);
        }
        __syncwarp();
        unsigned long long pos = idx;
        if (by_completion) {
            if (lane == 0) pos = atomicAdd(&a.ctl->qnext, 1ull);
            pos = shfl64(pos, 0);
            row = (size_t)((pos / a.epoch) % a.ring) * a.epoch + (size_t)(pos % a.epoch);
            const int len = (D > 0) ? min(D - 1, a.cap) : 0;
            __threadfence_block();
            for (int j = lane; j < len; j += 32) a.paths[row * (size_t)a.cap + j] = __ldcg(out + j);
            if (lane == 0 && pos < a.pidx_cap) a.pidx[pos] = idx;
        }
        if (lane == 0) {
            const int inc = (D > 0) ? D - 1 : 0;
            C.acc[5] += (unsigned long long)inc;
            C.acc[6]++;
            if (!calib) {
                a.plen[row] = (inc <= a.cap) ? inc : a.cap;
                a.pflag[row] = (sst == KAD_U64MAX) ? 1 : 0;
            }
            if (a.mode == KAD_MODE_RECORD) {
                a.rec_s[row] = C.s;
                a.rec_t[row] = C.t;
                a.rec_D[row] = D;
                a.rec_sst[row] = sst;
            }
            const long long now = clock64();
            C.acc[11] += (unsigned long long)(now - C.tmark);
            C.tmark = now;
        }
        __syncwarp();

        // ------------------------------------------------ reset the slot
        {
            const int t0 = min(C.tail[0], n), t1 = min(C.tail[1], n - t0);
            const int tot = t0 + t1;
            for (int j0 = lane; j0 < tot; j0 += 32 * 8) {
                int vr[8];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int j = j0 + 32 * k;
                    vr[k] = (j < tot) ? __ldcg(sl.list + ((j < t0) ? j : n - 1 - (j - t0))) : -1;
                }
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    if (vr[k] < 0) continue;
                    *(uint4 *)lab_at(sl.label, vr[k]) = make_uint4(0u, 0u, 0u, 0u);
                    if (!nobits) sl.bits[(vr[k] >> gs) >> 5] = 0u;
                }
            }
            if (D > 0 || C.abort) {
                const int mc = C.mcount;
                if (mc <= mcap + mext) {
                    for (int i = lane; i < mc; i += 32)
                        sl.sigma2[(i < mcap) ? C.m_id[i] : __ldcg(sl.mext_id + (i - mcap))] = 0ull;
                } else {
                    const int Y = 1 - X;
                    for (int j = C.fb[Y] + lane; j < C.fe[Y]; j += 32) sl.sigma2[__ldcg(sl.list + phys(Y, j, n))] = 0ull;
                }
            }
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) {
            const long long now = clock64();
            C.acc[12] += (unsigned long long)(now - C.tmark);
            C.tmark = now;
        }

        // ------------------------------------------------ epoch bookkeeping
        if (a.mode == KAD_MODE_RING && calib) {
            int publish = 0;
            if (lane == 0) {
                __threadfence();
                const unsigned long long done = atomicAdd(&a.ctl->calib_done, 1ull) + 1ull;
                __threadfence();
                publish = (done == a.calib_n) ? 1 : 0;
            }
            publish = __shfl_sync(FULL_MASK, publish, 0);
            if (publish) {
                for (int q = lane; q < a.nclass; q += 32) a.hpage->hist[q] = __ldcg(a.hist + q);
                __threadfence_system();
                __syncwarp();
                if (lane == 0) {
                    a.ctl->t_calib = global_ns();
                    *(volatile int *)&a.hpage->calib_flag = 1;
                    __threadfence_system();
                }
            }
        } else if (a.mode == KAD_MODE_RING) {
            int tc = 0;
            if (lane == 0) {
                const unsigned long long e = pos / a.epoch;
                const unsigned int old = atom_add_release(&a.epoch_done[e % a.ring], 1u);
                if (old + 1u == a.epoch) {
                    kad_fence_sc();
                    tc = 1;
                }
            }
            tc = __shfl_sync(FULL_MASK, tc, 0);
            if (tc) w_run_closer(a);
        }
        if (lane == 0) {
            const long long now = clock64();
            C.acc[13] += (unsigned long long)(now - C.tmark);
            C.tmark = now;
        }
    }
}

// A warp with no sample of its own (or whose samples are done) helps the
// block's jobs until every owner has finished.
__device__ void w_helper(const SampleArgs &a, WShared &S, int me) {
    unsigned long long deadline = 0;
    int last_active = -1;
    for (;;) {
        if (w_help_any(a, S, me)) {
            deadline = 0;
            continue;
        }
        const int act = vload(S.active);
        if (act == 0 && vload(S.arcmask) == 0u && vload(S.ctxmask) == 0u) break;
        if (act != last_active) {
            last_active = act;
            deadline = 0;
        }
        if (*(volatile int *)&a.ctl->err) break;
        if (wait_expired(deadline, a)) break;
        __nanosleep(64);
    }
}

__global__ void __launch_bounds__(W_THREADS, 1) k_wsample(const SampleArgs a) {
    __shared__ WShared S;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int nctx = a.nctx;
    if (!a.no_bits)
        for (int q = tid; q < nctx * a.nw; q += W_THREADS) w_bits_dyn[q] = 0u;
    if (tid == 0) {
        S.arcmask = 0u;
        S.ctxmask = 0u;
        S.active = nctx;
    }
    if (lane == 0) {
        S.w[wid].inflight = 0;
        S.w[wid].next = 0;
        S.c[wid].inflight = 0;
        S.c[wid].jnext = 0;
        S.c[wid].jend = 0;
    }
    if (lane < KAD_WORK_WORDS) S.c[wid].acc[lane] = 0;
    if (lane == 0) {
        S.c[wid].probe_score = 4;
        S.c[wid].probe_rounds = 0;
    }
    if (tid == 0 && a.mode == KAD_MODE_RING) atomicCAS(&a.ctl->t_start, 0ull, global_ns());
    __syncthreads();
    // a launch that continues a run first closes what an earlier launch completed
    if (a.mode == KAD_MODE_RING && blockIdx.x == 0 && wid == 0) w_run_closer(a);
    if (wid < nctx) {
        w_owner(a, S, wid);
        __syncwarp();
        if (lane == 0) {
            for (int i = 0; i < KAD_WORK_WORDS; i++)
                if (S.c[wid].acc[i]) atomicAdd(a.work + i, S.c[wid].acc[i]);
            __threadfence_block();
            atomicSub(&S.active, 1);
        }
    }
    __syncwarp();
    w_helper(a, S, wid);
    if (tid == 0 && a.mode == KAD_MODE_RING) atomicMax(&a.ctl->t_end, global_ns());
}

} // namespace

// ---------------------------------------------------------------- launchers
#if KAD_DIRECTED
cudaError_t kad_launch_wsample_directed(const SampleArgs &a, int blocks, size_t dyn_smem, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
#else
size_t kad_wsample_static_smem() { return sizeof(WShared); }

cudaError_t kad_launch_wsample(const SampleArgs &a, int blocks, size_t dyn_smem, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (a.rows[1] != a.rows[0]) return kad_launch_wsample_directed(a, blocks, dyn_smem, st);
#endif
    if (a.nctx < 1 || a.nctx > W_WARPS) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_wsample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
    if (e != cudaSuccess) return e;
    k_wsample<<<blocks, W_THREADS, dyn_smem, st>>>(a);
    return cudaGetLastError();
}

#if !KAD_DIRECTED

int kad_wsample_max_blocks_per_sm(size_t dyn_smem) {
    int nb = 0;
    if (cudaFuncSetAttribute(k_wsample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_wsample, W_THREADS, dyn_smem) != cudaSuccess) return 0;
    return nb;
}
#endif // !KAD_DIRECTED
