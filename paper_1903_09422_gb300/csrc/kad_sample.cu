// The KADABRA sampling kernel and the per-epoch fold/stop check (sm_103a).
//
// One resident thread block owns one sampling slot and computes samples one
// after another; sample indices are handed out by a device counter, and every
// random number of sample i comes from Philox4x32-10 keyed by the run's seed at
// counter (i, block, phase), so the result of a sample depends only on i.
//
// Per sample (Section 2.3 sample(), Appendix C.1):
//   1. pair draw: s = U(n), t = U(n-1) (+1 if >= s), uniform over ordered pairs;
//   2. same-component check (Appendix C.1);
//   3. balanced bidirectional BFS with shortest-path counts sigma (uint64,
//      saturating): each round expands the side whose frontier has the smaller
//      degree sum (s on ties); the round that reaches the other side's frontier
//      collects the meeting set M and the expanding side's counts at M;
//   4. meeting draw: w in M with probability sigma_X(w) sigma_Y(w) / sigma_st,
//      M walked in ascending vertex id (M is recorded during the search: a
//      rank selection for up to 256 members, else digit-wise selection);
//   5. trace-back from w to s, then to t, rebuilt from G and the per-vertex
//      level labels (no predecessor graph, Appendix C.1); the two sides are
//      traced at once by the two halves of the block, the t side's draws taken
//      from where the s side's end;
//   6. output of the D-1 interior vertices.
// A sample's labels and counts (one 16-byte record per vertex) and frontier
// lists live in global scratch of its slot and are cleared by walking the list
// of labelled vertices, so no Theta(n) reset is needed (the purpose of Appendix
// C.1's timestamps).  Once the run has stopped, a sample in flight gives up.
//
// Epochs (Algorithm 2's consistency requirement, Section 3.1, with the fixed
// sample-to-frame assignment of the indexed-frame algorithm, Appendix D.2):
// epoch k is the index range [kN, (k+1)N).  The block that completes the last
// sample of an epoch takes the closer role if free; the closer folds complete
// epochs strictly in index order into the counts (the associative operation of
// Algorithm 1 is integer addition) and evaluates the stop rule of Appendix B on
// the state after each epoch, so every check sees an integral prefix of samples.
// In completion order (the non-deterministic local-/shared-frame behaviour of
// Section 3.2) epoch k holds the (kN+1)-th to (k+1)N-th samples to complete
// instead: a sample takes its fold position once its path is complete.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "kad_device.cuh"

#define KAD_MCAP_MAX 256
#define KAD_ITEMS 4     // arcs per thread per expansion pass
#define KAD_PITEMS 8    // arcs per thread per probe pass
#define KAD_LCAP 64     // largest predecessor level searched from its list
#define KAD_DEG_SCAN 64 // adjacency lists up to this length are always scanned
#define KAD_PAIR_MIN_ARCS 1024 // rounds with fewer arcs always expand by scanning
#define KAD_WARP_SCAN 256       // adjacency lists up to this length are traced by one warp
#define KAD_TITEMS 2            // consecutive arcs per thread and pass of a team's adjacency scan
#define KAD_TBUF 64            // t-side trace steps team 1 can buffer (longer: team 0 traces both sides)

namespace {


// ---------------------------------------------------------------- block helpers
template <int BLOCK>
struct Smem {
    int32_t uid[BLOCK];
    int32_t rs[BLOCK];
    int32_t off[BLOCK];
    unsigned long long sig[BLOCK];
    int32_t m_id[KAD_MCAP_MAX];
    unsigned long long m_w[KAD_MCAP_MAX];
    int32_t wtmp[BLOCK / 32];
    unsigned long long wtmp64[BLOCK / 32];
    unsigned long long bin_lo[16], bin_hi[16];
    int tail[2], fb[2], fe[2], lev[2];
    int root_rs[2];
    int lvs[2][KAD_MAXLV + 2]; // logical list start of level l, l <= KAD_MAXLV + 1
    unsigned long long dsum[2];
    // per round r, slot r & 1: the next frontier's degree sum and the meeting
    // flag (two slots, so the next round's are cleared while this round's are read)
    unsigned long long next_dsum[2];
    volatile int met[2];
    int abort; // the run stopped while this (adaptive) sample was in its BFS
    // probe-first policy of this block: > 0 while probed rounds usually met;
    // large rounds counted, so that every 16th is probed whatever the score
    int probe_score, probe_rounds;
    int chunk_total; // arcs of a one-vertex chunk
    int mcount;    // members of M recorded (the first m_cap ids are in m_id)
    int mid;
    int D;
    int s, t;
    int try_close;
    int action;
    int calib; // the current sample is a calibration sample
    int publish;
    uint32_t dom;
    unsigned int prefix;
    unsigned long long P;
    unsigned long long r;
    // the stream after the meeting draw (for the t-side trace of team 1), the
    // stream positions that must agree, and team 1's buffered t-side vertices
    unsigned long long st_w0, st_w1;
    uint32_t st_blk;
    int st_pos;
    uint32_t st_end_blk, st_spec_blk;
    int st_end_pos, st_spec_pos;
    int tcount;
    unsigned long long wt1;
    // trace teams (team t = threads [t*BLOCK/2, (t+1)*BLOCK/2)): the step's random
    // number, per-warp partial sums, the first crossing position (two slots, by
    // pass parity) and the chosen predecessor with its row
    unsigned long long t_r[2];
    unsigned long long t_wsum[2][BLOCK / 64];
    int t_min[2][2];
    int t_p[2], t_rs[2], t_re[2];
    unsigned long long t_s[2];
    int32_t c_p[2][KAD_LCAP];           // predecessor candidates of a team step (-1: not adjacent)
    unsigned long long c_s[2][KAD_LCAP];
    int32_t tbuf_v[KAD_TBUF], tbuf_j[KAD_TBUF];
    unsigned long long sst;
    unsigned long long idx;
    unsigned long long qpos; // completion order: the sample's fold position
    unsigned long long k;
    unsigned long long ovf_acc;
    unsigned long long acc[KAD_WORK_WORDS];
    long long tmark;
    // the next sample's pair, drawn ahead by warp 1 while warp 0 draws a small
    // meeting set: the raw index, s and t, whether they share a component, the
    // bounds of their rows, and the stream after the two draws (pre_ok: set;
    // pre_use: the next sample is that index)
    unsigned long long pre_g, pre_w0, pre_w1;
    uint32_t pre_blk;
    int pre_pos, pre_ok, pre_use, pre_s, pre_t, pre_same;
    int pre_rs[2], pre_re[2];
};

// The sample a raw index g of the launch's counter stands for (~0: none):
// calibration samples first, then adaptive ones (RING); [i0, i1) in RECORD mode.
__device__ __forceinline__ unsigned long long sample_of(const SampleArgs &a, unsigned long long g, int &calib,
                                                        uint32_t &dom) {
    calib = 0;
    dom = a.domain;
    if (a.mode == KAD_MODE_RECORD) return (g < a.i1) ? g : ~0ull;
    if (g < a.calib_n) {
        calib = 1;
        dom = 1;
        return g;
    }
    dom = 0;
    return (a.i0 + (g - a.calib_n) < a.i1) ? a.i0 + (g - a.calib_n) : ~0ull;
}

// One thread draws the pair of the sample after this one (the same draws, in
// the same stream, as the pair draw at the start of a sample) and leaves it in
// shared memory with the loads the start of the sample needs.
template <int BLOCK>
__device__ __noinline__ void draw_ahead(const SampleArgs &a, Smem<BLOCK> &sm) {
    const int32_t n = a.n;
    const unsigned long long g = atomicAdd(&a.ctl->next, 1ull);
    int calib;
    uint32_t dom;
    const unsigned long long idx = sample_of(a, g, calib, dom);
    sm.pre_g = g;
    if (idx != ~0ull) {
        Stream ps;
        ps.init(a.key0, a.key1, idx, dom);
        const int s = (int)ps.uniform((unsigned long long)n, a.ctl);
        int t = (int)ps.uniform((unsigned long long)(n - 1), a.ctl);
        if (t >= s) t++;
        const int cs = __ldg(a.comp + s), ct = __ldg(a.comp + t);
        const int r0 = __ldg(a.rows[0] + s), r0e = __ldg(a.rows[0] + s + 1);
        const int r1 = __ldg(a.rows[1] + t), r1e = __ldg(a.rows[1] + t + 1);
        sm.pre_s = s;
        sm.pre_t = t;
        sm.pre_blk = ps.blk;
        sm.pre_pos = ps.pos;
        sm.pre_w0 = ps.w0;
        sm.pre_w1 = ps.w1;
        sm.pre_same = (cs == ct) ? 1 : 0;
        sm.pre_rs[0] = r0;
        sm.pre_re[0] = r0e;
        sm.pre_rs[1] = r1;
        sm.pre_re[1] = r1e;
    }
    sm.pre_ok = 1;
}

template <int BLOCK>
__device__ __forceinline__ int block_excl_scan(int v, int *wtmp, int &total) {
    // one barrier: every thread adds up the warp totals it needs (wtmp is not
    // written again before the caller's next barrier)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtmp[wid] = x;
    __syncthreads();
    int pre = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < BLOCK / 32; w++) {
        const int t = wtmp[w];
        pre += (w < wid) ? t : 0;
        tot += t;
    }
    total = tot;
    return pre + x - v;
}

// Saturating sum over the block (saturating addition is associative and
// commutative on [0, 2^64-1], so any order gives min(exact sum, 2^64-1)).
template <int BLOCK>
__device__ __forceinline__ unsigned long long block_sat_sum(unsigned long long v, unsigned long long *tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = kad_sat_add(v, __shfl_xor_sync(FULL_MASK, v, o));
    if (lane == 0) tmp[wid] = v;
    __syncthreads();
    unsigned long long r = 0;
#pragma unroll
    for (int i = 0; i < BLOCK / 32; i++) r = kad_sat_add(r, tmp[i]);
    __syncthreads();
    return r;
}


// The labelled-vertex bitmap of a slot lives in the block's dynamic shared
// memory when it fits (every check then costs a shared-memory read), else in
// global memory (read through L2).
extern __shared__ uint32_t kad_dyn_bits[];

__device__ __forceinline__ uint32_t bits_ld(bool sh, const uint32_t *g, int w) {
    return sh ? kad_dyn_bits[w] : __ldcg(g + w);
}
// b is a bit index: vertex v >> shift (one bit per 2^shift consecutive vertices;
// a set bit means that some vertex of the group may be labelled)
__device__ __forceinline__ void bits_set(bool sh, uint32_t *g, int b) {
    if (sh)
        atomicOr(kad_dyn_bits + (b >> 5), 1u << (b & 31));
    else
        atomicOr(g + (b >> 5), 1u << (b & 31));
}
__device__ __forceinline__ void bits_clear_word(bool sh, uint32_t *g, int w) {
    if (sh)
        kad_dyn_bits[w] = 0u;
    else
        g[w] = 0u;
}


// ---------------------------------------------------------------- trace-back
// One trace-back step at `cur` (on side z, distance d): among the neighbours p
// at distance d-1, in ascending id (CSR) order, pick the first whose running
// sum of sigma(p) exceeds r (Appendix C.1: the path is rebuilt from G and the
// distance labels).  Called by one warp; every lane returns the same choice.

// Scan adj(cur) 4 x 32 arcs per pass (all loads of a pass issued first).  Rows
// of up to 32 arcs read the labels directly; longer rows filter through the
// bitmap first.  The chosen predecessor's row bounds are fetched together with
// its path count, ready for the next step.
__device__ __forceinline__ void trace_scan(const SampleArgs &a, const uint32_t *label, bool bsh, bool nobits,
                                           int gs, const uint32_t *bits,
                                           int z, int d, int rsC, int reC,
                                           unsigned long long r, int &p_sel, unsigned long long &s_sel, int &rs_sel,
                                           int &re_sel, unsigned long long &w_trace) {
    const int lane = threadIdx.x & 31;
    const uint32_t key = (z ? KAD_SIDE : 0u) | (uint32_t)d; // level d-1
    const bool direct = nobits || reC - rsC <= 32;
    const int32_t *trow = trp(a, z), *tc = tcol(a, z);
    unsigned long long carry = 0;
    for (int base = rsC; base < reC; base += 128) {
        int pp[4];
        uint32_t lp[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int e = base + 32 * k + lane;
            pp[k] = (e < reC) ? __ldg(tc + e) : -1;
        }
        if (direct) {
#pragma unroll
            for (int k = 0; k < 4; k++) lp[k] = (pp[k] >= 0) ? kad_ld_u32(lab_at(label, pp[k])) : 0u;
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) lp[k] = (pp[k] >= 0) ? bits_ld(bsh, bits, (pp[k] >> gs) >> 5) : 0u;
#pragma unroll
            for (int k = 0; k < 4; k++)
                lp[k] = (pp[k] >= 0 && ((lp[k] >> ((pp[k] >> gs) & 31)) & 1u)) ? kad_ld_u32(lab_at(label, pp[k])) : 0u;
        }
        unsigned long long wk[4];
        int rk[4], ek[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            wk[k] = 0;
            rk[k] = ek[k] = 0;
            if (pp[k] >= 0 && (lp[k] & KAD_KEY) == key) {
                wk[k] = (lp[k] & KAD_OVF) ? KAD_U64MAX : kad_ld_u64(sig_at(label, pp[k]));
                rk[k] = __ldg(trow + pp[k]);
                ek[k] = __ldg(trow + pp[k] + 1);
            }
        }
        // the running sums item by item (a loop, so that the scan exists once)
#pragma unroll 1
        for (int k = 0; k < 4; k++) {
            unsigned long long wkk = wk[0];
            int ppk = pp[0], rkk = rk[0], ekk = ek[0];
#pragma unroll
            for (int q = 1; q < 4; q++)
                if (k == q) {
                    wkk = wk[q];
                    ppk = pp[q];
                    rkk = rk[q];
                    ekk = ek[q];
                }
            const unsigned long long incl = warp_incl_sat_scan(wkk);
            const unsigned long long cum = kad_sat_add(carry, incl);
            const unsigned hit = __ballot_sync(FULL_MASK, ppk >= 0 && cum > r);
            if (hit) {
                const int fl = __ffs(hit) - 1;
                p_sel = __shfl_sync(FULL_MASK, ppk, fl);
                s_sel = __shfl_sync(FULL_MASK, wkk, fl);
                rs_sel = __shfl_sync(FULL_MASK, rkk, fl);
                re_sel = __shfl_sync(FULL_MASK, ekk, fl);
                if (lane == 0) w_trace += (unsigned long long)(base + 32 * k + fl - rsC + 1);
                return;
            }
            carry = kad_sat_add(carry, __shfl_sync(FULL_MASK, incl, 31));
        }
    }
}

// Barrier of one trace team (named barrier t+1 over the team's BLOCK/2 threads).
__device__ __forceinline__ void team_bar(int t, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(t + 1), "r"(nthreads) : "memory");
}

// A trace step at `cur` (side z, distance d) when level d-1 has lcnt <= KAD_LCAP
// vertices: each of them is tested for adjacency to cur by G = BLOCK/128 threads
// of the team together (a search in the shorter of the two sorted rows with
// P = max(G-1, 1) probes per round, splitting the range into P+1 parts), the
// adjacent ones with their path counts go to shared memory, and the team's first
// warp selects among them in ascending id order: the same candidates, order and
// choice as scanning adj(cur).  Every thread of the team calls it; the choice is
// returned to the first warp.  The probes are counted into the trace counter.
template <int BLOCK>
__device__ __forceinline__ void team_from_level(const SampleArgs &a, Smem<BLOCK> &sm, int t, const uint32_t *label,
                                                const int32_t *list, int n, int z,
                                                int ls, int lcnt, int cur, int rsC, int reC, unsigned long long r,
                                                int &p_sel, unsigned long long &s_sel) {
    constexpr int TT = BLOCK / 2;
    constexpr int G = (TT / KAD_LCAP >= 2) ? TT / KAD_LCAP : 1; // threads per candidate (a power of two)
    constexpr int P = (G > 1) ? G - 1 : 1;                       // probes per round
    const int tl = (int)threadIdx.x - t * TT;
    const int lane = threadIdx.x & 31, tw = tl >> 5;
    const int j = tl / G, sub = tl % G;
    const bool mine = j < lcnt;
    // p precedes cur on side z when cur is in p's expansion row (side z's
    // direction), equivalently p in cur's trace row [rsC, reC): search the shorter
    int p = -1, lo = 0, hi = 0, key = 0;
    const int32_t *scol = tcol(a, z);
    if (mine) {
        p = __ldcg(list + phys(z, ls + j, n));
        const int32_t *xr = xrp(a, z);
        const int rsP = __ldg(xr + p), reP = __ldg(xr + p + 1);
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
    int probes = 0;
    while (__any_sync(FULL_MASK, !done)) {
        const int len = hi - lo;
        if (!done && len <= G) {
            // the last few positions: one per thread of the group
            found = sub < len && __ldg(scol + lo + sub) == key;
            probes += (sub < len) ? 1 : 0;
            done = true;
        }
        // the group's P probes split [lo, hi) into P+1 parts; every probe lies
        // inside the range, so each round shrinks it or finds the key
        int v = 0, q = 0;
        const bool probe = !done && sub < P;
        if (probe) {
            q = lo + (int)(((long long)len * (sub + 1)) / (P + 1));
            v = __ldg(scol + q);
            probes++;
        }
        int nlo = (probe && v < key) ? q + 1 : -0x7fffffff;
        int nhi = (probe && v > key) ? q : 0x7fffffff;
        int eq = (probe && v == key) ? 1 : 0;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            nlo = max(nlo, __shfl_xor_sync(FULL_MASK, nlo, o, G));
            nhi = min(nhi, __shfl_xor_sync(FULL_MASK, nhi, o, G));
            eq |= __shfl_xor_sync(FULL_MASK, eq, o, G);
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
    // the group's result (found by any of its threads)
    int f = found ? 1 : 0;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) f |= __shfl_xor_sync(FULL_MASK, f, o, G);
    if (mine && sub == 0) {
        sm.c_p[t][j] = f ? p : -1;
        if (f) {
            uint32_t lp;
            unsigned long long sp;
            ld_vs(label, p, lp, sp);
            sm.c_s[t][j] = sig_val(lp, sp);
        }
    }
    unsigned long long pr = probes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pr += __shfl_xor_sync(FULL_MASK, pr, o);
    if (lane == 0 && pr) atomicAdd(&sm.acc[4], pr);
    team_bar(t, TT);
    if (tw == 0) {
        int pc[2];
        unsigned long long wc[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int jj = lane + 32 * k;
            pc[k] = (jj < lcnt) ? sm.c_p[t][jj] : -1;
            wc[k] = (pc[k] >= 0) ? sm.c_s[t][jj] : 0ull;
        }
        // exclusive prefix of each candidate in id order
        unsigned long long ex[2] = {0ull, 0ull};
#pragma unroll
        for (int slot = 0; slot < 2; slot++) {
#pragma unroll 4
            for (int qq = 0; qq < 32; qq++) {
                const int pq = __shfl_sync(FULL_MASK, pc[slot], qq);
                const unsigned long long wq = __shfl_sync(FULL_MASK, wc[slot], qq);
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
                s_sel = __shfl_sync(FULL_MASK, wc[k], fl);
            }
        }
    }
}

// Trace one side z of the sample from the meeting vertex `cur` (distance d,
// path count sc) back to its root with team t (half of the
// block).  Per step the team leader draws a bounded number from the stream (its
// copy of it); each chosen vertex goes out directly (buf_v == nullptr) or into
// buf_v/buf_j for later.  The candidates of a step are the neighbours of cur at
// distance d-1, in ascending id (CSR) order, and the first whose running sum of
// sigma exceeds the draw is chosen (Appendix C.1: the path is rebuilt from G
// and the distance labels).  A short adjacency list is scanned by the team's
// first warp, a long one by the whole team (KAD_TITEMS consecutive arcs per
// thread and pass).  Called by every thread of the team; returns the number of
// buffered vertices, or -1 on error.
template <int BLOCK>
__device__ __forceinline__ int trace_side_team(const SampleArgs &a, Smem<BLOCK> &sm, Stream &st, int t,
                                               const uint32_t *label, bool bsh, bool nobits, int gs, const uint32_t *bits,
                                               const int32_t *list, int n, int z, int d,
                                               unsigned long long sc, int cur, int D, int32_t *out,
                                               int32_t *buf_v, int32_t *buf_j, unsigned long long &w_trace) {
    constexpr int TT = BLOCK / 2, TW = TT / 32;
    const int tl = (int)threadIdx.x - t * TT;
    const int lane = threadIdx.x & 31, tw = tl >> 5;
    const bool leader = tl == 0;
    // cur's row toward root z: its in-arcs on the s side, its out-arcs on the t side
    int rsC = __ldg(trp(a, z) + cur), reC = __ldg(trp(a, z) + cur + 1);
    int nb = 0, par = 0;
    while (d >= 1) {
        if (d == 1) {
            // The only vertex at distance 0 is the root.  Its draw, U(1), takes
            // exactly one word of the stream and cannot be rejected: the leader
            // just consumes the word, and the team needs no barrier.
            if (leader) st.next();
            break;
        }
        if (leader) sm.t_r[t] = st.uniform(sc, a.ctl);
        team_bar(t, TT);
        const unsigned long long r = sm.t_r[t];
        int p_sel = -1, rs_sel = 0, re_sel = 0;
        unsigned long long s_sel = 0;
        const int ls = (d <= KAD_MAXLV) ? sm.lvs[z][d - 1] : 0;
        const int lcnt = (d <= KAD_MAXLV) ? sm.lvs[z][d] - ls : KAD_LCAP + 1;
        if (!(a.debug & KAD_DEBUG_TRACE_SCAN) && reC - rsC > KAD_DEG_SCAN && lcnt <= KAD_LCAP) {
            // few vertices at distance d-1: the team tests each of them for
            // adjacency to cur
            team_from_level<BLOCK>(a, sm, t, label, list, n, z, ls, lcnt, cur, rsC, reC, r, p_sel, s_sel);
            if (tw == 0) {
                if (lane == 0) {
                    sm.t_p[t] = p_sel;
                    sm.t_s[t] = s_sel;
                    sm.t_rs[t] = (p_sel >= 0) ? __ldg(trp(a, z) + p_sel) : 0;
                    sm.t_re[t] = (p_sel >= 0) ? __ldg(trp(a, z) + p_sel + 1) : 0;
                }
            }
            team_bar(t, TT);
            p_sel = sm.t_p[t];
            s_sel = sm.t_s[t];
            rs_sel = sm.t_rs[t];
            re_sel = sm.t_re[t];
        } else if (reC - rsC <= KAD_WARP_SCAN) {
            // a short row: the team's first warp scans it
            if (tw == 0) {
                trace_scan(a, label, bsh, nobits, gs, bits, z, d, rsC, reC, r, p_sel, s_sel, rs_sel, re_sel, w_trace);
                if (lane == 0) {
                    sm.t_p[t] = p_sel;
                    sm.t_s[t] = s_sel;
                    sm.t_rs[t] = rs_sel;
                    sm.t_re[t] = re_sel;
                }
            }
            team_bar(t, TT);
            p_sel = sm.t_p[t];
            s_sel = sm.t_s[t];
            rs_sel = sm.t_rs[t];
            re_sel = sm.t_re[t];
        } else {
            // scan adj(cur): thread tl takes KAD_TITEMS consecutive arcs of each pass;
            // only vertices at distance d-1 on side z count
            const uint32_t key = (z ? KAD_SIDE : 0u) | (uint32_t)d;
            const bool direct = nobits || reC - rsC <= 32;
            unsigned long long carry = 0;
            for (int base = rsC; base < reC; base += KAD_TITEMS * TT) {
                const int e0 = base + KAD_TITEMS * tl;
                int pp[KAD_TITEMS];
                uint32_t lp[KAD_TITEMS];
                unsigned long long wk[KAD_TITEMS];
#pragma unroll
                for (int k = 0; k < KAD_TITEMS; k++) pp[k] = (e0 + k < reC) ? __ldg(tcol(a, z) + e0 + k) : -1;
                if (direct) {
#pragma unroll
                    for (int k = 0; k < KAD_TITEMS; k++) lp[k] = (pp[k] >= 0) ? kad_ld_u32(lab_at(label, pp[k])) : 0u;
                } else {
#pragma unroll
                    for (int k = 0; k < KAD_TITEMS; k++)
                        lp[k] = (pp[k] >= 0) ? bits_ld(bsh, bits, (pp[k] >> gs) >> 5) : 0u;
#pragma unroll
                    for (int k = 0; k < KAD_TITEMS; k++)
                        lp[k] = (pp[k] >= 0 && ((lp[k] >> ((pp[k] >> gs) & 31)) & 1u)) ? kad_ld_u32(lab_at(label, pp[k]))
                                                                                       : 0u;
                }
                unsigned long long mine = 0;
#pragma unroll
                for (int k = 0; k < KAD_TITEMS; k++) {
                    wk[k] = 0;
                    if (pp[k] >= 0 && (lp[k] & KAD_KEY) == key)
                        wk[k] = (lp[k] & KAD_OVF) ? KAD_U64MAX : kad_ld_u64(sig_at(label, pp[k]));
                    mine = kad_sat_add(mine, wk[k]);
                }
                // running sums in CSR order (saturating addition is associative):
                // warp scan, then the team's per-warp sums
                const unsigned long long incl = warp_incl_sat_scan(mine);
                unsigned long long excl = __shfl_up_sync(FULL_MASK, incl, 1);
                if (lane == 0) excl = 0;
                if (lane == 31) sm.t_wsum[t][tw] = incl;
                if (leader) sm.t_min[t][par] = 0x7fffffff;
                team_bar(t, TT);
                unsigned long long c = carry, tot = carry;
#pragma unroll
                for (int w = 0; w < TW; w++) {
                    const unsigned long long x = sm.t_wsum[t][w];
                    if (w < tw) c = kad_sat_add(c, x);
                    tot = kad_sat_add(tot, x);
                }
                c = kad_sat_add(c, excl);
                int hit = 0x7fffffff, hp = -1;
                unsigned long long hs = 0;
#pragma unroll
                for (int k = 0; k < KAD_TITEMS; k++) {
                    const unsigned long long c2 = kad_sat_add(c, wk[k]);
                    if (wk[k] && c2 > r && hit == 0x7fffffff) {
                        hit = e0 + k;
                        hp = pp[k];
                        hs = wk[k];
                    }
                    c = c2;
                }
                const int wmin = __reduce_min_sync(FULL_MASK, hit);
                if (lane == 0 && wmin != 0x7fffffff) atomicMin(&sm.t_min[t][par], wmin);
                team_bar(t, TT);
                const int sel = sm.t_min[t][par];
                par ^= 1;
                if (sel != 0x7fffffff) {
                    if (hit == sel) {
                        sm.t_p[t] = hp;
                        sm.t_s[t] = hs;
                        sm.t_rs[t] = __ldg(trp(a, z) + hp);
                        sm.t_re[t] = __ldg(trp(a, z) + hp + 1);
                    }
                    team_bar(t, TT);
                    p_sel = sm.t_p[t];
                    s_sel = sm.t_s[t];
                    rs_sel = sm.t_rs[t];
                    re_sel = sm.t_re[t];
                    if (leader) w_trace += (unsigned long long)(sel - rsC + 1);
                    break;
                }
                carry = tot;
            }
        }
        if (p_sel < 0) {
            if (leader) kad_set_err(a.ctl, KAD_DERR_TRACE);
            return -1;
        }
        d--;
        if (d >= 1) {
            const int j = (z == 0) ? d : D - d;
            if (leader) {
                if (!buf_v) {
                    emit(a, out, D, j, p_sel);
                } else {
                    buf_v[nb] = p_sel;
                    buf_j[nb] = j;
                }
            }
            nb++;
        }
        cur = p_sel;
        sc = s_sel;
        rsC = rs_sel;
        reC = re_sel;
    }
    return nb;
}

// ---------------------------------------------------------------- expansion
// What the warps of a block need to expand arcs of a frontier chunk: the slot's
// scratch and the round.  The chunk itself -- row starts, exclusive degree
// offsets and path counts of its cnt frontier vertices -- is in shared memory
// (sm.rs, sm.off, sm.sig), and so are the list tail, the next frontier's degree
// sum, the meeting flag and the recorded meeting set.
struct ExpandCtx {
    uint32_t *label; // 16-byte records: label, -, sigma
    unsigned long long *sigma2;
    int32_t *list;
    uint32_t *bits;
    int cnt, X, tailY, n, mcap;
    int32_t *mext_id; // this slot's meeting-set extension (mext entries after the first mcap)
    int mext;
    int rb; // round parity: slot of sm.met / sm.next_dsum
    uint32_t sideX, keyNext;
    bool bsh, watch;
    bool nobits; // no labelled-vertex bitmap: labels are read directly
    int gs;      // bitmap group shift: one bit per 2^gs vertices
    bool probe;  // look for arcs into the other side's frontier only (no claims)
};

// Expand the arcs first + k*stride (k < KAD_ITEMS) below `total` of the chunk.
// Called by whole warps.  All neighbour ids are loaded before any bitmap word,
// and those before any label or atomic, so each thread keeps several
// independent loads in flight.  No block barrier is needed: an unlabelled
// vertex can only become keyNext during the round (only side X labels, and
// every earlier label has its bit set), so claims and path-count pushes commute,
// and a fresh vertex's push need not wait for its claim's answer.  The arc that
// first marks a meeting vertex records it in M.  Returns true (for the whole
// warp) when the run has stopped and this sample may give up.
template <int BLOCK>
__device__ __forceinline__ bool expand_items(const SampleArgs &a, Smem<BLOCK> &sm, const ExpandCtx &c, int first,
                                             int stride, int total, unsigned long long &pred_next,
                                             unsigned long long &pred_m) {
    const int lane = threadIdx.x & 31;
    // lane 0 looks at the stop flag and every lane at the meeting flag (both
    // issued here, used below)
    int stop_now = 0;
    if (lane == 0 && c.watch) stop_now = *(volatile int *)&a.ctl->stop;
    const int met_before = sm.met[c.rb];
    int vv[KAD_ITEMS];
    int ix[KAD_ITEMS]; // frontier entry of the arc (its sigma is sm.sig[ix])
    uint32_t ll[KAD_ITEMS];
#pragma unroll
    for (int k = 0; k < KAD_ITEMS; k++) {
        const int e = first + k * stride;
        vv[k] = -1;
        ix[k] = 0;
        if (e < total) {
            // frontier entry owning arc e: last j with off[j] <= e
            int lo = 0, hi = c.cnt - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sm.off[mid] <= e)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            vv[k] = __ldg(xcol(a, c.X) + sm.rs[lo] + (e - sm.off[lo]));
            ix[k] = lo;
        }
    }
    bool fresh[KAD_ITEMS]; // unlabelled when the bitmap (or the label) was read
    if (c.nobits) {
        // no bitmap: every neighbour's label is read directly
#pragma unroll
        for (int k = 0; k < KAD_ITEMS; k++) ll[k] = (vv[k] >= 0) ? kad_ld_u32(lab_at(c.label, vv[k])) : 0u;
#pragma unroll
        for (int k = 0; k < KAD_ITEMS; k++) fresh[k] = vv[k] >= 0 && ll[k] == 0u;
    } else {
        uint32_t bw[KAD_ITEMS];
#pragma unroll
        for (int k = 0; k < KAD_ITEMS; k++) bw[k] = (vv[k] >= 0) ? bits_ld(c.bsh, c.bits, (vv[k] >> c.gs) >> 5) : 0u;
        // only vertices whose group bit is set may carry a label worth reading
#pragma unroll
        for (int k = 0; k < KAD_ITEMS; k++) {
            const bool set = vv[k] >= 0 && ((bw[k] >> ((vv[k] >> c.gs) & 31)) & 1u);
            ll[k] = set ? kad_ld_u32(lab_at(c.label, vv[k])) : 0u;
            fresh[k] = vv[k] >= 0 && ll[k] == 0u;
        }
    }
    // Does an arc of this warp reach the other side's frontier?  Then the round
    // meets and no new vertex needs claiming (other warps learn it through met).
    int reaches_y = 0;
#pragma unroll
    for (int k = 0; k < KAD_ITEMS; k++)
        if (ll[k] != 0u && (ll[k] & KAD_SIDE) != c.sideX) reaches_y = 1;
    const bool warp_meets = __any_sync(FULL_MASK, reaches_y) != 0;
    if (__shfl_sync(FULL_MASK, stop_now, 0)) return true;
    if (warp_meets && lane == 0) sm.met[c.rb] = 1;
    const bool meeting_seen = warp_meets || met_before != 0;
    uint32_t old[KAD_ITEMS];
    unsigned long long prev[KAD_ITEMS];
    int kind[KAD_ITEMS]; // 0 none, 1 next level of X, 2 other side's frontier
#pragma unroll
    for (int k = 0; k < KAD_ITEMS; k++) {
        old[k] = 0u;
        kind[k] = 0;
        prev[k] = 0;
        const int v = vv[k];
        if (fresh[k]) {
            if (meeting_seen || c.probe) continue;
            old[k] = atomicCAS(lab_at(c.label, v), 0u, c.keyNext);
            kind[k] = 1;
            prev[k] = atomicAdd(sig_at(c.label, v), sm.sig[ix[k]]);
        } else if (ll[k] != 0u) {
            const uint32_t lv = ll[k];
            if ((lv & KAD_KEY) == c.keyNext) {
                kind[k] = 1;
                prev[k] = atomicAdd(sig_at(c.label, v), sm.sig[ix[k]]);
            } else if ((lv & KAD_SIDE) != c.sideX) {
                kind[k] = 2; // handled below
            }
        }
    }
    // Arcs into the other side's frontier: the searches meet.  The arc that
    // first marks its head records it in M.  One at a time (a few per sample),
    // so that this code exists once.
    unsigned m2 = 0;
#pragma unroll
    for (int k = 0; k < KAD_ITEMS; k++)
        if (kind[k] == 2) m2 |= 1u << k;
    const bool any_m = m2 != 0;
    pred_m += (unsigned long long)__popc(m2);
    while (m2) {
        const int k = __ffs(m2) - 1;
        m2 &= m2 - 1;
        int v = vv[0], ixk = ix[0];
        uint32_t lv = ll[0];
#pragma unroll
        for (int q = 1; q < KAD_ITEMS; q++)
            if (k == q) {
                v = vv[q];
                ixk = ix[q];
                lv = ll[q];
            }
        if (!(lv & KAD_INM) && !(atomicOr(lab_at(c.label, v), KAD_INM) & KAD_INM)) {
            const int slot = atomicAdd(&sm.mcount, 1);
            if (slot < c.mcap) sm.m_id[slot] = v;
            else if (slot - c.mcap < c.mext) c.mext_id[slot - c.mcap] = v;
        }
        const unsigned long long add = sm.sig[ixk];
        const unsigned long long pv = atomicAdd(c.sigma2 + v, add);
        if (pv + add < pv) atomicOr(lab_at(c.label, v), KAD_OVF2);
    }
    int rs0[KAD_ITEMS], rs1[KAD_ITEMS];
#pragma unroll
    for (int k = 0; k < KAD_ITEMS; k++) {
        rs0[k] = rs1[k] = 0;
        if (fresh[k] && kind[k] == 1) {
            rs0[k] = __ldg(xrp(a, c.X) + vv[k]);
            rs1[k] = __ldg(xrp(a, c.X) + vv[k] + 1);
        }
    }
    bool claimed[KAD_ITEMS];
#pragma unroll
    for (int k = 0; k < KAD_ITEMS; k++) {
        claimed[k] = fresh[k] && kind[k] == 1 && old[k] == 0u;
        if (fresh[k] && kind[k] == 1 && old[k] != 0u && old[k] != c.keyNext)
            kad_set_err(a.ctl, KAD_DERR_LEVEL); // cannot happen (see above)
        if (claimed[k] && !c.nobits) bits_set(c.bsh, c.bits, vv[k] >> c.gs);
        if (kind[k] == 1) {
            pred_next++;
            if (prev[k] + sm.sig[ix[k]] < prev[k]) atomicOr(lab_at(c.label, vv[k]), KAD_OVF);
        }
    }
    if (any_m) sm.met[c.rb] = 1;
    // new vertices: one list reservation and one degree-sum update per warp
    unsigned mask[KAD_ITEMS];
    int nclaim = 0;
    unsigned long long mydeg = 0;
#pragma unroll
    for (int k = 0; k < KAD_ITEMS; k++) {
        mask[k] = __ballot_sync(FULL_MASK, claimed[k]);
        nclaim += __popc(mask[k]);
        if (claimed[k]) mydeg += (unsigned long long)(rs1[k] - rs0[k]);
    }
    if (nclaim) {
        int pos0 = 0;
        if (lane == 0) pos0 = atomicAdd(&sm.tail[c.X], nclaim);
        pos0 = __shfl_sync(FULL_MASK, pos0, 0);
#pragma unroll
        for (int k = 0; k < KAD_ITEMS; k++) {
            if (claimed[k]) {
                const int pos = pos0 + __popc(mask[k] & lanemask_lt());
                if (pos + c.tailY < c.n)
                    c.list[phys(c.X, pos, c.n)] = vv[k];
                else
                    kad_set_err(a.ctl, KAD_DERR_FRONTIER);
            }
            pos0 += __popc(mask[k]);
        }
        const unsigned long long ds = warp_sum_u64(mydeg);
        if (lane == 0) atomicAdd(&sm.next_dsum[c.rb], ds);
    }
    return false;
}

// The probe scan of a large round: arcs first + k*stride (k < KAD_PITEMS) below
// `total`.  Only an arc into the other side's frontier matters here (it marks
// its head as a member of M, recording it on first mark, and pushes sigma_X
// into sigma2); nothing is claimed, so a pass carries twice the arcs of a
// claiming one.  Returns true (for the whole warp) when the run has stopped.
template <int BLOCK>
__device__ __forceinline__ bool probe_items(const SampleArgs &a, Smem<BLOCK> &sm, const ExpandCtx &c, int first,
                                            int stride, int total, unsigned long long &pred_m) {
    const int lane = threadIdx.x & 31;
    int stop_now = 0;
    if (lane == 0 && c.watch) stop_now = *(volatile int *)&a.ctl->stop;
    int vv[KAD_PITEMS], ix[KAD_PITEMS];
#pragma unroll
    for (int k = 0; k < KAD_PITEMS; k++) {
        const int e = first + k * stride;
        vv[k] = -1;
        ix[k] = 0;
        if (e < total) {
            int lo = 0, hi = c.cnt - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sm.off[mid] <= e)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            vv[k] = __ldg(xcol(a, c.X) + sm.rs[lo] + (e - sm.off[lo]));
            ix[k] = lo;
        }
    }
    uint32_t ll[KAD_PITEMS];
    if (c.nobits) {
#pragma unroll
        for (int k = 0; k < KAD_PITEMS; k++) ll[k] = (vv[k] >= 0) ? kad_ld_u32(lab_at(c.label, vv[k])) : 0u;
    } else {
#pragma unroll
        for (int k = 0; k < KAD_PITEMS; k++) ll[k] = (vv[k] >= 0) ? bits_ld(c.bsh, c.bits, (vv[k] >> c.gs) >> 5) : 0u;
#pragma unroll
        for (int k = 0; k < KAD_PITEMS; k++)
            ll[k] = (vv[k] >= 0 && ((ll[k] >> ((vv[k] >> c.gs) & 31)) & 1u)) ? kad_ld_u32(lab_at(c.label, vv[k])) : 0u;
    }
    if (__shfl_sync(FULL_MASK, stop_now, 0)) return true;
    // arcs into the other side's frontier (a few per sample), handled one at a
    // time so that the code below exists once
    unsigned mk = 0;
#pragma unroll
    for (int k = 0; k < KAD_PITEMS; k++)
        if (ll[k] != 0u && (ll[k] & KAD_SIDE) != c.sideX) mk |= 1u << k;
    const bool any_m = mk != 0;
    while (mk) {
        const int k = __ffs(mk) - 1;
        mk &= mk - 1;
        int v = vv[0], ixk = ix[0];
        uint32_t lv = ll[0];
#pragma unroll
        for (int q = 1; q < KAD_PITEMS; q++)
            if (k == q) {
                v = vv[q];
                ixk = ix[q];
                lv = ll[q];
            }
        if (!(lv & KAD_INM) && !(atomicOr(lab_at(c.label, v), KAD_INM) & KAD_INM)) {
            const int slot = atomicAdd(&sm.mcount, 1);
            if (slot < c.mcap)
                sm.m_id[slot] = v;
            else if (slot - c.mcap < c.mext)
                c.mext_id[slot - c.mcap] = v;
        }
        const unsigned long long add = sm.sig[ixk];
        const unsigned long long prev = atomicAdd(c.sigma2 + v, add);
        if (prev + add < prev) atomicOr(lab_at(c.label, v), KAD_OVF2);
        pred_m++;
    }
    if (any_m) sm.met[c.rb] = 1;
    return false;
}

// Meeting draw for a large M (out of line: a minority of samples): select by id
// digits, 4 bits per pass from the top, with exact 128-bit bin sums, over the
// recorded members when all were recorded, else over the other side's
// frontier.  Sets sm.mid.  Called by every thread of the block.
template <int BLOCK>
__device__ __noinline__ void select_by_digits(const SampleArgs &a, Smem<BLOCK> &sm, bool from_rec, int mc, int mcap,
                                              const int32_t *mext_id, const unsigned long long *mext_w,
                                              const int32_t *list, const uint32_t *label,
                                              const unsigned long long *sigma2, int n, int Y, int yb, int ye,
                                              unsigned long long r) {
    const int tid = threadIdx.x;
    const int nb = 32 - __clz(max(n - 1, 1));
    const int top = ((nb + 3) / 4) * 4;
    unsigned int prefix = 0;
    unsigned long long P = 0;
    for (int shift = top - 4; shift >= 0; shift -= 4) {
        if (tid < 16) {
            sm.bin_lo[tid] = 0;
            sm.bin_hi[tid] = 0;
        }
        __syncthreads();
        if (from_rec) {
            for (int i = tid; i < mc; i += BLOCK) {
                const int v = (i < mcap) ? sm.m_id[i] : __ldcg(mext_id + (i - mcap));
                if (((unsigned long long)(unsigned)v >> (shift + 4)) !=
                    ((unsigned long long)prefix >> (shift + 4)))
                    continue;
                const unsigned long long w = (i < mcap) ? sm.m_w[i] : __ldcg(mext_w + (i - mcap));
                const int b = ((unsigned)v >> shift) & 15;
                const unsigned long long old = atomicAdd(&sm.bin_lo[b], w);
                if (old + w < old) atomicAdd(&sm.bin_hi[b], 1ull);
            }
        } else
        for (int j = yb + tid; j < ye; j += BLOCK) {
            const int v = __ldcg(list + phys(Y, j, n));
            const uint32_t lv = kad_ld_u32(lab_at(label, v));
            if (!(lv & KAD_INM)) continue;
            if (((unsigned long long)(unsigned)v >> (shift + 4)) !=
                ((unsigned long long)prefix >> (shift + 4)))
                continue;
            const unsigned long long sx = (lv & KAD_OVF2) ? KAD_U64MAX : kad_ld_u64(sigma2 + v);
            const unsigned long long sy = (lv & KAD_OVF) ? KAD_U64MAX : kad_ld_u64(sig_at(label, v));
            const unsigned long long w = kad_sat_mul(sx, sy);
            const int b = ((unsigned)v >> shift) & 15;
            const unsigned long long old = atomicAdd(&sm.bin_lo[b], w);
            if (old + w < old) atomicAdd(&sm.bin_hi[b], 1ull);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned long long cum = P;
            int chosen = -1;
            for (int b = 0; b < 16; b++) {
                const unsigned long long bw = sm.bin_hi[b] ? KAD_U64MAX : sm.bin_lo[b];
                const unsigned long long nc = kad_sat_add(cum, bw);
                if (nc > r) {
                    chosen = b;
                    break;
                }
                cum = nc;
            }
            if (chosen < 0) {
                kad_set_err(a.ctl, KAD_DERR_SELECT);
                chosen = 0;
            }
            sm.P = cum;
            sm.prefix = prefix | ((unsigned)chosen << shift);
        }
        __syncthreads();
        P = sm.P;
        prefix = sm.prefix;
    }
    if (tid == 0) sm.mid = (int)prefix;
}

// The block finishing the last calibration sample copies the histogram of c0
// to the mapped host page and raises the flag the host waits for (out of line:
// once per run).
template <int BLOCK>
__device__ __noinline__ void publish_histogram(const SampleArgs &a) {
    const int tid = threadIdx.x;
    for (int c = tid; c < a.nclass; c += BLOCK) a.hpage->hist[c] = __ldcg(a.hist + c);
    __threadfence_system();
    __syncthreads();
    if (tid == 0) {
        a.ctl->t_calib = global_ns();
        *(volatile int *)&a.hpage->calib_flag = 1;
        __threadfence_system();
    }
}

// The pairwise test when there are more pairs than half the block's threads (out
// of line: rare): four pairs per thread and step, their binary searches
// interleaved.  Called by every thread of the block.
template <int BLOCK>
__device__ __noinline__ void pairs_many(const SampleArgs &a, Smem<BLOCK> &sm, const int32_t *list, uint32_t *label,
                                        unsigned long long *sigma2, int32_t *mext_id, int mcap, int mext, int Y,
                                        int yb, int fx, long long np, int n, int rb, unsigned long long &pred_m) {
    const int tid = threadIdx.x;
    // u in F_X has an arc toward w in F_Y when w is in u's row (X's direction)
    // or u in w's row (Y's direction)
    const int32_t *xcX = xcol(a, 1 - Y), *xcY = xcol(a, Y), *xrY = xrp(a, Y);
    // four pairs per thread and step, their binary searches interleaved
    for (long long p0 = tid; p0 < np; p0 += 4ll * BLOCK) {
        int pi[4], pw[4], lo[4], hi[4], key[4];
        bool hit[4], inU[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const long long p = p0 + (long long)k * BLOCK;
            pi[k] = -1;
            pw[k] = -1;
            hit[k] = false;
            inU[k] = false;
            lo[k] = hi[k] = key[k] = 0;
            if (p < np) {
                pi[k] = (int)(p % fx);
                pw[k] = __ldcg(list + phys(Y, yb + (int)(p / fx), n));
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (pw[k] < 0) continue;
            const int rsW = __ldg(xrY + pw[k]), reW = __ldg(xrY + pw[k] + 1);
            const int rsU = sm.rs[pi[k]], reU = sm.off[pi[k]];
            if (reU - rsU <= reW - rsW) { // search w in the row of u
                lo[k] = rsU;
                hi[k] = reU;
                key[k] = pw[k];
                inU[k] = true;
            } else { // search u in the row of w
                lo[k] = rsW;
                hi[k] = reW;
                key[k] = sm.uid[pi[k]];
            }
        }
        for (int step = 0; step < 32; step++) {
            bool any = false;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (hit[k] || lo[k] >= hi[k]) continue;
                any = true;
                const int mid = (lo[k] + hi[k]) >> 1;
                const int v = __ldg((inU[k] ? xcX : xcY) + mid);
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
            if (!(atomicOr(lab_at(label, pw[k]), KAD_INM) & KAD_INM)) {
                const int slot = atomicAdd(&sm.mcount, 1);
                if (slot < mcap) sm.m_id[slot] = pw[k];
                else if (slot - mcap < mext) mext_id[slot - mcap] = pw[k];
            }
            prev[k] = atomicAdd(sigma2 + pw[k], sm.sig[pi[k]]);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (!hit[k]) continue;
            pred_m++;
            sm.met[rb] = 1;
            if (prev[k] + sm.sig[pi[k]] < prev[k]) atomicOr(lab_at(label, pw[k]), KAD_OVF2);
        }
    }
}

// ---------------------------------------------------------------- closer
// Fold epoch k (sample rows of ring slot k mod R) into the counts, then
// evaluate the stop rule on the consistent state after k+1 epochs.
template <int BLOCK>
__device__ __noinline__ void close_epoch(const SampleArgs &a, Smem<BLOCK> &sm, unsigned long long k) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const size_t rb = (size_t)(k % a.ring) * a.epoch;
    if (tid == 0) sm.ovf_acc = 0;
    __syncthreads();
    unsigned long long ovf = 0;
    for (uint32_t j = wid; j < a.epoch; j += BLOCK / 32) {
        const size_t row = rb + j;
        const int len = __ldcg(a.plen + row);
        if (lane == 0 && __ldcg(a.pflag + row)) ovf++;
        for (int t = lane; t < len; t += 32) {
            const int v = __ldcg(a.paths + row * (size_t)a.cap + t);
            const unsigned int c = atomicAdd(a.cnt + v, 1u) + 1u;
            atomicMax(a.classmax + __ldcg(a.c0 + v), (int)c);
        }
    }
    if (lane == 0 && ovf) atomicAdd(&sm.ovf_acc, ovf);
    __threadfence();
    __syncthreads();
    const unsigned long long tau = (k + 1) * (unsigned long long)a.epoch;
    int pass = 1;
    if (tau < a.omega) {
        // Appendix B: stop iff f <= eps and g <= eps for every vertex.  f and g
        // are non-decreasing in the count for a fixed L (every operation in
        // kad_fg_dev is correctly rounded, hence monotone), and L depends only on
        // the calibration count, so the largest count of each calibration class
        // decides for the whole class.
        for (int j = tid; j < a.nclass; j += BLOCK) {
            const int cm = __ldcg(a.classmax + j);
            if (cm >= 0) {
                const double L = __ldcg(a.ltab + j); // uploaded while this launch runs
                const double f = kad_fg_dev((unsigned long long)cm, L, tau, a.omega, false);
                const double g = kad_fg_dev((unsigned long long)cm, L, tau, a.omega, true);
                if (!(f <= a.eps && g <= a.eps)) pass = 0;
            }
        }
    }
    const int all = __syncthreads_and(pass);
    if (tid == 0) {
        if (a.ctl->t_first_close == 0) a.ctl->t_first_close = global_ns();
        a.ctl->overflow += sm.ovf_acc;
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
    __syncthreads();
}


// The closer role: at most one block holds it.  After releasing it the holder
// looks once more for a complete epoch, so a completion that raced with the
// release is never lost.  No thread ever waits for another block.
template <int BLOCK>
__device__ __noinline__ void run_closer(const SampleArgs &a, Smem<BLOCK> &sm) {
    bool holding = false;
    if (threadIdx.x == 0) holding = (atomicCAS(&a.ctl->closer, 0, 1) == 0);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int action = 0;
            for (int guard = 0; holding && guard < 4; guard++) {
                kad_fence_sc();
                unsigned long long k = *(volatile unsigned long long *)&a.ctl->closed;
                if (epoch_ready(a, k)) {
                    action = 1;
                    sm.k = k;
                    break;
                }
                atomicExch(&a.ctl->closer, 0);
                holding = false;
                kad_fence_sc();
                k = *(volatile unsigned long long *)&a.ctl->closed;
                if (epoch_ready(a, k) && atomicCAS(&a.ctl->closer, 0, 1) == 0) holding = true;
            }
            if (holding && action == 0) { // guard ran out: give the role back
                atomicExch(&a.ctl->closer, 0);
                holding = false;
            }
            sm.action = action;
        }
        __syncthreads();
        if (sm.action == 0) break;
        close_epoch<BLOCK>(a, sm, sm.k);
    }
}

// ---------------------------------------------------------------- the kernel
template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_sample(const SampleArgs a) {
    __shared__ Smem<BLOCK> sm;
    const int tid = threadIdx.x, lane = tid & 31;
    const int32_t n = a.n;
    const size_t soff = (size_t)blockIdx.x * (size_t)n;
    uint32_t *const label = a.label + 4 * soff; // 16-byte records (label, -, sigma)
    unsigned long long *const sigma2 = a.sigma2 + soff;
    int32_t *const list = a.list + soff;
    // meeting-set members beyond the shared-memory part go to this slot's row of
    // the global extension
    const int mext = a.mext_id ? a.mext : 0;
    int32_t *const mext_id = mext ? a.mext_id + (size_t)blockIdx.x * (size_t)mext : nullptr;
    unsigned long long *const mext_w = mext ? a.mext_w + (size_t)blockIdx.x * (size_t)mext : nullptr;
    uint32_t *const bits = a.bits + (size_t)blockIdx.x * (size_t)a.nw;
    const bool bsh = a.bits_smem != 0;
    const bool nobits = a.no_bits != 0 && !bsh;
    const int gs = a.bits_shift;
    if (bsh) {
        for (int w = tid; w < a.nw; w += BLOCK) kad_dyn_bits[w] = 0u;
        __syncthreads();
    }
    const int mcap = (a.mcap < KAD_MCAP_MAX) ? a.mcap : KAD_MCAP_MAX;

    // work counters (thread 0 except pred, which every thread counts)
    // Work counters kept by thread 0 live in shared memory (sm.acc, laid out as
    // the work buffer: expanded, scanned, labelled, -, trace arcs, increments,
    // samples, -, then SM cycles per stage: draw+init, BFS, meeting draw,
    // trace-back+output, reset, epoch close); every thread counts its own arcs
    // into the next level or meeting set.
    unsigned long long w_pred = 0;
    if (tid < KAD_WORK_WORDS) sm.acc[tid] = 0;
    if (tid == 0) {
        sm.probe_score = 4;
        sm.probe_rounds = 0;
        sm.pre_ok = 0;
    }
    if (tid == 0 && a.mode == KAD_MODE_RING) atomicCAS(&a.ctl->t_start, 0ull, global_ns());
    Stream st;

    // A launch that continues a run first closes the epochs an earlier launch
    // completed while the L table was not yet available.
    if (a.mode == KAD_MODE_RING && blockIdx.x == 0) run_closer<BLOCK>(a, sm);

    unsigned long long g_pre = ~0ull; // thread 0: an index fetched ahead (~0: none)
    for (;;) {
        // ---------------------------------------------------- next sample index
        if (tid == 0) {
            unsigned long long idx = ~0ull;
            int calib = 0;
            uint32_t dom = a.domain;
            const bool stopped = (a.mode == KAD_MODE_RING) && (*(volatile int *)&a.ctl->stop != 0);
            const bool ahead = sm.pre_ok != 0; // the index was taken (and its pair drawn) by draw_ahead
            if (!stopped) {
                const unsigned long long g =
                    (g_pre != ~0ull) ? g_pre : ahead ? sm.pre_g : atomicAdd(&a.ctl->next, 1ull);
                idx = sample_of(a, g, calib, dom);
            }
            g_pre = ~0ull;
            sm.pre_ok = 0;
            sm.pre_use = (ahead && idx != ~0ull) ? 1 : 0;
            sm.idx = idx;
            sm.calib = calib;
            sm.dom = dom;
        }
        __syncthreads();
        const unsigned long long idx = sm.idx;
        if (idx == ~0ull) break;
        const bool calib = sm.calib != 0;
        // adaptive samples of a run may be abandoned once the run has stopped
        const bool watch_stop = !calib && a.mode == KAD_MODE_RING;
        if (tid == 0) sm.tmark = clock64();

        // ---------------------------------------------------- pair draw
        if (tid == 0) {
            const bool ahead = sm.pre_use != 0;
            int s, t;
            if (ahead) {
                st.k0 = a.key0;
                st.k1 = a.key1;
                st.idx = idx;
                st.dom = sm.dom;
                st.blk = sm.pre_blk;
                st.pos = sm.pre_pos;
                st.w0 = sm.pre_w0;
                st.w1 = sm.pre_w1;
                s = sm.pre_s;
                t = sm.pre_t;
            } else {
                st.init(a.key0, a.key1, idx, sm.dom);
                s = (int)st.uniform((unsigned long long)n, a.ctl);
                t = (int)st.uniform((unsigned long long)(n - 1), a.ctl);
                if (t >= s) t++;
            }
            sm.s = s;
            sm.t = t;
            sm.tail[0] = sm.tail[1] = 0;
            sm.D = 0;
            sm.abort = 0;
            sm.mcount = 0;
            if (ahead ? sm.pre_same != 0 : __ldg(a.comp + s) == __ldg(a.comp + t)) {
                *(uint4 *)lab_at(label, s) = make_uint4(1u, 0u, 1u, 0u);            // s side, level 0, sigma 1
                *(uint4 *)lab_at(label, t) = make_uint4(KAD_SIDE | 1u, 0u, 1u, 0u); // t side, level 0, sigma 1
                if (!nobits) {
                    bits_set(bsh, bits, s >> gs);
                    bits_set(bsh, bits, t >> gs);
                }
                list[0] = s;
                list[n - 1] = t;
                sm.tail[0] = sm.tail[1] = 1;
                sm.fb[0] = sm.fb[1] = 0;
                sm.fe[0] = sm.fe[1] = 1;
                sm.lev[0] = sm.lev[1] = 0;
                sm.lvs[0][0] = sm.lvs[1][0] = 0;
                sm.lvs[0][1] = sm.lvs[1][1] = 1;
                // each root's row in its side's direction: out-arcs of s, in-arcs of t
                const int r0 = ahead ? sm.pre_rs[0] : __ldg(a.rows[0] + s);
                const int r1 = ahead ? sm.pre_rs[1] : __ldg(a.rows[1] + t);
                const int r0e = ahead ? sm.pre_re[0] : __ldg(a.rows[0] + s + 1);
                const int r1e = ahead ? sm.pre_re[1] : __ldg(a.rows[1] + t + 1);
                sm.root_rs[0] = r0;
                sm.root_rs[1] = r1;
                sm.dsum[0] = (unsigned long long)(r0e - r0);
                sm.dsum[1] = (unsigned long long)(r1e - r1);
                sm.D = -1; // searching
                // round 0: its flags, and its expansion counted ahead (one root)
                sm.met[0] = 0;
                sm.next_dsum[0] = 0;
                sm.acc[0] += 1ull;
                sm.acc[1] += (sm.dsum[0] <= sm.dsum[1]) ? sm.dsum[0] : sm.dsum[1];
            }
            __threadfence_block();
        }
        __syncthreads();

        if (tid == 0) {
            const long long now = clock64();
            sm.acc[8] += (unsigned long long)(now - sm.tmark);
            sm.tmark = now;
        }
        // ---------------------------------------------------- balanced bidirectional BFS
        // Barriers per round: the degree scan (one or two), the end of each
        // chunk, and the round's close.  The round's state is read without one:
        // thread 0 writes it only in the round's close, after a barrier, and the
        // next round's flags and counters are prepared there too (slot rb ^ 1).
        int X = 0;
        int rnd = 0;
        while (sm.D < 0) {
            const int rb = rnd & 1;
            X = (sm.dsum[0] <= sm.dsum[1]) ? 0 : 1;
            const int Y = 1 - X;
            const int fb = sm.fb[X], fe = sm.fe[X];
            const int levX = sm.lev[X];
            const int tailY = sm.tail[Y];
            if (fb == fe || levX + 2 > (int)KAD_LVL) {
                __syncthreads(); // everyone has read the round's state
                if (tid == 0) {
                    if (fb != fe) kad_set_err(a.ctl, KAD_DERR_LEVEL);
                    sm.D = 0; // no path
                }
                __syncthreads();
                break;
            }
            const uint32_t sideX = X ? KAD_SIDE : 0u;
            const uint32_t keyNext = sideX | (uint32_t)(levX + 2);
            const int yb = sm.fb[Y], fy = sm.fe[Y] - yb, fx = fe - fb;
            // Pairwise test: when both frontiers are small but X's rows are long,
            // testing every (u in F_X, w in F_Y) for adjacency finds exactly the
            // arcs from F_X into the other side's frontier -- M, and sigma_X on M
            // -- without reading X's rows.  No adjacent pair means no meeting in
            // this round, and the expansion below runs as usual.
            const bool pairs = !(a.debug & KAD_DEBUG_FULL_SCAN) && fx <= BLOCK && sm.dsum[X] >= KAD_PAIR_MIN_ARCS &&
                               (unsigned long long)fx * (unsigned long long)fy * (unsigned)a.pair_cost < sm.dsum[X];
            unsigned long long pred_next = 0, pred_m = 0;
            if (pairs) {
                if (tid < fx) {
                    const int u = __ldcg(list + phys(X, fb + tid, n));
                    uint32_t lu;
                    unsigned long long su;
                    ld_vs(label, u, lu, su);
                    sm.uid[tid] = u;
                    sm.rs[tid] = __ldg(xrp(a, X) + u);
                    sm.off[tid] = __ldg(xrp(a, X) + u + 1);
                    sm.sig[tid] = sig_val(lu, su);
                }
                __syncthreads();
                const long long np = (long long)fx * (long long)fy;
                if (np <= BLOCK / 2) {
                    // G threads per pair (G * np <= BLOCK): probes at G-1 points split
                    // the searched row into G parts per step; once at most 4G entries
                    // are left, the group reads all of them at once
                    int G = 1;
                    while (G < 32 && 2 * G * np <= BLOCK) G *= 2;
                    const int sub = tid & (G - 1);
                    const long long p = tid / G;
                    // an arc from u in F_X toward w in F_Y: w in u's row (X's
                    // direction) or u in w's row (Y's direction)
                    int pi = -1, pw = -1, lo = 0, hi = 0, key = 0;
                    bool inW = false; // searching w's row (else u's)
                    if (p < np) {
                        pi = (int)(p % fx);
                        pw = __ldcg(list + phys(Y, yb + (int)(p / fx), n));
                        const int rsW = __ldg(xrp(a, Y) + pw), reW = __ldg(xrp(a, Y) + pw + 1);
                        const int rsU = sm.rs[pi], reU = sm.off[pi];
                        if (reU - rsU <= reW - rsW) {
                            lo = rsU;
                            hi = reU;
                            key = pw;
                        } else {
                            lo = rsW;
                            hi = reW;
                            key = sm.uid[pi];
                            inW = true;
                        }
                    }
                    const int P = (G > 1) ? G - 1 : 1;
                    const int lgP1 = (G > 1) ? __ffs(G) - 1 : 1; // P + 1 = 2^lgP1
                    bool done = p >= np || lo >= hi, found = false;
                    while (__any_sync(FULL_MASK, !done)) {
                        const int len = hi - lo;
                        if (!done && len <= 4 * G) {
                            // every position left, four per thread
#pragma unroll
                            for (int k = 0; k < 4; k++) {
                                const int q = lo + sub + k * G;
                                if (q < hi && __ldg(xcol(a, inW ? Y : X) + q) == key) found = true;
                            }
                            done = true;
                        }
                        int v = 0, q = 0;
                        const bool probe = !done && sub < P;
                        if (probe) {
                            q = lo + (int)(((long long)len * (sub + 1)) >> lgP1);
                            v = __ldg(xcol(a, inW ? Y : X) + q);
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
                    if (f && sub == 0) {
                        if (!(atomicOr(lab_at(label, pw), KAD_INM) & KAD_INM)) {
                            const int slot = atomicAdd(&sm.mcount, 1);
                            if (slot < mcap) sm.m_id[slot] = pw;
                            else if (slot - mcap < mext) mext_id[slot - mcap] = pw;
                        }
                        const unsigned long long prev = atomicAdd(sigma2 + pw, sm.sig[pi]);
                        pred_m++;
                        sm.met[rb] = 1;
                        if (prev + sm.sig[pi] < prev) atomicOr(lab_at(label, pw), KAD_OVF2);
                    }
                } else {
                    pairs_many<BLOCK>(a, sm, list, label, sigma2, mext_id, mcap, mext, Y, yb, fx, np, n, rb, pred_m);
                }
                __syncthreads();
            }
            // A large round is probed first: one scan that only looks for arcs
            // into the other side's frontier (collecting M and sigma_X on M), and
            // claims new vertices only if it found none.  Almost all of a large
            // round's arcs are scanned in the meeting round, where claims are
            // wasted work; an ordinary large round is scanned twice.
            // Whether a large round is the meeting round depends on the graph:
            // on low-diameter graphs it usually is, on deep ones (grids) almost
            // never.  The block keeps a score of how its probes fared and probes
            // while it is positive, and every 16th large round regardless.
            const bool large = sm.dsum[X] > (unsigned long long)(BLOCK * KAD_ITEMS);
            const bool probe_first = !(a.debug & KAD_DEBUG_NO_PROBE) && large &&
                                     (sm.probe_score > 0 || (sm.probe_rounds & 15) == 0);
            for (int ph = probe_first ? 0 : 1; ph < 2; ph++) {
            // a meeting found by the pairwise test or the probe completes the round
            if (sm.met[rb] || sm.abort) break;
            const int expand_end = fe;
            for (int cb = fb; cb < expand_end; cb += BLOCK) {
                const int cnt = min(BLOCK, fe - cb);
                int d = 0;
                if (levX == 0) {
                    // level 0 is the root alone: its row is known and sigma = 1
                    if (tid == 0) {
                        sm.rs[0] = sm.root_rs[X];
                        sm.sig[0] = 1ull;
                        d = (int)sm.dsum[X];
                    }
                } else if (tid < cnt) {
                    const int u = __ldcg(list + phys(X, cb + tid, n));
                    const int rs = __ldg(xrp(a, X) + u), re = __ldg(xrp(a, X) + u + 1);
                    uint32_t lu;
                    unsigned long long su;
                    ld_vs(label, u, lu, su);
                    sm.rs[tid] = rs;
                    sm.sig[tid] = sig_val(lu, su);
                    d = re - rs;
                }
                // exclusive degree offsets of the chunk: a single vertex needs no scan
                int total;
                if (cnt == 1) {
                    if (tid == 0) {
                        sm.off[0] = 0;
                        sm.chunk_total = d;
                    }
                    __syncthreads();
                    total = sm.chunk_total;
                } else if (cnt <= 32) {
                    // every entry is in warp 0: a warp scan, one barrier
                    if (tid < 32) {
                        int x = d;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int y = __shfl_up_sync(FULL_MASK, x, o);
                            if (lane >= o) x += y;
                        }
                        if (tid < cnt) sm.off[tid] = x - d;
                        if (tid == 31) sm.chunk_total = x;
                    }
                    __syncthreads();
                    total = sm.chunk_total;
                } else {
                    const int excl = block_excl_scan<BLOCK>(d, sm.wtmp, total);
                    if (tid < cnt) sm.off[tid] = excl;
                    __syncthreads();
                }
                ExpandCtx ec;
                ec.label = label;
                ec.sigma2 = sigma2;
                ec.list = list;
                ec.bits = bits;
                ec.cnt = (levX == 0) ? 1 : cnt;
                ec.X = X;
                ec.tailY = tailY;
                ec.n = n;
                ec.sideX = sideX;
                ec.keyNext = keyNext;
                ec.mcap = mcap;
                ec.mext_id = mext_id;
                ec.mext = mext;
                ec.rb = rb;
                ec.bsh = bsh;
                ec.nobits = nobits;
                ec.gs = gs;
                ec.watch = watch_stop;
                ec.probe = ph == 0;
                long long tp = 0;
                if (tid == 0) tp = clock64();
                // a warp whose first arc of a pass (base + 32 w) is past the end has
                // none in it, nor in any later pass: it skips them (small rounds
                // then run on the warps that hold arcs)
                const int wfirst = tid & ~31;
                if (ec.probe) {
                    for (int base = 0; base + wfirst < total; base += BLOCK * KAD_PITEMS) {
                        if (probe_items<BLOCK>(a, sm, ec, base + tid, BLOCK, total, pred_m)) {
                            if (lane == 0) sm.abort = 1;
                            break;
                        }
                    }
                } else {
                    for (int base = 0; base + wfirst < total; base += BLOCK * KAD_ITEMS) {
                        if (expand_items<BLOCK>(a, sm, ec, base + tid, BLOCK, total, pred_next, pred_m)) {
                            if (lane == 0) sm.abort = 1;
                            break;
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) sm.acc[14] += (unsigned long long)(clock64() - tp);
                if (sm.abort) break;
            }
            }
            // every warp's passes ended at the chunk's barrier: this round's flag is final
            const int met = sm.met[rb];
            w_pred += met ? pred_m : pred_next;
            long long tc = 0;
            if (tid == 0) tc = clock64();
            if (tid == 0 && large) {
                sm.probe_rounds++;
                if (probe_first) sm.probe_score = met ? min(sm.probe_score + 1, 8) : sm.probe_score - 1;
            }
            if (tid == 0) {
                if (sm.abort) {
                    // An expansion pass saw the run's stop: this sample lies beyond
                    // the stop epoch and is never counted.  Give up (the reset below
                    // also clears sigma2 on the other side's frontier, where a
                    // meeting may have begun).
                    sm.D = 0;
                } else if (met) {
                    sm.D = sm.lev[X] + 1 + sm.lev[Y];
                } else {
                    const int tl = min(sm.tail[X], n - tailY);
                    sm.acc[2] += (unsigned long long)(tl - fe);
                    sm.fb[X] = fe;
                    sm.fe[X] = tl;
                    sm.lev[X] = levX + 1;
                    if (levX + 2 <= KAD_MAXLV + 1) sm.lvs[X][levX + 2] = tl;
                    sm.dsum[X] = sm.next_dsum[rb];
                    // the next round: its flags, and its expansion counted ahead
                    const int Xn = (sm.dsum[0] <= sm.dsum[1]) ? 0 : 1;
                    sm.met[rb ^ 1] = 0;
                    sm.next_dsum[rb ^ 1] = 0;
                    sm.acc[0] += (unsigned long long)(sm.fe[Xn] - sm.fb[Xn]);
                    sm.acc[1] += sm.dsum[Xn];
                }
            }
            __syncthreads();
            if (tid == 0) sm.acc[15] += (unsigned long long)(clock64() - tc);
            rnd++;
        }

        const int D = sm.D;
        // a small recorded M is drawn by warp 0 alone, and warp 1 draws the next
        // sample's pair meanwhile
        const bool small_m = D > 0 && sm.mcount <= 32 && sm.mcount <= mcap + mext;
        if (tid == 0) {
            const long long now = clock64();
            sm.acc[9] += (unsigned long long)(now - sm.tmark);
            sm.tmark = now;
            // the next sample's index, fetched while this one is finished (an
            // index taken after the run stopped is simply not computed: its
            // epoch lies beyond the stop epoch)
            if (!small_m) g_pre = atomicAdd(&a.ctl->next, 1ull);
        }
        unsigned long long sst = 0;
        // ---------------------------------------------------- meeting draw
        if (D > 0) {
            const int Y = 1 - X;
            const int yb = sm.fb[Y], ye = sm.fe[Y];
            // members recorded during the search: the first mcap in shared
            // memory, the next mext in the slot's extension
            const int mtot = mcap + mext;
            const int mc0 = sm.mcount; // final: the round ended at a barrier
            if (small_m) {
                // A small recorded M (most samples): warp 0 alone, one member per
                // lane -- weights, their saturating sum, the draw, and each
                // member's exclusive prefix in id order by shuffles.
                if (tid < 32) {
                    int id = 0x7fffffff;
                    unsigned long long w = 0;
                    if (lane < mc0) {
                        id = (lane < mcap) ? sm.m_id[lane] : __ldcg(mext_id + (lane - mcap));
                        uint32_t lv;
                        unsigned long long s1;
                        const unsigned long long s2 = kad_ld_u64(sigma2 + id);
                        ld_vs(label, id, lv, s1);
                        w = kad_sat_mul((lv & KAD_OVF2) ? KAD_U64MAX : s2, sig_val(lv, s1));
                    }
                    unsigned long long tot = w;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) tot = kad_sat_add(tot, __shfl_xor_sync(FULL_MASK, tot, o));
                    unsigned long long r = 0;
                    if (tid == 0) {
                        r = st.uniform(tot ? tot : 1ull, a.ctl);
                        sm.sst = tot;
                        sm.st_w0 = st.w0;
                        sm.st_w1 = st.w1;
                        sm.st_blk = st.blk;
                        sm.st_pos = st.pos;
                    }
                    r = __shfl_sync(FULL_MASK, r, 0);
                    unsigned long long ex = 0;
                    for (int q = 0; q < mc0; q++) {
                        const int iq = __shfl_sync(FULL_MASK, id, q);
                        const unsigned long long wq = __shfl_sync(FULL_MASK, w, q);
                        if (iq < id) ex = kad_sat_add(ex, wq);
                    }
                    const unsigned hit = __ballot_sync(FULL_MASK, lane < mc0 && ex <= r && kad_sat_add(ex, w) > r);
                    const int chosen = __shfl_sync(FULL_MASK, id, hit ? __ffs(hit) - 1 : 0);
                    if (tid == 0) sm.mid = hit ? chosen : -1;
                } else if (tid == 32) {
                    draw_ahead<BLOCK>(a, sm);
                }
                __syncthreads();
                sst = sm.sst;
            } else {
            const bool recorded = mc0 <= mtot;
            __syncthreads();
            if (tid == 0 && !recorded) sm.mcount = 0;
            __syncthreads();
            unsigned long long part = 0;
            if (recorded) {
                // M was recorded by the arcs that first reached its members
                for (int i = tid; i < sm.mcount; i += BLOCK) {
                    const int v = (i < mcap) ? sm.m_id[i] : __ldcg(mext_id + (i - mcap));
                    uint32_t lv;
                    unsigned long long s1;
                    const unsigned long long s2 = kad_ld_u64(sigma2 + v); // issued with the record's load
                    ld_vs(label, v, lv, s1);
                    const unsigned long long sx = (lv & KAD_OVF2) ? KAD_U64MAX : s2;
                    const unsigned long long sy = sig_val(lv, s1);
                    const unsigned long long w = kad_sat_mul(sx, sy);
                    part = kad_sat_add(part, w);
                    if (i < mcap)
                        sm.m_w[i] = w;
                    else
                        mext_w[i - mcap] = w;
                }
            } else
            for (int j = yb + tid; j < ye; j += BLOCK) {
                const int v = __ldcg(list + phys(Y, j, n));
                uint32_t lv;
                unsigned long long s1;
                ld_vs(label, v, lv, s1);
                if (lv & KAD_INM) {
                    const unsigned long long sx = (lv & KAD_OVF2) ? KAD_U64MAX : kad_ld_u64(sigma2 + v);
                    const unsigned long long sy = sig_val(lv, s1);
                    const unsigned long long w = kad_sat_mul(sx, sy);
                    part = kad_sat_add(part, w);
                    const int slot = atomicAdd(&sm.mcount, 1);
                    if (slot < mcap) {
                        sm.m_id[slot] = v;
                        sm.m_w[slot] = w;
                    }
                }
            }
            sst = block_sat_sum<BLOCK>(part, sm.wtmp64);
            if (tid == 0) {
                sm.sst = sst;
                sm.r = st.uniform(sst ? sst : 1ull, a.ctl);
                sm.mid = -1;
                sm.st_w0 = st.w0;
                sm.st_w1 = st.w1;
                sm.st_blk = st.blk;
                sm.st_pos = st.pos;
            }
            __syncthreads();
            const int mc = sm.mcount;
            const unsigned long long r = sm.r;
            if (mc <= mcap) {
                // Small M: the exclusive prefix of each member in id order is the
                // sum of the weights of the members with smaller ids.  P
                // consecutive lanes share a member (each sums every P-th other
                // member, in two independent exact sums) and combine by shuffles.
                int P = 1;
                while (P < 32 && 2 * P * mc <= BLOCK) P *= 2;
                const int per = BLOCK / P, p = tid & (P - 1);
                for (int base = 0; base < mc; base += per) {
                    const int i = base + tid / P;
                    int id = 0;
                    unsigned long long w = 0, e0 = 0, e1 = 0;
                    bool o0 = false, o1 = false; // an exact sum passed 2^64 - 1
                    if (i < mc) {
                        id = sm.m_id[i];
                        w = sm.m_w[i];
                        int j = p;
                        for (; j + P < mc; j += 2 * P) {
                            const unsigned long long a0 = (sm.m_id[j] < id) ? sm.m_w[j] : 0ull;
                            const unsigned long long a1 = (sm.m_id[j + P] < id) ? sm.m_w[j + P] : 0ull;
                            e0 += a0;
                            o0 |= e0 < a0;
                            e1 += a1;
                            o1 |= e1 < a1;
                        }
                        if (j < mc) {
                            const unsigned long long a0 = (sm.m_id[j] < id) ? sm.m_w[j] : 0ull;
                            e0 += a0;
                            o0 |= e0 < a0;
                        }
                    }
                    unsigned long long ex = (o0 || o1) ? KAD_U64MAX : kad_sat_add(e0, e1);
                    for (int o = 1; o < P; o <<= 1) ex = kad_sat_add(ex, __shfl_xor_sync(FULL_MASK, ex, o));
                    if (i < mc && p == 0 && ex <= r && kad_sat_add(ex, w) > r) sm.mid = id;
                }
            } else {
                select_by_digits<BLOCK>(a, sm, mc <= mtot, mc, mcap, mext_id, mext_w, list, label, sigma2, n, Y, yb,
                                        ye, r);
            }
            __syncthreads();
            }
        }

        if (tid == 0) {
            const long long now = clock64();
            sm.acc[10] += (unsigned long long)(now - sm.tmark);
            sm.tmark = now;
        }
        // ---------------------------------------------------- trace-back + output
        // In completion order the fold position (and with it the ring row) is
        // taken once the path is complete; the path is traced into the slot's
        // staging row meanwhile.
        const bool by_completion = a.mode == KAD_MODE_RING && a.fast && !calib;
        size_t row = 0;
        if (a.mode == KAD_MODE_RING)
            row = (size_t)((idx / a.epoch) % a.ring) * a.epoch + (size_t)(idx % a.epoch);
        else if (a.mode == KAD_MODE_RECORD)
            row = (size_t)(idx - a.i0);
        int32_t *const out = calib ? nullptr
                                   : (by_completion ? a.stage + (size_t)blockIdx.x * (size_t)a.cap
                                                    : a.paths + row * (size_t)a.cap);
        // The s side (team 0, the first half of the block) and the t side (team
        // 1) are traced at the same time.  The t side's draws follow the s side's
        // in the stream; team 1 starts where the s side ends if none of its draws
        // is rejected (each then takes one word) and buffers its vertices.  If
        // team 0 ends elsewhere (a rejection, probability below 2^-24 per draw
        // for counts under 2^40), team 0 traces the t side again from there.
        const int mid = sm.mid;
        const bool traced = D > 0 && mid >= 0 && mid < n;
        if (D > 0 && !traced && tid == 0) kad_set_err(a.ctl, KAD_DERR_SELECT);
        int dz[2] = {0, 0};
        unsigned long long gz[2] = {0, 0};
        constexpr int TT = BLOCK / 2;
        const int team = tid / TT, tl = tid - team * TT;
        if (traced) {
            // distance and path count of the meeting vertex on each side: side X
            // reaches it at level lev[X]+1 (count in sigma2), side Y holds it at
            // level lev[Y] (count in sigma)
            uint32_t lm;
            unsigned long long sm1;
            const unsigned long long sm2 = kad_ld_u64(sigma2 + mid);
            ld_vs(label, mid, lm, sm1);
            const int dX = sm.lev[X] + 1, dY = sm.lev[1 - X];
            const unsigned long long gX = (lm & KAD_OVF2) ? KAD_U64MAX : sm2;
            const unsigned long long gY = sig_val(lm, sm1);
            dz[0] = (X == 0) ? dX : dY;
            dz[1] = (X == 1) ? dX : dY;
            gz[0] = (X == 0) ? gX : gY;
            gz[1] = (X == 1) ? gX : gY;
        }
        const bool spec = traced && dz[1] <= KAD_TBUF && !(a.debug & KAD_DEBUG_SERIAL_TRACE);
        if (spec && team == 1 && tl == 0) {
            // team 1's stream: the one after the meeting draw, one word further per s-side step
            st.k0 = a.key0;
            st.k1 = a.key1;
            st.idx = idx;
            st.dom = sm.dom;
            st.blk = sm.st_blk;
            st.pos = sm.st_pos;
            st.w0 = sm.st_w0;
            st.w1 = sm.st_w1;
            for (int q = 0; q < dz[0]; q++) st.next();
            sm.st_spec_blk = st.blk;
            sm.st_spec_pos = st.pos;
        }
        // Two phases with one trace loop.  Phase 0: team 0 traces the s side and
        // team 1 the t side into its buffer.  Phase 1: the buffer goes out if the
        // stream positions agree; else (or without speculation) team 0 traces
        // the t side from its own stream.
        for (int ph = 0; ph < 2 && traced; ph++) {
            int z = -1;
            bool buffered = false;
            if (ph == 0) {
                if (team == 0) z = 0;
                if (team == 1 && spec) {
                    z = 1;
                    buffered = true;
                }
            } else if (team == 0) {
                if (!spec || sm.st_end_blk != sm.st_spec_blk || sm.st_end_pos != sm.st_spec_pos) z = 1;
            } else if (spec && sm.st_end_blk == sm.st_spec_blk && sm.st_end_pos == sm.st_spec_pos) {
                if (tl < sm.tcount) emit(a, out, D, sm.tbuf_j[tl], sm.tbuf_v[tl]);
                if (tl == 0) atomicAdd(&sm.acc[4], sm.wt1);
            }
            if (z >= 0) {
                unsigned long long wt = 0;
                if (z == 0 && tl == 0) emit(a, out, D, dz[0], mid);
                const int nb = trace_side_team<BLOCK>(a, sm, st, team, label, bsh, nobits, gs, bits, list, n, z,
                                                      z ? dz[1] : dz[0], z ? gz[1] : gz[0], mid, D, out,
                                                      buffered ? sm.tbuf_v : nullptr, buffered ? sm.tbuf_j : nullptr, wt);
                if (tl == 0) {
                    if (buffered) {
                        sm.tcount = nb;
                        sm.wt1 = wt;
                    } else {
                        atomicAdd(&sm.acc[4], wt);
                    }
                    if (ph == 0 && z == 0) {
                        sm.st_end_blk = st.blk;
                        sm.st_end_pos = st.pos;
                    }
                }
            }
            __syncthreads();
        }
        unsigned long long pos = idx; // the sample's fold position (its index, or its completion rank)
        if (by_completion) {
            if (tid == 0) sm.qpos = atomicAdd(&a.ctl->qnext, 1ull);
            __syncthreads();
            pos = sm.qpos;
            row = (size_t)((pos / a.epoch) % a.ring) * a.epoch + (size_t)(pos % a.epoch);
            const int len = (D > 0) ? min(D - 1, a.cap) : 0;
            for (int j = tid; j < len; j += BLOCK) a.paths[row * (size_t)a.cap + j] = __ldcg(out + j);
            if (tid == 0 && pos < a.pidx_cap) a.pidx[pos] = idx;
        }
        if (tid == 0) {
            const int inc = (D > 0) ? D - 1 : 0;
            sm.acc[5] += (unsigned long long)inc;
            sm.acc[6]++;
            if (!calib) {
                a.plen[row] = (inc <= a.cap) ? inc : a.cap;
                a.pflag[row] = (sst == KAD_U64MAX) ? 1 : 0;
            }
            if (a.mode == KAD_MODE_RECORD) {
                a.rec_s[row] = sm.s;
                a.rec_t[row] = sm.t;
                a.rec_D[row] = D;
                a.rec_sst[row] = sst;
            }
        }
        __syncthreads();

        if (tid == 0) {
            const long long now = clock64();
            sm.acc[11] += (unsigned long long)(now - sm.tmark);
            sm.tmark = now;
        }
        // ---------------------------------------------------- reset the slot
        // Every vertex this sample labelled is on the list: clear its label, path
        // count and bitmap word.  sigma2 is nonzero only on the meeting set, which
        // lies in the non-expanding side's final frontier.
        {
            const int t0 = min(sm.tail[0], n), t1 = min(sm.tail[1], n - t0);
            const int tot = t0 + t1;
            for (int j0 = tid; j0 < tot; j0 += 4 * BLOCK) {
                int vr[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int j = j0 + k * BLOCK;
                    vr[k] = (j < tot) ? __ldcg(list + ((j < t0) ? j : n - 1 - (j - t0))) : -1;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (vr[k] < 0) continue;
                    *(uint4 *)lab_at(label, vr[k]) = make_uint4(0u, 0u, 0u, 0u);
                    // every set bit of the word is a group with a listed vertex
                    if (!nobits) bits_clear_word(bsh, bits, (vr[k] >> gs) >> 5);
                }
            }
            if (D > 0 || sm.abort) {
                // every vertex with a nonzero sigma2 was counted into mcount when
                // it joined M; if all were recorded, clear just those
                const int mc = sm.mcount;
                if (mc <= mcap + mext) {
                    for (int i = tid; i < mc; i += BLOCK)
                        sigma2[(i < mcap) ? sm.m_id[i] : __ldcg(mext_id + (i - mcap))] = 0ull;
                } else {
                    const int Y = 1 - X;
                    for (int j = sm.fb[Y] + tid; j < sm.fe[Y]; j += BLOCK) sigma2[__ldcg(list + phys(Y, j, n))] = 0ull;
                }
            }
        }
        __threadfence_block();
        __syncthreads();

        if (tid == 0) {
            const long long now = clock64();
            sm.acc[12] += (unsigned long long)(now - sm.tmark);
            sm.tmark = now;
        }
        // ---------------------------------------------------- epoch bookkeeping
        if (a.mode == KAD_MODE_RING && calib) {
            // The block finishing the last calibration sample publishes the
            // histogram to the mapped host page and raises the flag the host
            // waits for; the host then computes the L table while sampling goes on.
            if (tid == 0) {
                __threadfence();
                const unsigned long long done = atomicAdd(&a.ctl->calib_done, 1ull) + 1ull;
                __threadfence();
                sm.publish = (done == a.calib_n) ? 1 : 0;
            }
            __syncthreads();
            if (sm.publish) publish_histogram<BLOCK>(a);
        } else if (a.mode == KAD_MODE_RING) {
            if (tid == 0) {
                // Publish this sample's path (release); the block completing an
                // epoch tries the closer role.  Epochs completed before the L table
                // arrived are closed by the next completion (or the next launch).
                const unsigned long long e = pos / a.epoch;
                const unsigned int old = atom_add_release(&a.epoch_done[e % a.ring], 1u);
                int tc = 0;
                if (old + 1u == a.epoch) {
                    kad_fence_sc();
                    tc = 1;
                }
                sm.try_close = tc;
            }
            __syncthreads();
            if (sm.try_close) run_closer<BLOCK>(a, sm);
        }
        if (tid == 0) {
            const long long now = clock64();
            sm.acc[13] += (unsigned long long)(now - sm.tmark);
            sm.tmark = now;
        }
    }

    // ---------------------------------------------------- work counters
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w_pred += __shfl_xor_sync(FULL_MASK, w_pred, o);
    if (lane == 0 && w_pred) atomicAdd(a.work + 3, w_pred);
    if (tid == 0) {
        for (int i = 0; i < KAD_WORK_WORDS; i++)
            if (i != 3 && sm.acc[i]) atomicAdd(a.work + i, sm.acc[i]);
        if (a.mode == KAD_MODE_RING) atomicMax(&a.ctl->t_end, global_ns());
    }
}

// ---------------------------------------------------------------- small kernels
// b~(v) = c(v)/tau (Section 2.3), correctly rounded division.
__global__ void k_finalize(const uint32_t *__restrict__ cnt, int32_t n, unsigned long long tau, double *__restrict__ bc) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        bc[v] = __ddiv_rn((double)__ldg(cnt + v), (double)tau);
}

__global__ void k_fg(const uint32_t *__restrict__ counts, const uint32_t *__restrict__ c0,
                     const double *__restrict__ ltab, int32_t n, unsigned long long tau, unsigned long long omega,
                     double *__restrict__ f, double *__restrict__ g) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const double L = ltab[c0[v]];
        f[v] = kad_fg_dev(counts[v], L, tau, omega, false);
        g[v] = kad_fg_dev(counts[v], L, tau, omega, true);
    }
}

} // namespace

// ---------------------------------------------------------------- launchers
// Sampling-kernel variants: threads per block x resident blocks per SM the
// register budget is sized for (64K registers per SM).
#define KAD_VARIANTS(X) X(128, 4) X(128, 8) X(256, 2) X(256, 4) X(512, 1) X(512, 2) X(1024, 1)

#if KAD_DIRECTED
cudaError_t kad_launch_sample_directed(const SampleArgs &a, int blocks, int threads, int per_sm, size_t dyn_smem,
                                       cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
#else
cudaError_t kad_launch_sample(const SampleArgs &a, int blocks, int threads, int per_sm, size_t dyn_smem,
                              cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (a.rows[1] != a.rows[0]) return kad_launch_sample_directed(a, blocks, threads, per_sm, dyn_smem, st);
#endif
#define KAD_LAUNCH(T, B)                                                                                              \
    if (threads == T && per_sm == B) {                                                                                \
        if (dyn_smem > 0) {                                                                                           \
            const cudaError_t e =                                                                                     \
                cudaFuncSetAttribute(k_sample<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);     \
            if (e != cudaSuccess) return e;                                                                           \
        }                                                                                                             \
        k_sample<T, B><<<blocks, T, dyn_smem, st>>>(a);                                                               \
        return cudaGetLastError();                                                                                    \
    }
    KAD_VARIANTS(KAD_LAUNCH)
#undef KAD_LAUNCH
    return cudaErrorInvalidConfiguration;
}

#if !KAD_DIRECTED // one copy of the queries and the other kernels' launchers

bool kad_sample_variant_exists(int threads, int per_sm) {
#define KAD_HAS(T, B)                                                                                                 \
    if (threads == T && per_sm == B) return true;
    KAD_VARIANTS(KAD_HAS)
#undef KAD_HAS
    return false;
}

size_t kad_sample_static_smem(int threads, int per_sm) {
    cudaFuncAttributes fa;
    memset(&fa, 0, sizeof(fa));
#define KAD_ATTR(T, B)                                                                                                \
    if (threads == T && per_sm == B && cudaFuncGetAttributes(&fa, k_sample<T, B>) == cudaSuccess) return fa.sharedSizeBytes;
    KAD_VARIANTS(KAD_ATTR)
#undef KAD_ATTR
    return 0;
}

int kad_sample_max_blocks_per_sm(int threads, int per_sm, size_t dyn_smem) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidConfiguration;
#define KAD_OCC(T, B)                                                                                                 \
    if (threads == T && per_sm == B) {                                                                                \
        if (dyn_smem > 0)                                                                                             \
            cudaFuncSetAttribute(k_sample<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);         \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sample<T, B>, T, dyn_smem);                         \
    }
    KAD_VARIANTS(KAD_OCC)
#undef KAD_OCC
    return (e == cudaSuccess) ? nb : 0;
}

cudaError_t kad_launch_finalize(const uint32_t *cnt, int32_t n, unsigned long long tau, double *bc, cudaStream_t st) {
    const int threads = 256;
    int blocks = (n + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_finalize<<<blocks, threads, 0, st>>>(cnt, n, tau, bc);
    return cudaGetLastError();
}

cudaError_t kad_launch_fg(const uint32_t *counts, const uint32_t *c0, const double *ltab, int32_t n,
                          unsigned long long tau, unsigned long long omega, double *f, double *g, cudaStream_t st) {
    const int threads = 256;
    int blocks = (n + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_fg<<<blocks, threads, 0, st>>>(counts, c0, ltab, n, tau, omega, f, g);
    return cudaGetLastError();
}
#endif // !KAD_DIRECTED
