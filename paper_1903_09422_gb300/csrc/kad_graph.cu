// Graph set-up on the device: CSR validation, connected components and the
// vertex-diameter bound that fixes omega (Section 2.3 preprocessing: "mostly
// computing an upper bound on the diameter"; Appendix C.1: components are
// computed with it so that pairs in different components can be skipped).
// Directed graphs (Section 5: KADABRA also covers them) get their in-arc rows,
// weak components and a bound through the strongly connected components
// (setup_directed below).
//
// Undirected:
// VD = max over components C of 2 ecc_C(v0_C) + 1, with v0_C the vertex of
// largest degree in C (smallest id on ties).  One multi-source BFS from all
// v0_C at once computes every ecc_C, since the components are disjoint.  The
// BFS is level-synchronous and direction-optimising (top-down while the
// frontier's arcs are few, bottom-up once they are a large share of the graph).
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kad_internal.cuh"

namespace {

#define GERR_RANGE 1
#define GERR_SELF 2
#define GERR_ORDER 4
#define GERR_SYM 8
#define GERR_ROWPTR 16
#define GERR_CC 32

// Row pointers non-decreasing within [0, m] (thread per vertex), and every arc
// (v, w) with 0 <= w < n, w != v, and w above its predecessor in the row.  The
// arcs are checked 32 consecutive ones per thread (the row of the first found
// by binary search in row_ptr), so a hub's row is spread over many threads;
// with a bad row_ptr those reads stay in bounds and the row_ptr flag decides.
#define KAD_ROW_CHUNK 32
__global__ void k_validate_rows(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                                int64_t m, int *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t v = t0; v < n; v += stride) {
        const int a = rp[v], b = rp[v + 1];
        if (a > b || a < 0 || (int64_t)b > m) atomicOr(err, GERR_ROWPTR);
    }
    const int64_t chunks = (m + KAD_ROW_CHUNK - 1) / KAD_ROW_CHUNK;
    for (int64_t c = t0; c < chunks; c += stride) {
        const int64_t e0 = c * KAD_ROW_CHUNK;
        const int64_t e1 = (e0 + KAD_ROW_CHUNK < m) ? e0 + KAD_ROW_CHUNK : m;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)rp[mid] <= e0)
                lo = mid;
            else
                hi = mid - 1;
        }
        int v = lo;
        int64_t vbeg = rp[v], vend = rp[v + 1];
        int prev = -1;
        for (int64_t e = e0; e < e1; e++) {
            while (vend <= e && v < n - 1) {
                v++;
                vbeg = rp[v];
                vend = rp[v + 1];
            }
            const int w = col[e];
            if (w < 0 || w >= n) {
                atomicOr(err, GERR_RANGE);
            } else {
                if (w == v) atomicOr(err, GERR_SELF);
                if (e > vbeg && (e == e0 ? col[e - 1] : prev) >= w) atomicOr(err, GERR_ORDER);
            }
            prev = w;
        }
    }
}

// Symmetry, given sorted duplicate-free rows.  Rank the vertices by (degree,
// id) and call an arc (v, w) "up" when v ranks above w.  The graph is symmetric
// iff every up arc has its reverse (v in row w) and there are as many up arcs as
// down arcs: the reverse map sends up arcs into down arcs injectively, and equal
// counts make it a bijection, so every down arc has its reverse as well.  Only
// up arcs are searched for, so every search runs in the shorter of the two rows
// (on skewed graphs most arcs end at a hub, whose row is never searched).
// Arc-parallel: each thread takes 32 consecutive arcs, finds the row of the
// first by binary search in row_ptr and walks on, so a hub's row is spread over
// many threads.  counts[0] += up arcs, counts[1] += down arcs.  Runs after
// k_validate_rows has accepted row_ptr.
#define KAD_SYM_CHUNK 32
__global__ void k_validate_sym(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                               int64_t m, int *err, unsigned long long *counts) {
    unsigned long long up = 0, down = 0;
    const int64_t chunks = (m + KAD_SYM_CHUNK - 1) / KAD_SYM_CHUNK;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = c * KAD_SYM_CHUNK;
        const int64_t e1 = (e0 + KAD_SYM_CHUNK < m) ? e0 + KAD_SYM_CHUNK : m;
        // the row holding arc e0: the last v with rp[v] <= e0
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)rp[mid] <= e0)
                lo = mid;
            else
                hi = mid - 1;
        }
        int v = lo;
        int vend = rp[v + 1];
        // four arcs at a time, their binary searches interleaved, so that each
        // thread keeps four independent loads in flight
        for (int64_t e = e0; e < e1; e += 4) {
            int wk[4], vk[4], a[4], b[4], bend[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                wk[k] = -1;
                vk[k] = v;
                a[k] = b[k] = bend[k] = 0;
                if (e + k >= e1) continue;
                while ((int64_t)vend <= e + k && v < n - 1) {
                    v++;
                    vend = rp[v + 1];
                }
                vk[k] = v;
                const int w = col[e + k];
                if (w < 0 || w >= n) continue;
                wk[k] = w;
                a[k] = rp[w];
                b[k] = bend[k] = rp[w + 1];
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (wk[k] < 0) continue;
                // the arc is "up" when its tail ranks above its head by (degree,
                // id); only up arcs are searched, in the head's (shorter) row
                const int dv = rp[vk[k] + 1] - rp[vk[k]], dw = bend[k] - a[k];
                const bool upward = dv > dw || (dv == dw && vk[k] > wk[k]);
                if (upward) {
                    up++;
                } else {
                    down++;
                    wk[k] = -1;
                    a[k] = b[k] = 0;
                }
            }
            for (;;) {
                bool any = false;
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (a[k] >= b[k]) continue;
                    any = true;
                    const int mid = (a[k] + b[k]) >> 1;
                    if (col[mid] < vk[k])
                        a[k] = mid + 1;
                    else
                        b[k] = mid;
                }
                if (!any) break;
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (wk[k] >= 0 && (a[k] >= bend[k] || col[a[k]] != vk[k])) atomicOr(err, GERR_SYM);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        up += __shfl_xor_sync(0xffffffffu, up, o);
        down += __shfl_xor_sync(0xffffffffu, down, o);
    }
    if ((threadIdx.x & 31) == 0 && (up || down)) {
        atomicAdd(counts, up);
        atomicAdd(counts + 1, down);
    }
}

__global__ void k_check_ends(const int32_t *__restrict__ rp, int32_t n, int64_t m, int *err) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || (int64_t)rp[n] != m)) atomicOr(err, GERR_ROWPTR);
}

// ------------------------------------------------ connected components
// Union-find with hooking of the larger root under the smaller one, so the
// final root of a component is its smallest vertex id.
__global__ void k_cc_init(int32_t *parent, int32_t n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) parent[v] = v;
}

__device__ __forceinline__ int cc_find(int32_t *parent, int x, int32_t n) {
    // Pointer jumping; every value written is an ancestor, so races are benign.
    // Parent ids strictly decrease along a chain, so n steps always suffice.
    for (int guard = 0; guard <= n; guard++) {
        const int p = *(volatile int32_t *)(parent + x);
        if (p == x) return x;
        const int gp = *(volatile int32_t *)(parent + p);
        if (gp != p) *(volatile int32_t *)(parent + x) = gp;
        x = p;
    }
    return x;
}

// Join the trees of x and y: the larger root goes under the smaller (bounded
// retries; a run-out sets GERR_CC).
__device__ __forceinline__ void cc_link(int32_t *parent, int x, int y, int32_t n, int *err) {
    int guard = 0;
    for (;;) {
        int rx = cc_find(parent, x, n), ry = cc_find(parent, y, n);
        if (rx == ry) return;
        if (rx < ry) {
            const int t = rx;
            rx = ry;
            ry = t;
        }
        if (atomicCAS(parent + rx, rx, ry) == rx) return;
        x = rx;
        y = ry;
        if (++guard > (1 << 20)) {
            atomicOr(err, GERR_CC);
            return;
        }
    }
}

// Components by neighbour sampling (the order of links does not matter: every
// tree's root is its smallest id).  Rounds 0 and 1 link each vertex with its
// r-th neighbour; after compression, the most frequent root in a sample of
// vertices is taken as the large component, and only vertices outside it link
// with all their neighbours.  Every edge between two trees is then seen from a
// vertex outside the large one, so the result is the connected components.
__global__ void k_cc_sample(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                            int32_t *parent, int *err, int r) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (rp[v + 1] - rp[v] > r) cc_link(parent, v, col[rp[v] + r], n, err);
}

__global__ void k_cc_compress(int32_t *parent, int32_t n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        parent[v] = cc_find(parent, v, n);
}

// roots of `count` vertices spread evenly over the ids
__global__ void k_cc_probe(const int32_t *parent, int32_t n, int32_t *out, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = parent[(int)(((int64_t)i * n) / count)];
}

// `skip`: leading arcs of each row already linked by the sampling rounds (the
// in-arc rows of a directed graph had none linked: 0).
__global__ void k_cc_rest(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                          int32_t *parent, int *err, int big, int skip) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        if (*(volatile int32_t *)(parent + v) == big) continue; // inside the large tree
        const int a = rp[v], b = rp[v + 1];
        for (int e = a + skip + lane; e < b; e += 32) cc_link(parent, v, col[e], n, err);
    }
}

__global__ void k_cc_flatten(int32_t *parent, int32_t *comp, int32_t n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        comp[v] = cc_find(parent, v, n);
}

// best[root] = max over the component of (deg << 32) | (~v & 0xffffffff):
// largest degree, then smallest id.
__global__ void k_best_root(const int32_t *__restrict__ rp, const int32_t *__restrict__ comp, int32_t n,
                            unsigned long long *best) {
    // one atomic per warp when its vertices share a component (the common case:
    // one large component), else one per vertex
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        const bool in = v < n;
        const int c = in ? comp[v] : -1;
        const unsigned long long key =
            in ? (((unsigned long long)(uint32_t)(rp[v + 1] - rp[v]) << 32) | (0xffffffffu - (uint32_t)v)) : 0ull;
        const int c0 = __shfl_sync(0xffffffffu, c, 0);
        if (__all_sync(0xffffffffu, c == c0)) {
            unsigned long long k = key;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, k, o);
                k = (y > k) ? y : k;
            }
            if (lane == 0 && c0 >= 0) atomicMax(best + c0, k);
        } else if (in) {
            atomicMax(best + c, key);
        }
    }
}

// one BFS source per component (its best root); also the largest degree overall
__global__ void k_bfs_seed(const int32_t *__restrict__ comp, const unsigned long long *__restrict__ best, int32_t n,
                           int32_t *dist, int32_t *queue, int *qlen, int *ncomp, int *maxdeg) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (comp[v] == v) {
            const int src = (int)(0xffffffffu - (uint32_t)(best[v] & 0xffffffffull));
            dist[src] = 0;
            queue[atomicAdd(qlen, 1)] = src;
            atomicAdd(ncomp, 1);
            atomicMax(maxdeg, (int)(best[v] >> 32));
        }
    }
}

__global__ void k_fill(int32_t *p, int32_t n, int32_t val) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) p[v] = val;
}

// top-down: warp per frontier vertex, coalesced neighbour loads
__global__ void k_bfs_td(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                         const int32_t *__restrict__ q, int qlen, int parts, int32_t *dist, int32_t *nq, int *nqlen,
                         unsigned long long *narcs, int level) {
    // `parts` warps share each frontier vertex's row (a small frontier of hubs
    // would otherwise leave one warp with a whole hub row)
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)qlen * parts;
    for (int64_t it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += warps) {
        const int i = (int)(it / parts), part = (int)(it % parts);
        const int u = q[i];
        const int a = rp[u], b = rp[u + 1];
        for (int e = a + 32 * part + lane; e < b; e += 32 * parts) {
            const int w = col[e];
            if (*(volatile int32_t *)(dist + w) < 0 && atomicCAS(dist + w, -1, level + 1) == -1) {
                nq[atomicAdd(nqlen, 1)] = w;
                atomicAdd(narcs, (unsigned long long)(rp[w + 1] - rp[w]));
            }
        }
    }
}

// bottom-up: thread per unvisited vertex, stop at the first parent found
__global__ void k_bfs_bu(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n, int32_t *dist,
                         int32_t *nq, int *nqlen, unsigned long long *narcs, int level) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (dist[v] >= 0) continue;
        const int a = rp[v], b = rp[v + 1];
        for (int e = a; e < b; e++) {
            if (*(volatile int32_t *)(dist + col[e]) == level) {
                dist[v] = level + 1;
                nq[atomicAdd(nqlen, 1)] = v;
                atomicAdd(narcs, (unsigned long long)(b - a));
                break;
            }
        }
    }
}

// ------------------------------------------------ directed graphs
// The in-arc rows (the rows the t side expands along): a count of each head's
// arcs, a scan, a scatter, and a sort of every row, so that rows are ascending
// like the out-arc rows (the trace-back walks them in id order).

__global__ void k_tr_count(const int32_t *__restrict__ col, int64_t m, int32_t *cnt1) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt1 + col[e], 1);
}

// In-place inclusive scan of x[0, len) in tiles of KAD_SCAN_TILE (1024 threads x
// 4 items): tiles scanned alone, then the tile sums, then the offsets added.
#define KAD_SCAN_TILE 4096
__device__ __forceinline__ int block_excl_scan_1024(int v, int *wsum, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w; // inclusive per warp
    }
    __syncthreads();
    total = wsum[31];
    const int before = (wid > 0) ? wsum[wid - 1] : 0;
    __syncthreads(); // wsum is reused by the next call
    return before + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(int32_t *x, int64_t len, int32_t *tile_sum) {
    __shared__ int wsum[32];
    const int64_t base = (int64_t)blockIdx.x * KAD_SCAN_TILE + 4 * threadIdx.x;
    int v[4], run = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = (base + k < len) ? x[base + k] : 0;
        run += v[k];
        v[k] = run; // inclusive within the thread
    }
    int total;
    const int off = block_excl_scan_1024(run, wsum, total);
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (base + k < len) x[base + k] = v[k] + off;
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// one block: tile sums to exclusive offsets
__global__ void __launch_bounds__(1024) k_scan_sums(int32_t *tile_sum, int ntiles) {
    __shared__ int wsum[32];
    int carry = 0;
    for (int b = 0; b < ntiles; b += 1024) {
        const int i = b + (int)threadIdx.x;
        const int v = (i < ntiles) ? tile_sum[i] : 0;
        int total;
        const int ex = block_excl_scan_1024(v, wsum, total);
        if (i < ntiles) tile_sum[i] = carry + ex;
        carry += total;
    }
}

__global__ void k_scan_add(int32_t *x, int64_t len, const int32_t *__restrict__ tile_sum) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += tile_sum[i / KAD_SCAN_TILE];
}

// every arc u -> v into a free place of row v (warp per tail u)
__global__ void k_tr_fill(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                          const int32_t *__restrict__ rpT, int32_t *cursor, int32_t *colT) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps)
        for (int e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            const int v = col[e];
            colT[rpT[v] + atomicAdd(cursor + v, 1)] = u;
        }
}

// Rows of up to 32 arcs are sorted by their thread (insertion sort); longer
// ones are listed for the warp sort (up to KAD_SORT_WARP arcs), the block sort
// (up to KAD_SORT_MID) or the bitmap sort.
#define KAD_SORT_WARP 256
#define KAD_SORT_MID 4096
__global__ void k_tr_sort_small(const int32_t *__restrict__ rpT, int32_t *colT, int32_t n, int32_t *wl, int *nwl,
                                int32_t *mid, int *nmid, int32_t *big, int *nbig) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int a = rpT[v], len = rpT[v + 1] - a;
        if (len > KAD_SORT_MID) {
            big[atomicAdd(nbig, 1)] = v;
        } else if (len > KAD_SORT_WARP) {
            mid[atomicAdd(nmid, 1)] = v;
        } else if (len > 32) {
            wl[atomicAdd(nwl, 1)] = v;
        } else if (len > 1) {
            int buf[32];
            for (int i = 0; i < len; i++) {
                const int x = colT[a + i];
                int j = i;
                while (j > 0 && buf[j - 1] > x) {
                    buf[j] = buf[j - 1];
                    j--;
                }
                buf[j] = x;
            }
            for (int i = 0; i < len; i++) colT[a + i] = buf[i];
        }
    }
}

// a warp per listed row of at most KAD_SORT_WARP arcs: the row goes to shared
// memory, and each element is written at its rank, the number of smaller
// elements (the ids of a row are distinct)
__global__ void __launch_bounds__(256) k_tr_sort_warp(const int32_t *__restrict__ rpT, int32_t *colT,
                                                      const int32_t *__restrict__ wl, int nwl) {
    __shared__ int sh[8][KAD_SORT_WARP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nwl; r += warps) {
        const int v = wl[r];
        const int a = rpT[v], len = rpT[v + 1] - a;
        for (int i = lane; i < len; i += 32) sh[w][i] = colT[a + i];
        __syncwarp();
        for (int i = lane; i < len; i += 32) {
            const int x = sh[w][i];
            int rank = 0;
            for (int j = 0; j < len; j++) rank += (sh[w][j] < x) ? 1 : 0;
            colT[a + rank] = x;
        }
        __syncwarp();
    }
}

// a block per listed row: bitonic sort in shared memory, padded to a power of two
__global__ void __launch_bounds__(1024) k_tr_sort_mid(const int32_t *__restrict__ rpT, int32_t *colT,
                                                      const int32_t *__restrict__ mid, int nmid) {
    __shared__ int sh[KAD_SORT_MID];
    for (int r = blockIdx.x; r < nmid; r += gridDim.x) {
        const int v = mid[r];
        const int a = rpT[v], len = rpT[v + 1] - a;
        int P = 64;
        while (P < len) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = (i < len) ? colT[a + i] : 0x7fffffff;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const int x = sh[i], y = sh[ixj];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) {
                            sh[i] = y;
                            sh[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x) colT[a + i] = sh[i];
        __syncthreads();
    }
}

// a block per listed long row: the row's ids marked in a bitmap over all n
// vertices (its own slice of `bits`), then read back in id order
__global__ void __launch_bounds__(1024) k_tr_sort_big(const int32_t *__restrict__ rpT, int32_t *colT,
                                                      const int32_t *__restrict__ big, int nbig, int32_t n,
                                                      uint32_t *bits) {
    __shared__ int wsum[32];
    const int words = (n + 31) >> 5;
    uint32_t *mine = bits + (size_t)blockIdx.x * (size_t)words;
    for (int r = blockIdx.x; r < nbig; r += gridDim.x) {
        const int v = big[r];
        const int a = rpT[v], len = rpT[v + 1] - a;
        for (int i = threadIdx.x; i < words; i += blockDim.x) mine[i] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            const int x = colT[a + i];
            atomicOr(mine + (x >> 5), 1u << (x & 31));
        }
        __syncthreads();
        int carry = 0;
        for (int b = 0; b < words; b += 1024) {
            const int i = b + (int)threadIdx.x;
            const uint32_t w = (i < words) ? mine[i] : 0u;
            int total;
            int pos = carry + block_excl_scan_1024(__popc(w), wsum, total);
            for (uint32_t q = w; q; q &= q - 1) colT[a + pos++] = (i << 5) + __ffs(q) - 1;
            carry += total;
        }
        __syncthreads();
    }
}

// ------------------------------------------------ strongly connected components
// scc[v] = -1 while unassigned, else the id of its component's colour root.
// A component is assigned whole, so a vertex whose unassigned in-neighbours (or
// out-neighbours) are none is a component of its own (trim).
__device__ __forceinline__ bool any_unassigned(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                               const int32_t *scc, int v) {
    for (int e = rp[v]; e < rp[v + 1]; e++)
        if (*(volatile const int32_t *)(scc + col[e]) < 0) return true;
    return false;
}

__global__ void k_scc_trim(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const int32_t *__restrict__ rpT, const int32_t *__restrict__ colT, int32_t n, int32_t *scc,
                           int *count) {
    int c = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (scc[v] >= 0) continue;
        if (!any_unassigned(rpT, colT, scc, v) || !any_unassigned(rp, col, scc, v)) {
            scc[v] = v;
            c++;
        }
    }
    if (c) atomicAdd(count, c);
}

// colour[v] = v for the unassigned; all of them start active
__global__ void k_scc_color_init(const int32_t *__restrict__ scc, int32_t n, int32_t *color, int32_t *q, int *qlen) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (scc[v] < 0) {
            color[v] = v;
            q[atomicAdd(qlen, 1)] = v;
        }
}

// colours flow forward along arcs between unassigned vertices, the larger one
// winning: at the fixed point colour[v] is the largest id among the unassigned
// vertices that reach v (warp per active vertex; a raised vertex is active in
// the next step, once: stamp)
__global__ void k_scc_color_push(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const int32_t *__restrict__ q, int qlen, const int32_t *scc, int32_t *color,
                                 int32_t *stamp, int step, int32_t *nq, int *nqlen) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < qlen; i += warps) {
        const int u = q[i];
        const int c = *(volatile int32_t *)(color + u);
        for (int e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            const int x = col[e];
            if (*(volatile const int32_t *)(scc + x) >= 0 || *(volatile int32_t *)(color + x) >= c) continue;
            if (atomicMax(color + x, c) < c && atomicExch(stamp + x, step) != step) nq[atomicAdd(nqlen, 1)] = x;
        }
    }
}

// the roots: unassigned vertices that keep their own colour
__global__ void k_scc_roots(int32_t *scc, const int32_t *__restrict__ color, int32_t n, int32_t *q, int *qlen) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (scc[v] < 0 && color[v] == v) {
            scc[v] = v;
            q[atomicAdd(qlen, 1)] = v;
        }
}

// backward from every root among vertices of its colour: the vertices of that
// colour that reach the root are exactly its strongly connected component
__global__ void k_scc_back(const int32_t *__restrict__ rpT, const int32_t *__restrict__ colT,
                           const int32_t *__restrict__ q, int qlen, int32_t *scc, const int32_t *__restrict__ color,
                           int32_t *nq, int *nqlen) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < qlen; i += warps) {
        const int v = q[i];
        const int c = color[v];
        for (int e = rpT[v] + lane; e < rpT[v + 1]; e += 32) {
            const int u = colT[e];
            if (color[u] == c && *(volatile int32_t *)(scc + u) < 0 && atomicCAS(scc + u, -1, c) == -1)
                nq[atomicAdd(nqlen, 1)] = u;
        }
    }
}

// The forward-backward step for the component of the pivot p, the unassigned
// vertex of largest out- plus in-degree (smallest id on ties; so p is r_S of
// its component): the vertices reached from p and reaching p, over unassigned
// vertices, are its component, and their distances from and to p are within it
// (a path between two vertices of one component never leaves it), so they give
// ecc_out(p) and ecc_in(p) directly.
__global__ void k_scc_pivot(const int32_t *__restrict__ rp, const int32_t *__restrict__ rpT,
                            const int32_t *__restrict__ scc, int32_t n, unsigned long long *key) {
    unsigned long long best = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (scc[v] < 0) {
            const uint32_t d = (uint32_t)(rp[v + 1] - rp[v]) + (uint32_t)(rpT[v + 1] - rpT[v]);
            const unsigned long long k = ((unsigned long long)d << 32) | (0xffffffffu - (uint32_t)v);
            best = (k > best) ? k : best;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
        best = (y > best) ? y : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

__global__ void k_pivot_seed(const unsigned long long *__restrict__ key, int32_t *dist, int32_t *q) {
    const int p = (int)(0xffffffffu - (uint32_t)(*key & 0xffffffffull));
    dist[p] = 0;
    q[0] = p;
}

// one BFS level over unassigned vertices (warp per frontier vertex, `parts`
// warps per row when the frontier is small)
__global__ void k_reach_bfs(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ scc, const int32_t *__restrict__ q, int qlen, int parts,
                            int32_t *dist, int level, int32_t *nq, int *nqlen, unsigned long long *narcs) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)qlen * parts;
    for (int64_t it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += warps) {
        const int i = (int)(it / parts), part = (int)(it % parts);
        const int u = q[i];
        for (int e = rp[u] + 32 * part + lane; e < rp[u + 1]; e += 32 * parts) {
            const int x = col[e];
            if (scc[x] < 0 && *(volatile int32_t *)(dist + x) < 0 && atomicCAS(dist + x, -1, level + 1) == -1) {
                nq[atomicAdd(nqlen, 1)] = x;
                atomicAdd(narcs, (unsigned long long)(rp[x + 1] - rp[x]));
            }
        }
    }
}

// the same level bottom-up: each unvisited unassigned vertex looks for a parent
// at `level` among the tails of its rows in the other direction (rpo/colo);
// rp gives the degrees counted for the direction switch
__global__ void k_reach_bu(const int32_t *__restrict__ rp, const int32_t *__restrict__ rpo,
                           const int32_t *__restrict__ colo, const int32_t *__restrict__ scc, int32_t n, int32_t *dist,
                           int level, int32_t *nq, int *nqlen, unsigned long long *narcs) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        if (dist[x] >= 0 || scc[x] >= 0) continue;
        for (int e = rpo[x]; e < rpo[x + 1]; e++) {
            if (*(volatile int32_t *)(dist + colo[e]) == level) {
                dist[x] = level + 1;
                nq[atomicAdd(nqlen, 1)] = x;
                atomicAdd(narcs, (unsigned long long)(rp[x + 1] - rp[x]));
                break;
            }
        }
    }
}

// the pivot's component: reached both ways; its eccentricities from the distances
__global__ void k_scc_fwbw(int32_t *scc, const int32_t *__restrict__ df, const int32_t *__restrict__ db, int32_t n,
                           const unsigned long long *__restrict__ key, int32_t *e_out, int32_t *e_in, int *count) {
    const int p = (int)(0xffffffffu - (uint32_t)(*key & 0xffffffffull));
    int c = 0, mf = 0, mb = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (scc[v] < 0 && df[v] >= 0 && db[v] >= 0) {
            scc[v] = p;
            c++;
            mf = (df[v] > mf) ? df[v] : mf;
            mb = (db[v] > mb) ? db[v] : mb;
        }
    c = __reduce_add_sync(0xffffffffu, c);
    mf = __reduce_max_sync(0xffffffffu, mf);
    mb = __reduce_max_sync(0xffffffffu, mb);
    if ((threadIdx.x & 31) == 0 && c) {
        atomicAdd(count, c);
        atomicMax(e_out + p, mf);
        atomicMax(e_in + p, mb);
    }
}

// per component (indexed by its label): size, and the root r_S of largest
// out- plus in-degree, smallest id on ties, as (deg << 32) | ~v
__global__ void k_scc_stats(const int32_t *__restrict__ rp, const int32_t *__restrict__ rpT,
                            const int32_t *__restrict__ scc, int32_t n, int32_t *size, unsigned long long *best,
                            int *maxdeg, int *err) {
    // one atomic per warp when its vertices share a component (most of a large
    // component's vertices), else one per vertex
    const int lane = threadIdx.x & 31;
    int md = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        int s = -1;
        unsigned long long key = 0;
        if (v < n) {
            s = scc[v];
            if (s < 0 || s >= n) { // every vertex is assigned by now; checked, not assumed
                atomicOr(err, GERR_CC);
                s = -1;
            } else {
                const uint32_t d = (uint32_t)(rp[v + 1] - rp[v]) + (uint32_t)(rpT[v + 1] - rpT[v]);
                key = ((unsigned long long)d << 32) | (0xffffffffu - (uint32_t)v);
                md = ((int)d > md) ? (int)d : md;
            }
        }
        const int s0 = __shfl_sync(0xffffffffu, s, 0);
        if (__all_sync(0xffffffffu, s == s0)) {
            unsigned long long k = key;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, k, o);
                k = (y > k) ? y : k;
            }
            if (lane == 0 && s0 >= 0) {
                atomicAdd(size + s0, 32);
                atomicMax(best + s0, k);
            }
        } else if (s >= 0) {
            atomicAdd(size + s, 1);
            atomicMax(best + s, key);
        }
    }
    md = __reduce_max_sync(0xffffffffu, md);
    if (lane == 0 && md) atomicMax(maxdeg, md);
}

// how many v have lab[v] == v (component labels: one per component)
__global__ void k_count_self(const int32_t *__restrict__ lab, int32_t n, int *count) {
    int c = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) c += (lab[v] == v);
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// BFS sources: the roots of components of two or more vertices, except the
// pivot's (its eccentricities are known; a single vertex has none)
__global__ void k_scc_seed(const int32_t *__restrict__ scc, const unsigned long long *__restrict__ best,
                           const int32_t *__restrict__ size, const unsigned long long *__restrict__ pivot, int32_t n,
                           int32_t *dist, int32_t *q, int *qlen) {
    const int p = *pivot ? (int)(0xffffffffu - (uint32_t)(*pivot & 0xffffffffull)) : -1;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (scc[v] == v && size[v] > 1 && v != p) {
            const int r = (int)(0xffffffffu - (uint32_t)(best[v] & 0xffffffffull));
            dist[r] = 0;
            q[atomicAdd(qlen, 1)] = r;
        }
}

// one BFS level from every component's root at once, over arcs inside the
// component (rows: out-arcs for ecc_out, in-arcs for ecc_in); ecc[label] is
// raised to the level reached
__global__ void k_scc_bfs(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                          const int32_t *__restrict__ scc, const int32_t *__restrict__ q, int qlen, int parts,
                          int32_t *dist, int level, int32_t *ecc, int32_t *nq, int *nqlen) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int64_t items = (int64_t)qlen * parts;
    for (int64_t it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += warps) {
        const int i = (int)(it / parts), part = (int)(it % parts);
        const int u = q[i];
        const int s = scc[u];
        bool any = false;
        for (int e = rp[u] + 32 * part + lane; e < rp[u + 1]; e += 32 * parts) {
            const int x = col[e];
            if (scc[x] == s && *(volatile int32_t *)(dist + x) < 0 && atomicCAS(dist + x, -1, level + 1) == -1) {
                nq[atomicAdd(nqlen, 1)] = x;
                any = true;
            }
        }
        if (__any_sync(0xffffffffu, any) && lane == 0) atomicMax(ecc + s, level + 1);
    }
}

// w(S) = min(|S|, ecc_in + ecc_out + 1); B(S) starts at w(S)
__global__ void k_scc_weight(const int32_t *__restrict__ scc, int32_t n, const int32_t *__restrict__ size,
                             const int32_t *__restrict__ e_out, const int32_t *__restrict__ e_in, int32_t *w,
                             int32_t *B) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (scc[v] == v) {
            const int64_t x = (int64_t)e_out[v] + e_in[v] + 1;
            w[v] = (x < size[v]) ? (int32_t)x : size[v];
            B[v] = w[v];
        }
}

// every arc e as pairs[e] = (S, S') when it joins two components, else (-1, -1)
// (warp per vertex; each arc keeps its own slot, so no counter is shared)
__global__ void k_chain_arcs(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const int32_t *__restrict__ scc, int32_t n, int2 *pairs) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int su = scc[u];
        for (int e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            const int sv = scc[col[e]];
            const bool cross = su >= 0 && su < n && sv != su && sv >= 0 && sv < n;
            pairs[e] = cross ? make_int2(su, sv) : make_int2(-1, -1);
        }
    }
}

// one relaxation of B(S) = w(S) + B(S') over the arcs between components; sets
// *changed when some B grew.  Repeated until nothing changes: the components'
// graph is acyclic, so B stops at the heaviest chain below S.
__global__ void k_chain_relax(const int2 *__restrict__ pairs, int64_t npairs, const int32_t *__restrict__ w,
                              int32_t *B, int *changed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npairs; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 p = pairs[i];
        if (p.x < 0) continue;
        const int cand = w[p.x] + *(volatile int32_t *)(B + p.y);
        if (cand > *(volatile int32_t *)(B + p.x) && atomicMax(B + p.x, cand) < cand) atomicOr(changed, 1);
    }
}

// one relaxation of B(S) = w(S) + max over arcs S -> S' of B(S') (warp per
// vertex); sets *changed when some B grew.  Repeated until nothing changes: the
// components' graph is acyclic, so B stops at the heaviest chain below S.
__global__ void k_scc_chain(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ scc, int32_t n, const int32_t *__restrict__ w, int32_t *B,
                            int *changed) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int su = scc[u];
        if (su < 0 || su >= n) continue; // (k_scc_stats has flagged it)
        int best = 0;
        for (int e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            const int sv = scc[col[e]];
            if (sv != su && sv >= 0 && sv < n) {
                const int b = *(volatile int32_t *)(B + sv);
                best = (b > best) ? b : best;
            }
        }
        best = __reduce_max_sync(0xffffffffu, best);
        if (lane == 0 && best > 0) {
            const int cand = w[su] + best;
            if (cand > *(volatile int32_t *)(B + su) && atomicMax(B + su, cand) < cand) atomicOr(changed, 1);
        }
    }
}

__global__ void k_scc_vd(const int32_t *__restrict__ scc, const int32_t *__restrict__ B, int32_t n, int *vd,
                         int *nscc) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (scc[v] == v) {
            atomicMax(vd, B[v]);
            atomicAdd(nscc, 1);
        }
}

// ------------------------------------------------ double sweep (opt-in)
// key[comp root] = max over the component of (dist << 32) | ~v: the farthest
// vertex, smallest id on ties (dist >= 0 for every vertex after a BFS from
// every component)
__global__ void k_far(const int32_t *__restrict__ comp, const int32_t *__restrict__ dist, int32_t n,
                      unsigned long long *key) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        const bool in = v < n && dist[v] >= 0;
        const int c = in ? comp[v] : -1;
        const unsigned long long k =
            in ? (((unsigned long long)(uint32_t)dist[v] << 32) | (0xffffffffu - (uint32_t)v)) : 0ull;
        const int c0 = __shfl_sync(0xffffffffu, c, 0);
        if (__all_sync(0xffffffffu, c == c0)) {
            unsigned long long x = k;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
                x = (y > x) ? y : x;
            }
            if (lane == 0 && c0 >= 0) atomicMax(key + c0, x);
        } else if (in) {
            atomicMax(key + c, k);
        }
    }
}

// one BFS source per component: the vertex in the low word of key[root], stored
// as ~v (inverted = 1, from k_far) or as v (inverted = 0, from k_mid)
__global__ void k_seed_key(const int32_t *__restrict__ comp, const unsigned long long *__restrict__ key, int32_t n,
                           int inverted, int32_t *dist, int32_t *q, int *qlen) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (comp[v] == v) {
            const uint32_t lo = (uint32_t)(key[v] & 0xffffffffull);
            const int src = (int)(inverted ? 0xffffffffu - lo : lo);
            if (src < 0 || src >= n) continue; // cannot happen: every component has a vertex
            dist[src] = 0;
            q[atomicAdd(qlen, 1)] = src;
        }
}

// key_m[root] = min over the component's midpoints x (d(a,x) + d(x,b) = d(a,b)
// and d(a,x) = ceil(d(a,b)/2)) of (d(v0,x) << 32) | x
__global__ void k_mid(const int32_t *__restrict__ comp, const int32_t *__restrict__ d0, const int32_t *__restrict__ da,
                      const int32_t *__restrict__ db, const unsigned long long *__restrict__ key_b, int32_t n,
                      unsigned long long *key_m) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int c = comp[v];
        const int d = (int)(key_b[c] >> 32);
        if (da[v] + db[v] == d && da[v] == (d + 1) / 2)
            atomicMin(key_m + c, ((unsigned long long)(uint32_t)d0[v] << 32) | (uint32_t)v);
    }
}

// VD = max over components of 2 min(ecc(v0), ecc(m)) + 1
__global__ void k_tight_vd(const int32_t *__restrict__ comp, const unsigned long long *__restrict__ key_a,
                           const unsigned long long *__restrict__ key_e, int32_t n, int *vd) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (comp[v] == v) {
            const int e0 = (int)(key_a[v] >> 32), em = (int)(key_e[v] >> 32);
            atomicMax(vd, 2 * (em < e0 ? em : e0) + 1);
        }
}

int grid_for(int64_t work, int threads, int cap) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

} // namespace

#define GCHK(x)                                                                                                       \
    do {                                                                                                              \
        cudaError_t e_ = (x);                                                                                         \
        if (e_ != cudaSuccess) {                                                                                      \
            *cerr = e_;                                                                                               \
            status = KAD_ERR_CUDA;                                                                                    \
            goto done;                                                                                                \
        }                                                                                                             \
    } while (0)

// Directed graph set-up, after the out-arc rows were validated: the in-arc rows
// (sorted), the weak components (the pair check of Appendix C.1: no path joins
// two of them), and the vertex-diameter bound through the strongly connected
// components -- a shortest path runs through a chain S_1 -> ... -> S_k of the
// components' DAG and spends at most w(S) = min(|S|, ecc_in(r_S) + ecc_out(r_S) + 1)
// vertices in each, r_S the vertex of largest out- plus in-degree (smallest id
// on ties), so VD = the heaviest chain.  The components: trim vertices with no
// unassigned in- or out-neighbour (components of their own) until none is left,
// which removes every vertex on no cycle (a chain of n costs about n/2 passes); one
// forward-backward step from the unassigned vertex of largest out+in degree
// (its component, on skewed graphs the large one, with its eccentricities); the
// rest by colour propagation (each unassigned vertex takes the largest id that
// reaches it; the vertices of a colour that reach its root form the root's
// component).  Every loop below ends: each pass of the outer loop assigns at
// least the largest unassigned id, and each inner loop runs until its frontier
// is empty.
static kad_status setup_directed(KadGraphDev &gd, cudaStream_t st, int32_t *vd_out, int32_t *ncomp_out, int32_t *maxdeg_out,
                          cudaError_t *cerr) {
    const int32_t n = gd.n;
    const int64_t m = gd.m;
    const int T = 256;
    const int gv = grid_for(n, T, 65535);
    const int gw = grid_for((int64_t)n * 32, T, 65535);
    const int ga = grid_for(m, T, 65535);
    const int ntiles = (int)(((int64_t)n + 1 + KAD_SCAN_TILE - 1) / KAD_SCAN_TILE);
    const size_t a4 = (((size_t)n * 4) + 255) & ~(size_t)255, a8 = (((size_t)n * 8) + 255) & ~(size_t)255;
    const size_t at = (((size_t)ntiles * 4) + 255) & ~(size_t)255;
    kad_status status = KAD_OK;
    char *scratch = nullptr;
    uint32_t *bits = nullptr;
    int2 *pairs = nullptr; // the arcs between components, for the heaviest chain
    int *d_cnt = nullptr; // [0] error flags, [1..3] counters, [4] changed, [5] vd, [6] count, [7] largest degree
    unsigned long long *pivot = nullptr; // the forward-backward pivot's key (after the counters)
    unsigned long long *d_arcs = nullptr; // arcs of a BFS frontier (direction switch)
    int32_t *parent, *scc, *color, *stamp, *q0, *q1, *dist, *size, *e_out, *e_in, *wt, *B, *tiles;
    unsigned long long *best;
    int h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int nmid = 0, nbig = 0, remaining = n, step = 0, qlen = 0, level = 0;
    int32_t *qa, *qb;
    if (kad_pool_alloc((void **)&scratch, 256 + 12 * a4 + a8 + at, st) != cudaSuccess ||
        kad_pool_alloc((void **)&gd.rpT, ((size_t)n + 1) * 4, st) != cudaSuccess ||
        kad_pool_alloc((void **)&gd.colT, (size_t)(m > 0 ? m : 1) * 4, st) != cudaSuccess) {
        cudaGetLastError();
        status = KAD_ERR_OOM;
        goto done;
    }
    d_cnt = (int *)scratch;
    pivot = (unsigned long long *)(scratch + 64);
    d_arcs = (unsigned long long *)(scratch + 72);
    parent = (int32_t *)(scratch + 256);
    scc = (int32_t *)(scratch + 256 + a4);
    color = (int32_t *)(scratch + 256 + 2 * a4);
    stamp = (int32_t *)(scratch + 256 + 3 * a4);
    q0 = (int32_t *)(scratch + 256 + 4 * a4);
    q1 = (int32_t *)(scratch + 256 + 5 * a4);
    dist = (int32_t *)(scratch + 256 + 6 * a4);
    size = (int32_t *)(scratch + 256 + 7 * a4);
    e_out = (int32_t *)(scratch + 256 + 8 * a4);
    e_in = (int32_t *)(scratch + 256 + 9 * a4);
    wt = (int32_t *)(scratch + 256 + 10 * a4);
    B = (int32_t *)(scratch + 256 + 11 * a4);
    best = (unsigned long long *)(scratch + 256 + 12 * a4);
    tiles = (int32_t *)(scratch + 256 + 12 * a4 + a8);
    GCHK(cudaMemsetAsync(d_cnt, 0, 8 * sizeof(int), st));

    // ---- in-arc rows: counts, scan, scatter, per-row sort
    GCHK(cudaMemsetAsync(gd.rpT, 0, ((size_t)n + 1) * 4, st));
    k_tr_count<<<ga, T, 0, st>>>(gd.col, m, gd.rpT + 1);
    k_scan_tiles<<<ntiles, 1024, 0, st>>>(gd.rpT, (int64_t)n + 1, tiles);
    k_scan_sums<<<1, 1024, 0, st>>>(tiles, ntiles);
    k_scan_add<<<grid_for((int64_t)n + 1, T, 65535), T, 0, st>>>(gd.rpT, (int64_t)n + 1, tiles);
    GCHK(cudaMemsetAsync(parent, 0, (size_t)n * 4, st)); // the scatter cursors
    k_tr_fill<<<gw, T, 0, st>>>(gd.rp, gd.col, n, gd.rpT, parent, gd.colT);
    k_tr_sort_small<<<gv, T, 0, st>>>(gd.rpT, gd.colT, n, dist, d_cnt + 3, q0, d_cnt + 1, q1, d_cnt + 2);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_cnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    nmid = h[1];
    nbig = h[2];
    if (h[3] > 0) k_tr_sort_warp<<<grid_for((int64_t)h[3] * 32, T, 65535), T, 0, st>>>(gd.rpT, gd.colT, dist, h[3]);
    if (nmid > 0) k_tr_sort_mid<<<(nmid < 2048 ? nmid : 2048), 1024, 0, st>>>(gd.rpT, gd.colT, q0, nmid);
    if (nbig > 0) {
        const int gb = nbig < 64 ? nbig : 64;
        if (kad_pool_alloc((void **)&bits, (size_t)gb * (size_t)((n + 31) / 32) * 4, st) != cudaSuccess) {
            cudaGetLastError();
            status = KAD_ERR_OOM;
            goto done;
        }
        k_tr_sort_big<<<gb, 1024, 0, st>>>(gd.rpT, gd.colT, q1, nbig, n, bits);
    }
    GCHK(cudaGetLastError());

    // ---- weak components: union-find over the out-arc and the in-arc rows
    k_cc_init<<<gv, T, 0, st>>>(parent, n);
    for (int r = 0; r < 2; r++) k_cc_sample<<<gv, T, 0, st>>>(gd.rp, gd.col, n, parent, d_cnt, r);
    k_cc_compress<<<gv, T, 0, st>>>(parent, n);
    {
        const int probes = (n < 1024) ? n : 1024;
        int32_t h_probe[1024];
        k_cc_probe<<<(probes + T - 1) / T, T, 0, st>>>(parent, n, q0, probes);
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h_probe, q0, (size_t)probes * 4, cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        std::sort(h_probe, h_probe + probes);
        int big = h_probe[0], best_run = 0;
        for (int i = 0; i < probes;) {
            int j = i;
            while (j < probes && h_probe[j] == h_probe[i]) j++;
            if (j - i > best_run) {
                best_run = j - i;
                big = h_probe[i];
            }
            i = j;
        }
        // an arc with an endpoint outside the large tree is linked from that
        // endpoint: from the tail's out-arc row or from the head's in-arc row
        k_cc_rest<<<gw, T, 0, st>>>(gd.rp, gd.col, n, parent, d_cnt, big, 2);
        k_cc_rest<<<gw, T, 0, st>>>(gd.rpT, gd.colT, n, parent, d_cnt, big, 0);
    }
    k_cc_flatten<<<gv, T, 0, st>>>(parent, gd.comp, n);
    k_count_self<<<gv, T, 0, st>>>(gd.comp, n, d_cnt + 6);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_cnt, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    if (h[0] & GERR_CC) {
        status = KAD_ERR_INTERNAL;
        goto done;
    }
    *ncomp_out = h[6];

    // ---- strongly connected components
    k_fill<<<gv, T, 0, st>>>(scc, n, -1);
    k_fill<<<gv, T, 0, st>>>(stamp, n, -1);
    GCHK(cudaMemsetAsync(e_out, 0, (size_t)n * 4, st));
    GCHK(cudaMemsetAsync(e_in, 0, (size_t)n * 4, st));
    GCHK(cudaMemsetAsync(pivot, 0, sizeof(unsigned long long), st));
    GCHK(cudaGetLastError());
    for (int pass = 0; pass <= n && remaining > 0; pass++) { // to the fixed point
        GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
        k_scc_trim<<<gv, T, 0, st>>>(gd.rp, gd.col, gd.rpT, gd.colT, n, scc, d_cnt + 1);
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        remaining -= h[1];
        if (h[1] == 0) break;
    }
    if (remaining > 0) {
        // forward-backward from the pivot (on skewed graphs: the large component)
        k_scc_pivot<<<gv, T, 0, st>>>(gd.rp, gd.rpT, scc, n, pivot);
        for (int z = 0; z < 2; z++) {
            const int32_t *rows = z ? gd.rpT : gd.rp, *cols = z ? gd.colT : gd.col;
            int32_t *dz = z ? dist : color;
            k_fill<<<gv, T, 0, st>>>(dz, n, -1);
            k_pivot_seed<<<1, 1, 0, st>>>(pivot, dz, q0);
            GCHK(cudaGetLastError());
            qlen = 1;
            qa = q0;
            qb = q1;
            unsigned long long arcs = 0; // unknown for the seed level: start top-down
            for (level = 0; qlen > 0; level++) {
                GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
                GCHK(cudaMemsetAsync(d_arcs, 0, sizeof(unsigned long long), st));
                if ((int64_t)arcs * 14 > m && qlen > n / 64) {
                    // a frontier with a large share of the arcs: bottom-up over the
                    // other direction's rows
                    k_reach_bu<<<gv, T, 0, st>>>(rows, z ? gd.rp : gd.rpT, z ? gd.col : gd.colT, scc, n, dz, level,
                                                 qb, d_cnt + 1, d_arcs);
                } else {
                    const int parts = (qlen >= 9728) ? 1 : (9728 + qlen - 1) / qlen;
                    k_reach_bfs<<<grid_for((int64_t)qlen * parts * 32, T, 65535), T, 0, st>>>(
                        rows, cols, scc, qa, qlen, parts, dz, level, qb, d_cnt + 1, d_arcs);
                }
                GCHK(cudaGetLastError());
                GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
                GCHK(cudaMemcpyAsync(&arcs, d_arcs, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
                GCHK(cudaStreamSynchronize(st));
                qlen = h[1];
                int32_t *t = qa;
                qa = qb;
                qb = t;
            }
        }
        GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
        k_scc_fwbw<<<gv, T, 0, st>>>(scc, color, dist, n, pivot, e_out, e_in, d_cnt + 1);
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        remaining -= h[1];
    }
    // the rest by colour propagation
    for (int outer = 0; remaining > 0; outer++) {
        if (outer > n) { // cannot happen: every pass assigns the largest unassigned id
            status = KAD_ERR_INTERNAL;
            goto done;
        }
        for (int pass = 0; pass <= n && remaining > 0; pass++) { // to the fixed point
            GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
            k_scc_trim<<<gv, T, 0, st>>>(gd.rp, gd.col, gd.rpT, gd.colT, n, scc, d_cnt + 1);
            GCHK(cudaGetLastError());
            GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
            GCHK(cudaStreamSynchronize(st));
            remaining -= h[1];
            if (h[1] == 0) break;
        }
        if (remaining <= 0) break;
        GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
        k_scc_color_init<<<gv, T, 0, st>>>(scc, n, color, q0, d_cnt + 1);
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        qlen = h[1];
        qa = q0;
        qb = q1;
        while (qlen > 0) {
            GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
            k_scc_color_push<<<grid_for((int64_t)qlen * 32, T, 65535), T, 0, st>>>(gd.rp, gd.col, qa, qlen, scc, color,
                                                                                   stamp, step++, qb, d_cnt + 1);
            GCHK(cudaGetLastError());
            GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
            GCHK(cudaStreamSynchronize(st));
            qlen = h[1];
            int32_t *t = qa;
            qa = qb;
            qb = t;
        }
        GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
        k_scc_roots<<<gv, T, 0, st>>>(scc, color, n, q0, d_cnt + 1);
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        qlen = h[1];
        remaining -= qlen;
        qa = q0;
        qb = q1;
        while (qlen > 0) {
            GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
            k_scc_back<<<grid_for((int64_t)qlen * 32, T, 65535), T, 0, st>>>(gd.rpT, gd.colT, qa, qlen, scc, color, qb,
                                                                             d_cnt + 1);
            GCHK(cudaGetLastError());
            GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
            GCHK(cudaStreamSynchronize(st));
            qlen = h[1];
            remaining -= qlen;
            int32_t *t = qa;
            qa = qb;
            qb = t;
        }
    }

    // ---- per component: size, root, eccentricities within it, weight
    GCHK(cudaMemsetAsync(size, 0, (size_t)n * 4, st));
    GCHK(cudaMemsetAsync(best, 0, (size_t)n * 8, st));
    k_scc_stats<<<gv, T, 0, st>>>(gd.rp, gd.rpT, scc, n, size, best, d_cnt + 7, d_cnt);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    if (h[0]) {
        status = KAD_ERR_INTERNAL;
        goto done;
    }
    for (int z = 0; z < 2; z++) {
        const int32_t *rows = z ? gd.rpT : gd.rp, *cols = z ? gd.colT : gd.col;
        k_fill<<<gv, T, 0, st>>>(dist, n, -1);
        GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
        k_scc_seed<<<gv, T, 0, st>>>(scc, best, size, pivot, n, dist, q0, d_cnt + 1);
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        qlen = h[1];
        qa = q0;
        qb = q1;
        for (level = 0; qlen > 0; level++) {
            const int parts = (qlen >= 9728) ? 1 : (9728 + qlen - 1) / qlen;
            GCHK(cudaMemsetAsync(d_cnt + 1, 0, sizeof(int), st));
            k_scc_bfs<<<grid_for((int64_t)qlen * parts * 32, T, 65535), T, 0, st>>>(
                rows, cols, scc, qa, qlen, parts, dist, level, z ? e_in : e_out, qb, d_cnt + 1);
            GCHK(cudaGetLastError());
            GCHK(cudaMemcpyAsync(h + 1, d_cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
            GCHK(cudaStreamSynchronize(st));
            qlen = h[1];
            int32_t *t = qa;
            qa = qb;
            qb = t;
        }
    }
    k_scc_weight<<<gv, T, 0, st>>>(scc, n, size, e_out, e_in, wt, B);
    GCHK(cudaGetLastError());

    // ---- the heaviest chain, over the arcs between components (marked once)
    if (m > 0 && kad_pool_alloc((void **)&pairs, (size_t)m * sizeof(int2), st) != cudaSuccess) {
        cudaGetLastError();
        pairs = nullptr; // no room for the list: relax over the CSR itself
    }
    if (pairs) k_chain_arcs<<<gw, T, 0, st>>>(gd.rp, gd.col, scc, n, pairs);
    for (int pass = 0;; pass++) {
        if (pass > n) { // cannot happen: each pass lengthens the chains it changes
            status = KAD_ERR_INTERNAL;
            goto done;
        }
        GCHK(cudaMemsetAsync(d_cnt + 4, 0, sizeof(int), st));
        if (pairs) {
            k_chain_relax<<<ga, T, 0, st>>>(pairs, m, wt, B, d_cnt + 4);
        } else {
            k_scc_chain<<<gw, T, 0, st>>>(gd.rp, gd.col, scc, n, wt, B, d_cnt + 4);
        }
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h + 4, d_cnt + 4, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        if (!h[4]) break;
    }
    GCHK(cudaMemsetAsync(d_cnt + 5, 0, 2 * sizeof(int), st));
    k_scc_vd<<<gv, T, 0, st>>>(scc, B, n, d_cnt + 5, d_cnt + 6);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_cnt, 8 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    *vd_out = h[5] > 1 ? h[5] : 1;
    *maxdeg_out = h[7];

done:
    if (pairs) cudaFreeAsync(pairs, st);
    if (bits) cudaFreeAsync(bits, st);
    if (scratch) cudaFreeAsync(scratch, st);
    return status;
}

// Level-synchronous multi-source BFS from the qlen sources in q0 (dist 0 there,
// -1 everywhere else): top-down while the frontier's arcs are few, bottom-up
// once they are a large share of the graph.  *levels = the largest distance
// reached.  q0 and q1 are frontier buffers of n entries; d_cnt one int and
// d_arcs one u64 of device scratch.
static cudaError_t bfs_multi(const KadGraphDev &gd, int32_t *dist, int32_t *q0, int32_t *q1, int qlen, int *d_cnt,
                      unsigned long long *d_arcs, cudaStream_t st, int *levels) {
    const int32_t n = gd.n;
    const int T = 256;
    const int gv = grid_for(n, T, 65535);
    int32_t *qa = q0, *qb = q1;
    unsigned long long arcs = 0; // unknown for the seed level: start top-down
    cudaError_t e = cudaSuccess;
    int level = 0;
    for (;; level++) {
        if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(int), st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(d_arcs, 0, 8, st)) != cudaSuccess) return e;
        const bool bottom_up = (int64_t)arcs * 14 > gd.m && qlen > n / 64;
        if (bottom_up)
            k_bfs_bu<<<gv, T, 0, st>>>(gd.rp, gd.col, n, dist, qb, d_cnt, d_arcs, level);
        else {
            // about 152 SMs x 64 warps in flight: split rows when the frontier is small
            const int parts = (qlen >= 9728) ? 1 : (9728 + qlen - 1) / qlen;
            k_bfs_td<<<grid_for((int64_t)qlen * parts * 32, T, 65535), T, 0, st>>>(gd.rp, gd.col, qa, qlen, parts,
                                                                                  dist, qb, d_cnt, d_arcs, level);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&qlen, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&arcs, d_arcs, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (qlen == 0) break;
        int32_t *t = qa;
        qa = qb;
        qb = t;
    }
    *levels = level;
    return cudaSuccess;
}

// The opt-in double-sweep bound (KAD_GRAPH_TIGHT_VD), after the BFS from each
// component's v0 left its distances in d0: per component a = the farthest
// vertex from v0, b = the farthest from a (smallest ids on ties), m = the
// midpoint of an a-b shortest path nearest v0 (d(a,m) = ceil(d(a,b)/2), then
// smallest d(v0,m), then smallest id), and the bound 2 min(ecc(v0), ecc(m)) + 1;
// VD is the maximum over components.  Every vertex's diameter bound 2 ecc(x)
// holds, so any m gives an upper bound; the double sweep looks for a central one.
// Four more multi-source BFSs, all components at once.
static kad_status tighten_vd(const KadGraphDev &gd, const int32_t *d0, int32_t *q0, int32_t *q1, int *d_flags,
                      unsigned long long *d_arcs, cudaStream_t st, int32_t *vd_out, cudaError_t *cerr) {
    const int32_t n = gd.n;
    const int T = 256;
    const int gv = grid_for(n, T, 65535);
    const size_t a4 = (((size_t)n * 4) + 255) & ~(size_t)255, a8 = (((size_t)n * 8) + 255) & ~(size_t)255;
    kad_status status = KAD_OK;
    char *scratch = nullptr;
    int32_t *da, *db;
    unsigned long long *key_a, *key_b, *key_m, *key_e;
    int h[2] = {0, 0};
    int qlen = 0, level = 0;
    if (kad_pool_alloc((void **)&scratch, 2 * a4 + 4 * a8, st) != cudaSuccess) {
        cudaGetLastError();
        return KAD_ERR_OOM;
    }
    da = (int32_t *)scratch;
    db = (int32_t *)(scratch + a4);
    key_a = (unsigned long long *)(scratch + 2 * a4);
    key_b = (unsigned long long *)(scratch + 2 * a4 + a8);
    key_m = (unsigned long long *)(scratch + 2 * a4 + 2 * a8);
    key_e = (unsigned long long *)(scratch + 2 * a4 + 3 * a8);
    GCHK(cudaMemsetAsync(key_a, 0, 2 * a8, st));         // key_a, key_b: maxima
    GCHK(cudaMemsetAsync(key_m, 0xff, a8, st));          // key_m: minimum
    GCHK(cudaMemsetAsync(key_e, 0, a8, st));
    k_far<<<gv, T, 0, st>>>(gd.comp, d0, n, key_a);
    // from a
    k_fill<<<gv, T, 0, st>>>(da, n, -1);
    GCHK(cudaMemsetAsync(d_flags + 1, 0, sizeof(int), st));
    k_seed_key<<<gv, T, 0, st>>>(gd.comp, key_a, n, 1, da, q0, d_flags + 1);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    qlen = h[0];
    GCHK(bfs_multi(gd, da, q0, q1, qlen, d_flags + 1, d_arcs, st, &level));
    k_far<<<gv, T, 0, st>>>(gd.comp, da, n, key_b);
    // from b
    k_fill<<<gv, T, 0, st>>>(db, n, -1);
    GCHK(cudaMemsetAsync(d_flags + 1, 0, sizeof(int), st));
    k_seed_key<<<gv, T, 0, st>>>(gd.comp, key_b, n, 1, db, q0, d_flags + 1);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    qlen = h[0];
    GCHK(bfs_multi(gd, db, q0, q1, qlen, d_flags + 1, d_arcs, st, &level));
    // the midpoint nearest v0, then from it (its distances replace a's)
    k_mid<<<gv, T, 0, st>>>(gd.comp, d0, da, db, key_b, n, key_m);
    k_fill<<<gv, T, 0, st>>>(da, n, -1);
    GCHK(cudaMemsetAsync(d_flags + 1, 0, sizeof(int), st));
    k_seed_key<<<gv, T, 0, st>>>(gd.comp, key_m, n, 0, da, q0, d_flags + 1);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    qlen = h[0];
    GCHK(bfs_multi(gd, da, q0, q1, qlen, d_flags + 1, d_arcs, st, &level));
    k_far<<<gv, T, 0, st>>>(gd.comp, da, n, key_e);
    GCHK(cudaMemsetAsync(d_flags + 1, 0, sizeof(int), st));
    k_tight_vd<<<gv, T, 0, st>>>(gd.comp, key_a, key_e, n, d_flags + 1);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h, d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    *vd_out = (h[0] > 1) ? h[0] : 1;
done:
    if (scratch) cudaFreeAsync(scratch, st);
    return status;
}

kad_status kad_graph_setup(KadGraphDev &gd, uint32_t flags, cudaStream_t st, int32_t *vd_out, int32_t *ncomp_out,
                           int32_t *maxdeg_out,
                           cudaError_t *cerr) {
    const int32_t n = gd.n;
    kad_status status = KAD_OK;
    int *d_flags = nullptr; // [0] err, [1] qlen, [2] ncomp, [3] largest degree, [4..7] two u64 arc counts,
                            // [16] the symmetry check's flag, [18..21] its two u64 counts
    cudaStream_t side = nullptr; // the symmetry check's stream
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int32_t *parent = nullptr, *dist = nullptr, *q0 = nullptr, *q1 = nullptr;
    unsigned long long *best = nullptr, *d_arcs = nullptr;
    int h_flags[4] = {0, 0, 0, 0};
    unsigned long long h_counts[2] = {0, 0};
    const int T = 256;
    const int gw = grid_for((int64_t)n * 32, T, 65535); // warp-per-vertex kernels
    const int gv = grid_for(n, T, 65535);
    int level = 0, qlen = 0;
    // one stream-ordered block from the graph pool, cut into the scratch arrays
    // (each start rounded up to 256 bytes)
    char *scratch = nullptr;
    const size_t a4 = (((size_t)n * 4) + 255) & ~(size_t)255, a8 = (((size_t)n * 8) + 255) & ~(size_t)255;
    if (kad_pool_alloc((void **)&scratch, 256 + 4 * a4 + a8 + 256, st) != cudaSuccess) {
        cudaGetLastError();
        status = KAD_ERR_OOM;
        goto done;
    }
    d_flags = (int *)scratch;
    parent = (int32_t *)(scratch + 256);
    dist = (int32_t *)(scratch + 256 + a4);
    q0 = (int32_t *)(scratch + 256 + 2 * a4);
    q1 = (int32_t *)(scratch + 256 + 3 * a4);
    best = (unsigned long long *)(scratch + 256 + 4 * a4);
    d_arcs = (unsigned long long *)(scratch + 256 + 4 * a4 + a8);
    GCHK(cudaMemsetAsync(d_flags, 0, 8 * sizeof(int), st));
    k_check_ends<<<1, 32, 0, st>>>(gd.rp, n, gd.m, d_flags);
    k_validate_rows<<<grid_for(((gd.m > n ? gd.m : n) + KAD_ROW_CHUNK - 1) / KAD_ROW_CHUNK + 1, T, 65535), T, 0, st>>>(
        gd.rp, gd.col, n, gd.m, d_flags);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h_flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    if (h_flags[0]) {
        status = KAD_ERR_BAD_CSR;
        goto done;
    }
    if (gd.directed) {
        status = setup_directed(gd, st, vd_out, ncomp_out, maxdeg_out, cerr);
        goto done;
    }
    if (!(flags & KAD_GRAPH_TRUSTED)) {
        // The symmetry check runs on a side stream, concurrently with the
        // components and the BFS (both are safe on any CSR that passed the row
        // checks, and their result is discarded if the check fails); its flag
        // and counts (d_flags[16], d_flags + 18) are read once both are done.
        GCHK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        GCHK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        GCHK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        GCHK(cudaMemsetAsync(d_flags + 16, 0, 8 * sizeof(int), st));
        GCHK(cudaEventRecord(ev_fork, st));
        GCHK(cudaStreamWaitEvent(side, ev_fork, 0));
        k_validate_sym<<<grid_for((gd.m + KAD_SYM_CHUNK - 1) / KAD_SYM_CHUNK, T, 65535), T, 0, side>>>(
            gd.rp, gd.col, n, gd.m, d_flags + 16, (unsigned long long *)(d_flags + 18));
        GCHK(cudaGetLastError());
    }

    // components
    k_cc_init<<<gv, T, 0, st>>>(parent, n);
    for (int r = 0; r < 2; r++) k_cc_sample<<<gv, T, 0, st>>>(gd.rp, gd.col, n, parent, d_flags, r);
    k_cc_compress<<<gv, T, 0, st>>>(parent, n);
    {
        const int probes = (n < 1024) ? n : 1024;
        int32_t *d_probe = q1; // free until the BFS
        int32_t h_probe[1024];
        k_cc_probe<<<(probes + T - 1) / T, T, 0, st>>>(parent, n, d_probe, probes);
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h_probe, d_probe, (size_t)probes * 4, cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        std::sort(h_probe, h_probe + probes);
        int big = h_probe[0], best_run = 0;
        for (int i = 0; i < probes;) {
            int j = i;
            while (j < probes && h_probe[j] == h_probe[i]) j++;
            if (j - i > best_run) {
                best_run = j - i;
                big = h_probe[i];
            }
            i = j;
        }
        k_cc_rest<<<gw, T, 0, st>>>(gd.rp, gd.col, n, parent, d_flags, big, 2);
    }
    k_cc_flatten<<<gv, T, 0, st>>>(parent, gd.comp, n);
    GCHK(cudaGetLastError());
    GCHK(cudaMemsetAsync(best, 0, (size_t)n * 8, st));
    k_best_root<<<gv, T, 0, st>>>(gd.rp, gd.comp, n, best);
    k_fill<<<gv, T, 0, st>>>(dist, n, -1);
    k_bfs_seed<<<gv, T, 0, st>>>(gd.comp, best, n, dist, q0, d_flags + 1, d_flags + 2, d_flags + 3);
    GCHK(cudaGetLastError());
    GCHK(cudaMemcpyAsync(h_flags, d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GCHK(cudaStreamSynchronize(st));
    if (h_flags[0] & GERR_CC) {
        status = KAD_ERR_INTERNAL;
        goto done;
    }
    qlen = h_flags[1];
    *ncomp_out = h_flags[2];
    *maxdeg_out = h_flags[3];

    // multi-source BFS from every component's v0
    GCHK(bfs_multi(gd, dist, q0, q1, qlen, d_flags + 1, d_arcs, st, &level));
    // `level` is now the largest distance reached from any source
    *vd_out = 2 * level + 1;
    if (flags & KAD_GRAPH_TIGHT_VD) status = tighten_vd(gd, dist, q0, q1, d_flags, d_arcs, st, vd_out, cerr);
    if (status == KAD_OK && side) {
        GCHK(cudaEventRecord(ev_join, side));
        GCHK(cudaStreamWaitEvent(st, ev_join, 0));
        GCHK(cudaMemcpyAsync(h_flags, d_flags + 16, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaMemcpyAsync(h_counts, d_flags + 18, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        if (h_flags[0] || h_counts[0] != h_counts[1]) status = KAD_ERR_BAD_CSR;
    }

done:
    if (side) {
        // whatever happened, the side stream's work ends before the scratch is freed
        cudaEventRecord(ev_join, side);
        cudaStreamWaitEvent(st, ev_join, 0);
        cudaStreamDestroy(side);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (scratch) cudaFreeAsync(scratch, st); // after the set-up's last kernel, in stream order
    return status;
}
