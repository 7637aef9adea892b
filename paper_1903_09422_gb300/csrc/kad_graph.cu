// Graph set-up on the device: CSR validation, connected components and the
// vertex-diameter bound that fixes omega (Section 2.3 preprocessing: "mostly
// computing an upper bound on the diameter"; Appendix C.1: components are
// computed with it so that pairs in different components can be skipped).
//
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

__global__ void k_cc_rest(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                          int32_t *parent, int *err, int big) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        if (*(volatile int32_t *)(parent + v) == big) continue; // inside the large tree
        const int a = rp[v], b = rp[v + 1];
        for (int e = a + 2 + lane; e < b; e += 32) cc_link(parent, v, col[e], n, err);
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

kad_status kad_graph_setup(KadGraphDev &gd, uint32_t flags, cudaStream_t st, int32_t *vd_out, int32_t *ncomp_out,
                           int32_t *maxdeg_out,
                           cudaError_t *cerr) {
    const int32_t n = gd.n;
    kad_status status = KAD_OK;
    int *d_flags = nullptr; // [0] err, [1] qlen, [2] ncomp, [3] largest degree, [4..7] two u64 arc counts
    int32_t *parent = nullptr, *dist = nullptr, *q0 = nullptr, *q1 = nullptr;
    unsigned long long *best = nullptr, *d_arcs = nullptr;
    int h_flags[4] = {0, 0, 0, 0};
    unsigned long long h_counts[2] = {0, 0};
    const int T = 256;
    const int gw = grid_for((int64_t)n * 32, T, 65535); // warp-per-vertex kernels
    const int gv = grid_for(n, T, 65535);
    int level = 0, qlen = 0;
    unsigned long long arcs = 0;
    int32_t *qa, *qb;
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
    if (!(flags & KAD_GRAPH_TRUSTED)) {
        k_validate_sym<<<grid_for((gd.m + KAD_SYM_CHUNK - 1) / KAD_SYM_CHUNK, T, 65535), T, 0, st>>>(
            gd.rp, gd.col, n, gd.m, d_flags, (unsigned long long *)(d_flags + 4));
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h_flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaMemcpyAsync(h_counts, d_flags + 4, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        if (h_flags[0] || h_counts[0] != h_counts[1]) {
            status = KAD_ERR_BAD_CSR;
            goto done;
        }
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
        k_cc_rest<<<gw, T, 0, st>>>(gd.rp, gd.col, n, parent, d_flags, big);
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

    // multi-source BFS, level by level
    qa = q0;
    qb = q1;
    arcs = 0; // unknown for the seed level: start top-down
    for (level = 0;; level++) {
        GCHK(cudaMemsetAsync(d_flags + 1, 0, sizeof(int), st));
        GCHK(cudaMemsetAsync(d_arcs, 0, 8, st));
        const bool bottom_up = (int64_t)arcs * 14 > gd.m && qlen > n / 64;
        if (bottom_up)
            k_bfs_bu<<<gv, T, 0, st>>>(gd.rp, gd.col, n, dist, qb, d_flags + 1, d_arcs, level);
        else {
            // about 152 SMs x 64 warps in flight: split rows when the frontier is small
            const int parts = (qlen >= 9728) ? 1 : (9728 + qlen - 1) / qlen;
            k_bfs_td<<<grid_for((int64_t)qlen * parts * 32, T, 65535), T, 0, st>>>(gd.rp, gd.col, qa, qlen, parts,
                                                                                  dist, qb, d_flags + 1, d_arcs, level);
        }
        GCHK(cudaGetLastError());
        GCHK(cudaMemcpyAsync(h_flags + 1, d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        GCHK(cudaMemcpyAsync(&arcs, d_arcs, 8, cudaMemcpyDeviceToHost, st));
        GCHK(cudaStreamSynchronize(st));
        qlen = h_flags[1];
        if (qlen == 0) break;
        int32_t *t = qa;
        qa = qb;
        qb = t;
    }
    // `level` is now the largest distance reached from any source
    *vd_out = 2 * level + 1;

done:
    if (scratch) cudaFreeAsync(scratch, st); // after the set-up's last kernel, in stream order
    return status;
}
