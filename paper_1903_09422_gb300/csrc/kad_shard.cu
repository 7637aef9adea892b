// Device side of the sharded run (kad_run_sharded): folding the path rows that
// all ranks computed for one epoch (or for the calibration phase) into the
// sampling state, and the stop check on that state (sm_103a).
//
// Sharding splits each epoch's sample-index range among the ranks; every rank
// then receives all of the epoch's rows, folds them with integer atomics (the
// associative operation of Algorithm 1 is integer addition, so the order of the
// rows does not matter) and evaluates the stop rule of Appendix B on the same
// state as every other rank -- the distributed reduction the paper names as
// future work (Section 6), bit-exact with the single-GPU run.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kad_internal.cuh"

namespace {

// blocks: `world` blocks of rows, each [maxc lengths][maxc flags][maxc x cap
// vertices]; a row with length < 0 is absent (a rank's chunk can be shorter
// than maxc).  Calibration rows count every interior vertex into c0 and move it
// one histogram bin up; adaptive rows count into cnt and raise the running
// maximum count of the vertex's calibration class.
__global__ void k_fold_rows(const int32_t *__restrict__ blocks, int world, int maxc, int cap, int calib,
                            uint32_t *c0w, uint32_t *hist, uint32_t *cnt, int32_t *classmax,
                            const uint32_t *__restrict__ c0, unsigned long long *ovf) {
    const size_t bstride = (size_t)maxc * (size_t)(2 + cap);
    const long long rows = (long long)world * maxc;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < rows;
         q += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(q / maxc), j = (int)(q % maxc);
        const int32_t *blk = blocks + (size_t)b * bstride;
        const int len = blk[j];
        if (len < 0) continue;
        if (!calib && blk[maxc + j]) atomicAdd(ovf, 1ull);
        const int32_t *path = blk + 2 * (size_t)maxc + (size_t)j * cap;
        for (int t = 0; t < len && t < cap; t++) {
            const int v = path[t];
            if (calib) {
                const unsigned int c = atomicAdd(c0w + v, 1u);
                atomicSub(hist + c, 1u);
                atomicAdd(hist + c + 1, 1u);
            } else {
                const unsigned int c = atomicAdd(cnt + v, 1u) + 1u;
                atomicMax(classmax + c0[v], (int)c);
            }
        }
    }
}

// Appendix B per calibration class: f and g are non-decreasing in the count for
// a fixed L, so the largest count of each class decides for all of it.  Sets
// *fail when some class fails f <= eps and g <= eps.
__global__ void k_check_classes(const int32_t *__restrict__ classmax, const double *__restrict__ ltab, int nclass,
                                unsigned long long tau, unsigned long long omega, double eps, int *fail) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nclass; j += gridDim.x * blockDim.x) {
        const int cm = classmax[j];
        if (cm < 0) continue;
        const double L = ltab[j];
        const double f = kad_fg_dev((unsigned long long)cm, L, tau, omega, false);
        const double g = kad_fg_dev((unsigned long long)cm, L, tau, omega, true);
        if (!(f <= eps && g <= eps)) atomicOr(fail, 1);
    }
}

} // namespace

cudaError_t kad_launch_fold_rows(const int32_t *blocks, int world, int maxc, int cap, int calib, uint32_t *c0w,
                                 uint32_t *hist, uint32_t *cnt, int32_t *classmax, const uint32_t *c0,
                                 unsigned long long *ovf, cudaStream_t st) {
    const long long rows = (long long)world * maxc;
    if (rows <= 0) return cudaSuccess;
    int blocks_n = (int)((rows + 255) / 256);
    if (blocks_n > 4096) blocks_n = 4096;
    k_fold_rows<<<blocks_n, 256, 0, st>>>(blocks, world, maxc, cap, calib, c0w, hist, cnt, classmax, c0, ovf);
    return cudaGetLastError();
}

cudaError_t kad_launch_check_classes(const int32_t *classmax, const double *ltab, int nclass, unsigned long long tau,
                                     unsigned long long omega, double eps, int *fail, cudaStream_t st) {
    int blocks_n = (nclass + 255) / 256;
    if (blocks_n > 1024) blocks_n = 1024;
    if (blocks_n < 1) blocks_n = 1;
    k_check_classes<<<blocks_n, 256, 0, st>>>(classmax, ltab, nclass, tau, omega, eps, fail);
    return cudaGetLastError();
}
