// iwpp_skiz.cu -- the per-pixel steps of the influence zones and their
// skeleton (SKIZ) of labelled sources inside a mask.
//
// The zones (named in Section 1 among the IWPP algorithms, with the
// watershed) are computed from three wavefront propagations of the
// persistent kernels, with these streaming kernels around them:
//   1. prep: the sources' uint8 plane (labels != 0) for the shortest-path
//      propagation, which gives every free pixel its least path cost from a
//      source (8 moves, cost 5 / 7);
//   2. label init: the shortest-path in-edges -- neighbour q of a reached,
//      free, non-source pixel p when q is free and reached and
//      dist(q) + cost(q, p) = dist(p) -- and two value planes: the labels
//      and the negated labels at the sources, INT_MAX elsewhere.  One
//      launch of the label propagation then runs both planes: each pixel
//      receives the least label, and the least negated label (the greatest
//      label), among the sources on whose shortest paths it lies;
//   3. finish: zones = the least label (0 where none reaches), skiz = 1
//      where the least and the greatest differ (two zones equally near).
// One thread per pixel.
#include <climits>
#include <cstdint>

#include "iwpp_internal.h"

namespace iwpp {
namespace {

constexpr int SK_BX = 256;

__global__ void skiz_prep_kernel(const SkizArgs a) {
    const int x = blockIdx.x * SK_BX + threadIdx.x;
    if (x >= a.w) return;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y)
        a.seeds[(int64_t)y * a.w + x] = a.labels[(int64_t)y * a.pl + x] != 0;
}

__global__ void skiz_label_init_kernel(const SkizArgs a) {
    const int x = blockIdx.x * SK_BX + threadIdx.x;
    if (x >= a.w) return;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        const int64_t p = (int64_t)y * a.w + x;
        const bool free_p = a.mask[(int64_t)y * a.pmask + x] != 0;
        const int32_t lab = a.labels[(int64_t)y * a.pl + x];
        const int32_t d = a.dist[p];
        const bool source = free_p && lab != 0;
        unsigned bits = 0;
        if (free_p && !source && d != INT_MAX) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int qy = y + nb8_dy(k), qx = x + nb8_dx(k);
                if (qy < 0 || qy >= a.h || qx < 0 || qx >= a.w) continue;
                if (!a.mask[(int64_t)qy * a.pmask + qx]) continue;
                const int32_t dq = a.dist[(int64_t)qy * a.w + qx];
                const int cost = (nb8_dy(k) != 0 && nb8_dx(k) != 0) ? 7 : 5;
                if (dq != INT_MAX && (int64_t)dq + cost == d) bits |= 1u << k;
            }
        }
        a.E[p] = (uint8_t)bits;
        a.zones[p] = source ? lab : INT_MAX;
        a.neg[p] = source ? -lab : INT_MAX;
    }
}

__global__ void skiz_finish_kernel(const SkizArgs a) {
    const int x = blockIdx.x * SK_BX + threadIdx.x;
    if (x >= a.w) return;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        const int64_t p = (int64_t)y * a.w + x;
        const int32_t lo = a.zones[p];
        const bool reached = lo != INT_MAX;
        if (a.skiz) a.skiz[p] = reached && lo != -a.neg[p];
        if (!reached) a.zones[p] = 0;
    }
}

cudaError_t launch_one(void (*k)(const SkizArgs), const SkizArgs &a, cudaStream_t s) {
    (void)cudaGetLastError();
    const dim3 grid((a.w + SK_BX - 1) / SK_BX, a.h < 8192 ? a.h : 8192);
    k<<<grid, SK_BX, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_skiz_prep(const SkizArgs &a, cudaStream_t s) { return launch_one(skiz_prep_kernel, a, s); }
cudaError_t launch_skiz_label_init(const SkizArgs &a, cudaStream_t s) {
    return launch_one(skiz_label_init_kernel, a, s);
}
cudaError_t launch_skiz_finish(const SkizArgs &a, cudaStream_t s) { return launch_one(skiz_finish_kernel, a, s); }

}  // namespace iwpp
