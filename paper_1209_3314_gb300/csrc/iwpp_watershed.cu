// iwpp_watershed.cu -- the per-pixel steps of the watershed from markers.
//
// The watershed (named in Section 1 among the IWPP algorithms) is computed
// as three wavefront propagations of the persistent kernels, with these
// streaming kernels between them:
//   1. complement: A = ~relief at marker pixels and the type's bottom
//      elsewhere, B = ~relief.  The flooding level -- the least, over the
//      paths from a marker, of the highest relief value on the path -- is
//      the reconstruction by erosion of (relief at the markers, top
//      elsewhere) above the relief, i.e. ~(reconstruction by dilation of A
//      under B), which the reconstruction family computes in place in A;
//   2. plateau init: the levels c = ~A; the in-edges between neighbours of
//      equal level; plateau distance 0 at entry pixels (markers and pixels
//      with a lower neighbour), WS_DINF elsewhere; the plateau-distance
//      propagation then gives every pixel its breadth-first distance from
//      the entry of its level region;
//   3. label init: the optimal in-edges (a lower neighbour into an entry
//      pixel, or an equal-level neighbour one plateau step closer to the
//      entry; none into a marker pixel) and labels = the markers; the
//      label propagation then gives every pixel the least marker value that
//      reaches it along optimal edges.
// Every kernel here reads a pixel's 3x3 neighbourhood from global memory
// (through L1) and writes the pixel: one thread per pixel, rows of 256.
#include <climits>
#include <cstdint>

#include "iwpp_internal.h"

namespace iwpp {
namespace {

constexpr int WS_BX = 256;

template <typename T>
struct Range;
template <>
struct Range<uint8_t> {
    static constexpr uint8_t bottom = 0;
};
template <>
struct Range<int32_t> {
    static constexpr int32_t bottom = INT_MIN;
};

// order-reversing complement of the type (255 - v for uint8, -1 - v for int32)
__device__ __forceinline__ uint8_t cpl(uint8_t v) { return (uint8_t)~v; }
__device__ __forceinline__ int32_t cpl(int32_t v) { return ~v; }

template <typename T>
__global__ void ws_complement_kernel(const WsArgs a) {
    const int x = blockIdx.x * WS_BX + threadIdx.x;
    if (x >= a.w) return;
    const T *f = (const T *)a.relief;
    T *A = (T *)a.A, *B = (T *)a.B;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        const T v = f[(int64_t)y * a.pf + x];
        const int64_t p = (int64_t)y * a.w + x;
        A[p] = a.markers[(int64_t)y * a.pm + x] ? cpl(v) : Range<T>::bottom;
        B[p] = cpl(v);
    }
}

template <typename T>
__global__ void ws_plateau_init_kernel(const WsArgs a) {
    const int x = blockIdx.x * WS_BX + threadIdx.x;
    if (x >= a.w) return;
    const T *A = (const T *)a.A;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        const int64_t p = (int64_t)y * a.w + x;
        const T c = cpl(A[p]);
        if (a.levels) ((T *)a.levels)[p] = c;
        unsigned bits = 0;
        bool lower = a.markers[(int64_t)y * a.pm + x] != 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int qy = y + nb8_dy(k), qx = x + nb8_dx(k);
            if (qy < 0 || qy >= a.h || qx < 0 || qx >= a.w) continue;
            const T cq = cpl(A[(int64_t)qy * a.w + qx]);
            if (cq == c) bits |= 1u << k;
            if (cq < c) lower = true;
        }
        // an entry pixel is at distance 0 already: it needs no in-edge
        a.E[p] = lower ? 0 : (uint8_t)bits;
        a.D[p] = lower ? 0 : WS_DINF;
    }
}

template <typename T>
__global__ void ws_label_init_kernel(const WsArgs a) {
    const int x = blockIdx.x * WS_BX + threadIdx.x;
    if (x >= a.w) return;
    const T *A = (const T *)a.A;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        const int64_t p = (int64_t)y * a.w + x;
        const int32_t m = a.markers[(int64_t)y * a.pm + x];
        unsigned bits = 0;
        if (m == 0) {
            const T c = cpl(A[p]);
            const int32_t d = a.D[p];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int qy = y + nb8_dy(k), qx = x + nb8_dx(k);
                if (qy < 0 || qy >= a.h || qx < 0 || qx >= a.w) continue;
                const int64_t q = (int64_t)qy * a.w + qx;
                const T cq = cpl(A[q]);
                if ((cq < c && d == 0) || (cq == c && a.D[q] + 1 == d)) bits |= 1u << k;
            }
        }
        a.E[p] = (uint8_t)bits;
        a.labels[p] = m;
    }
}

template <typename T>
cudaError_t launch_one(void (*k)(const WsArgs), const WsArgs &a, cudaStream_t s) {
    (void)cudaGetLastError();
    const dim3 grid((a.w + WS_BX - 1) / WS_BX, a.h < 8192 ? a.h : 8192);
    k<<<grid, WS_BX, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ws_complement(const WsArgs &a, cudaStream_t s) {
    return a.dtype == DT_U8 ? launch_one<uint8_t>(ws_complement_kernel<uint8_t>, a, s)
                            : launch_one<int32_t>(ws_complement_kernel<int32_t>, a, s);
}

cudaError_t launch_ws_plateau_init(const WsArgs &a, cudaStream_t s) {
    return a.dtype == DT_U8 ? launch_one<uint8_t>(ws_plateau_init_kernel<uint8_t>, a, s)
                            : launch_one<int32_t>(ws_plateau_init_kernel<int32_t>, a, s);
}

cudaError_t launch_ws_label_init(const WsArgs &a, cudaStream_t s) {
    return a.dtype == DT_U8 ? launch_one<uint8_t>(ws_label_init_kernel<uint8_t>, a, s)
                            : launch_one<int32_t>(ws_label_init_kernel<int32_t>, a, s);
}

}  // namespace iwpp
