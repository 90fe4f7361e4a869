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
//      entry; none into a marker pixel) and labels = the markers (INT_MAX
//      where there is none); the label propagation then gives every pixel
//      the least marker value that reaches it along optimal edges;
//   4. label finish: INT_MAX (reached by no marker) becomes 0.
// The init kernels read a pixel's 3x3 neighbourhood from global memory
// (through L1) and write the pixel.  All of them handle four pixels per
// thread with vector loads and stores where the width allows, else one
// pixel per thread.
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
        a.labels[p] = m ? m : INT_MAX;
    }
}

__global__ void ws_label_finish_kernel(const WsArgs a) {
    const int x = blockIdx.x * WS_BX + threadIdx.x;
    if (x >= a.w) return;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        int32_t *l = a.labels + (int64_t)y * a.w + x;
        if (*l == INT_MAX) *l = 0;
    }
}

// ---- four pixels per thread (w % 4 == 0, outputs aligned): the planes'
// rows then start on 16-byte boundaries (int32) / 4-byte boundaries (uint8),
// so a thread loads the 3 x 6 neighbourhood of its 4 pixels with one vector
// and two scalar loads per row and writes vectors.  Comparisons work on the
// complemented values: a lower level is a larger complement.

template <typename T>
struct Vec4;
template <>
struct Vec4<uint8_t> {
    typedef uchar4 type;
};
template <>
struct Vec4<int32_t> {
    typedef int4 type;
};

// row[x-1 .. x+4] -> v[0 .. 5]; v[0] / v[5] are 0 where the image has no
// such column (the callers never compare them)
template <typename T>
__device__ __forceinline__ void load6(const T *row, int x, bool has_l, bool has_r, T (&v)[6]) {
    const typename Vec4<T>::type m = *(const typename Vec4<T>::type *)(row + x);
    v[0] = has_l ? row[x - 1] : T(0);
    v[1] = m.x;
    v[2] = m.y;
    v[3] = m.z;
    v[4] = m.w;
    v[5] = has_r ? row[x + 4] : T(0);
}

template <typename T>
__device__ __forceinline__ void store4(T *dst, const T (&v)[4]) {
    typename Vec4<T>::type m;
    m.x = v[0];
    m.y = v[1];
    m.z = v[2];
    m.w = v[3];
    *(typename Vec4<T>::type *)dst = m;
}

template <typename T>
__global__ void ws_complement_x4(const WsArgs a) {
    const int x = (blockIdx.x * WS_BX + threadIdx.x) * 4;
    if (x >= a.w) return;
    const T *f = (const T *)a.relief;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        T va[4], vb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T v = f[(int64_t)y * a.pf + x + j];
            vb[j] = cpl(v);
            va[j] = a.markers[(int64_t)y * a.pm + x + j] ? vb[j] : Range<T>::bottom;
        }
        store4((T *)a.A + (int64_t)y * a.w + x, va);
        store4((T *)a.B + (int64_t)y * a.w + x, vb);
    }
}

template <typename T>
__global__ void ws_plateau_init_x4(const WsArgs a) {
    const int x = (blockIdx.x * WS_BX + threadIdx.x) * 4;
    if (x >= a.w) return;
    const T *A = (const T *)a.A;
    const bool has_l = x > 0, has_r = x + 4 < a.w;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        T c[3][6];
        bool rv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int yy = y - 1 + i;
            rv[i] = yy >= 0 && yy < a.h;
            if (rv[i]) load6(A + (int64_t)yy * a.w, x, has_l, has_r, c[i]);
        }
        uint8_t e[4];
        int32_t d[4];
        T lv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T ap = c[1][j + 1];
            lv[j] = cpl(ap);
            unsigned bits = 0;
            bool lower = a.markers[(int64_t)y * a.pm + x + j] != 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int ri = 1 + nb8_dy(k), ci = j + 1 + nb8_dx(k);
                const bool ok = rv[ri] && (ci > 0 || has_l) && (ci < 5 || has_r);
                if (ok && c[ri][ci] == ap) bits |= 1u << k;
                if (ok && c[ri][ci] > ap) lower = true;
            }
            e[j] = lower ? 0 : (uint8_t)bits;
            d[j] = lower ? 0 : WS_DINF;
        }
        const int64_t p = (int64_t)y * a.w + x;
        *(uchar4 *)(a.E + p) = make_uchar4(e[0], e[1], e[2], e[3]);
        *(int4 *)(a.D + p) = make_int4(d[0], d[1], d[2], d[3]);
        if (a.levels) store4((T *)a.levels + p, lv);
    }
}

template <typename T>
__global__ void ws_label_init_x4(const WsArgs a) {
    const int x = (blockIdx.x * WS_BX + threadIdx.x) * 4;
    if (x >= a.w) return;
    const T *A = (const T *)a.A;
    const bool has_l = x > 0, has_r = x + 4 < a.w;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        T c[3][6];
        int32_t dd[3][6];
        bool rv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int yy = y - 1 + i;
            rv[i] = yy >= 0 && yy < a.h;
            if (rv[i]) {
                load6(A + (int64_t)yy * a.w, x, has_l, has_r, c[i]);
                load6(a.D + (int64_t)yy * a.w, x, has_l, has_r, dd[i]);
            }
        }
        uint8_t e[4];
        int32_t lab[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int32_t m = a.markers[(int64_t)y * a.pm + x + j];
            const T ap = c[1][j + 1];
            const int32_t dp = dd[1][j + 1];
            unsigned bits = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int ri = 1 + nb8_dy(k), ci = j + 1 + nb8_dx(k);
                const bool ok = rv[ri] && (ci > 0 || has_l) && (ci < 5 || has_r);
                if (ok && ((c[ri][ci] > ap && dp == 0) || (c[ri][ci] == ap && dd[ri][ci] + 1 == dp)))
                    bits |= 1u << k;
            }
            e[j] = m ? 0 : (uint8_t)bits;
            lab[j] = m ? m : INT_MAX;
        }
        const int64_t p = (int64_t)y * a.w + x;
        *(uchar4 *)(a.E + p) = make_uchar4(e[0], e[1], e[2], e[3]);
        *(int4 *)(a.labels + p) = make_int4(lab[0], lab[1], lab[2], lab[3]);
    }
}

__global__ void ws_label_finish_x4(const WsArgs a) {
    const int x = (blockIdx.x * WS_BX + threadIdx.x) * 4;
    if (x >= a.w) return;
    for (int y = blockIdx.y; y < a.h; y += gridDim.y) {
        int4 *l = (int4 *)(a.labels + (int64_t)y * a.w + x);
        int4 v = *l;
        if (v.x == INT_MAX || v.y == INT_MAX || v.z == INT_MAX || v.w == INT_MAX) {
            v.x = v.x == INT_MAX ? 0 : v.x;
            v.y = v.y == INT_MAX ? 0 : v.y;
            v.z = v.z == INT_MAX ? 0 : v.z;
            v.w = v.w == INT_MAX ? 0 : v.w;
            *l = v;
        }
    }
}

// the four-pixel kernels need whole quads in every row and vector-aligned
// outputs (the context's planes are 256-byte aligned and dense)
bool quads(const WsArgs &a) {
    const size_t es = a.dtype == DT_U8 ? 1 : 4;
    return a.w % 4 == 0 && (uintptr_t)a.labels % 16 == 0 && (!a.levels || (uintptr_t)a.levels % (4 * es) == 0);
}

cudaError_t launch_one(void (*k)(const WsArgs), const WsArgs &a, bool x4, cudaStream_t s) {
    (void)cudaGetLastError();
    const int cols = x4 ? WS_BX * 4 : WS_BX;
    const dim3 grid((a.w + cols - 1) / cols, a.h < 8192 ? a.h : 8192);
    k<<<grid, WS_BX, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ws_complement(const WsArgs &a, cudaStream_t s) {
    const bool x4 = quads(a);
    if (a.dtype == DT_U8)
        return launch_one(x4 ? ws_complement_x4<uint8_t> : ws_complement_kernel<uint8_t>, a, x4, s);
    return launch_one(x4 ? ws_complement_x4<int32_t> : ws_complement_kernel<int32_t>, a, x4, s);
}

cudaError_t launch_ws_plateau_init(const WsArgs &a, cudaStream_t s) {
    const bool x4 = quads(a);
    if (a.dtype == DT_U8)
        return launch_one(x4 ? ws_plateau_init_x4<uint8_t> : ws_plateau_init_kernel<uint8_t>, a, x4, s);
    return launch_one(x4 ? ws_plateau_init_x4<int32_t> : ws_plateau_init_kernel<int32_t>, a, x4, s);
}

cudaError_t launch_ws_label_init(const WsArgs &a, cudaStream_t s) {
    const bool x4 = quads(a);
    if (a.dtype == DT_U8)
        return launch_one(x4 ? ws_label_init_x4<uint8_t> : ws_label_init_kernel<uint8_t>, a, x4, s);
    return launch_one(x4 ? ws_label_init_x4<int32_t> : ws_label_init_kernel<int32_t>, a, x4, s);
}

cudaError_t launch_ws_label_finish(const WsArgs &a, cudaStream_t s) {
    const bool x4 = quads(a);
    return launch_one(x4 ? ws_label_finish_x4 : ws_label_finish_kernel, a, x4, s);
}

}  // namespace iwpp
