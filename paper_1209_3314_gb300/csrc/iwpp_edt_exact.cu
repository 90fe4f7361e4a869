// Exact Euclidean distance transform on the GPU: the separable method
// (a column pass that finds, for every pixel, the nearest feature in its own
// column, then a row pass that takes the lower envelope of the parabolas
// (x - i)^2 + dy(i)^2 over the columns i of the row).  This is not the
// paper's propagation method: it is the exact transform the paper measures
// its departures against (Section 2.2, Figure 3), offered beside the
// propagation EDT as an exact variant and a speed comparison.
//
// All arithmetic is integer: squared distances are exact and every
// comparison of parabola intersections is done by cross-multiplication in
// 64 bits, so the result equals the definition min over features f of
// |p - f|^2 bit for bit.  Nearest-feature ties may go to any of the equally
// near features.

#include <climits>
#include <cstdint>

#include "iwpp_internal.h"

namespace iwpp {

namespace {

constexpr int XT = 128;  // columns per CTA in the column kernels
constexpr int BH = 256;  // rows per band in the column pass

__device__ __forceinline__ bool feature_px(uint8_t b, int flags) {
    return (flags & 1) ? b != 0 : b == 0;
}

// Per (column, band): first and last feature rows inside the band (-1: none).
__global__ void band_ends_kernel(ExactArgs a) {
    const int x = blockIdx.x * XT + threadIdx.x, b = blockIdx.y;
    if (x >= a.w) return;
    const int r0 = b * BH, r1 = min(a.h, r0 + BH);
    int first = -1, last = -1;
    for (int r = r0; r < r1; ++r) {
        if (feature_px(__ldg(a.bin + (int64_t)r * a.pitch + x), a.flags)) {
            if (first < 0) first = r;
            last = r;
        }
    }
    a.first[(int64_t)b * a.w + x] = first;
    a.last[(int64_t)b * a.w + x] = last;
}

// Per column: the nearest feature row above each band (the last feature of
// the bands above) and below it (the first feature of the bands below).
__global__ void band_links_kernel(ExactArgs a) {
    const int x = blockIdx.x * XT + threadIdx.x;
    if (x >= a.w) return;
    int run = -1;
    for (int b = 0; b < a.nb; ++b) {
        a.above[(int64_t)b * a.w + x] = run;
        const int l = a.last[(int64_t)b * a.w + x];
        if (l >= 0) run = l;
    }
    run = -1;
    for (int b = a.nb - 1; b >= 0; --b) {
        a.below[(int64_t)b * a.w + x] = run;
        const int f = a.first[(int64_t)b * a.w + x];
        if (f >= 0) run = f;
    }
}

// Per (column, band): the row of the nearest feature in the pixel's column
// (-1: the column has none), written to G.  Downward pass: the last
// feature at or above; upward pass: the first at or below; the nearer wins
// (the upper one on a tie).
__global__ void columns_kernel(ExactArgs a) {
    const int x = blockIdx.x * XT + threadIdx.x, b = blockIdx.y;
    if (x >= a.w) return;
    const int r0 = b * BH, r1 = min(a.h, r0 + BH);
    int up = a.above[(int64_t)b * a.w + x];
    for (int r = r0; r < r1; ++r) {
        if (feature_px(__ldg(a.bin + (int64_t)r * a.pitch + x), a.flags)) up = r;
        a.G[(int64_t)r * a.w + x] = up;
    }
    int dn = a.below[(int64_t)b * a.w + x];
    for (int r = r1 - 1; r >= r0; --r) {
        if (feature_px(__ldg(a.bin + (int64_t)r * a.pitch + x), a.flags)) dn = r;
        const int u = a.G[(int64_t)r * a.w + x];
        a.G[(int64_t)r * a.w + x] = (u >= 0 && (dn < 0 || r - u <= dn - r)) ? u : dn;
    }
}

// stack entry: column v (15 bits) and signed row offset dy of its nearest
// column feature (16 bits)
__device__ __forceinline__ uint32_t site_pack(int v, int dy) { return (uint32_t)v | ((uint32_t)(dy & 0xFFFF) << 16); }
__device__ __forceinline__ int site_v(uint32_t e) { return (int)(e & 0xFFFFu); }
__device__ __forceinline__ int site_dy(uint32_t e) { return (int)(int16_t)(e >> 16); }

// Intersection of the parabolas of sites a and b (va < vb) as the fraction
// num / den, den > 0:  ((vb^2 + fb) - (va^2 + fa)) / (2 (vb - va)).
__device__ __forceinline__ void cross(uint32_t ea, uint32_t eb, long long &num, long long &den) {
    const long long va = site_v(ea), vb = site_v(eb);
    const long long fa = (long long)site_dy(ea) * site_dy(ea), fb = (long long)site_dy(eb) * site_dy(eb);
    num = (vb * vb + fb) - (va * va + fa);
    den = 2 * (vb - va);
}

// One thread per row: the lower envelope of the row's sites (Felzenszwalb
// and Huttenlocher's sweep, with exact rational comparisons), then the
// nearest site of every pixel.  The row's G values are all read before its
// outputs are written, so G may be the nearest-index output itself.
__global__ void rows_kernel(ExactArgs a) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= a.h) return;
    const int w = a.w;
    const int32_t *Grow = a.G + (int64_t)y * w;
    uint32_t *S = a.stack + (int64_t)y * w;
    int k = -1;
    for (int q = 0; q < w; ++q) {
        const int g = Grow[q];
        if (g < 0) continue;
        const uint32_t e = site_pack(q, y - g);
        // pop the top while the new site's parabola overtakes it no later
        // than the top overtook the entry below it
        while (k >= 1) {
            long long n1, d1, n2, d2;
            cross(S[k], e, n1, d1);
            cross(S[k - 1], S[k], n2, d2);
            if (n1 * d2 <= n2 * d1) --k;
            else break;
        }
        S[++k] = e;
    }
    int32_t *sq = a.sqdist + (int64_t)y * w;
    int32_t *nn = a.nearest + (int64_t)y * w;
    if (k < 0) {
        for (int x = 0; x < w; ++x) {
            sq[x] = INT_MAX;
            nn[x] = -1;
        }
        return;
    }
    int j = 0;
    for (int x = 0; x < w; ++x) {
        while (j < k) {
            long long n, d;
            cross(S[j], S[j + 1], n, d);
            if (n <= (long long)x * d) ++j;  // the next site is at least as near from x on
            else break;
        }
        const int v = site_v(S[j]), dy = site_dy(S[j]);
        sq[x] = (x - v) * (x - v) + dy * dy;
        nn[x] = (y - dy) * w + v;
    }
}

}  // namespace

int exact_bands(int h) { return (h + BH - 1) / BH; }

cudaError_t launch_edt_exact(const ExactArgs &a, cudaStream_t s) {
    cudaGetLastError();
    const dim3 gx((a.w + XT - 1) / XT), gxb((a.w + XT - 1) / XT, a.nb);
    band_ends_kernel<<<gxb, XT, 0, s>>>(a);
    band_links_kernel<<<gx, XT, 0, s>>>(a);
    columns_kernel<<<gxb, XT, 0, s>>>(a);
    rows_kernel<<<(a.h + 31) / 32, 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace iwpp
