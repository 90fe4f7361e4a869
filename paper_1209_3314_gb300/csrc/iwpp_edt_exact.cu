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
constexpr int SW = 256;   // pixels per row segment in the windowed row passes (threads per CTA)
constexpr int WB = 256;   // search radius of the first windowed row pass
constexpr int SR = 8;     // rows per CTA in the first windowed row pass
constexpr int WB2 = 4096; // search radius of the second windowed row pass
constexpr int UNSETTLED = -2;  // sqdist marker of a pixel left to the next pass

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

// Outward search from pixel x of row y over the staged column-pass
// results g (g[i] is column base + i; -1: no site), one column offset d at
// a time up to radius rad, keeping the nearest site.  Once d^2 is no
// smaller than the best squared distance found, no site farther out can be
// nearer, so the pixel is settled exactly; it is also settled when the
// window covers the whole row.  Returns settled; best / bc / bg describe
// the nearest site found (bc < 0: none).
__device__ __forceinline__ bool window_search(const int *g, int base, int x, int y, int w, int rad, long long &best,
                                              int &bc, int &bg) {
    best = LLONG_MAX;
    bc = bg = -1;
    int d = 0;
    for (; d <= rad; ++d) {
        const long long dd = (long long)d * d;
        if (dd >= best) break;
        const int gl = g[x - base - d];
        if (gl >= 0) {
            const long long c = dd + (long long)(y - gl) * (y - gl);
            if (c < best) { best = c; bc = x - d; bg = gl; }
        }
        if (d > 0) {
            const int gr = g[x - base + d];
            if (gr >= 0) {
                const long long c = dd + (long long)(y - gr) * (y - gr);
                if (c < best) { best = c; bc = x + d; bg = gr; }
            }
        }
    }
    // d is the offset the loop stopped at (rad + 1 when it ran out)
    return (long long)d * d >= best || (x - rad <= 0 && x + rad >= w - 1);
}

// Stages columns base .. base + n - 1 of G's row y (-1 outside the image).
__device__ __forceinline__ void stage_row(int *g, const int32_t *Grow, int base, int n, int w) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int c = base + i;
        g[i] = (c >= 0 && c < w) ? Grow[c] : -1;
    }
}

__device__ __forceinline__ void write_site(const ExactArgs &a, int y, int x, long long best, int bc, int bg) {
    const int64_t o = (int64_t)y * a.w + x;
    a.sqdist[o] = bc < 0 ? INT_MAX : (int)best;
    a.nearest[o] = bc < 0 ? -1 : bg * a.w + bc;
}

// First windowed row pass: a CTA takes SW pixels of SR rows, stages the
// column-pass results of those columns and WB columns on either side, and
// searches with radius WB.  A pixel left unsettled is marked in sqdist and
// flags its row (rowflag 1) for the second pass.
__global__ void rows_window_kernel(ExactArgs a) {
    __shared__ int g[SW + 2 * WB];
    const int x0 = blockIdx.x * SW, x = x0 + threadIdx.x;
    const int base = x0 - WB;  // column of g[0]
    for (int rr = 0; rr < SR; ++rr) {
        const int y = blockIdx.y * SR + rr;
        if (y >= a.h) break;
        __syncthreads();
        stage_row(g, a.G + (int64_t)y * a.w, base, SW + 2 * WB, a.w);
        __syncthreads();
        if (x >= a.w) continue;
        long long best;
        int bc, bg;
        if (window_search(g, base, x, y, a.w, WB, best, bc, bg)) {
            write_site(a, y, x, best, bc, bg);
        } else {
            a.sqdist[(int64_t)y * a.w + x] = UNSETTLED;
            a.rowflag[y] = 1;
        }
    }
}

// Second windowed row pass, on flagged rows only: radius WB2 for the
// marked pixels; a pixel still unsettled flags its row (rowflag 2) for the
// exact envelope pass.
__global__ void rows_window2_kernel(ExactArgs a) {
    extern __shared__ int g2[];
    const int x0 = blockIdx.x * SW, x = x0 + threadIdx.x;
    const int base = x0 - WB2;
    for (int rr = 0; rr < SR; ++rr) {
        const int y = blockIdx.y * SR + rr;
        if (y >= a.h) break;
        if (a.rowflag[y] == 0) continue;  // block-uniform
        const int64_t o = (int64_t)y * a.w + x;
        const bool mine = x < a.w && a.sqdist[o] == UNSETTLED;
        if (!__syncthreads_or(mine)) continue;
        stage_row(g2, a.G + (int64_t)y * a.w, base, SW + 2 * WB2, a.w);
        __syncthreads();
        if (mine) {
            long long best;
            int bc, bg;
            if (window_search(g2, base, x, y, a.w, WB2, best, bc, bg)) write_site(a, y, x, best, bc, bg);
            else a.rowflag[y] = 2;
        }
        __syncthreads();  // g2 is restaged for the next row
    }
}

// One thread per row: the lower envelope of the row's sites (Felzenszwalb
// and Huttenlocher's sweep, with exact rational comparisons), then the
// nearest site of every pixel.  Runs on the rows the windowed passes left
// unsettled (rowflag 2).
__global__ void rows_kernel(ExactArgs a) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= a.h || a.rowflag[y] != 2) return;
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
    cudaError_t e = cudaMemsetAsync(a.rowflag, 0, (size_t)a.h * sizeof(int), s);
    if (e != cudaSuccess) return e;
    band_ends_kernel<<<gxb, XT, 0, s>>>(a);
    band_links_kernel<<<gx, XT, 0, s>>>(a);
    columns_kernel<<<gxb, XT, 0, s>>>(a);
    rows_window_kernel<<<dim3((a.w + SW - 1) / SW, (a.h + SR - 1) / SR), SW, 0, s>>>(a);
    const int smem2 = (SW + 2 * WB2) * (int)sizeof(int);
    e = cudaFuncSetAttribute(rows_window2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2);
    if (e != cudaSuccess) return e;
    rows_window2_kernel<<<dim3((a.w + SW - 1) / SW, (a.h + SR - 1) / SR), SW, smem2, s>>>(a);
    rows_kernel<<<(a.h + 31) / 32, 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace iwpp
