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
constexpr int BH = 128;  // rows per band in the column pass

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
// feature at or above, kept in shared memory (16 bits: rows < 32768);
// upward pass: the first at or below; the nearer wins (the upper one on a
// tie), and G is written once.
__global__ void columns_kernel(ExactArgs a) {
    __shared__ int16_t U[BH][XT];
    const int x = blockIdx.x * XT + threadIdx.x, b = blockIdx.y;
    if (x >= a.w) return;  // no barrier below: each thread keeps to its own column of U
    const int r0 = b * BH, r1 = min(a.h, r0 + BH);
    int up = a.above[(int64_t)b * a.w + x];
    for (int r = r0; r < r1; ++r) {
        if (feature_px(__ldg(a.bin + (int64_t)r * a.pitch + x), a.flags)) up = r;
        U[r - r0][threadIdx.x] = (int16_t)up;
    }
    int dn = a.below[(int64_t)b * a.w + x];
    for (int r = r1 - 1; r >= r0; --r) {
        if (feature_px(__ldg(a.bin + (int64_t)r * a.pitch + x), a.flags)) dn = r;
        const int u = U[r - r0][threadIdx.x];
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

// Row pass geometry: a CTA of ET threads takes one row; thread t owns the
// chunk of C columns starting at t*C, C = 32 or 64 with ET*C >= w (sides up
// to 32768).  Chunk t's sites sit at S[t*(C+1) ...] and the owners of its
// pixels (as positions in S) at own[t*(C+2) ...]: the gaps keep the lanes
// of a warp on distinct banks when they step through their chunks in
// lockstep.
constexpr int ET = 512;

int env_chunk(int w) { return w <= 32 * ET ? 32 : 64; }

size_t env_smem(int w) {
    const size_t C = env_chunk(w);
    return ET * (C + 1) * sizeof(uint32_t) + ET * (C + 2) * sizeof(uint16_t) + (4 * ET + 64) * sizeof(int);
}

// For sites p < q < r (by column): q owns no abscissa once r overtakes q
// no later than q overtakes p, x(q, r) <= x(p, q).
__device__ __forceinline__ bool dominated(uint32_t p, uint32_t q, uint32_t r) {
    long long n1, d1, n2, d2;
    cross(q, r, n1, d1);
    cross(p, q, n2, d2);
    return n1 * d2 <= n2 * d1;
}

// The pops of merge_envelopes (below), from A's last non-empty chunk ca and
// B's first cb; A spans chunks ca0 .. ca, B chunks cb .. cend - 1.
__device__ __forceinline__ void merge_sides(const uint32_t *S, int *lo, int *hi, int ca0, int ca, int cb, int cend) {
    // a1: A's last (chunk ca); a0: the one before (chunk cp, pa0 < 0: none)
    int pa1 = hi[ca] - 1, cp = ca, pa0 = -1;
    if (pa1 > lo[ca]) pa0 = pa1 - 1;
    else {
        for (cp = ca - 1; cp >= ca0 && lo[cp] == hi[cp]; --cp) {}
        if (cp >= ca0) pa0 = hi[cp] - 1;
    }
    // b0: B's first (chunk cb); b1: the one after (chunk cn, pb1 < 0: none)
    int pb0 = lo[cb], cn = cb, pb1 = -1;
    if (pb0 + 1 < hi[cb]) pb1 = pb0 + 1;
    else {
        for (cn = cb + 1; cn < cend && lo[cn] == hi[cn]; ++cn) {}
        if (cn < cend) pb1 = lo[cn];
    }
    for (;;) {
        if (pa0 >= 0 && dominated(S[pa0], S[pa1], S[pb0])) {
            hi[ca] = pa1;  // a1 was the last live entry of chunk ca
            ca = cp;
            pa1 = pa0;
            if (pa1 > lo[ca]) pa0 = pa1 - 1;
            else {
                for (cp = ca - 1; cp >= ca0 && lo[cp] == hi[cp]; --cp) {}
                pa0 = cp >= ca0 ? hi[cp] - 1 : -1;
            }
        } else if (pb1 >= 0 && dominated(S[pa1], S[pb0], S[pb1])) {
            lo[cb] = pb0 + 1;  // b0 was the first live entry of chunk cb
            cb = cn;
            pb0 = pb1;
            if (pb0 + 1 < hi[cb]) pb1 = pb0 + 1;
            else {
                for (cn = cb + 1; cn < cend && lo[cn] == hi[cn]; ++cn) {}
                pb1 = cn < cend ? lo[cn] : -1;
            }
        } else {
            break;
        }
    }
}

// Merges the envelopes of the chunk groups A = [ca0, cb0) and B = [cb0, cend)
// (A's columns all left of B's).  Subtracting x^2 turns each parabola into
// a line whose slope falls with the site's column, so the union's envelope
// is a prefix of A's followed by a suffix of B's: pop A's last site while
// the pair (A's second-to-last, B's first) covers it, or B's first while
// (A's last, B's second) covers it, until neither applies.  Each pop drops
// a site that owns no abscissa, and at the end both triples across the
// junction are valid, so the sequence is the union's lower envelope.  lo
// and hi hold each chunk's live range as positions in S; gf / gl, indexed
// by a group's first chunk, its first / last non-empty chunk (-1: none).
// A group's first site and its last are never popped (each is the only
// site that owns the abscissae far enough to its side), so gf and gl of
// the merged group follow from the two groups'.
__device__ __forceinline__ void merge_envelopes(const uint32_t *S, int *lo, int *hi, int *gf, int *gl, int ca0, int cb0,
                                int cend) {
    const int ca = gl[ca0], cb = gf[cb0];
    gf[ca0] = ca >= 0 ? gf[ca0] : cb;
    gl[ca0] = cb >= 0 ? gl[cb0] : ca;
    if (ca < 0 || cb < 0) return;  // one side empty: nothing to pop
    merge_sides(S, lo, hi, ca0, ca, cb, cend);
}

// The row pass: one CTA per row builds the lower envelope of the row's
// sites (Felzenszwalb and Huttenlocher's construction, exact rational
// comparisons) in parallel and colours every pixel of the row with its
// site.  Its cost does not depend on the distances.
//  0. The row's column-pass results are staged in chunk layout, each
//     warp its own lanes' chunks, eight loads per thread in flight.
//  1. Each thread builds its chunk's envelope with the sequential sweep,
//     in place over the staged entries.
//  2. log2(ET) rounds merge neighbouring groups of chunks pairwise.
//  3. The surviving sites, in chunk order, are the row's envelope; each
//     thread finds the owner of its chunk's first pixel by binary search on
//     the breakpoints, walks forward across its chunk and records each
//     pixel's owner; then each warp writes its lanes' chunks, coalesced.
__global__ void __launch_bounds__(ET) rows_envelope_kernel(ExactArgs a, int C) {
    extern __shared__ uint32_t S[];
    uint16_t *own = (uint16_t *)(S + (size_t)ET * (C + 1));
    int *lo = (int *)(own + (size_t)ET * (C + 2));
    int *hi = lo + ET;
    // during the merges: each group's first / last non-empty chunk (indexed
    // by the group's first chunk); from step 3: the last non-empty chunk at
    // or before c (-1: none) / the first at or after c (ET: none)
    int *prv = hi + ET;
    int *nxt = prv + ET;
    int *wsum = nxt + ET;  // per-warp partial results of the scans
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, w = a.w;
    const int CO = C + 2, CP = C >> 5;  // CP: 32-column parts per chunk (1 or 2)
    constexpr int UB = 8;
    for (int y = blockIdx.x; y < a.h; y += gridDim.x) {
        __syncthreads();  // shared arrays are reused per row
        const int32_t *Grow = a.G + (int64_t)y * w;
        // 0. each warp stages its own 32 chunks (its lanes' chunks), so the
        // phases up to the wide merges need only warp barriers
        for (int u0 = 0; u0 < 32; u0 += UB) {
            uint32_t v[UB][2];
#pragma unroll
            for (int u = 0; u < UB; ++u)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int c = warp * 32 + u0 + u, q = c * C + p * 32 + lane;
                    v[u][p] = (p < CP && q < w) ? (uint32_t)__ldg(Grow + q) : 0xFFFFFFFFu;
                }
#pragma unroll
            for (int u = 0; u < UB; ++u)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const int c = warp * 32 + u0 + u;
                    if (p < CP) S[c * (C + 1) + p * 32 + lane] = v[u][p];
                }
        }
        __syncwarp();
        // 1. the chunk's envelope, written over its own staged entries
        {
            uint32_t *my = S + (size_t)tid * (C + 1);
            const int x0 = tid * C, n = min(C, w - x0);
            int k = -1;
            for (int i = 0; i < n; ++i) {
                const int g = (int)my[i];
                if (g < 0) continue;
                const uint32_t e = site_pack(x0 + i, y - g);
                while (k >= 1 && dominated(my[k - 1], my[k], e)) --k;
                my[++k] = e;
            }
            lo[tid] = tid * (C + 1);
            hi[tid] = tid * (C + 1) + k + 1;
            prv[tid] = nxt[tid] = k >= 0 ? tid : -1;  // the chunk's group: its first / last non-empty chunk
        }
        // 2. pairwise merges, each by the thread of the group's first chunk:
        // up to groups of 32 chunks, a merge reads only what lanes of its
        // own warp wrote, so a warp barrier orders the rounds
        for (int span = 1; span < ET; span <<= 1) {
            if (span < 32) __syncwarp();
            else __syncthreads();
            if ((tid & (2 * span - 1)) == 0) merge_envelopes(S, lo, hi, prv, nxt, tid, tid + span, tid + 2 * span);
        }
        __syncthreads();
        // 3. the neighbouring non-empty chunks of every chunk (a max scan
        // and a min scan of the non-empty chunks' indices)
        const bool live = hi[tid] > lo[tid];
        int pm = live ? tid : -1, nm = live ? tid : ET;
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, pm, d);
            const int v = __shfl_down_sync(0xffffffffu, nm, d);
            if (lane >= d) pm = max(pm, u);
            if (lane + d < 32) nm = min(nm, v);
        }
        if (lane == 31) wsum[warp] = pm;
        if (lane == 0) wsum[32 + warp] = nm;
        __syncthreads();
        for (int q = 0; q < ET / 32; ++q) {
            if (q < warp) pm = max(pm, wsum[q]);
            if (q > warp) nm = min(nm, wsum[32 + q]);
        }
        prv[tid] = pm;
        nxt[tid] = nm;
        __syncthreads();
        int32_t *sq = a.sqdist + (int64_t)y * w;
        int32_t *nn = a.nearest + (int64_t)y * w;
        if (prv[ET - 1] < 0) {  // block-uniform: no feature in any column
            for (int x = tid; x < w; x += ET) {
                sq[x] = INT_MAX;
                nn[x] = -1;
            }
            continue;
        }
        // bp(p, q) <= x: from x on, the envelope's site at q is at least as
        // near as its predecessor at p
        auto reached = [&](int p, int q, int x) {
            long long n, d;
            cross(S[p], S[q], n, d);
            return n <= (long long)x * d;
        };
        // the first site of non-empty chunk c owns an abscissa <= x
        auto starts_by = [&](int c, int x) {
            const int pc = c > 0 ? prv[c - 1] : -1;
            return pc < 0 || reached(hi[pc] - 1, lo[c], x);
        };
        const int x0 = tid * C, x1 = min(w, x0 + C);
        if (x0 < w) {
            // the owner of x0: in the last non-empty chunk whose first site
            // starts by x0 (breakpoints increase along the envelope; the
            // first non-empty chunk always qualifies), ...
            int l = nxt[0], r = ET - 1;
            while (l < r) {
                const int m = (l + r + 1) >> 1;
                if (starts_by(prv[m], x0)) l = m;
                else r = m - 1;
            }
            int c = prv[l];
            // ... at its last site that starts by x0
            int pl = lo[c], pr = hi[c] - 1;
            while (pl < pr) {
                const int m = (pl + pr + 1) >> 1;
                if (reached(m - 1, m, x0)) pl = m;
                else pr = m - 1;
            }
            // the site after pos (chunk c): nx in chunk cn, nx < 0: none
            int pos = pl, cn = c, nx = -1;
            auto advance_next = [&]() {
                if (pos + 1 < hi[c]) {
                    cn = c;
                    nx = pos + 1;
                } else {
                    cn = c + 1 < ET ? nxt[c + 1] : ET;
                    nx = cn < ET ? lo[cn] : -1;
                }
            };
            advance_next();
            for (int x = x0; x < x1; ++x) {
                while (nx >= 0 && reached(pos, nx, x)) {
                    pos = nx;
                    c = cn;
                    advance_next();
                }
                own[tid * CO + (x - x0)] = (uint16_t)pos;
            }
        }
        __syncwarp();  // each warp writes out its own lanes' chunks
        for (int c = warp * 32; c < warp * 32 + 32; ++c)
            for (int p = 0; p < CP; ++p) {
                const int k = p * 32 + lane, x = c * C + k;
                if (x >= w) break;
                const uint32_t e = S[own[c * CO + k]];
                const int v = site_v(e), dy = site_dy(e);
                sq[x] = (x - v) * (x - v) + dy * dy;
                nn[x] = (y - dy) * w + v;
            }
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
    const int C = env_chunk(a.w);
    const int smem = (int)env_smem(a.w);
    cudaError_t e = cudaFuncSetAttribute(rows_envelope_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // one wave of resident CTAs, each taking rows blockIdx.x + k * grid
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_envelope_kernel, ET, smem)) != cudaSuccess)
        return e;
    rows_envelope_kernel<<<min(a.h, max(1, sms * per_sm)), ET, smem, s>>>(a, C);
    return cudaGetLastError();
}

}  // namespace iwpp
