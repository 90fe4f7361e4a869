// iwpp_kernels.cu -- the persistent tile-wavefront kernel of libiwpp.
//
// One kernel drains a queue of image tiles.  Visiting a tile means:
//   1. stage the tile plus a 1-pixel halo in shared memory (the halo holds
//      the current values of the neighbouring tiles, read only);
//   2. seed sweeps (reconstruction): raster and anti-raster passes inside
//      the tile, each split into a row pass and a column pass as in
//      Algorithm 5 (N^{+,0}, N^{0,+}, N^{-,0}, N^{0,-});
//   3. seed scan: every pixel of tile+halo that can still propagate into a
//      tile pixel is queued (the full-neighbourhood test of Algorithm 5 for
//      reconstruction; Algorithm 6's initial wavefront generalised to a
//      partial result for the distance transform);
//   4. wavefront propagation inside the tile in rounds over in/out queues
//      (Algorithm 4): atomicMax updates for reconstruction (Algorithm 5),
//      compare-and-swap retry updates for the distance transform
//      (Algorithm 6); warp-aggregated enqueue into per-warp, per-block
//      (shared) and per-CTA global spill queues (Section 3.2);
//   5. store the tile, then test every tile-border pixel against the
//      neighbouring tiles' current values; a neighbour that could still be
//      updated is re-queued (the border-propagation step of Section 4, done
//      on one device without a separate stage).
// Tiles only ever write their own pixels, and values only move in one
// direction (up for reconstruction, closer features for the distance
// transform), so any interleaving of visits converges to the same fixpoint
// as the sequential algorithms.
#include <climits>
#include <cstdint>

#include "iwpp_internal.h"

namespace iwpp {

constexpr int NT = 256;      // threads per CTA
constexpr int NW = NT / 32;  // warps per CTA

// shared header slots
enum : int {
    H_TILE = 0,
    H_CNT0 = 1,   // round-queue counters (2)
    H_RESCAN = 3,
    H_SRC = 4,    // 3x3 neighbour tiles: 1 if visited (9)
    H_FLAG = 13,  // 3x3 neighbour tiles: needs a visit (9)
    H_PUSH = 22,
    H_SPILL = 23,
    H_RESC = 24,
    H_SEEDS = 25,
    H_WORDS = 64,
};

template <int TS>
struct Geo {
    static constexpr int R = TS + 2;                       // staged rows/cols
    static constexpr int P = (R % 2 == 0) ? R + 1 : R;     // odd pitch (words)
    static constexpr int CELLS = R * P;
    static constexpr int QCAP = TS * TS;                   // BQ entries per buffer
    static constexpr int WORDS = H_WORDS + 2 * CELLS + 2 * QCAP + NW * 64;
};

struct Smem {
    int *hdr, *A, *B, *Q0, *Q1, *WQ;
};

template <int TS>
__device__ __forceinline__ Smem carve(int *base) {
    using G = Geo<TS>;
    Smem s;
    s.hdr = base;
    s.A = base + H_WORDS;
    s.B = s.A + G::CELLS;
    s.Q0 = s.B + G::CELLS;
    s.Q1 = s.Q0 + G::QCAP;
    s.WQ = s.Q1 + G::QCAP;
    return s;
}

template <int CONN> struct Nb;
template <> struct Nb<8> {
    static __device__ __forceinline__ int dr(int k) { return k < 3 ? -1 : (k < 5 ? 0 : 1); }
    static __device__ __forceinline__ int dc(int k) {
        const int t[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
        return t[k];
    }
};
template <> struct Nb<4> {
    static __device__ __forceinline__ int dr(int k) { return k == 0 ? -1 : (k == 3 ? 1 : 0); }
    static __device__ __forceinline__ int dc(int k) { return k == 1 ? -1 : (k == 2 ? 1 : 0); }
};

template <typename T> struct Low;
template <> struct Low<uint8_t> { static constexpr int v = -1; };
template <> struct Low<int32_t> { static constexpr int v = INT_MIN; };

__device__ __forceinline__ int ldcg_val(const uint8_t *p) { return (int)__ldcg(p); }
__device__ __forceinline__ int ldcg_val(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ int ldg_val(const uint8_t *p) { return (int)__ldg(p); }
__device__ __forceinline__ int ldg_val(const int32_t *p) { return __ldg(p); }

__device__ __forceinline__ JobDesc job_of(const KArgs &ka, int t) {
    if (ka.njobs == 1) return ka.job0;
    int lo = 0, hi = ka.njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&ka.jobs[mid].tile_base) <= t) lo = mid; else hi = mid - 1;
    }
    return ka.jobs[lo];
}

// Enumerates the 4*(TS+1) halo cells: top row, bottom row, left and right
// columns (corners belong to the rows).
template <int TS>
__device__ __forceinline__ void halo_cell(int i, int &r, int &c) {
    constexpr int R = TS + 2;
    if (i < R) { r = 0; c = i; }
    else if (i < 2 * R) { r = R - 1; c = i - R; }
    else if (i < 2 * R + TS) { r = i - 2 * R + 1; c = 0; }
    else { r = i - 2 * R - TS + 1; c = R - 1; }
}

__device__ __forceinline__ int region(int v, int last) { return v == 0 ? 0 : (v == last ? 2 : 1); }

// Loads the 3x3 'visited' flags of the tile neighbourhood into hdr[H_SRC..].
__device__ __forceinline__ void load_sources(const KArgs &ka, const JobDesc &jd, int tx, int ty, Smem s) {
    const int tid = threadIdx.x;
    if (tid < 9) {
        const int ny = ty + tid / 3 - 1, nx = tx + tid % 3 - 1;
        int v = 0;
        if (ny >= 0 && ny < jd.tiles_y && nx >= 0 && nx < jd.tiles_x)
            v = ld_acquire(ka.tq.visited + jd.tile_base + ny * jd.tiles_x + nx);
        s.hdr[H_SRC + tid] = v;
    }
}

// Publishes the tile's stores, re-queues flagged neighbours, marks the tile
// visited.  Thread 0 only; all stores of the CTA precede it (barrier).
__device__ __forceinline__ void finish_tile(const KArgs &ka, const JobDesc &jd, int gt, int tx, int ty, Smem s) {
    __threadfence();
    if (!s.hdr[H_SRC + 4]) st_release(ka.tq.visited + gt, 1);
    for (int k = 0; k < 9; ++k) {
        if (k == 4 || !s.hdr[H_FLAG + k]) continue;
        const int ny = ty + k / 3 - 1, nx = tx + k % 3 - 1;
        tq_push(ka.tq, ka.ctl, jd.tile_base + ny * jd.tiles_x + nx);
    }
    tq_finish(ka.tq, ka.ctl, gt);
}

// =====================================================================
// Reconstruction by dilation (Section 2.1; Algorithms 2, 4, 5)
// =====================================================================

template <int CONN, int TS>
__device__ void recon_seed_scan(const int *J, const int *I, WarpQueue &wq, const RoundQueue &rq) {
    using G = Geo<TS>;
    constexpr int R = G::R, P = G::P;
    for (int base = 0; base < R * R; base += NT) {
        const int i = base + threadIdx.x;
        bool seed = false;
        int p = 0;
        if (i < R * R) {
            const int r = i / R, c = i - r * R;
            p = r * P + c;
            const int jp = J[p];
#pragma unroll
            for (int k = 0; k < CONN; ++k) {
                const int rr = r + Nb<CONN>::dr(k), cc = c + Nb<CONN>::dc(k);
                if (rr >= 1 && rr <= TS && cc >= 1 && cc <= TS) {
                    const int q = rr * P + cc;
                    seed |= J[q] < min(jp, I[q]);
                }
            }
        }
        wq.push(seed, p, rq);
    }
    wq.drain(rq);
}

template <typename T, int CONN, int TS>
__device__ void recon_tile(const KArgs &ka, const JobDesc &jd, int gt, Smem s) {
    using G = Geo<TS>;
    constexpr int R = G::R, P = G::P;
    constexpr int LOW = Low<T>::v;
    const int tid = threadIdx.x;
    const int lt = gt - jd.tile_base;
    const int tx = lt % jd.tiles_x, ty = lt / jd.tiles_x;
    const int oy = ty * TS - 1, ox = tx * TS - 1;  // image coords of staged cell (0,0)
    const T *mk = (const T *)jd.a;
    const T *ms = (const T *)jd.b;
    T *out = (T *)jd.out;
    int *J = s.A;
    const int *I = s.B;
    volatile int *VJ = s.A;

    load_sources(ka, jd, tx, ty, s);
    if (tid < 9) s.hdr[H_FLAG + tid] = 0;
    if (tid == 0) {
        s.hdr[H_CNT0] = 0; s.hdr[H_CNT0 + 1] = 0; s.hdr[H_RESCAN] = 0;
        s.hdr[H_PUSH] = 0; s.hdr[H_SPILL] = 0; s.hdr[H_RESC] = 0;
    }
    __syncthreads();

    // 1. stage marker-or-current (clipped by the mask) and mask, tile + halo
    for (int i = tid; i < R * R; i += NT) {
        const int r = i / R, c = i - r * R;
        const int gy = oy + r, gx = ox + c;
        int jv = LOW, iv = LOW;
        if (gy >= 0 && gy < jd.h && gx >= 0 && gx < jd.w) {
            iv = ldg_val(ms + (int64_t)gy * jd.pb + gx);
            const bool cur = s.hdr[H_SRC + region(r, R - 1) * 3 + region(c, R - 1)] != 0;
            const int v = cur ? ldcg_val(out + (int64_t)gy * jd.po + gx)
                              : ldcg_val(mk + (int64_t)gy * jd.pa + gx);
            jv = min(v, iv);
        }
        s.A[r * P + c] = jv;
        s.B[r * P + c] = iv;
    }
    __syncthreads();

    // 2. seed sweeps: raster (rows L->R, then columns top->bottom over the
    //    upper neighbours) and anti-raster (rows R->L, columns bottom->top).
    for (int sp = 0; sp < ka.sweeps; ++sp) {
        if (tid < TS) {
            const int r = tid + 1;
            int run = VJ[r * P];
            for (int c = 1; c <= TS; ++c) {
                const int v = min(max(VJ[r * P + c], run), I[r * P + c]);
                VJ[r * P + c] = v;
                run = v;
            }
        }
        __syncthreads();
        if (tid < TS) {
            const int c = tid + 1;
            int up = VJ[c];
            for (int r = 1; r <= TS; ++r) {
                int v = max(VJ[r * P + c], up);
                if (CONN == 8) v = max(v, max(VJ[(r - 1) * P + c - 1], VJ[(r - 1) * P + c + 1]));
                v = min(v, I[r * P + c]);
                VJ[r * P + c] = v;
                up = v;
            }
        }
        __syncthreads();
        if (tid < TS) {
            const int r = tid + 1;
            int run = VJ[r * P + TS + 1];
            for (int c = TS; c >= 1; --c) {
                const int v = min(max(VJ[r * P + c], run), I[r * P + c]);
                VJ[r * P + c] = v;
                run = v;
            }
        }
        __syncthreads();
        if (tid < TS) {
            const int c = tid + 1;
            int dn = VJ[(TS + 1) * P + c];
            for (int r = TS; r >= 1; --r) {
                int v = max(VJ[r * P + c], dn);
                if (CONN == 8) v = max(v, max(VJ[(r + 1) * P + c - 1], VJ[(r + 1) * P + c + 1]));
                v = min(v, I[r * P + c]);
                VJ[r * P + c] = v;
                dn = v;
            }
        }
        __syncthreads();
    }

    // 3. seed scan into round queue 0
    int *spill = ka.spill + (int64_t)blockIdx.x * 2 * ka.spill_cap;
    WarpQueue wq{s.WQ + (tid >> 5) * 64, 0, 0u};
    {
        RoundQueue rq{s.Q0, spill, s.hdr + H_CNT0, s.hdr + H_RESCAN, G::QCAP, ka.spill_cap};
        recon_seed_scan<CONN, TS>(J, I, wq, rq);
    }
    __syncthreads();
    if (tid == 0) s.hdr[H_SEEDS] = s.hdr[H_CNT0];

    // 4. propagation rounds (Algorithm 5, wavefront phase)
    int cur = 0;
    unsigned spilled = 0, rescans = 0;
    while (true) {
        __syncthreads();
        const int n_raw = s.hdr[H_CNT0 + cur];
        const int resc = s.hdr[H_RESCAN];
        const int n_in = min(n_raw, G::QCAP + ka.spill_cap);
        if (n_in == 0 && !resc) break;
        __syncthreads();
        if (tid == 0) {
            s.hdr[H_CNT0 + (cur ^ 1)] = 0;
            s.hdr[H_RESCAN] = 0;
            spilled += n_in > G::QCAP ? n_in - G::QCAP : 0;
            rescans += resc ? 1 : 0;
        }
        __syncthreads();
        const int *qin_s = cur ? s.Q1 : s.Q0;
        const int *qin_g = spill + cur * ka.spill_cap;
        RoundQueue rq{cur ? s.Q0 : s.Q1, spill + (cur ^ 1) * ka.spill_cap,
                      s.hdr + H_CNT0 + (cur ^ 1), s.hdr + H_RESCAN, G::QCAP, ka.spill_cap};
        {
            for (int base = 0; base < n_in; base += NT) {
                const int i = base + tid;
                const bool valid = i < n_in;
                const int p = valid ? rq_load(qin_s, qin_g, G::QCAP, i) : (P + 1);
                const int pr = p / P, pc = p - pr * P;
                const int jp = valid ? VJ[p] : LOW;
#pragma unroll
                for (int k = 0; k < CONN; ++k) {
                    const int rr = pr + Nb<CONN>::dr(k), cc = pc + Nb<CONN>::dc(k);
                    const int q = rr * P + cc;
                    bool pred = false;
                    if (valid && rr >= 1 && rr <= TS && cc >= 1 && cc <= TS) {
                        const int v = min(jp, I[q]);
                        if (VJ[q] < v) pred = atomicMax(J + q, v) < v;
                    }
                    wq.push(pred, q, rq);
                }
            }
            wq.drain(rq);
        }
        if (resc) {
            // the in-queue of this round was truncated (items dropped): the
            // items that fitted were processed above, which guarantees
            // progress; the next queue is rebuilt from a full scan of the
            // partial result (the restart rule of Section 3.2)
            __syncthreads();
            if (tid == 0) { s.hdr[H_CNT0 + (cur ^ 1)] = 0; s.hdr[H_RESCAN] = 0; }
            __syncthreads();
            recon_seed_scan<CONN, TS>(J, I, wq, rq);
        }
        cur ^= 1;
    }

    // 5. store the tile
    for (int i = tid; i < TS * TS; i += NT) {
        const int r = i / TS + 1, c = i - (i / TS) * TS + 1;
        const int gy = oy + r, gx = ox + c;
        if (gy < jd.h && gx < jd.w) out[(int64_t)gy * jd.po + gx] = (T)J[r * P + c];
    }
    if ((tid & 31) == 0) atomicAdd(s.hdr + H_PUSH, (int)wq.pushed);
    __syncthreads();
    if (tid == 0) __threadfence();
    load_sources(ka, jd, tx, ty, s);  // fresh flags for the border test
    __syncthreads();

    // 6. border test against the neighbours' current values
    for (int i = tid; i < 4 * (TS + 1); i += NT) {
        int r, c;
        halo_cell<TS>(i, r, c);
        const int gy = oy + r, gx = ox + c;
        if (gy < 0 || gy >= jd.h || gx < 0 || gx >= jd.w) continue;
        const int reg = region(r, R - 1) * 3 + region(c, R - 1);
        const int iq = I[r * P + c];
        const int v = s.hdr[H_SRC + reg] ? ldcg_val(out + (int64_t)gy * jd.po + gx)
                                         : ldcg_val(mk + (int64_t)gy * jd.pa + gx);
        const int jq = min(v, iq);
        bool need = false;
#pragma unroll
        for (int k = 0; k < CONN; ++k) {
            const int pr = r + Nb<CONN>::dr(k), pc = c + Nb<CONN>::dc(k);
            if (pr >= 1 && pr <= TS && pc >= 1 && pc <= TS) need |= jq < min(J[pr * P + pc], iq);
        }
        if (need) s.hdr[H_FLAG + reg] = 1;
    }
    __syncthreads();
    if (tid == 0) {
        s.hdr[H_SPILL] = (int)spilled;
        s.hdr[H_RESC] = (int)rescans;
        finish_tile(ka, jd, gt, tx, ty, s);
    }
}

// =====================================================================
// Distance transform by nearest-feature propagation (Section 2.2;
// Algorithms 3 and 6).  Shared memory holds the Voronoi assignment VR as
// packed image coordinates (y << 16 | x); 0xFFFFFFFF is the virtual 'inf'
// pixel, farther than any real pixel.
// =====================================================================

enum : unsigned { VR_INF = 0xFFFFFFFFu };

__device__ __forceinline__ unsigned pack_yx(int y, int x) { return ((unsigned)y << 16) | (unsigned)x; }

// squared distance from (y, x) to packed feature f; VR_INF for 'inf'
__device__ __forceinline__ unsigned d2(int y, int x, unsigned f) {
    if (f == VR_INF) return VR_INF;
    const int dy = y - (int)(f >> 16), dx = x - (int)(f & 0xFFFFu);
    return (unsigned)(dy * dy + dx * dx);
}

__device__ __forceinline__ bool is_feature(uint8_t b, int flags) {
    return (flags & 1) ? b != 0 : b == 0;
}

// current VR of image pixel (gy, gx): from the stored result of a visited
// tile, else from the binary input (Algorithm 6 initialisation)
__device__ __forceinline__ unsigned vr_fetch(const JobDesc &jd, bool visited, int gy, int gx) {
    if (visited) {
        const int idx = __ldcg(jd.nearest + (int64_t)gy * jd.w + gx);
        if (idx < 0) return VR_INF;
        const int fy = idx / jd.w;
        return pack_yx(fy, idx - fy * jd.w);
    }
    const uint8_t b = __ldg((const uint8_t *)jd.a + (int64_t)gy * jd.pa + gx);
    return is_feature(b, jd.flags) ? pack_yx(gy, gx) : VR_INF;
}

template <int TS>
__device__ void edt_seed_scan(const unsigned *V, int oy, int ox, WarpQueue &wq, const RoundQueue &rq) {
    using G = Geo<TS>;
    constexpr int R = G::R, P = G::P;
    for (int base = 0; base < R * R; base += NT) {
        const int i = base + threadIdx.x;
        bool seed = false;
        int p = 0;
        if (i < R * R) {
            const int r = i / R, c = i - r * R;
            p = r * P + c;
            const unsigned f = V[p];
            if (f != VR_INF) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int rr = r + Nb<8>::dr(k), cc = c + Nb<8>::dc(k);
                    if (rr >= 1 && rr <= TS && cc >= 1 && cc <= TS) {
                        const int y = oy + rr, x = ox + cc;
                        seed |= d2(y, x, f) < d2(y, x, V[rr * P + cc]);
                    }
                }
            }
        }
        wq.push(seed, p, rq);
    }
    wq.drain(rq);
}

template <int TS>
__device__ void edt_tile(const KArgs &ka, const JobDesc &jd, int gt, Smem s) {
    using G = Geo<TS>;
    constexpr int R = G::R, P = G::P;
    const int tid = threadIdx.x;
    const int lt = gt - jd.tile_base;
    const int tx = lt % jd.tiles_x, ty = lt / jd.tiles_x;
    const int oy = ty * TS - 1, ox = tx * TS - 1;
    unsigned *V = (unsigned *)s.A;
    volatile unsigned *VV = V;

    load_sources(ka, jd, tx, ty, s);
    if (tid < 9) s.hdr[H_FLAG + tid] = 0;
    if (tid == 0) {
        s.hdr[H_CNT0] = 0; s.hdr[H_CNT0 + 1] = 0; s.hdr[H_RESCAN] = 0;
        s.hdr[H_PUSH] = 0; s.hdr[H_SPILL] = 0; s.hdr[H_RESC] = 0;
    }
    __syncthreads();

    // 1. stage VR of tile + halo
    for (int i = tid; i < R * R; i += NT) {
        const int r = i / R, c = i - r * R;
        const int gy = oy + r, gx = ox + c;
        unsigned v = VR_INF;
        if (gy >= 0 && gy < jd.h && gx >= 0 && gx < jd.w) {
            const bool visited = s.hdr[H_SRC + region(r, R - 1) * 3 + region(c, R - 1)] != 0;
            v = vr_fetch(jd, visited, gy, gx);
        }
        V[r * P + c] = v;
    }
    __syncthreads();

    // 2. seed scan (Algorithm 6 lines 2-5, generalised to partial results)
    int *spill = ka.spill + (int64_t)blockIdx.x * 2 * ka.spill_cap;
    WarpQueue wq{s.WQ + (tid >> 5) * 64, 0, 0u};
    {
        RoundQueue rq{s.Q0, spill, s.hdr + H_CNT0, s.hdr + H_RESCAN, G::QCAP, ka.spill_cap};
        edt_seed_scan<TS>(V, oy, ox, wq, rq);
    }
    __syncthreads();
    if (tid == 0) s.hdr[H_SEEDS] = s.hdr[H_CNT0];

    // 3. propagation rounds with CAS retry (Algorithm 6, wavefront phase)
    int cur = 0;
    unsigned spilled = 0, rescans = 0;
    while (true) {
        __syncthreads();
        const int n_raw = s.hdr[H_CNT0 + cur];
        const int resc = s.hdr[H_RESCAN];
        const int n_in = min(n_raw, G::QCAP + ka.spill_cap);
        if (n_in == 0 && !resc) break;
        __syncthreads();
        if (tid == 0) {
            s.hdr[H_CNT0 + (cur ^ 1)] = 0;
            s.hdr[H_RESCAN] = 0;
            spilled += n_in > G::QCAP ? n_in - G::QCAP : 0;
            rescans += resc ? 1 : 0;
        }
        __syncthreads();
        const int *qin_s = cur ? s.Q1 : s.Q0;
        const int *qin_g = spill + cur * ka.spill_cap;
        RoundQueue rq{cur ? s.Q0 : s.Q1, spill + (cur ^ 1) * ka.spill_cap,
                      s.hdr + H_CNT0 + (cur ^ 1), s.hdr + H_RESCAN, G::QCAP, ka.spill_cap};
        {
            for (int base = 0; base < n_in; base += NT) {
                const int i = base + tid;
                const bool valid = i < n_in;
                const int p = valid ? rq_load(qin_s, qin_g, G::QCAP, i) : (P + 1);
                const int pr = p / P, pc = p - pr * P;
                const unsigned f = valid ? VV[p] : VR_INF;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int rr = pr + Nb<8>::dr(k), cc = pc + Nb<8>::dc(k);
                    const int q = rr * P + cc;
                    bool pred = false;
                    if (f != VR_INF && rr >= 1 && rr <= TS && cc >= 1 && cc <= TS) {
                        const int y = oy + rr, x = ox + cc;
                        const unsigned dn = d2(y, x, f);
                        unsigned cq = VV[q];
                        while (dn < d2(y, x, cq)) {
                            const unsigned old = atomicCAS(V + q, cq, f);
                            if (old == cq) { pred = true; break; }
                            cq = old;
                        }
                    }
                    wq.push(pred, q, rq);
                }
            }
            wq.drain(rq);
        }
        if (resc) {  // truncated in-queue: processed what fitted, now rescan
            __syncthreads();
            if (tid == 0) { s.hdr[H_CNT0 + (cur ^ 1)] = 0; s.hdr[H_RESCAN] = 0; }
            __syncthreads();
            edt_seed_scan<TS>(V, oy, ox, wq, rq);
        }
        cur ^= 1;
    }

    // 4. store VR (as linear index) and the squared distance (Algorithm 6,
    //    final loop)
    for (int i = tid; i < TS * TS; i += NT) {
        const int r = i / TS + 1, c = i - (i / TS) * TS + 1;
        const int gy = oy + r, gx = ox + c;
        if (gy < jd.h && gx < jd.w) {
            const unsigned f = V[r * P + c];
            const int64_t o = (int64_t)gy * jd.w + gx;
            if (f == VR_INF) {
                jd.nearest[o] = -1;
                jd.sqdist[o] = INT_MAX;
            } else {
                jd.nearest[o] = (int)(f >> 16) * jd.w + (int)(f & 0xFFFFu);
                jd.sqdist[o] = (int)d2(gy, gx, f);
            }
        }
    }
    if ((tid & 31) == 0) atomicAdd(s.hdr + H_PUSH, (int)wq.pushed);
    __syncthreads();
    if (tid == 0) __threadfence();
    load_sources(ka, jd, tx, ty, s);
    __syncthreads();

    // 5. border test
    for (int i = tid; i < 4 * (TS + 1); i += NT) {
        int r, c;
        halo_cell<TS>(i, r, c);
        const int gy = oy + r, gx = ox + c;
        if (gy < 0 || gy >= jd.h || gx < 0 || gx >= jd.w) continue;
        const int reg = region(r, R - 1) * 3 + region(c, R - 1);
        const unsigned cq = vr_fetch(jd, s.hdr[H_SRC + reg] != 0, gy, gx);
        const unsigned dq = d2(gy, gx, cq);
        bool need = false;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int pr = r + Nb<8>::dr(k), pc = c + Nb<8>::dc(k);
            if (pr >= 1 && pr <= TS && pc >= 1 && pc <= TS) need |= d2(gy, gx, V[pr * P + pc]) < dq;
        }
        if (need) s.hdr[H_FLAG + reg] = 1;
    }
    __syncthreads();
    if (tid == 0) {
        s.hdr[H_SPILL] = (int)spilled;
        s.hdr[H_RESC] = (int)rescans;
        finish_tile(ka, jd, gt, tx, ty, s);
    }
}

// =====================================================================
// kernels
// =====================================================================

template <int TS>
__global__ void __launch_bounds__(NT) persistent_kernel(const __grid_constant__ KArgs ka) {
    extern __shared__ int smem_raw[];
    Smem s = carve<TS>(smem_raw);
    if (ld_volatile(&ka.ctl->done)) return;
    const unsigned long long deadline = globaltimer_ns() + ka.timeout_ns;
    while (true) {
        if (threadIdx.x == 0) s.hdr[H_TILE] = tq_claim(ka.tq, ka.ctl, deadline);
        __syncthreads();
        const int t = s.hdr[H_TILE];
        if (t < 0) break;
        const JobDesc jd = job_of(ka, t);
        if (jd.op == OP_RECON) {
            if (jd.dtype == DT_U8) {
                if (jd.conn == 8) recon_tile<uint8_t, 8, TS>(ka, jd, t, s);
                else recon_tile<uint8_t, 4, TS>(ka, jd, t, s);
            } else {
                if (jd.conn == 8) recon_tile<int32_t, 8, TS>(ka, jd, t, s);
                else recon_tile<int32_t, 4, TS>(ka, jd, t, s);
            }
        } else {
            edt_tile<TS>(ka, jd, t, s);
        }
        if (threadIdx.x == 0) {
            atomicAdd(&ka.ctl->tiles_processed, 1ull);
            atomicAdd(&ka.ctl->seeds, (unsigned long long)s.hdr[H_SEEDS]);
            atomicAdd(&ka.ctl->pushes, (unsigned long long)s.hdr[H_PUSH]);
            atomicAdd(&ka.ctl->spills, (unsigned long long)s.hdr[H_SPILL]);
            atomicAdd(&ka.ctl->rescans, (unsigned long long)s.hdr[H_RESC]);
            __threadfence();
            atomicSub(ka.tq.pending, 1);
        }
        __syncthreads();
    }
}

// Slot of tile t in the initial queue: colour class (x mod 2, y mod 2)
// first, so that tiles visited at the same time are never adjacent.
__device__ __forceinline__ int initial_slot(const JobDesc &jd, int t) {
    const int lt = t - jd.tile_base;
    const int x = lt % jd.tiles_x, y = lt / jd.tiles_x;
    const int a = x & 1, b = y & 1;
    const int nx = (jd.tiles_x - a + 1) >> 1;
    return jd.color_base[b * 2 + a] + (y >> 1) * nx + (x >> 1);
}

__global__ void fill_queue_kernel(const __grid_constant__ KArgs ka, int first) {
    if (!first && !ld_volatile(&ka.ctl->want_reset)) return;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)ka.tq.cap; i += stride) {
        if (i < ka.ntiles) {
            const JobDesc jd = job_of(ka, i);
            ka.tq.slots[initial_slot(jd, i)] = i;
            ka.tq.state[i] = TS_QUEUED;
            if (first) ka.tq.visited[i] = 0;
        } else {
            ka.tq.slots[i] = -1;
        }
    }
    if (first && blockIdx.x == 0 && threadIdx.x == 0) {
        *ka.tq.head = 0;
        *ka.tq.tail = (unsigned)ka.ntiles;
        *ka.tq.pending = ka.ntiles;
        ka.ctl->status = 0;
        ka.ctl->sticky = 0;
        ka.ctl->done = 0;
        ka.ctl->want_reset = 0;
    }
}

// Between attempts: decide whether the persistent kernel must run again
// (tile queue overflowed) and reset the queue counters for it.  The final
// call records the outcome of the whole sequence in `errors`.
__global__ void decide_kernel(const __grid_constant__ KArgs ka, int final_step) {
    Control *c = ka.ctl;
    if (final_step) {
        if (!c->done) c->errors |= ST_OVERFLOW;
        c->errors |= c->sticky & ST_TIMEOUT;
        c->want_reset = 0;
        return;
    }
    if (c->done) { c->want_reset = 0; return; }
    if (c->status & ST_TIMEOUT) {
        c->want_reset = 0;
        c->done = 1;  // a timeout is final; the host reports it
        return;
    }
    if (c->status & ST_OVERFLOW) {
        c->want_reset = 1;
        c->status = 0;
        c->relaunches += 1;
        *ka.tq.head = 0;
        *ka.tq.tail = (unsigned)ka.ntiles;
        *ka.tq.pending = ka.ntiles;
    } else {
        c->done = 1;
        c->want_reset = 0;
    }
}

int smem_bytes(int tile) {
    switch (tile) {
        case 32: return Geo<32>::WORDS * 4;
        case 64: return Geo<64>::WORDS * 4;
        default: return -1;
    }
}

template <int TS>
static cudaError_t setup_attr() {
    return cudaFuncSetAttribute(persistent_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                Geo<TS>::WORDS * 4);
}

int max_blocks_per_sm(int tile, int *out) {
    cudaError_t e;
    int n = 0;
    if (tile == 32) {
        if ((e = setup_attr<32>()) != cudaSuccess) return (int)e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_kernel<32>, NT, Geo<32>::WORDS * 4);
    } else if (tile == 64) {
        if ((e = setup_attr<64>()) != cudaSuccess) return (int)e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_kernel<64>, NT, Geo<64>::WORDS * 4);
    } else {
        return (int)cudaErrorInvalidValue;
    }
    *out = n;
    return (int)e;
}

cudaError_t launch_init(const KArgs &ka, int first_attempt, cudaStream_t s) {
    int blocks = (int)((ka.tq.cap + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    fill_queue_kernel<<<blocks, 256, 0, s>>>(ka, first_attempt);
    return cudaGetLastError();
}

cudaError_t launch_persistent(const KArgs &ka, int tile, int grid, cudaStream_t s) {
    if (tile == 32) {
        persistent_kernel<32><<<grid, NT, Geo<32>::WORDS * 4, s>>>(ka);
    } else if (tile == 64) {
        persistent_kernel<64><<<grid, NT, Geo<64>::WORDS * 4, s>>>(ka);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_decide(const KArgs &ka, int final_step, cudaStream_t s) {
    decide_kernel<<<1, 1, 0, s>>>(ka, final_step);
    return cudaGetLastError();
}

cudaError_t launch_reset(const KArgs &ka, cudaStream_t s) {
    int blocks = (int)((ka.tq.cap + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    fill_queue_kernel<<<blocks, 256, 0, s>>>(ka, 0);
    return cudaGetLastError();
}

}  // namespace iwpp
