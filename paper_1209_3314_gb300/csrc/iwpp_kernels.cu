// iwpp_kernels.cu -- the persistent tile-wavefront kernels of libiwpp.
//
// The image is cut into 64x64 tiles.  A persistent kernel drains a queue of
// tiles (the tile-level form of the wavefront loop of Algorithms 1 and 4: a
// tile is queued again whenever a neighbour can still propagate into it,
// which is the border-propagation step of Section 4 done on one device).
//
// Visiting a tile:
//   1. stage tile + 1-pixel halo in shared memory with TMA boxes (plain
//      loads when the image pitch does not meet TMA alignment);
//   2. reconstruction, first visit: raster and anti-raster sweeps, each
//      split into a row and a column pass as in Algorithm 5 (N^{+,0},
//      N^{0,+}, N^{-,0}, N^{0,-}), then one elementary geodesic dilation
//      step whose changed pixels seed the queue (afterwards every pixel that
//      can still propagate is queued: the role of Algorithm 5's
//      full-neighbourhood seed test);
//      distance transform, first visit: Algorithm 6's initialisation, with
//      the features that can improve a neighbour as the wavefront;
//      any later visit: only the halo can have changed (the interior was
//      left stable), so the halo pixels that can propagate inward are the
//      seeds;
//   3. wavefront propagation inside the tile in rounds over in/out queues
//      (Algorithm 4): a max-update for reconstruction (Algorithm 5), a
//      min-update of the packed (squared distance, feature) word for the
//      distance transform (Algorithm 6's compare-and-swap, done as one
//      64-bit atomicMin); each thread keeps the up to 8 neighbours it
//      queues as a bit mask (the per-thread queue of Section 3.2), a warp
//      prefix sum over those counts reserves the warp's block-queue space
//      with one shared atomic, and a block queue that is full spills to the
//      CTA's global queue; items beyond both are dropped and the tile is
//      rescanned (Section 3.2's restart from a partial result);
//   4. store the tile, then test each border pixel against the neighbouring
//      tiles' current values and queue every neighbour that could change.
// Tiles only write their own pixels and values move one way (up for
// reconstruction, towards closer features for the distance transform), so
// every interleaving of visits reaches a fixpoint of the propagation rule.
#include <climits>
#include <cstdint>

#include "iwpp_internal.h"
#include "iwpp_tma.cuh"

namespace iwpp {

constexpr int TS = TILE;       // 64
constexpr int RR = TS + 2;     // staged rows / columns
constexpr int QCAP_R = 1024;   // int32 reconstruction block-queue entries per buffer
constexpr int QCAP_U8 = 512;   // uint8 reconstruction block-queue entries per buffer
constexpr int QCAP_E = 2048;   // distance-transform block-queue entries per buffer

// u8 TMA box: columns x0-16 .. x0+79 (96), rows y0-1 .. y0+64 (66)
constexpr int BU8_W = 96, BU8_BYTES = BU8_W * RR, BU8_PAD = 6400;
// int32 TMA box: columns x0-4 .. x0+67 (72), rows y0-1 .. y0+64
constexpr int BI32_W = 72, BI32_BYTES = BI32_W * RR * 4, BI32_PAD = 19072;
// u8 working layout = the u8 TMA box: row stride 96 bytes, cell (r, c) at
// byte r*96 + c + 15, so the 64 interior cells of a row are four aligned
// 16-byte words (bytes 16 .. 79).
constexpr int WU8_P = BU8_W, WU8_C0 = 15;
// distance-transform working array: the int32 TMA box layout (stride 72,
// cell (r, c) at word r*72 + c + 3), holding packed feature coordinates

// shared header (ints)
enum : int {
    H_TILE = 0, H_CNT0 = 1, H_CNT1 = 2, H_RESCAN = 3,
    H_SRC = 4,    // 3x3 neighbourhood: 0 unvisited tile, 1 visited, 2 outside the image
    H_FLAG = 13,  // 3x3 neighbourhood: needs a visit
    H_PUSH = 22, H_SPILL = 23, H_RESC = 24, H_SEEDS = 25, H_ROUNDS = 26,
    H_OFF = 32,   // 9 neighbour offsets of the current layout
    H_CHG = 44,   // the visit lowered a value (watershed-family visits)
    H_PH = 48,    // 4 phase durations of the visit (ns, low 32 bits)
    H_SETS = 52,  // sweep sets the visit ran
};
constexpr int HDR_BYTES = 512;  // header ints, mbarrier at byte 256, CTA counters at byte 320
constexpr int HDR_STATS = 320;  // 12 x u64: tiles, seeds, pushes, spills, rescans, rounds, phase[4], sets, revisits

// byte offsets of the layouts.  The uint8 reconstruction works in its two
// TMA boxes and keeps short block queues (overflow spills to global): its
// visits are latency-bound, so shared memory per CTA -- which sets the
// resident CTAs per SM -- is what its throughput follows.
constexpr int RU8_JW = HDR_BYTES, RU8_IW = RU8_JW + BU8_PAD, RU8_U = RU8_IW + BU8_PAD;
constexpr int RU8_BYTES = RU8_U + 2 * QCAP_U8 * 2;
constexpr int RI32_J = HDR_BYTES, RI32_I = RI32_J + BI32_PAD, RI32_U = RI32_I + BI32_PAD;
constexpr int RI32_BYTES = RI32_U + 2 * QCAP_R * 2;
constexpr int E_W = HDR_BYTES, E_U = E_W + BI32_PAD;
constexpr int E_BYTES = E_U + 2 * QCAP_E * 2;
static_assert(RU8_JW % 128 == 0 && RU8_IW % 128 == 0 && RI32_J % 128 == 0 && RI32_I % 128 == 0 && RI32_U % 128 == 0 &&
                  E_U % 128 == 0 && E_W % 128 == 0,
              "TMA destinations must be 128-byte aligned");
static_assert(
                  BU8_PAD <= 2 * QCAP_E * 2,
              "queues must fit the staging union");
// the distance transform's sweep change flags (320 bytes at the end of the
// second queue buffer) must not overlap the binary box or the first buffer
static_assert(BU8_BYTES <= 2 * QCAP_E * 2 - 320 && QCAP_E * 2 <= 2 * QCAP_E * 2 - 320, "EDT change flags");
// the wide-window pass's box (tile + 8-pixel halo, int32) fits the layout
static_assert(E_W + (TS + 16) * (TS + 16) * 4 + 32 <= E_BYTES, "EDT wide-window box and its change masks");

constexpr int cmax(int a, int b) { return a > b ? a : b; }
// geodesic distance: D as the int32 box layout (stride 72, cell (r, c) at
// word r*72 + c + 3), the mask as a uint8 box (stride 96, cell (r, c) at
// byte r*96 + c + 15), then the block queues: 30,080 bytes, so that 7 CTAs
// fit an SM (the sources are read from global memory when needed)
constexpr int QCAP_G = 1024;
constexpr int G_D = HDR_BYTES, G_M = G_D + BI32_PAD, G_U = 25984;
constexpr int G_BYTES = G_U + 2 * QCAP_G * 2;
static_assert(G_M + BU8_BYTES <= G_U && G_U % 128 == 0 && G_M % 128 == 0, "geodesic layout");
// watershed propagations: the same V / E boxes, the block queues after them
constexpr int WS_BYTES = G_U + 2 * QCAP_G * 2;
constexpr int FAM_SMEM[FAM_COUNT] = {RU8_BYTES, RI32_BYTES, E_BYTES,
                                     cmax(cmax(RU8_BYTES, RI32_BYTES), E_BYTES), G_BYTES, WS_BYTES};
constexpr int FAM_NT[FAM_COUNT] = {64, 64, 128, 128, 64, 64};
// resident CTAs per SM that each family's shared memory allows; the
// register budget is sized for them
constexpr int FAM_MINB[FAM_COUNT] = {14, 5, 8, 5, 7, 7};

// neighbourhood offsets (dy, dx); 8-connected: the first 4 are N+ (raster)
__device__ __forceinline__ int nb_dy(int conn, int k) {
    return conn == 8 ? (k < 3 ? -1 : (k < 5 ? 0 : 1)) : (k == 0 ? -1 : (k == 3 ? 1 : 0));
}
__device__ __forceinline__ int nb_dx(int conn, int k) {
    return conn == 8 ? ((k == 0 || k == 3 || k == 5) ? -1 : ((k == 2 || k == 4 || k == 7) ? 1 : 0))
                     : (k == 1 ? -1 : (k == 2 ? 1 : 0));
}

__device__ __forceinline__ const JobDesc *job_of(const KArgs &ka, int t) {
    if (ka.njobs == 1) return &ka.job0;
    int lo = 0, hi = ka.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&ka.jobs[mid].tile_base) <= t) lo = mid; else hi = mid - 1;
    }
    return ka.jobs + lo;
}

__device__ __forceinline__ int region(int v) { return v == 0 ? 0 : (v == RR - 1 ? 2 : 1); }

// the k-th of the 4*(TS+1) halo cells: top row, bottom row, left, right
__device__ __forceinline__ void halo_cell(int k, int &r, int &c) {
    if (k < RR) { r = 0; c = k; }
    else if (k < 2 * RR) { r = RR - 1; c = k - RR; }
    else if (k < 2 * RR + TS) { r = k - 2 * RR + 1; c = 0; }
    else { r = k - 2 * RR - TS + 1; c = RR - 1; }
}

// 3x3 'visited' states of the tile neighbourhood -> hdr[H_SRC..]
__device__ __forceinline__ void load_sources(const KArgs &ka, const JobDesc *jd, int tx, int ty, int *hdr) {
    const int tid = threadIdx.x;
    if (tid < 9) {
        const int ny = ty + tid / 3 - 1, nx = tx + tid % 3 - 1;
        int v = 2;
        if (ny >= 0 && ny < jd->tiles_y && nx >= 0 && nx < jd->tiles_x)
            v = ld_acquire(ka.tq.visited + jd->tile_base + ny * jd->tiles_x + nx) ? 1 : 0;
        hdr[H_SRC + tid] = v;
    }
}

__device__ __forceinline__ void begin_visit(int *hdr) {
    const int tid = threadIdx.x;
    if (tid < 9) hdr[H_FLAG + tid] = 0;
    if (tid == 0) {
        hdr[H_CNT0] = 0; hdr[H_CNT1] = 0; hdr[H_RESCAN] = 0;
        hdr[H_PUSH] = 0; hdr[H_SPILL] = 0; hdr[H_RESC] = 0; hdr[H_SEEDS] = 0; hdr[H_ROUNDS] = 0;
        hdr[H_PH] = hdr[H_PH + 1] = hdr[H_PH + 2] = hdr[H_PH + 3] = 0;
        hdr[H_SETS] = 0;
    }
}

// Marks the tile visited once its result is stored (thread 0; the barrier
// before it completed every thread's stores).
__device__ __forceinline__ void publish_tile(const KArgs &ka, int gt, int *hdr) {
    if (threadIdx.x == 0 && hdr[H_SRC + 4] != 1) {
        __threadfence();
        st_release(ka.tq.visited + gt, 1);
    }
}

// Queues the flagged neighbours (threads 0..8, one neighbour each) and, in
// parallel on thread 4, ends the tile's own visit (tq_finish: a fence, then
// the state change, which re-queues the tile if a neighbour asked
// meanwhile).  Called by all threads after the border test; the barrier at
// the end precedes the caller's fenced pending-count decrement, so every
// push is performed before it.
__device__ __forceinline__ void finish_tile(const KArgs &ka, const JobDesc *jd, int gt, int tx, int ty, int *hdr) {
    const int k = threadIdx.x;
    if (k == 4) {
        tq_finish(ka.tq, ka.ctl, gt);
    } else if (k < 9 && hdr[H_FLAG + k]) {
        __threadfence();
        tq_push(ka.tq, ka.ctl, jd->tile_base + (ty + k / 3 - 1) * jd->tiles_x + tx + k % 3 - 1);
    }
    __syncthreads();
}

// Per-visit phase timing (thread 0): mark(i) closes phase i.
struct PhaseClock {
    unsigned long long t;
    __device__ __forceinline__ void start() { if (threadIdx.x == 0) t = globaltimer_ns(); }
    __device__ __forceinline__ void mark(int *hdr, int i) {
        if (threadIdx.x == 0) {
            const unsigned long long n = globaltimer_ns();
            hdr[H_PH + i] += (int)(n - t);
            t = n;
        }
    }
};

// neighbour offsets in a layout with row pitch P -> hdr[H_OFF..]; entry 8
// is 0 (the pixel itself)
template <int CONN, int P>
__device__ __forceinline__ void make_offsets(int *hdr) {
    if (threadIdx.x < 9) {
        const int n = threadIdx.x;
        hdr[H_OFF + n] = n < CONN ? nb_dy(CONN, n) * P + nb_dx(CONN, n) : 0;
    }
}

// ------------------------------------------------------------ the queues

// Round queue: virtual array [block queue in shared memory | CTA spill
// queue in global memory]; entries past both are dropped (rescan flag).
struct RQ {
    uint16_t *s;
    uint16_t *g;
    int *count;
    int *rescan;
    int cap_s, cap_g;
    int per_thread;  // queue ablation: one shared atomic per pushing thread
};

__device__ __forceinline__ void rq_put(const RQ &q, int pos, int item) {
    if (pos < q.cap_s) q.s[pos] = (uint16_t)item;
    else if (pos - q.cap_s < q.cap_g) q.g[pos - q.cap_s] = (uint16_t)item;
    else *q.rescan = 1;
}

__device__ __forceinline__ int rq_get(const uint16_t *s, const uint16_t *g, int cap_s, int i) {
    return i < cap_s ? s[i] : __ldcg(g + (i - cap_s));
}

// Warp-aggregated enqueue: each lane holds up to 9 items as a neighbour bit
// mask (its per-thread queue; bit 8 is the pixel itself); an inclusive warp
// scan of the counts gives each lane its slots and the last lane reserves
// the warp's total with one shared atomic.  Called by all 32 lanes.  With
// q.per_thread (queue ablation) every pushing lane reserves its own slots.
__device__ __forceinline__ unsigned warp_enqueue(unsigned mask, int p, const int *off, const RQ &q) {
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(mask);
    if (!__any_sync(0xffffffffu, cnt)) return 0;
    if (q.per_thread) {
        if (cnt) {
            int pos = atomicAdd(q.count, cnt);
            while (mask) {
                const int k = __ffs(mask) - 1;
                mask &= mask - 1;
                rq_put(q, pos++, p + off[k]);
            }
        }
        return __reduce_add_sync(0xffffffffu, (unsigned)cnt);
    }
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (lane == 31) base = atomicAdd(q.count, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    int pos = base + incl - cnt;
    while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1;
        rq_put(q, pos++, p + off[k]);
    }
    return (unsigned)total;
}

// Propagation rounds until the queue is empty (the loop of Algorithm 4).
// proc(p, n): tests / updates neighbour n of item p, true if it raised it;
// rescan(q): re-seeds the whole tile into q, returns the count.
template <int NT, int NB, typename Proc, typename Rescan>
__device__ void run_rounds(int *hdr, uint16_t *Q0, uint16_t *Q1, int qcap, uint16_t *spill, int spill_cap,
                           const int *off, Proc proc, Rescan rescan, unsigned long long deadline, Control *ctl,
                           int per_thread) {
    const int tid = threadIdx.x;
    int cur = 0;
    unsigned pushed = 0, spilled = 0, rescans = 0, rounds = 0;
    while (true) {
        // every round makes progress, so the loop ends; the deadline is a
        // last guard that turns a defect into a reported timeout
        if (tid == 0 && (rounds & 63) == 63 && globaltimer_ns() > deadline) {
            atomicOr(&ctl->status, ST_TIMEOUT);
            atomicOr(&ctl->sticky, ST_TIMEOUT);
            hdr[H_CNT0 + cur] = 0;
            hdr[H_RESCAN] = 0;
        }
        __syncthreads();
        const int n_raw = hdr[H_CNT0 + cur];
        const int resc = hdr[H_RESCAN];
        const int n_in = min(n_raw, qcap + spill_cap);
        if (n_in == 0 && !resc) break;
        __syncthreads();
        if (tid == 0) {
            hdr[H_CNT0 + (cur ^ 1)] = 0;
            hdr[H_RESCAN] = 0;
        }
        spilled += n_in > qcap ? n_in - qcap : 0;
        rescans += resc ? 1 : 0;
        ++rounds;
        __syncthreads();
        const uint16_t *qs = cur ? Q1 : Q0;
        const uint16_t *qg = spill + cur * spill_cap;
        RQ out{cur ? Q0 : Q1, spill + (cur ^ 1) * spill_cap, hdr + H_CNT0 + (cur ^ 1), hdr + H_RESCAN, qcap,
               spill_cap, per_thread};
        // neighbour-parallel: lane task k handles neighbour k % NB of item
        // k / NB, so small frontiers still fill the lanes and each lane's
        // critical path is one neighbour test
        for (int base = 0; base < n_in * NB; base += NT) {
            const int k = base + tid;
            const int item = k / NB, n = k - item * NB;
            const int p = item < n_in ? rq_get(qs, qg, qcap, item) : -1;
            const unsigned m = (p >= 0 && proc(p, n)) ? 1u << n : 0u;
            pushed += warp_enqueue(m, p, off, out);
        }
        if (resc) {
            // the in-queue was truncated: what fitted was processed (progress),
            // the next queue comes from a scan of the partial result
            __syncthreads();
            if (tid == 0) { hdr[H_CNT0 + (cur ^ 1)] = 0; hdr[H_RESCAN] = 0; }
            __syncthreads();
            pushed += rescan(out);
        }
        cur ^= 1;
    }
    if ((tid & 31) == 0) atomicAdd(hdr + H_PUSH, (int)pushed);
    if (tid == 0) {
        hdr[H_SPILL] = (int)spilled;
        hdr[H_RESC] = (int)rescans;
        hdr[H_ROUNDS] = (int)rounds;
    }
}

// Plain (non-TMA) staging of a box with zero fill outside the image.
template <typename T, int BW>
__device__ void stage_plain(T *dst, const T *src, int64_t pitch, int h, int w, int bx, int by, int nt) {
    for (int i = threadIdx.x; i < BW * RR; i += nt) {
        const int r = i / BW, c = i - r * BW;
        const int gy = by + r, gx = bx + c;
        T v = 0;
        if (gy >= 0 && gy < h && gx >= 0 && gx < w) v = __ldcg(src + (int64_t)gy * pitch + gx);
        dst[i] = v;
    }
}

// Waits for the visit's TMA boxes; on a timeout raises ST_TIMEOUT, gives the
// copies a second bounded wait and tells the caller to abandon the kernel.
__device__ __forceinline__ bool wait_boxes(uint64_t *bar, uint32_t &phase, unsigned long long deadline,
                                           Control *ctl) {
    const bool ok = mbar_wait(bar, phase, deadline);
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicOr(&ctl->status, ST_TIMEOUT);
            atomicOr(&ctl->sticky, ST_TIMEOUT);
        }
        mbar_wait(bar, phase, globaltimer_ns() + 1000000000ull);
    }
    phase ^= 1;
    return __syncthreads_and(ok) != 0;
}

// =====================================================================
// Reconstruction by dilation (Section 2.1; Algorithms 2, 4, 5)
// =====================================================================

// Row passes (N^{+,0} left to right, then N^{-,0} right to left) of one
// uint8 working row, owned by one thread.  The 64 interior cells of J and I
// are handled as four 16-byte chunks: each chunk comes with one shared load
// per image, its 16 cells are worked on in registers (bytes extracted and
// re-inserted) and it is stored back only if it changed.  The running
// value's dependency chain is one max and one min per cell; the chunk loop
// stays rolled to keep the kernel's instruction footprint small.
template <int DIR>
__device__ __forceinline__ bool u8_row_pass(uint8_t *__restrict__ J, const uint8_t *__restrict__ I, int base) {
    uint4 *jp = (uint4 *)(J + base + 1);  // cells 1 .. 64
    const uint4 *ip = (const uint4 *)(I + base + 1);
    int run = J[base + (DIR > 0 ? 0 : TS + 1)];
    uint32_t diff = 0;
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
        const int k = DIR > 0 ? s : 3 - s;
        const uint4 a = jp[k], bm = ip[k];
        const uint32_t j[4] = {a.x, a.y, a.z, a.w}, m[4] = {bm.x, bm.y, bm.z, bm.w};
        uint32_t nw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int c = DIR > 0 ? q : 15 - q, w = c >> 2, b = c & 3;
            run = min((int)((m[w] >> (8 * b)) & 0xFFu), max((int)((j[w] >> (8 * b)) & 0xFFu), run));
            nw[w] |= (uint32_t)run << (8 * b);
        }
        const uint32_t d = (nw[0] ^ j[0]) | (nw[1] ^ j[1]) | (nw[2] ^ j[2]) | (nw[3] ^ j[3]);
        if (d) jp[k] = make_uint4(nw[0], nw[1], nw[2], nw[3]);
        diff |= d;
    }
    return diff != 0;
}

__device__ __forceinline__ bool u8_row_passes(uint8_t *__restrict__ J, const uint8_t *__restrict__ I, int r) {
    const int base = r * WU8_P + WU8_C0;  // cell 0
    const bool a = u8_row_pass<+1>(J, I, base);
    const bool b = u8_row_pass<-1>(J, I, base);
    return a || b;
}

// Row passes for int32 rows (one thread per row).  The 64 interior cells
// (16-byte aligned: a row is 288 bytes and cell 1 sits at word 4) come as
// 16-byte chunks of four cells, worked on in registers and stored back
// only if changed; the chunk loop stays rolled.
template <int DIR>
__device__ __forceinline__ bool i32_row_pass(int *__restrict__ J, const int *__restrict__ I, int base) {
    int4 *jp = (int4 *)(J + base + 1);  // cells 1 .. 64
    const int4 *ip = (const int4 *)(I + base + 1);
    int run = J[base + (DIR > 0 ? 0 : TS + 1)];
    bool ch = false;
#pragma unroll 1
    for (int s = 0; s < TS / 4; ++s) {
        const int k = DIR > 0 ? s : TS / 4 - 1 - s;
        const int4 a = jp[k], m = ip[k];
        int v[4] = {a.x, a.y, a.z, a.w};
        const int mm[4] = {m.x, m.y, m.z, m.w};
        bool d = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = DIR > 0 ? q : 3 - q;
            const int nv = min(mm[c], max(v[c], run));
            d |= nv != v[c];
            v[c] = nv;
            run = nv;
        }
        if (d) jp[k] = make_int4(v[0], v[1], v[2], v[3]);
        ch |= d;
    }
    return ch;
}

__device__ __forceinline__ bool i32_row_passes(int *__restrict__ J, const int *__restrict__ I, int base) {
    const bool a = i32_row_pass<+1>(J, I, base);
    const bool b = i32_row_pass<-1>(J, I, base);
    return a || b;
}

// Column pass (N^{0,+} downwards when DIR = +1, N^{0,-} upwards when -1) for
// the column of this thread: one thread per column, rows in sequence.  The
// vertical neighbour is this thread's own running value; the two diagonal
// neighbours of the previous row are read from shared memory, where the
// neighbouring columns' threads may or may not have stored their new value
// yet -- either is a valid lower bound, and keeping the diagonals off the
// running value's dependency chain leaves two operations per row on it.
// When a whole sweep set changes nothing, every value read was the current
// one, so the stability argument is unaffected.
template <int CONN, int DIR, typename T>
__device__ __forceinline__ bool column_pass(T *__restrict__ J, const T *__restrict__ I, int P, int c0) {
    const int c = threadIdx.x + 1;
    const int r0 = DIR > 0 ? 0 : RR - 1;
    int up = J[r0 * P + c0 + c];
    bool ch = false;
#pragma unroll 4
    for (int s = 1; s <= TS; ++s) {
        const int r = DIR > 0 ? s : RR - 1 - s;
        const int i = r * P + c0 + c;
        const int o = J[i];
        int w = o;
        if (CONN == 8) {
            const int ip = i - DIR * P;
            w = max(w, max((int)J[ip - 1], (int)J[ip + 1]));
        }
        const int v = min(max(w, up), (int)I[i]);
        if (v != o) {
            J[i] = (T)v;
            ch = true;
        }
        up = v;
    }
    return ch;
}

// One raster + anti-raster sweep set (rows both ways, then columns down and
// up); returns whether any pixel changed (block-uniform).  A set that
// changes nothing has compared every pixel with every neighbour at their
// current values, so the tile is then stable.
template <int CONN>
__device__ bool sweep_set_u8(uint8_t *J, const uint8_t *I) {
    const int t = threadIdx.x;
    bool ch = false;
    if (t < TS) ch |= u8_row_passes(J, I, t + 1);
    __syncthreads();
    if (t < TS) {
        ch |= column_pass<CONN, +1>(J, I, WU8_P, WU8_C0);
        ch |= column_pass<CONN, -1>(J, I, WU8_P, WU8_C0);
    }
    return __syncthreads_or(ch) != 0;
}

template <int CONN>
__device__ bool sweep_set_i32(int *J, const int *I) {
    const int t = threadIdx.x;
    bool ch = false;
    if (t < TS) ch |= i32_row_passes(J, I, (t + 1) * BI32_W + 3);
    __syncthreads();
    if (t < TS) {
        ch |= column_pass<CONN, +1>(J, I, BI32_W, 3);
        ch |= column_pass<CONN, -1>(J, I, BI32_W, 3);
    }
    return __syncthreads_or(ch) != 0;
}

// One elementary geodesic dilation over the tile interior (each pixel takes
// the max of its neighbourhood, clipped by the mask); every pixel that
// changes is queued.  Afterwards every pixel that can still raise a
// neighbour is in the queue (a pixel that did not change was seen by all its
// neighbours, which are therefore no longer below it where the mask allows).
// One thread per column slides a 3-row window down the tile; each pixel is
// written only by its own thread.
template <int CONN, int NT, typename T>
__device__ unsigned dilate_seed(T *__restrict__ J, const T *__restrict__ I, int P, int c0, const RQ &q, const int *off) {
    unsigned pushed = 0;
    const int t = threadIdx.x;
    if (t >= ((TS + 31) / 32) * 32) return 0;  // whole warps only
    const int c = t + 1;
    const int col = c0 + c;
    auto hmax = [&](int r) -> int {
        const int i = r * P + col;
        return CONN == 8 ? max(J[i], max(J[i - 1], J[i + 1])) : (int)J[i];
    };
    int hp = hmax(0), hc = hmax(1);
    for (int r = 1; r <= TS; ++r) {
        const int hn = hmax(r + 1);
        const int i = r * P + col;
        const int o = J[i];
        int m = max(hp, max(hc, hn));
        if (CONN == 4) m = max(m, max((int)J[i - 1], (int)J[i + 1]));
        const int v = min(m, (int)I[i]);
        unsigned bit = 0;
        if (v > o) {
            J[i] = (T)v;
            bit = 1u << 8;
        }
        pushed += warp_enqueue(bit, i, off, q);
        hp = hc;
        hc = hn;
    }
    return pushed;
}

// Access policy for the two value layouts.
struct U8Grid {  // uint8 images: the TMA box layout, stride 96 bytes
    uint8_t *J;
    const uint8_t *I;
    static constexpr int P = WU8_P, C0 = WU8_C0, QCAP = QCAP_U8;
    static __device__ __forceinline__ int cell(int r, int c) { return r * P + c + C0; }
    __device__ __forceinline__ int j(int i) const { return ((volatile uint8_t *)J)[i]; }
    __device__ __forceinline__ int iv(int i) const { return I[i]; }
    __device__ __forceinline__ void set(int i, int v) const { ((volatile uint8_t *)J)[i] = (uint8_t)v; }
    // raises J[i] to v if below; true if this call raised it
    __device__ __forceinline__ bool raise(int i, int v) const {
        unsigned *w = (unsigned *)(J + (i & ~3));
        const int sh = (i & 3) * 8;
        unsigned old = *(volatile unsigned *)w;
        while (true) {
            if ((int)((old >> sh) & 0xFFu) >= v) return false;
            const unsigned nw = (old & ~(0xFFu << sh)) | ((unsigned)v << sh);
            const unsigned prev = atomicCAS(w, old, nw);
            if (prev == old) return true;
            old = prev;
        }
    }
    __device__ __forceinline__ bool sweep(int conn) const {
        return conn == 8 ? sweep_set_u8<8>(J, I) : sweep_set_u8<4>(J, I);
    }
    template <int CONN, int NT>
    __device__ __forceinline__ unsigned dilate(const RQ &q, const int *off) const {
        return dilate_seed<CONN, NT, uint8_t>(J, I, P, C0, q, off);
    }
};

struct I32Grid {  // int32 images: TMA box layout, stride 72 words
    int *J;
    const int *I;
    static constexpr int P = BI32_W, C0 = 3, QCAP = QCAP_R;
    static __device__ __forceinline__ int cell(int r, int c) { return r * P + c + C0; }
    __device__ __forceinline__ int j(int i) const { return ((volatile int *)J)[i]; }
    __device__ __forceinline__ int iv(int i) const { return I[i]; }
    __device__ __forceinline__ void set(int i, int v) const { ((volatile int *)J)[i] = v; }
    __device__ __forceinline__ bool raise(int i, int v) const { return atomicMax(J + i, v) < v; }
    __device__ __forceinline__ bool sweep(int conn) const {
        return conn == 8 ? sweep_set_i32<8>(J, I) : sweep_set_i32<4>(J, I);
    }
    template <int CONN, int NT>
    __device__ __forceinline__ unsigned dilate(const RQ &q, const int *off) const {
        return dilate_seed<CONN, NT, int>(J, I, P, 3, q, off);
    }
};

template <typename G>
__device__ __forceinline__ bool interior(int i) {
    const int r = i / G::P, c = i - r * G::P - G::C0;
    return r >= 1 && r <= TS && c >= 1 && c <= TS;
}

// Halo pixels that can raise an interior neighbour (later visits).
template <int CONN, int NT, typename G>
__device__ unsigned halo_seed(const G &g, const RQ &q, const int *off) {
    unsigned pushed = 0;
    for (int base = 0; base < 4 * (TS + 1); base += NT) {
        const int k = base + threadIdx.x;
        unsigned m = 0;
        int i = 0;
        if (k < 4 * (TS + 1)) {
            int r, c;
            halo_cell(k, r, c);
            i = G::cell(r, c);
            const int jp = g.j(i);
#pragma unroll
            for (int n = 0; n < CONN; ++n) {
                const int rr = r + nb_dy(CONN, n), cc = c + nb_dx(CONN, n);
                if (rr >= 1 && rr <= TS && cc >= 1 && cc <= TS) {
                    const int qi = i + off[n];
                    if (g.j(qi) < min(jp, g.iv(qi))) m = 1u << 8;
                }
            }
        }
        pushed += warp_enqueue(m, i, off, q);
    }
    return pushed;
}

template <int CONN, int NT, typename G>
__device__ void recon_propagate(const KArgs &ka, const G &g, int *hdr, uint16_t *Q0, uint16_t *Q1, bool first,
                                const int *off, PhaseClock &pc, unsigned long long deadline) {
    uint16_t *spill = ka.spill + (int64_t)blockIdx.x * 2 * ka.spill_cap;
    // block-queue capacity: 0 in the global-only queue ablation
    const int qcap = (ka.queue_mode & 2) ? 0 : G::QCAP;
    RQ q0{Q0, spill, hdr + H_CNT0, hdr + H_RESCAN, qcap, ka.spill_cap, ka.queue_mode & 1};
    auto sweeps_then_dilate = [&](const RQ &q, int sets) -> unsigned {
        bool changed = true;
        int s = 0;
        for (; s < sets && changed; ++s) changed = g.sweep(CONN);
        if (threadIdx.x == 0) hdr[H_SETS] += s;
        // a sweep set that changed nothing proves the tile stable
        if (!changed && sets > 0) return 0u;
        return g.template dilate<CONN, NT>(q, off);
    };
    unsigned seeds;
    if (first) {
        seeds = sweeps_then_dilate(q0, ka.sweeps);
    } else {
        // later visit: only the halo changed.  A few entry points are
        // cheapest as queue seeds; many mean a bulk change, which the
        // sweeps carry further per operation than the queue.
        seeds = halo_seed<CONN, NT>(g, q0, off);
        __syncthreads();
        if (hdr[H_CNT0] > ka.revisit_sweep_min) {
            __syncthreads();
            if (threadIdx.x == 0) { hdr[H_CNT0] = 0; hdr[H_RESCAN] = 0; }
            __syncthreads();
            seeds = sweeps_then_dilate(q0, ka.revisit_sweeps);
        }
    }
    if ((threadIdx.x & 31) == 0) atomicAdd(hdr + H_SEEDS, (int)seeds);
    pc.mark(hdr, 1);
    auto proc = [&](int p, int n) -> bool {
        const int pr = p / G::P, pc = p - pr * G::P - G::C0;
        const int rr = pr + nb_dy(CONN, n), cc = pc + nb_dx(CONN, n);
        if (rr < 1 || rr > TS || cc < 1 || cc > TS) return false;
        const int qi = p + off[n];
        const int v = min(g.j(p), g.iv(qi));
        return g.j(qi) < v && g.raise(qi, v);
    };
    auto rescan = [&](const RQ &q) -> unsigned { return g.template dilate<CONN, NT>(q, off); };
    run_rounds<NT, CONN>(hdr, Q0, Q1, qcap, spill, ka.spill_cap, off, proc, rescan, deadline, ka.ctl,
                         ka.queue_mode & 1);
    pc.mark(hdr, 2);
}

// Border test against the neighbours' current values; flags hdr[H_FLAG..].
// Each thread first issues all its halo loads from global memory, then
// tests, so the loads' latencies overlap instead of adding up.
template <typename T, int CONN, int NT, typename G>
__device__ void recon_border(const JobDesc *jd, const G &g, int *hdr, int x0, int y0) {
    constexpr int HN = 4 * (TS + 1), HPT = (HN + NT - 1) / NT;
    const T *mk = (const T *)jd->a;
    const T *out = (const T *)jd->out;
    int val[HPT];
#pragma unroll
    for (int u = 0; u < HPT; ++u) {
        const int k = threadIdx.x + u * NT;
        val[u] = 0;
        if (k >= HN) continue;
        int r, c;
        halo_cell(k, r, c);
        const int gy = y0 - 1 + r, gx = x0 - 1 + c;
        if (gy < 0 || gy >= jd->h || gx < 0 || gx >= jd->w) continue;
        const int reg = region(r) * 3 + region(c);
        val[u] = hdr[H_SRC + reg] == 1 ? (int)__ldcg(out + (int64_t)gy * jd->po + gx)
                                       : (int)__ldcg(mk + (int64_t)gy * jd->pa + gx);
    }
#pragma unroll
    for (int u = 0; u < HPT; ++u) {
        const int k = threadIdx.x + u * NT;
        if (k >= HN) continue;
        int r, c;
        halo_cell(k, r, c);
        const int gy = y0 - 1 + r, gx = x0 - 1 + c;
        if (gy < 0 || gy >= jd->h || gx < 0 || gx >= jd->w) continue;
        const int i = G::cell(r, c);
        const int iq = g.iv(i);
        const int jq = min(val[u], iq);
        bool need = false;
#pragma unroll
        for (int n = 0; n < CONN; ++n) {
            const int pr = r + nb_dy(CONN, n), pc = c + nb_dx(CONN, n);
            if (pr >= 1 && pr <= TS && pc >= 1 && pc <= TS) need |= jq < min(g.j(G::cell(pr, pc)), iq);
        }
        if (need) hdr[H_FLAG + region(r) * 3 + region(c)] = 1;
    }
}

// Halo cells of neighbour tiles whose J lives in the other buffer (marker
// vs current result): fetch() reads them from global memory into registers
// -- all loads issued before any is used, and before the visit waits for
// its TMA boxes, so their latency overlaps the copies -- and apply() writes
// them into the staged J box and clips every halo cell by the mask (halo
// pixels are sources only, so no later step clips them).
template <typename T, int NT>
struct HaloVals {
    static constexpr int HN = 4 * (TS + 1), HPT = (HN + NT - 1) / NT;
    T val[HPT];
    bool got[HPT];
    __device__ __forceinline__ void fetch(const JobDesc *jd, const int *hdr, bool first, int x0, int y0) {
        const T *mk = (const T *)jd->a;
        const T *out = (const T *)jd->out;
#pragma unroll
        for (int u = 0; u < HPT; ++u) {
            const int k = threadIdx.x + u * NT;
            got[u] = false;
            val[u] = 0;
            if (k >= HN) continue;
            int r, c;
            halo_cell(k, r, c);
            const int src = hdr[H_SRC + region(r) * 3 + region(c)];
            const int gy = y0 - 1 + r, gx = x0 - 1 + c;
            if (src != 2 && src != (first ? 0 : 1) && gy >= 0 && gy < jd->h && gx >= 0 && gx < jd->w) {
                val[u] = src == 1 ? __ldcg(out + (int64_t)gy * jd->po + gx) : __ldcg(mk + (int64_t)gy * jd->pa + gx);
                got[u] = true;
            }
        }
    }
    template <typename Cell>
    __device__ __forceinline__ void apply(T *J, const T *I, Cell cell) {
#pragma unroll
        for (int u = 0; u < HPT; ++u) {
            const int k = threadIdx.x + u * NT;
            if (k >= HN) continue;
            int r, c;
            halo_cell(k, r, c);
            const int i = cell(r, c);
            if (got[u]) J[i] = val[u];
            if (J[i] > I[i]) J[i] = I[i];
        }
    }
};

template <int CONN, int NT>
__device__ bool recon_u8_visit(const KArgs &ka, const JobDesc *jd, int gt, char *sm, uint32_t &phase,
                               unsigned long long deadline) {
    int *hdr = (int *)sm;
    uint64_t *bar = (uint64_t *)(sm + 256);
    uint8_t *JW = (uint8_t *)(sm + RU8_JW);
    uint8_t *IW = (uint8_t *)(sm + RU8_IW);
    uint16_t *Q0 = (uint16_t *)(sm + RU8_U), *Q1 = Q0 + QCAP_U8;
    const int tid = threadIdx.x;
    const int lt = gt - jd->tile_base, tx = lt % jd->tiles_x, ty = lt / jd->tiles_x;
    const int x0 = tx * TS, y0 = ty * TS;
    const uint8_t *mk = (const uint8_t *)jd->a, *ms = (const uint8_t *)jd->b;
    uint8_t *out = (uint8_t *)jd->out;

    PhaseClock pc;
    pc.start();
    load_sources(ka, jd, tx, ty, hdr);
    begin_visit(hdr);
    make_offsets<CONN, WU8_P>(hdr);
    __syncthreads();
    const bool first = hdr[H_SRC + 4] == 0;
    const uint8_t *jsrc = first ? mk : out;
    const int64_t jpitch = first ? jd->pa : jd->po;

    // 1. stage the mask box and the box of the tile's own J source (marker
    //    on a first visit, the current result later); the boxes are the
    //    working layout.  Cells outside the image are zero in J and I (zero
    //    fill) and so never raise or get raised.  The halo cells that live
    //    in the other buffer are fetched from global memory while the boxes
    //    are in flight.
    HaloVals<uint8_t, NT> hv;
    if (jd->use_tma) {
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, 2 * BU8_BYTES);
            tma_load_2d(IW, &jd->tm[1], x0 - 16, y0 - 1, bar);
            tma_load_2d(JW, &jd->tm[first ? 0 : 2], x0 - 16, y0 - 1, bar);
        }
        hv.fetch(jd, hdr, first, x0, y0);
        if (!wait_boxes(bar, phase, deadline, ka.ctl)) return false;
    } else {
        stage_plain<uint8_t, BU8_W>(IW, ms, jd->pb, jd->h, jd->w, x0 - 16, y0 - 1, NT);
        stage_plain<uint8_t, BU8_W>(JW, jsrc, jpitch, jd->h, jd->w, x0 - 16, y0 - 1, NT);
        hv.fetch(jd, hdr, first, x0, y0);
        __syncthreads();
    }
    // halo cells from the other buffer, halo clipped by the mask; the
    // interior is clipped here on a first visit without sweeps (otherwise
    // the first row pass clips every interior pixel)
    hv.apply(JW, IW, U8Grid::cell);
    if (first && ka.sweeps == 0)
        for (int k = tid; k < TS * TS; k += NT) {
            const int i = U8Grid::cell(k / TS + 1, k % TS + 1);
            if (JW[i] > IW[i]) JW[i] = IW[i];
        }
    __syncthreads();

    pc.mark(hdr, 0);
    U8Grid g{JW, IW};
    const int *off = hdr + H_OFF;

    // 2. sweeps, 3. seeds + propagation
    recon_propagate<CONN, NT>(ka, g, hdr, Q0, Q1, first, off, pc, deadline);
    __syncthreads();

    // 4. store the interior rows (16-byte vector stores when aligned); the
    //    neighbourhood states for the border test are fetched meanwhile
    load_sources(ka, jd, tx, ty, hdr);
    {
        const bool vec = jd->use_tma != 0;  // TMA maps imply 16-byte aligned base and pitch
        for (int i = tid; i < TS * 4; i += NT) {
            const int r = i >> 2, q = i & 3;
            const int gy = y0 + r, gx = x0 + q * 16;
            if (gy >= jd->h || gx >= jd->w) continue;
            const uint32_t *src = (const uint32_t *)(JW + (r + 1) * WU8_P + WU8_C0 + 1 + q * 16);
            uint8_t *dst = out + (int64_t)gy * jd->po + gx;
            if (vec && gx + 16 <= jd->w) {
                *(uint4 *)dst = make_uint4(src[0], src[1], src[2], src[3]);
            } else {
                const int n = min(16, jd->w - gx);
                for (int b = 0; b < n; ++b) dst[b] = JW[(r + 1) * WU8_P + WU8_C0 + 1 + q * 16 + b];
            }
        }
    }
    __syncthreads();
    publish_tile(ka, gt, hdr);
    recon_border<uint8_t, CONN, NT>(jd, g, hdr, x0, y0);
    __syncthreads();
    finish_tile(ka, jd, gt, tx, ty, hdr);
    pc.mark(hdr, 3);
    return true;
}

template <int CONN, int NT>
__device__ bool recon_i32_visit(const KArgs &ka, const JobDesc *jd, int gt, char *sm, uint32_t &phase,
                                unsigned long long deadline) {
    int *hdr = (int *)sm;
    uint64_t *bar = (uint64_t *)(sm + 256);
    int *JB = (int *)(sm + RI32_J);
    int *IB = (int *)(sm + RI32_I);
    uint16_t *Q0 = (uint16_t *)(sm + RI32_U), *Q1 = Q0 + QCAP_R;
    const int tid = threadIdx.x;
    const int lt = gt - jd->tile_base, tx = lt % jd->tiles_x, ty = lt / jd->tiles_x;
    const int x0 = tx * TS, y0 = ty * TS;
    const int *mk = (const int *)jd->a, *ms = (const int *)jd->b;
    int *out = (int *)jd->out;

    PhaseClock pc;
    pc.start();
    load_sources(ka, jd, tx, ty, hdr);
    begin_visit(hdr);
    make_offsets<CONN, BI32_W>(hdr);
    __syncthreads();
    const bool first = hdr[H_SRC + 4] == 0;
    const int *jsrc = first ? mk : out;
    const int64_t jpitch = first ? jd->pa : jd->po;

    // 1. stage the mask box and the box of the tile's own J source (marker
    //    on a first visit, the current result later); the boxes are the
    //    working layout.  The halo cells that live in the other buffer are
    //    fetched from global memory while the boxes are in flight.
    HaloVals<int, NT> hv;
    if (jd->use_tma) {
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, 2 * BI32_BYTES);
            tma_load_2d(IB, &jd->tm[1], x0 - 4, y0 - 1, bar);
            tma_load_2d(JB, &jd->tm[first ? 0 : 2], x0 - 4, y0 - 1, bar);
        }
        hv.fetch(jd, hdr, first, x0, y0);
        if (!wait_boxes(bar, phase, deadline, ka.ctl)) return false;
    } else {
        stage_plain<int, BI32_W>(IB, ms, jd->pb, jd->h, jd->w, x0 - 4, y0 - 1, NT);
        stage_plain<int, BI32_W>(JB, jsrc, jpitch, jd->h, jd->w, x0 - 4, y0 - 1, NT);
        hv.fetch(jd, hdr, first, x0, y0);
        __syncthreads();
    }
    // cells outside the image take the lowest value in J and I, so they
    // never raise or get raised; only tiles at the image edge have them
    if (x0 == 0 || y0 == 0 || x0 + TS >= jd->w || y0 + TS >= jd->h) {
        for (int i = tid; i < RR * BI32_W; i += NT) {
            const int r = i / BI32_W, c = i - r * BI32_W - 3;
            const int gy = y0 - 1 + r, gx = x0 - 1 + c;
            if (gy < 0 || gy >= jd->h || gx < 0 || gx >= jd->w) {
                JB[i] = INT_MIN;
                IB[i] = INT_MIN;
            }
        }
        __syncthreads();
    }
    // halo cells from the other buffer, halo clipped by the mask; the
    // interior is clipped here on a first visit without sweeps (otherwise
    // the first row pass clips every interior pixel)
    hv.apply(JB, IB, I32Grid::cell);
    if (first && ka.sweeps == 0)
        for (int k = tid; k < TS * TS; k += NT) {
            const int i = I32Grid::cell(k / TS + 1, k % TS + 1);
            if (JB[i] > IB[i]) JB[i] = IB[i];
        }
    __syncthreads();

    pc.mark(hdr, 0);
    I32Grid g{JB, IB};
    const int *off = hdr + H_OFF;
    recon_propagate<CONN, NT>(ka, g, hdr, Q0, Q1, first, off, pc, deadline);
    __syncthreads();
    // store the interior rows, four pixels per 16-byte store where the
    // TMA maps guarantee 16-byte aligned rows
    load_sources(ka, jd, tx, ty, hdr);
    {
        const bool vec = jd->use_tma != 0;
        for (int i = tid; i < TS * TS / 4; i += NT) {
            const int r = i >> 4, q = i & 15;
            const int gy = y0 + r, gx = x0 + 4 * q;
            if (gy >= jd->h || gx >= jd->w) continue;
            const int4 v = *(const int4 *)(JB + I32Grid::cell(r + 1, 4 * q + 1));
            int *dst = out + (int64_t)gy * jd->po + gx;
            if (vec && gx + 4 <= jd->w) {
                *(int4 *)dst = v;
            } else {
                const int vv[4] = {v.x, v.y, v.z, v.w};
                for (int b = 0; b < 4 && gx + b < jd->w; ++b) dst[b] = vv[b];
            }
        }
    }
    __syncthreads();
    publish_tile(ka, gt, hdr);
    recon_border<int, CONN, NT>(jd, g, hdr, x0, y0);
    __syncthreads();
    finish_tile(ka, jd, gt, tx, ty, hdr);
    pc.mark(hdr, 3);
    return true;
}

// =====================================================================
// Distance transform (Section 2.2; Algorithms 3 and 6).  Each staged pixel
// holds VR, the packed coordinates (y << 16 | x) of its assigned feature;
// all ones is the virtual 'inf' pixel, farther than any real pixel.  VR(q)
// takes feature f when f is strictly closer, or equally close with smaller
// packed coordinates (a fixed tie rule in place of the arrival order); the
// update is Algorithm 6's compare-and-swap loop.
// =====================================================================

constexpr unsigned VR_INF = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned pack_yx(int y, int x) { return ((unsigned)y << 16) | (unsigned)x; }

// squared distance from (y, x) to packed feature f (f != VR_INF)
__device__ __forceinline__ unsigned d2(int y, int x, unsigned f) {
    const int dy = y - (int)(f >> 16), dx = x - (int)(f & 0xFFFFu);
    return (unsigned)(dy * dy + dx * dx);
}

// does feature f (distance dn from q) beat q's current feature c?
__device__ __forceinline__ bool better(unsigned dn, unsigned f, int qy, int qx, unsigned c) {
    if (c == VR_INF) return true;
    const unsigned dc = d2(qy, qx, c);
    return dn < dc || (dn == dc && f < c);
}

__device__ __forceinline__ bool is_feature(uint8_t b, int flags) { return (flags & 1) ? b != 0 : b == 0; }

constexpr int EP = BI32_W;  // VR row stride (words)

// row of a linear feature index (0 <= idx < 2^31) through the job's
// multiply-and-shift divisor
__device__ __forceinline__ int div_w(const JobDesc *jd, int idx) {
    return (int)(((unsigned long long)(unsigned)idx * jd->wdiv_m) >> jd->wdiv_s);
}
__device__ __forceinline__ int ecell(int r, int c) { return r * EP + c + 3; }

// Can the feature of cell (pr, pc) improve its interior neighbour n?  With
// commit, performs the compare-and-swap update and reports whether this call
// made it.
__device__ __forceinline__ bool edt_try(unsigned *V, int oy, int ox, int pr, int pc, unsigned f, int n,
                                        bool commit) {
    const int rr = pr + nb_dy(8, n), cc = pc + nb_dx(8, n);
    if (rr < 1 || rr > TS || cc < 1 || cc > TS) return false;
    const int qi = ecell(rr, cc);
    const int qy = oy + rr, qx = ox + cc;
    const unsigned self = pack_yx(qy, qx);
    const unsigned dn = d2(qy, qx, f);
    unsigned c = ((volatile unsigned *)V)[qi];
    while (true) {
        if (c == self || !better(dn, f, qy, qx, c)) return false;  // a feature is its own nearest
        if (!commit) return true;
        const unsigned old = atomicCAS(V + qi, c, f);
        if (old == c) return true;
        c = old;
    }
}

// Best of the current feature and candidates for pixel (y, x): the strictly
// closer one, or the one with smaller packed coordinates when equally close
// (the same rule as the compare-and-swap updates).  The rule is one
// lexicographic comparison of 64-bit keys (squared distance << 32 | packed
// feature): squared distances stay below 2^31 for sides up to 32768, and
// 'inf' is the largest key.
__device__ __forceinline__ unsigned long long ekey(unsigned d, unsigned f) {
    return ((unsigned long long)d << 32) | f;
}
constexpr unsigned long long KEY_INF = ~0ull;

struct Pick {
    unsigned long long key;
    __device__ __forceinline__ Pick(unsigned f, int y, int x) : key(f == VR_INF ? KEY_INF : ekey(d2(y, x, f), f)) {}
    __device__ __forceinline__ void consider(unsigned cand, int y, int x) {
        if (cand != VR_INF) key = min(key, ekey(d2(y, x, cand), cand));
    }
    // a candidate whose squared distance is already known
    __device__ __forceinline__ void consider_d(unsigned cand, unsigned d) {
        if (cand != VR_INF) key = min(key, ekey(d, cand));
    }
    __device__ __forceinline__ unsigned best() const { return (unsigned)key; }
    __device__ __forceinline__ unsigned dist() const { return (unsigned)(key >> 32); }
};

// A running candidate of a sweep pass: feature f, its squared distance d to
// the current pixel and the increment t to the next pixel along the pass.
// One step along an axis changes the offset o to the feature by one, so
// (o + 1)^2 = o^2 + (2o + 1): d grows by t, and t by 2.  When the pass
// takes a new feature at offset o (pixel minus feature, signed along the
// pass direction), t = 2o + 1.
struct Run {
    unsigned f, d;
    int t;
    __device__ __forceinline__ void step() { d += (unsigned)t; t += 2; }
    __device__ __forceinline__ void take(unsigned nf, unsigned nd, int o) { f = nf; d = nd; t = 2 * o + 1; }
};

// Row pass of the distance-transform sweep (one thread per row, DIR +1
// left to right, -1 right to left): each pixel keeps the better of its own
// feature and the previous pixel's, as Danielsson's raster vector
// propagation does.  The features are read four cells at a time with
// 16-byte loads (cell 1 sits at word r*72 + 4): the threads of a warp own
// rows 72 words apart, which scalar loads would put on 4 banks.  Only the
// cells a pass improves are stored.  The previous pixel's feature carries
// its squared distance along (Run), so only the pixel's own feature needs a
// distance computation.
template <int DIR>
__device__ __forceinline__ bool edt_row_pass(unsigned *__restrict__ V, int r, int oy, int ox, uint8_t *RF,
                                             uint8_t *CF) {
    const int base = r * EP + 3, y = oy + r;
    const uint4 *vp = (const uint4 *)(V + base + 1);
    bool ch = false;
    const int c0 = DIR > 0 ? 0 : TS + 1;
    Run run;
    {
        const unsigned f = V[base + c0];
        if (f == VR_INF) {
            run.f = VR_INF;
            run.d = 0;
            run.t = 0;
        } else {
            const int x = ox + c0;
            run.take(f, d2(y, x, f), DIR * (x - (int)(f & 0xFFFFu)));
        }
    }
    const unsigned self1 = pack_yx(y, ox + 1);  // cell 1; ox + 1 = x0 >= 0
#pragma unroll 1
    for (int s = 0; s < TS / 4; ++s) {
        const int k = DIR > 0 ? s : TS / 4 - 1 - s;
        const uint4 q = vp[k];
        const unsigned f4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int jj = DIR > 0 ? j : 3 - j;
            const int c = 4 * k + jj + 1;
            const unsigned f = f4[jj];
            run.step();
            if (f == self1 + (unsigned)(c - 1)) {  // a feature is its own nearest
                run.f = f;
                run.d = 0;
                run.t = 1;
                continue;
            }
            Pick p(f, y, ox + c);
            p.consider_d(run.f, run.d);
            const unsigned b = p.best();
            if (b != f) {
                V[base + c] = b;
                CF[c] = 1;
                ch = true;
            }
            if (b != run.f) run.take(b, p.dist(), DIR * (ox + c - (int)(b & 0xFFFFu)));
        }
    }
    if (ch) RF[r] = 1;
    return ch;
}

// Column pass of the distance-transform sweep (DIR +1 downwards over the
// upper neighbours, -1 upwards over the lower ones), one thread per column.
// The vertical candidate is this thread's running feature, which carries
// its squared distance along (Run); the diagonal ones are read from shared
// memory, where the neighbouring columns' threads may or may not have
// stored their new feature yet -- either is a valid candidate, and keeping
// them off the running feature's dependency chain leaves only the vertical
// candidate's test on it.  The row loop stays rolled: with the two halves
// of the CTA running the two directions' code at once, a smaller
// instruction footprint measured 6 % faster than two-fold unrolling.
template <int DIR>
__device__ __forceinline__ bool edt_column_pass(unsigned *__restrict__ V, int oy, int ox, int t, uint8_t *RF,
                                                uint8_t *CF) {
    const int c = t + 1, x = ox + c;
    const int r0 = DIR > 0 ? 0 : RR - 1;
    Run up;
    {
        const unsigned f = V[ecell(r0, c)];
        if (f == VR_INF) {
            up.f = VR_INF;
            up.d = 0;
            up.t = 0;
        } else {
            const int y = oy + r0;
            up.take(f, d2(y, x, f), DIR * (y - (int)(f >> 16)));
        }
    }
    bool ch = false;
#pragma unroll 1
    for (int s = 1; s <= TS; ++s) {
        const int r = DIR > 0 ? s : RR - 1 - s;
        const int i = ecell(r, c), y = oy + r, ip = i - DIR * EP;
        const unsigned f = V[i];
        up.step();
        if (f == pack_yx(y, x)) {  // a feature is its own nearest
            up.f = f;
            up.d = 0;
            up.t = 1;
            continue;
        }
        Pick p(f, y, x);
        p.consider(V[ip - 1], y, x);
        p.consider(V[ip + 1], y, x);
        p.consider_d(up.f, up.d);
        const unsigned b = p.best();
        if (b != f) {
            V[i] = b;
            RF[r] = 1;
            ch = true;
        }
        if (b != up.f) up.take(b, p.dist(), DIR * (y - (int)(b >> 16)));
    }
    if (ch) CF[c] = 1;
    return ch;
}

// One sweep set on 128 threads: threads 0..63 run the left-to-right row
// pass and then the downward column pass, threads 64..127 the right-to-left
// row pass and then the upward column pass, at the same time.  A pixel
// written by both halves keeps one of the two candidates (a valid feature
// either way; later steps use compare-and-swap and so only improve it).
// Block-uniform "changed" result: a set that changes nothing wrote nothing,
// so every pixel was compared with all 8 neighbours' current features and
// the tile is stable.  RF[r] / CF[c] (cleared by the caller) are set for
// every row / column in which the set wrote a pixel.
template <int NT>
__device__ bool edt_sweep_set(unsigned *V, int oy, int ox, uint8_t *RF, uint8_t *CF) {
    const int t = threadIdx.x;
    bool ch = false;
    if (NT >= 2 * TS) {
        if (t < TS) {
            ch |= edt_row_pass<+1>(V, t + 1, oy, ox, RF, CF);
            ch |= edt_column_pass<+1>(V, oy, ox, t, RF, CF);
        } else if (t < 2 * TS) {
            ch |= edt_row_pass<-1>(V, t - TS + 1, oy, ox, RF, CF);
            ch |= edt_column_pass<-1>(V, oy, ox, t - TS, RF, CF);
        }
    } else {
        if (t < TS) {
            ch |= edt_row_pass<+1>(V, t + 1, oy, ox, RF, CF);
            ch |= edt_row_pass<-1>(V, t + 1, oy, ox, RF, CF);
        }
        __syncthreads();
        if (t < TS) {
            ch |= edt_column_pass<+1>(V, oy, ox, t, RF, CF);
            ch |= edt_column_pass<-1>(V, oy, ox, t, RF, CF);
        }
    }
    return __syncthreads_or(ch) != 0;
}

// One propagation step over the interior: each pixel takes the best feature
// of its 8-neighbourhood; pixels that change are queued.  Afterwards every
// pixel that can still improve a neighbour is queued (a pixel that did not
// change was seen by all its neighbours).  Each pixel is written only by its
// own thread.
//
// After a sweep set, only pixels with a pixel written by that set in their
// 3x3 neighbourhood can be improved by a neighbour: any other pixel and all
// its neighbours kept their features through the set, whose passes compared
// the pixel with each neighbour's feature, so none is strictly better (nor
// equally near with smaller coordinates).  NR[r] / NC[c] (rows / columns
// within one of a written one) select those pixels; the others are
// skipped.  The argument for the queue holds unchanged: a skipped pixel
// can only become improvable by a neighbour that changes in this step,
// and that neighbour is queued.
template <int NT>
__device__ unsigned edt_dilate_seed(unsigned *V, int oy, int ox, const RQ &q, const int *off, const uint8_t *NR,
                                    const uint8_t *NC) {
    unsigned pushed = 0;
    for (int base = 0; base < TS * TS; base += NT) {
        const int k = base + threadIdx.x;
        unsigned m = 0;
        int i = 0;
        if (k < TS * TS) {
            const int r = k / TS + 1, c = k - (k / TS) * TS + 1;
            const int y = oy + r, x = ox + c;
            i = ecell(r, c);
            const unsigned f = V[i];
            if ((NR[r] & NC[c]) && f != pack_yx(y, x)) {  // features stay
                Pick p(f, y, x);
#pragma unroll
                for (int n = 0; n < 8; ++n) p.consider(V[i + off[n]], y, x);
                if (p.best() != f) {
                    V[i] = p.best();
                    m = 1u << 8;
                }
            }
        }
        pushed += warp_enqueue(m, i, off, q);
    }
    return pushed;
}

template <int NT>
__device__ unsigned edt_seed_scan(unsigned *V, int oy, int ox, const RQ &q, bool all, const int *off) {
    unsigned pushed = 0;
    const int ncell = all ? RR * RR : 4 * (TS + 1);
    for (int base = 0; base < ncell; base += NT) {
        const int k = base + threadIdx.x;
        unsigned m = 0;
        int i = 0;
        if (k < ncell) {
            int r, c;
            if (all) { r = k / RR; c = k - r * RR; }
            else halo_cell(k, r, c);
            i = ecell(r, c);
            const unsigned f = V[i];
            if (f != VR_INF) {
                if (f == pack_yx(oy + r, ox + c)) {
                    // a feature improves exactly its interior neighbours that
                    // are not features themselves
#pragma unroll
                    for (int n = 0; n < 8; ++n) {
                        const int rr = r + nb_dy(8, n), cc = c + nb_dx(8, n);
                        if (rr >= 1 && rr <= TS && cc >= 1 && cc <= TS &&
                            V[ecell(rr, cc)] != pack_yx(oy + rr, ox + cc))
                            m = 1u << 8;
                    }
                } else {
#pragma unroll
                    for (int n = 0; n < 8; ++n)
                        if (edt_try(V, oy, ox, r, c, f, n, false)) m = 1u << 8;
                }
            }
        }
        pushed += warp_enqueue(m, i, off, q);
    }
    return pushed;
}

template <int NT>
__device__ bool edt_visit(const KArgs &ka, const JobDesc *jd, int gt, char *sm, uint32_t &phase,
                          unsigned long long deadline) {
    int *hdr = (int *)sm;
    uint64_t *bar = (uint64_t *)(sm + 256);
    unsigned *V = (unsigned *)(sm + E_W);  // also the landing zone of the nearest box
    uint8_t *BB = (uint8_t *)(sm + E_U);   // binary box (then the queues)
    uint16_t *Q0 = (uint16_t *)(sm + E_U), *Q1 = Q0 + QCAP_E;
    const int tid = threadIdx.x;
    const int lt = gt - jd->tile_base, tx = lt % jd->tiles_x, ty = lt / jd->tiles_x;
    const int x0 = tx * TS, y0 = ty * TS;
    const int oy = y0 - 1, ox = x0 - 1;

    PhaseClock pc;
    pc.start();
    load_sources(ka, jd, tx, ty, hdr);
    begin_visit(hdr);
    make_offsets<8, EP>(hdr);
    __syncthreads();
    int need_b = 0, need_n = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        need_b |= hdr[H_SRC + k] == 0;
        need_n |= hdr[H_SRC + k] == 1;
    }
    const bool first = hdr[H_SRC + 4] == 0;
    if (jd->use_tma) {
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, need_b * BU8_BYTES + need_n * BI32_BYTES);
            if (need_b) tma_load_2d(BB, &jd->tm[0], x0 - 16, oy, bar);
            if (need_n) tma_load_2d(V, &jd->tm[2], x0 - 4, oy, bar);
        }
        if (!wait_boxes(bar, phase, deadline, ka.ctl)) return false;
    } else {
        if (need_b)
            stage_plain<uint8_t, BU8_W>(BB, (const uint8_t *)jd->a, jd->pa, jd->h, jd->w, x0 - 16, oy, NT);
        if (need_n) stage_plain<int, BI32_W>((int *)V, jd->nearest, jd->w, jd->h, jd->w, x0 - 4, oy, NT);
        __syncthreads();
    }
    // A first visit of a tile whose pixels are all features (inside the
    // image) has its result already: each pixel is its own nearest feature
    // at distance 0, and no neighbour can ever improve it, so neighbours
    // never ask for a second visit.  Such a tile skips steps 1-3; its store
    // and border test use its own coordinates directly.
    bool trivial = false;
    if (first && x0 + TS <= jd->w && y0 + TS <= jd->h) {
        bool all = true;
        for (int k = tid; k < TS * 4; k += NT) {  // 16-byte chunks of the interior rows
            const uint4 b = *(const uint4 *)(BB + (k / 4 + 1) * BU8_W + 16 + (k & 3) * 16);
            const unsigned w4[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const unsigned v = w4[j];
                // FEATURE_ZERO: every byte 0; FEATURE_NONZERO: no byte 0
                all &= (jd->flags & 1) ? ((v - 0x01010101u) & ~v & 0x80808080u) == 0 : v == 0;
            }
        }
        trivial = __syncthreads_and(all) != 0;
    }
    if (!trivial) {
    // 1. VR of tile + halo, converted in place: linear nearest indices of
    //    visited regions -> packed coordinates; unvisited regions from the
    //    binary image (Algorithm 6 initialisation); outside the image 'inf'
    if (!need_b && x0 > 0 && y0 > 0 && x0 + TS < jd->w && y0 + TS < jd->h) {
        // every cell lies in the image and comes from visited regions: a
        // plain index conversion over the whole box (its padding columns
        // too), no region lookups
        uint4 *V4 = (uint4 *)V;
        for (int i = tid; i < RR * EP / 4; i += NT) {
            const uint4 w4 = V4[i];
            unsigned v[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int idx = (int)v[b];
                v[b] = VR_INF;
                if (idx >= 0) {
                    const int fy = div_w(jd, idx);
                    v[b] = pack_yx(fy, idx - fy * jd->w);
                }
            }
            V4[i] = make_uint4(v[0], v[1], v[2], v[3]);
        }
    } else {
        // four cells per step: words 4q .. 4q+3 of a row hold cells
        // 4q-3 .. 4q, which lie in one column region (q = 0: the left halo
        // and padding; q = 17: the right halo and padding; else interior),
        // and their binary bytes are one aligned 32-bit word of the box
        for (int g = tid; g < RR * (EP / 4); g += NT) {
            const int r = g / (EP / 4), q = g - r * (EP / 4);
            const int gy = oy + r, c0 = 4 * q - 3;
            const int src = hdr[H_SRC + region(r) * 3 + (q == 0 ? 0 : (q == EP / 4 - 1 ? 2 : 1))];
            uint4 *vp = (uint4 *)(V + r * EP + 4 * q);
            unsigned v[4] = {VR_INF, VR_INF, VR_INF, VR_INF};
            if (gy >= 0 && gy < jd->h) {
                if (src == 1) {
                    const uint4 w4 = *vp;
                    const int idx[4] = {(int)w4.x, (int)w4.y, (int)w4.z, (int)w4.w};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = c0 + b, gx = ox + c;
                        if (c >= 0 && c < RR && gx >= 0 && gx < jd->w && idx[b] >= 0) {
                            const int fy = div_w(jd, idx[b]);
                            v[b] = pack_yx(fy, idx[b] - fy * jd->w);
                        }
                    }
                } else {
                    const unsigned bw = *(const unsigned *)(BB + r * BU8_W + 4 * q + 12);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = c0 + b, gx = ox + c;
                        if (c >= 0 && c < RR && gx >= 0 && gx < jd->w &&
                            is_feature((uint8_t)(bw >> (8 * b)), jd->flags))
                            v[b] = pack_yx(gy, gx);
                    }
                }
            }
            *vp = make_uint4(v[0], v[1], v[2], v[3]);
        }
    }
    __syncthreads();
    pc.mark(hdr, 0);
    const int *off = hdr + H_OFF;

    // 2. seeds.  First visit: raster / anti-raster vector-propagation sweeps
    //    (Danielsson-style, the same rule as the queue updates) until a set
    //    changes nothing or the set budget is spent, then one propagation
    //    step whose changed pixels seed the queue.  Later visit: only the
    //    halo changed; a few entry points seed the queue directly, many
    //    mean a bulk change handled as on a first visit.
    uint16_t *spill = ka.spill + (int64_t)blockIdx.x * 2 * ka.spill_cap;
    const int qcap = (ka.queue_mode & 2) ? 0 : QCAP_E;
    RQ q0{Q0, spill, hdr + H_CNT0, hdr + H_RESCAN, qcap, ka.spill_cap, ka.queue_mode & 1};
    // change flags of the last sweep set: rows RF, columns CF; NR / NC mark
    // the rows / columns within one of a flagged one.  They live in the
    // second queue buffer, which is free until the propagation rounds.
    uint8_t *RF = (uint8_t *)(sm + E_U + 2 * QCAP_E * 2 - 320), *CF = RF + 72, *NR = RF + 144, *NC = RF + 216;
    auto sweeps_then_dilate = [&]() -> unsigned {
        bool changed = true;
        int s = 0;
        for (; s < ka.edt_sweeps && changed; ++s) {
            if (tid < RR) { RF[tid] = 0; CF[tid] = 0; }
            __syncthreads();
            changed = edt_sweep_set<NT>(V, oy, ox, RF, CF);
        }
        if (tid == 0) hdr[H_SETS] += s;
        if (!changed) return 0u;
        if (tid >= 1 && tid <= TS) {
            NR[tid] = RF[tid - 1] | RF[tid] | RF[tid + 1];
            NC[tid] = CF[tid - 1] | CF[tid] | CF[tid + 1];
        }
        __syncthreads();
        return edt_dilate_seed<NT>(V, oy, ox, q0, off, NR, NC);
    };
    unsigned seeds;
    if (first && ka.edt_sweeps > 0) {
        seeds = sweeps_then_dilate();
    } else {
        seeds = edt_seed_scan<NT>(V, oy, ox, q0, first, off);
        __syncthreads();
        if (!first && hdr[H_CNT0] > ka.edt_revisit_sweep_min && ka.edt_sweeps > 0) {
            __syncthreads();
            if (tid == 0) { hdr[H_CNT0] = 0; hdr[H_RESCAN] = 0; }
            __syncthreads();
            seeds = sweeps_then_dilate();
        }
    }
    if ((tid & 31) == 0) atomicAdd(hdr + H_SEEDS, (int)seeds);
    pc.mark(hdr, 1);

    // 3. propagation rounds
    auto proc = [&](int p, int n) -> bool {
        const unsigned f = ((volatile unsigned *)V)[p];
        if (f == VR_INF) return false;
        const int pr = p / EP, pc2 = p - pr * EP - 3;
        return edt_try(V, oy, ox, pr, pc2, f, n, true);
    };
    auto rescan = [&](const RQ &q) -> unsigned { return edt_seed_scan<NT>(V, oy, ox, q, true, off); };
    run_rounds<NT, 8>(hdr, Q0, Q1, qcap, spill, ka.spill_cap, off, proc, rescan, deadline, ka.ctl,
                      ka.queue_mode & 1);
    __syncthreads();
    }  // !trivial
    pc.mark(hdr, 2);

    // 4. store nearest (linear index) and squared distance, four pixels per
    //    16-byte store where rows are 16-byte aligned; the neighbourhood
    //    states for the border test are fetched meanwhile
    load_sources(ka, jd, tx, ty, hdr);
    {
        const bool vec = (jd->w & 3) == 0 && ((reinterpret_cast<uintptr_t>(jd->nearest) |
                                                reinterpret_cast<uintptr_t>(jd->sqdist)) & 15) == 0;
        for (int i = tid; i < TS * TS / 4; i += NT) {
            const int r = i >> 4, q = i & 15;
            const int gy = y0 + r, gx = x0 + 4 * q;
            if (gy >= jd->h || gx >= jd->w) continue;
            int nv[4], dv[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const unsigned f = trivial ? pack_yx(gy, gx + b) : V[ecell(r + 1, 4 * q + b + 1)];
                nv[b] = f == VR_INF ? -1 : (int)(f >> 16) * jd->w + (int)(f & 0xFFFFu);
                dv[b] = f == VR_INF ? INT_MAX : (int)d2(gy, gx + b, f);
            }
            const int64_t o = (int64_t)gy * jd->w + gx;
            if (vec && gx + 4 <= jd->w) {
                *(int4 *)(jd->nearest + o) = make_int4(nv[0], nv[1], nv[2], nv[3]);
                *(int4 *)(jd->sqdist + o) = make_int4(dv[0], dv[1], dv[2], dv[3]);
            } else {
                for (int b = 0; b < 4 && gx + b < jd->w; ++b) {
                    jd->nearest[o + b] = nv[b];
                    jd->sqdist[o + b] = dv[b];
                }
            }
        }
    }
    __syncthreads();
    publish_tile(ka, gt, hdr);

    // 5. border test (strict distance rule across tiles); every halo load
    //    is issued before any is used
    {
        constexpr int HN = 4 * (TS + 1), HPT = (HN + NT - 1) / NT;
        int raw[HPT];
#pragma unroll
        for (int u = 0; u < HPT; ++u) {
            const int k = tid + u * NT;
            raw[u] = 0;
            if (k >= HN) continue;
            int r, c;
            halo_cell(k, r, c);
            const int gy = oy + r, gx = ox + c;
            if (gy < 0 || gy >= jd->h || gx < 0 || gx >= jd->w) continue;
            raw[u] = hdr[H_SRC + region(r) * 3 + region(c)] == 1
                         ? __ldcg(jd->nearest + (int64_t)gy * jd->w + gx)
                         : (int)__ldcg((const uint8_t *)jd->a + (int64_t)gy * jd->pa + gx);
        }
#pragma unroll
        for (int u = 0; u < HPT; ++u) {
            const int k = tid + u * NT;
            if (k >= HN) continue;
            int r, c;
            halo_cell(k, r, c);
            const int gy = oy + r, gx = ox + c;
            if (gy < 0 || gy >= jd->h || gx < 0 || gx >= jd->w) continue;
            const int reg = region(r) * 3 + region(c);
            unsigned cq;
            if (hdr[H_SRC + reg] == 1) {
                const int idx = raw[u];
                const int fy = div_w(jd, idx);
                cq = idx < 0 ? (unsigned)VR_INF : pack_yx(fy, idx - fy * jd->w);
            } else {
                cq = is_feature((uint8_t)raw[u], jd->flags) ? pack_yx(gy, gx) : (unsigned)VR_INF;
            }
            const unsigned dq = cq == VR_INF ? (unsigned)VR_INF : d2(gy, gx, cq);
            bool need = false;
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int pr = r + nb_dy(8, n), pcc = c + nb_dx(8, n);
                if (pr < 1 || pr > TS || pcc < 1 || pcc > TS) continue;
                const unsigned fp = trivial ? pack_yx(oy + pr, ox + pcc) : V[ecell(pr, pcc)];
                if (fp != VR_INF && d2(gy, gx, fp) < dq) need = true;
            }
            if (need) hdr[H_FLAG + reg] = 1;
        }
    }
    __syncthreads();
    finish_tile(ka, jd, gt, tx, ty, hdr);
    pc.mark(hdr, 3);
    return true;
}

// =====================================================================
// Distance transform, second wavefront with a wide window (Section 2.2: a
// sufficiently large neighbourhood makes the propagation exact).  It starts
// from the fixpoint of the 8-neighbour propagation (the nearest indices the
// first launch stored) and runs the same update rule with the window of
// all offsets (dy, dx) with |dy|, |dx| <= k in place of the 8 neighbours:
// a pixel takes the feature of any window pixel that is strictly closer
// (equally close with smaller packed coordinates), until no pixel changes.
// The half-width k of a pixel's window grows with its current squared
// distance U (KArgs::wide_u[]: k = 1 + the number of the K - 1 thresholds
// U reaches): the 8-neighbour rule departs from the exact distance only at
// pixels far from their features (Figure 3), and the farther, the wider
// the window the correction needs.
// =====================================================================

template <int K>
struct Wide {
    static constexpr int B = TS + 2 * K;  // box side: tile + K-pixel halo
    static __device__ __forceinline__ int cell(int r, int c) { return r * B + c; }  // box coordinates
};

// A pixel within k of the tile border changed: the neighbouring tiles whose
// pixels see it in their windows must be visited again (hdr[H_FLAG..]).
__device__ __forceinline__ void wide_flag(int *hdr, const JobDesc *jd, int tx, int ty, int ri, int ci, int k) {
    const int ry0 = ri < k ? 0 : 1, ry1 = ri >= TS - k ? 2 : 1;
    const int rx0 = ci < k ? 0 : 1, rx1 = ci >= TS - k ? 2 : 1;
    for (int ry = ry0; ry <= ry1; ++ry)
        for (int rx = rx0; rx <= rx1; ++rx) {
            if (ry == 1 && rx == 1) continue;
            const int ny = ty + ry - 1, nx = tx + rx - 1;
            if (ny >= 0 && ny < jd->tiles_y && nx >= 0 && nx < jd->tiles_x) hdr[H_FLAG + ry * 3 + rx] = 1;
        }
}

template <int NT, int K>
__device__ bool edt_wide_visit(const KArgs &ka, const JobDesc *jd, int gt, char *sm, uint32_t &phase,
                               unsigned long long deadline) {
    using G = Wide<K>;
    constexpr int B = G::B;
    int *hdr = (int *)sm;
    uint64_t *bar = (uint64_t *)(sm + 256);
    unsigned *V = (unsigned *)(sm + E_W);  // B x B packed features (the nearest box, converted)
    const int tid = threadIdx.x;
    const int lt = gt - jd->tile_base, tx = lt % jd->tiles_x, ty = lt / jd->tiles_x;
    const int x0 = tx * TS, y0 = ty * TS;
    const int by = y0 - K, bx = x0 - K;  // global coordinates of box cell (0, 0)

    PhaseClock pc;
    pc.start();
    begin_visit(hdr);
    if (tid == 0) hdr[H_SRC + 4] = ld_acquire(ka.tq.visited + gt);  // 0 on the tile's first visit
    __syncthreads();
    // On its first visit a tile holds the 8-neighbour fixpoint, so an inner
    // pixel (all 8 neighbours in the tile) whose window is the
    // 8-neighbourhood (k = 1) cannot change in the first pass and is
    // skipped there; border pixels, later passes and later visits test
    // every pixel (a neighbour may have changed meanwhile).
    const bool first = hdr[H_SRC + 4] == 0;
    // 1. stage the nearest indices of tile + K-pixel halo, then convert them
    //    to packed coordinates ('inf' outside the image and without feature)
    if (jd->use_tma) {
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, B * B * 4);
            tma_load_2d(V, &jd->tm[1], bx, by, bar);
        }
        if (!wait_boxes(bar, phase, deadline, ka.ctl)) return false;
    } else {
        for (int i = tid; i < B * B; i += NT) {
            const int r = i / B, c = i - r * B;
            const int gy = by + r, gx = bx + c;
            int v = -1;
            if (gy >= 0 && gy < jd->h && gx >= 0 && gx < jd->w) v = __ldcg(jd->nearest + (int64_t)gy * jd->w + gx);
            V[i] = (unsigned)v;
        }
        __syncthreads();
    }
    for (int i = tid; i < B * B; i += NT) {
        const int r = i / B, c = i - r * B;
        const int gy = by + r, gx = bx + c;
        unsigned v = VR_INF;
        if (gy >= 0 && gy < jd->h && gx >= 0 && gx < jd->w) {
            const int idx = (int)V[i];
            if (idx >= 0) {
                const int fy = div_w(jd, idx);
                v = pack_yx(fy, idx - fy * jd->w);
            }
        }
        V[i] = v;
    }
    __syncthreads();
    pc.mark(hdr, 0);

    // 2. window passes until one changes nothing.  Each pixel is written
    //    only by its own thread; a window cell read while its owner updates
    //    it gives the old or the new feature, both valid candidates, and a
    //    pass that changes nothing has compared every pixel with every
    //    window cell at its final value.  After the first pass, a pixel
    //    whose window held no pixel the previous pass changed saw all its
    //    window cells at their present values then, so it cannot change
    //    and is skipped; the rows and columns the pass changed pixels in
    //    (64-bit masks CH[0] / CH[1]; CH[2] / CH[3] for the pass running)
    //    bound the windows that did.
    unsigned long long *CH = (unsigned long long *)(sm + E_W + B * B * 4);
    if (tid < 4) CH[tid] = 0;
    __syncthreads();
    bool any = false;
    int sets = 0;
    while (true) {
        bool ch = false;
        const unsigned long long prow = CH[0], pcol = CH[1];
        for (int k = tid; k < TS * TS; k += NT) {
            const int ri = k / TS, ci = k - ri * TS;
            if (y0 + ri >= jd->h || x0 + ci >= jd->w) continue;
            const int y = y0 + ri, x = x0 + ci;
            const int i = G::cell(ri + K, ci + K);
            const unsigned f = V[i];
            if (f == pack_yx(y, x)) continue;  // a feature is its own nearest
            Pick p(f, y, x);
            const unsigned u = p.dist();
            int kw = 1;
#pragma unroll
            for (int j = 0; j < K - 1; ++j) kw += u >= (unsigned)ka.wide_u[j] ? 1 : 0;
            if (kw == 1 && first && sets == 0 && ri > 0 && ri < TS - 1 && ci > 0 && ci < TS - 1) continue;
            if (sets > 0) {
                const int r0 = max(0, ri - kw), r1 = min(TS - 1, ri + kw);
                const int c0 = max(0, ci - kw), c1 = min(TS - 1, ci + kw);
                const unsigned long long mr = (~0ull >> (63 - (r1 - r0))) << r0;
                const unsigned long long mc = (~0ull >> (63 - (c1 - c0))) << c0;
                if (!(prow & mr) || !(pcol & mc)) continue;
            }
            unsigned last = VR_INF;
            for (int dy = -kw; dy <= kw; ++dy) {
                const unsigned *row = V + i + dy * B;
                for (int dx = -kw; dx <= kw; ++dx) {
                    const unsigned g = row[dx];
                    if (g == last) continue;  // runs of one feature are tested once
                    last = g;
                    p.consider(g, y, x);
                }
            }
            const unsigned b = p.best();
            if (b != f) {
                V[i] = b;
                ch = true;
                atomicOr(CH + 2, 1ull << ri);
                atomicOr(CH + 3, 1ull << ci);
                wide_flag(hdr, jd, tx, ty, ri, ci, K);
            }
        }
        ++sets;
        if (!__syncthreads_or(ch)) break;
        any = true;
        if (tid == 0) {  // this pass's masks become the previous pass's
            CH[0] = CH[2];
            CH[1] = CH[3];
            CH[2] = 0;
            CH[3] = 0;
        }
        __syncthreads();
        // a guard only (every pass that changes something improves a pixel,
        // so the loop ends); thread 0 decides for the whole block
        if (__syncthreads_or(tid == 0 && globaltimer_ns() > deadline)) {
            if (tid == 0) {
                atomicOr(&ka.ctl->status, ST_TIMEOUT);
                atomicOr(&ka.ctl->sticky, ST_TIMEOUT);
            }
            return false;
        }
    }
    if (tid == 0) hdr[H_SETS] = sets;
    pc.mark(hdr, 1);
    pc.mark(hdr, 2);

    // 3. store what changed: nearest (linear index) and squared distance
    if (any) {
        const bool vec = (jd->w & 3) == 0 && ((reinterpret_cast<uintptr_t>(jd->nearest) |
                                                reinterpret_cast<uintptr_t>(jd->sqdist)) & 15) == 0;
        for (int i = tid; i < TS * TS / 4; i += NT) {
            const int r = i >> 4, q = i & 15;
            const int gy = y0 + r, gx = x0 + 4 * q;
            if (gy >= jd->h || gx >= jd->w) continue;
            int nv[4], dv[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const unsigned f = V[G::cell(r + K, 4 * q + b + K)];
                nv[b] = f == VR_INF ? -1 : (int)(f >> 16) * jd->w + (int)(f & 0xFFFFu);
                dv[b] = f == VR_INF ? INT_MAX : (int)d2(gy, gx + b, f);
            }
            const int64_t o = (int64_t)gy * jd->w + gx;
            if (vec && gx + 4 <= jd->w) {
                *(int4 *)(jd->nearest + o) = make_int4(nv[0], nv[1], nv[2], nv[3]);
                *(int4 *)(jd->sqdist + o) = make_int4(dv[0], dv[1], dv[2], dv[3]);
            } else {
                for (int b = 0; b < 4 && gx + b < jd->w; ++b) {
                    jd->nearest[o + b] = nv[b];
                    jd->sqdist[o + b] = dv[b];
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0 && first) {
        __threadfence();
        st_release(ka.tq.visited + gt, 1);
    }
    finish_tile(ka, jd, gt, tx, ty, hdr);
    pc.mark(hdr, 3);
    return true;
}

// =====================================================================
// Shortest paths on a grid with obstacles (Section 1's further IWPP use)
// =====================================================================
//
// D(p) = least cost of a path from a source to p through free pixels, with
// 8 moves costing 5 (straight) or 7 (diagonal).  Wavefront element: a pixel
// whose D may lower a free neighbour; update: D(q) = D(p) + w (atomicMin).
// Sweeps: Algorithm 2's raster / anti-raster passes with min-plus in place
// of max-min.  Obstacles and pixels outside the image keep GD_INF.

constexpr int GD_INF = 0x3FFFFFFF;  // > any path cost; GD_INF + 7 still fits

__device__ __forceinline__ int gcell(int r, int c) { return r * BI32_W + c + 3; }
__device__ __forceinline__ int gmask(int r, int c) { return r * BU8_W + c + 15; }
__device__ __forceinline__ int gstep(int n) { return (nb_dy(8, n) != 0 && nb_dx(8, n) != 0) ? 7 : 5; }

// Row pass (one thread per row) over an int32 working row and its uint8
// companion row (mask / in-edge bits): the 64 interior cells of both are
// 16-byte aligned (int32 cell 1 at word r*72 + 4, uint8 cell 1 at byte
// r*96 + 16), so each 16-cell chunk comes with four int4 and one uint4
// shared loads, is worked on in registers and is stored back by the int4
// that changed.  Threads of a warp own rows 72 words apart, so scalar
// accesses would fall on 4 banks; 16-byte ones spread over them.
// relax(run, old, byte) gives a cell's new value.
template <int DIR, typename Relax>
__device__ __forceinline__ bool i32_u8_row_pass(int *__restrict__ V, const uint8_t *__restrict__ M, int r,
                                                Relax relax) {
    int4 *vp = (int4 *)(V + gcell(r, 1));
    const uint4 *mp = (const uint4 *)(M + gmask(r, 1));
    int run = V[gcell(r, DIR > 0 ? 0 : TS + 1)];
    bool ch = false;
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
        const int k = DIR > 0 ? s : 3 - s;
        const uint4 mw = mp[k];
        const uint32_t m[4] = {mw.x, mw.y, mw.z, mw.w};
        int v[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int4 a = vp[4 * k + q];
            v[4 * q] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
        unsigned changed = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int c = DIR > 0 ? j : 15 - j;
            const int nv = relax(run, v[c], (m[c >> 2] >> (8 * (c & 3))) & 0xFFu);
            changed |= (nv != v[c] ? 1u : 0u) << (c >> 2);
            v[c] = nv;
            run = nv;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (changed & (1u << q)) vp[4 * k + q] = make_int4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        ch |= changed != 0;
    }
    return ch;
}

template <int DIR>
__device__ __forceinline__ bool gdt_row_pass(int *__restrict__ D, const uint8_t *__restrict__ M, int r) {
    return i32_u8_row_pass<DIR>(D, M, r, [](int run, int o, unsigned m) { return m ? min(o, run + 5) : o; });
}

// column pass; the diagonal neighbours of the previous row are read from
// shared memory (old or new: both are valid upper bounds)
template <int DIR>
__device__ __forceinline__ bool gdt_column_pass(int *__restrict__ D, const uint8_t *__restrict__ M, int t) {
    const int c = t + 1;
    const int r0 = DIR > 0 ? 0 : RR - 1;
    int up = D[gcell(r0, c)];
    bool ch = false;
#pragma unroll 4
    for (int s = 1; s <= TS; ++s) {
        const int r = DIR > 0 ? s : RR - 1 - s;
        const int i = gcell(r, c), ip = i - DIR * BI32_W;
        const int o = D[i];
        int v = o;
        if (M[gmask(r, c)]) v = min(o, min(up + 5, min(D[ip - 1], D[ip + 1]) + 7));
        if (v != o) { D[i] = v; ch = true; }
        up = v;
    }
    return ch;
}

__device__ bool gdt_sweep_set(int *D, const uint8_t *M) {
    const int t = threadIdx.x;
    bool ch = false;
    if (t < TS) {
        ch |= gdt_row_pass<+1>(D, M, t + 1);
        ch |= gdt_row_pass<-1>(D, M, t + 1);
    }
    __syncthreads();
    if (t < TS) {
        ch |= gdt_column_pass<+1>(D, M, t);
        ch |= gdt_column_pass<-1>(D, M, t);
    }
    return __syncthreads_or(ch) != 0;
}

// One relaxation step over the interior (each free pixel takes the least
// neighbour D plus step cost); the pixels it lowers are queued.  Afterwards
// every pixel that can still lower a neighbour is queued (a pixel that did
// not change was seen by each neighbour during the step).
template <int NT>
__device__ unsigned gdt_dilate_seed(int *D, const uint8_t *M, const RQ &q, const int *off) {
    unsigned pushed = 0;
    for (int base = 0; base < TS * TS; base += NT) {
        const int k = base + threadIdx.x;
        unsigned m = 0;
        int i = 0;
        if (k < TS * TS) {
            const int r = k / TS + 1, c = k - (k / TS) * TS + 1;
            i = gcell(r, c);
            if (M[gmask(r, c)]) {
                const int o = D[i];
                int v = o;
#pragma unroll
                for (int n = 0; n < 8; ++n) v = min(v, D[i + off[n]] + gstep(n));
                if (v < o) {
                    D[i] = v;
                    m = 1u << 8;
                }
            }
        }
        pushed += warp_enqueue(m, i, off, q);
    }
    return pushed;
}

// later visits: halo pixels that can lower a free interior neighbour
template <int NT>
__device__ unsigned gdt_halo_seed(int *D, const uint8_t *M, const RQ &q, const int *off) {
    unsigned pushed = 0;
    for (int base = 0; base < 4 * (TS + 1); base += NT) {
        const int k = base + threadIdx.x;
        unsigned m = 0;
        int i = 0;
        if (k < 4 * (TS + 1)) {
            int r, c;
            halo_cell(k, r, c);
            i = gcell(r, c);
            const int dp = D[i];
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int rr = r + nb_dy(8, n), cc = c + nb_dx(8, n);
                if (rr >= 1 && rr <= TS && cc >= 1 && cc <= TS && M[gmask(rr, cc)] &&
                    dp + gstep(n) < D[i + off[n]])
                    m = 1u << 8;
            }
        }
        pushed += warp_enqueue(m, i, off, q);
    }
    return pushed;
}

template <int NT>
__device__ bool gdt_visit(const KArgs &ka, const JobDesc *jd, int gt, char *sm, uint32_t &phase,
                          unsigned long long deadline) {
    int *hdr = (int *)sm;
    uint64_t *bar = (uint64_t *)(sm + 256);
    int *D = (int *)(sm + G_D);
    uint8_t *M = (uint8_t *)(sm + G_M);
    uint16_t *Q0 = (uint16_t *)(sm + G_U), *Q1 = Q0 + QCAP_G;
    const int tid = threadIdx.x;
    const int lt = gt - jd->tile_base, tx = lt % jd->tiles_x, ty = lt / jd->tiles_x;
    const int x0 = tx * TS, y0 = ty * TS;
    const uint8_t *mk = (const uint8_t *)jd->a, *sd = (const uint8_t *)jd->b;
    int *out = (int *)jd->out;

    PhaseClock pc;
    pc.start();
    load_sources(ka, jd, tx, ty, hdr);
    begin_visit(hdr);
    make_offsets<8, BI32_W>(hdr);
    // 1. stage the mask box (zero, i.e. obstacle, outside the image) and
    //    the current result's box (visited regions); in unvisited regions a
    //    free pixel starts at 0 if it is a source (read from global memory:
    //    a sources box would cost the CTA per SM that its 6 KB take),
    //    else at GD_INF
    __syncthreads();
    const bool first = hdr[H_SRC + 4] == 0;
    int need_o = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) need_o |= hdr[H_SRC + k] == 1;
    if (jd->use_tma) {
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, BU8_BYTES + need_o * BI32_BYTES);
            tma_load_2d(M, &jd->tm[0], x0 - 16, y0 - 1, bar);
            if (need_o) tma_load_2d(D, &jd->tm[2], x0 - 4, y0 - 1, bar);
        }
        if (!wait_boxes(bar, phase, deadline, ka.ctl)) return false;
    } else {
        stage_plain<uint8_t, BU8_W>(M, mk, jd->pa, jd->h, jd->w, x0 - 16, y0 - 1, NT);
        if (need_o) stage_plain<int, BI32_W>(D, out, jd->po, jd->h, jd->w, x0 - 4, y0 - 1, NT);
        __syncthreads();
    }
    int all_visited = 1;
#pragma unroll
    for (int k = 0; k < 9; ++k) all_visited &= hdr[H_SRC + k] == 1;
    if (all_visited && x0 > 0 && y0 > 0 && x0 + TS < jd->w && y0 + TS < jd->h) {
        // every cell of the box lies in the image and comes from the
        // current result: only 'unreachable' (INT32_MAX) maps to GD_INF,
        // four cells per 16-byte access (the box's padding columns too)
        int4 *D4 = (int4 *)D;
        for (int i = tid; i < RR * BI32_W / 4; i += NT) {
            int4 v = D4[i];
            v.x = min(v.x, GD_INF);
            v.y = min(v.y, GD_INF);
            v.z = min(v.z, GD_INF);
            v.w = min(v.w, GD_INF);
            D4[i] = v;
        }
    } else {
        // four cells per step: words 4q .. 4q+3 of a row hold cells
        // 4q-3 .. 4q, which lie in one column region, and their mask bytes
        // are one aligned 32-bit word of the mask box; the sources' bytes
        // are read from global memory, all four loads in flight at once
        for (int g = tid; g < RR * (BI32_W / 4); g += NT) {
            const int r = g / (BI32_W / 4), q = g - r * (BI32_W / 4);
            const int gy = y0 - 1 + r, c0 = 4 * q - 3;
            const int src = hdr[H_SRC + region(r) * 3 + (q == 0 ? 0 : (q == BI32_W / 4 - 1 ? 2 : 1))];
            int4 *dp = (int4 *)(D + r * BI32_W + 4 * q);
            int v[4] = {GD_INF, GD_INF, GD_INF, GD_INF};
            if (gy >= 0 && gy < jd->h) {
                if (src == 1) {
                    const int4 o4 = *dp;
                    const int o[4] = {o4.x, o4.y, o4.z, o4.w};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = c0 + b, gx = x0 - 1 + c;
                        if (c >= 0 && c < RR && gx >= 0 && gx < jd->w) v[b] = min(o[b], GD_INF);
                    }
                } else {
                    const unsigned mw = *(const unsigned *)(M + r * BU8_W + 4 * q + 12);
                    uint8_t sv[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = c0 + b, gx = x0 - 1 + c;
                        if (c >= 0 && c < RR && gx >= 0 && gx < jd->w && ((mw >> (8 * b)) & 0xFFu))
                            sv[b] = __ldg(sd + (int64_t)gy * jd->pb + gx);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (sv[b]) v[b] = 0;
                }
            }
            *dp = make_int4(v[0], v[1], v[2], v[3]);
        }
    }
    __syncthreads();
    pc.mark(hdr, 0);
    const int *off = hdr + H_OFF;

    // 2. seeds: sweep sets then one relaxation step (first visit, or a
    //    later visit whose halo changed in many places); else halo seeds
    uint16_t *spill = ka.spill + (int64_t)blockIdx.x * 2 * ka.spill_cap;
    const int qcap = (ka.queue_mode & 2) ? 0 : QCAP_G;
    RQ q0{Q0, spill, hdr + H_CNT0, hdr + H_RESCAN, qcap, ka.spill_cap, ka.queue_mode & 1};
    auto sweeps_then_seed = [&]() -> unsigned {
        bool changed = true;
        int s = 0;
        for (; s < ka.gdt_sweeps && changed; ++s) changed = gdt_sweep_set(D, M);
        if (tid == 0) hdr[H_SETS] += s;
        if (!changed && ka.gdt_sweeps > 0) return 0u;
        return gdt_dilate_seed<NT>(D, M, q0, off);
    };
    unsigned seeds;
    if (first) {
        seeds = sweeps_then_seed();
    } else {
        seeds = gdt_halo_seed<NT>(D, M, q0, off);
        __syncthreads();
        if (hdr[H_CNT0] > ka.gdt_revisit_sweep_min) {
            __syncthreads();
            if (tid == 0) { hdr[H_CNT0] = 0; hdr[H_RESCAN] = 0; }
            __syncthreads();
            seeds = sweeps_then_seed();
        }
    }
    if ((tid & 31) == 0) atomicAdd(hdr + H_SEEDS, (int)seeds);
    pc.mark(hdr, 1);

    // 3. propagation rounds (atomicMin updates of free interior pixels)
    auto proc = [&](int p, int n) -> bool {
        const int pr = p / BI32_W, pcol = p - pr * BI32_W - 3;
        const int rr = pr + nb_dy(8, n), cc = pcol + nb_dx(8, n);
        if (rr < 1 || rr > TS || cc < 1 || cc > TS || !M[gmask(rr, cc)]) return false;
        const int cand = ((volatile int *)D)[p] + gstep(n);
        return atomicMin(D + p + off[n], cand) > cand;
    };
    auto rescan = [&](const RQ &q) -> unsigned { return gdt_dilate_seed<NT>(D, M, q, off); };
    run_rounds<NT, 8>(hdr, Q0, Q1, qcap, spill, ka.spill_cap, off, proc, rescan, deadline, ka.ctl,
                      ka.queue_mode & 1);
    __syncthreads();
    pc.mark(hdr, 2);

    // 4. store the interior (unreachable: INT32_MAX), four pixels per
    //    16-byte store where the TMA maps guarantee 16-byte aligned rows
    load_sources(ka, jd, tx, ty, hdr);
    {
        const bool vec = jd->use_tma != 0;
        for (int i = tid; i < TS * TS / 4; i += NT) {
            const int r = i >> 4, q = i & 15;
            const int gy = y0 + r, gx = x0 + 4 * q;
            if (gy >= jd->h || gx >= jd->w) continue;
            const int4 v4 = *(const int4 *)(D + gcell(r + 1, 4 * q + 1));
            int vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int b = 0; b < 4; ++b) vv[b] = vv[b] >= GD_INF ? INT_MAX : vv[b];
            int *dst = out + (int64_t)gy * jd->po + gx;
            if (vec && gx + 4 <= jd->w) {
                *(int4 *)dst = make_int4(vv[0], vv[1], vv[2], vv[3]);
            } else {
                for (int b = 0; b < 4 && gx + b < jd->w; ++b) dst[b] = vv[b];
            }
        }
    }
    __syncthreads();
    publish_tile(ka, gt, hdr);

    // 5. border test: can an interior pixel lower a free halo pixel's
    //    current value (its tile's result, or its source value)?
    for (int k = tid; k < 4 * (TS + 1); k += NT) {
        int r, c;
        halo_cell(k, r, c);
        const int gy = y0 - 1 + r, gx = x0 - 1 + c;
        if (gy < 0 || gy >= jd->h || gx < 0 || gx >= jd->w || !M[gmask(r, c)]) continue;
        const int reg = region(r) * 3 + region(c);
        int cur;
        if (hdr[H_SRC + reg] == 1) {
            const int o = __ldcg(out + (int64_t)gy * jd->po + gx);
            cur = o < GD_INF ? o : GD_INF;
        } else {
            cur = __ldcg(sd + (int64_t)gy * jd->pb + gx) ? 0 : GD_INF;
        }
        bool need = false;
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int pr = r + nb_dy(8, n), pcc = c + nb_dx(8, n);
            if (pr < 1 || pr > TS || pcc < 1 || pcc > TS) continue;
            if (D[gcell(pr, pcc)] + gstep(n) < cur) need = true;
        }
        if (need) hdr[H_FLAG + reg] = 1;
    }
    __syncthreads();
    finish_tile(ka, jd, gt, tx, ty, hdr);
    pc.mark(hdr, 3);
    return true;
}

// =====================================================================
// Watershed from markers (Section 1's further IWPP use): plateau
// distances and labels
// =====================================================================
//
// Two min-propagations along fixed directed edges, given per pixel as an
// in-edge mask E (bit k: neighbour k may lower the pixel) that the
// per-pixel kernels of iwpp_watershed.cu build from the flooding levels:
//   plateau distance (PLAT): V(q) = min(V(q), V(p) + 1) over edges between
//     neighbours of equal level; entry pixels start at 0, the rest at
//     WS_DINF;
//   labels: V(q) = min(V(q), V(p)) over the optimal edges; marker pixels
//     have no in-edges and keep their value; a pixel without a label holds
//     INT_MAX until the last per-pixel kernel writes 0 there.
// Wavefront element: a pixel whose value can lower an out-neighbour.  The
// sweeps, seeding, queue rounds and border test follow the shortest-path
// family with the edge mask in place of the obstacle mask.  Pixels outside
// the image are never an in-neighbour (their bits are 0 in every mask), so
// the staged boxes need no fill values: the halo is used as loaded.

template <bool PLAT>
__device__ __forceinline__ int ws_cand(int v) { return PLAT ? v + 1 : v; }

template <int DIR, bool PLAT>
__device__ __forceinline__ bool ws_row_pass(int *__restrict__ V, const uint8_t *__restrict__ E, int r) {
    constexpr unsigned FROM = DIR > 0 ? 1u << 3 : 1u << 4;  // the left / right neighbour
    return i32_u8_row_pass<DIR>(V, E, r, [](int run, int o, unsigned e) {
        return (e & FROM) ? min(o, ws_cand<PLAT>(run)) : o;
    });
}

// column pass; the diagonal neighbours of the previous row are read from
// shared memory (old or new: both are values the pixel held)
template <int DIR, bool PLAT>
__device__ __forceinline__ bool ws_column_pass(int *__restrict__ V, const uint8_t *__restrict__ E, int t) {
    // in-edge bits of the previous row's straight, left and right neighbours
    constexpr unsigned BS = DIR > 0 ? 1u << 1 : 1u << 6;
    constexpr unsigned BL = DIR > 0 ? 1u << 0 : 1u << 5;
    constexpr unsigned BR = DIR > 0 ? 1u << 2 : 1u << 7;
    const int c = t + 1;
    int up = V[gcell(DIR > 0 ? 0 : RR - 1, c)];
    bool ch = false;
#pragma unroll 4
    for (int s = 1; s <= TS; ++s) {
        const int r = DIR > 0 ? s : RR - 1 - s;
        const int i = gcell(r, c), ip = i - DIR * BI32_W;
        const unsigned e = E[gmask(r, c)];
        const int o = V[i];
        int v = o;
        if (e & BS) v = min(v, ws_cand<PLAT>(up));
        if (e & BL) v = min(v, ws_cand<PLAT>(V[ip - 1]));
        if (e & BR) v = min(v, ws_cand<PLAT>(V[ip + 1]));
        if (v != o) { V[i] = v; ch = true; }
        up = v;
    }
    return ch;
}

template <bool PLAT>
__device__ bool ws_sweep_set(int *V, const uint8_t *E) {
    const int t = threadIdx.x;
    bool ch = false;
    if (t < TS) {
        ch |= ws_row_pass<+1, PLAT>(V, E, t + 1);
        ch |= ws_row_pass<-1, PLAT>(V, E, t + 1);
    }
    __syncthreads();
    if (t < TS) {
        ch |= ws_column_pass<+1, PLAT>(V, E, t);
        ch |= ws_column_pass<-1, PLAT>(V, E, t);
    }
    return __syncthreads_or(ch) != 0;
}

// One relaxation step over the interior (each pixel takes the least
// candidate of its in-neighbours); the pixels it lowers are queued, after
// which every pixel that can still lower a neighbour is queued.
template <int NT, bool PLAT>
__device__ unsigned ws_dilate_seed(int *V, const uint8_t *E, const RQ &q, const int *off) {
    unsigned pushed = 0;
    for (int base = 0; base < TS * TS; base += NT) {
        const int k = base + threadIdx.x;
        unsigned m = 0;
        int i = 0;
        if (k < TS * TS) {
            const int r = k / TS + 1, c = k - (k / TS) * TS + 1;
            i = gcell(r, c);
            const unsigned e = E[gmask(r, c)];
            if (e) {
                const int o = V[i];
                int v = o;
#pragma unroll
                for (int n = 0; n < 8; ++n)
                    if (e & (1u << n)) v = min(v, ws_cand<PLAT>(V[i + off[n]]));
                if (v < o) {
                    V[i] = v;
                    m = 1u << 8;
                }
            }
        }
        pushed += warp_enqueue(m, i, off, q);
    }
    return pushed;
}

// later visits: halo pixels that can lower an interior neighbour (the
// neighbour's in-edge from the halo pixel is its mirror bit 7 - n)
template <int NT, bool PLAT>
__device__ unsigned ws_halo_seed(int *V, const uint8_t *E, const RQ &q, const int *off) {
    unsigned pushed = 0;
    for (int base = 0; base < 4 * (TS + 1); base += NT) {
        const int k = base + threadIdx.x;
        unsigned m = 0;
        int i = 0;
        if (k < 4 * (TS + 1)) {
            int r, c;
            halo_cell(k, r, c);
            i = gcell(r, c);
            const int cv = ws_cand<PLAT>(V[i]);
#pragma unroll
            for (int n = 0; n < 8; ++n) {
                const int rr = r + nb_dy(8, n), cc = c + nb_dx(8, n);
                if (rr >= 1 && rr <= TS && cc >= 1 && cc <= TS && (E[gmask(rr, cc)] & (1u << (7 - n))) &&
                    cv < V[i + off[n]])
                    m = 1u << 8;
            }
        }
        pushed += warp_enqueue(m, i, off, q);
    }
    return pushed;
}

template <int NT, bool PLAT>
__device__ bool ws_visit(const KArgs &ka, const JobDesc *jd, int gt, char *sm, uint32_t &phase,
                         unsigned long long deadline) {
    int *hdr = (int *)sm;
    uint64_t *bar = (uint64_t *)(sm + 256);
    int *V = (int *)(sm + G_D);
    uint8_t *E = (uint8_t *)(sm + G_M);
    uint16_t *Q0 = (uint16_t *)(sm + G_U), *Q1 = Q0 + QCAP_G;
    const int tid = threadIdx.x;
    const int lt = gt - jd->tile_base, tx = lt % jd->tiles_x, ty = lt / jd->tiles_x;
    const int x0 = tx * TS, y0 = ty * TS;
    int *out = (int *)jd->out;

    PhaseClock pc;
    pc.start();
    load_sources(ka, jd, tx, ty, hdr);
    begin_visit(hdr);
    if (tid == 0) hdr[H_CHG] = 0;
    make_offsets<8, BI32_W>(hdr);
    // 1. stage the in-edge masks (0 outside the image: no edges) and the
    //    current values (the plane always holds valid values: the per-pixel
    //    kernels initialised it; values outside the image are never read as
    //    candidates)
    __syncthreads();
    const bool first = hdr[H_SRC + 4] == 0;
    if (jd->use_tma) {
        if (tid == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, BU8_BYTES + BI32_BYTES);
            tma_load_2d(E, &jd->tm[0], x0 - 16, y0 - 1, bar);
            tma_load_2d(V, &jd->tm[2], x0 - 4, y0 - 1, bar);
        }
        if (!wait_boxes(bar, phase, deadline, ka.ctl)) return false;
    } else {
        stage_plain<uint8_t, BU8_W>(E, (const uint8_t *)jd->a, jd->pa, jd->h, jd->w, x0 - 16, y0 - 1, NT);
        stage_plain<int, BI32_W>(V, out, jd->po, jd->h, jd->w, x0 - 4, y0 - 1, NT);
        __syncthreads();
    }
    pc.mark(hdr, 0);
    const int *off = hdr + H_OFF;

    // 2. seeds: sweep sets then one relaxation step (first visit, or a
    //    later visit whose halo changed in many places); else halo seeds
    uint16_t *spill = ka.spill + (int64_t)blockIdx.x * 2 * ka.spill_cap;
    const int qcap = (ka.queue_mode & 2) ? 0 : QCAP_G;
    RQ q0{Q0, spill, hdr + H_CNT0, hdr + H_RESCAN, qcap, ka.spill_cap, ka.queue_mode & 1};
    auto sweeps_then_seed = [&]() -> unsigned {
        bool changed = true;
        for (int s = 0; s < ka.ws_sweeps && changed; ++s) {
            changed = ws_sweep_set<PLAT>(V, E);
            if (changed && tid == 0) hdr[H_CHG] = 1;
        }
        if (!changed && ka.ws_sweeps > 0) return 0u;
        const unsigned lowered = ws_dilate_seed<NT, PLAT>(V, E, q0, off);
        if (lowered) hdr[H_CHG] = 1;  // the pixels it queues are the ones it lowered
        return lowered;
    };
    unsigned seeds;
    if (first) {
        seeds = sweeps_then_seed();
    } else {
        seeds = ws_halo_seed<NT, PLAT>(V, E, q0, off);
        __syncthreads();
        if (hdr[H_CNT0] > ka.ws_revisit_sweep_min) {
            __syncthreads();
            if (tid == 0) { hdr[H_CNT0] = 0; hdr[H_RESCAN] = 0; }
            __syncthreads();
            seeds = sweeps_then_seed();
        }
    }
    if ((tid & 31) == 0) atomicAdd(hdr + H_SEEDS, (int)seeds);
    pc.mark(hdr, 1);

    // 3. propagation rounds (atomicMin along the in-edges of interior pixels)
    auto proc = [&](int p, int n) -> bool {
        const int pr = p / BI32_W, pcol = p - pr * BI32_W - 3;
        const int rr = pr + nb_dy(8, n), cc = pcol + nb_dx(8, n);
        if (rr < 1 || rr > TS || cc < 1 || cc > TS || !(E[gmask(rr, cc)] & (1u << (7 - n)))) return false;
        const int cand = ws_cand<PLAT>(((volatile int *)V)[p]);
        return atomicMin(V + p + off[n], cand) > cand;
    };
    auto rescan = [&](const RQ &q) -> unsigned { return ws_dilate_seed<NT, PLAT>(V, E, q, off); };
    run_rounds<NT, 8>(hdr, Q0, Q1, qcap, spill, ka.spill_cap, off, proc, rescan, deadline, ka.ctl,
                      ka.queue_mode & 1);
    __syncthreads();
    pc.mark(hdr, 2);

    // A visit that lowered nothing (no sweep change, no relaxation, no
    // queue update) leaves the plane as it was: the store is not needed,
    // and neither is the border test -- every neighbour saw these values
    // when it staged its halo, or will when it is visited.
    if (!hdr[H_CHG] && hdr[H_PUSH] == 0) {
        publish_tile(ka, gt, hdr);
        finish_tile(ka, jd, gt, tx, ty, hdr);
        pc.mark(hdr, 3);
        return true;
    }

    // 4. store the interior; 16-byte stores when the tile is whole and the
    //    plane meets TMA's alignment
    if (jd->use_tma && x0 + TS <= jd->w) {
        for (int i = tid; i < TS * TS / 4; i += NT) {
            const int r = i / (TS / 4), c4 = i - r * (TS / 4);
            const int gy = y0 + r;
            if (gy >= jd->h) continue;
            *(int4 *)(out + (int64_t)gy * jd->po + x0 + 4 * c4) = *(const int4 *)(V + gcell(r + 1, 1 + 4 * c4));
        }
    } else {
        for (int i = tid; i < TS * TS; i += NT) {
            const int r = i / TS, c = i - r * TS;
            const int gy = y0 + r, gx = x0 + c;
            if (gy >= jd->h || gx >= jd->w) continue;
            out[(int64_t)gy * jd->po + gx] = V[gcell(r + 1, c + 1)];
        }
    }
    __syncthreads();
    publish_tile(ka, gt, hdr);

    // 5. border test: can an interior pixel lower a halo pixel's current
    //    value along one of the halo pixel's in-edges?
    for (int k = tid; k < 4 * (TS + 1); k += NT) {
        int r, c;
        halo_cell(k, r, c);
        const int gy = y0 - 1 + r, gx = x0 - 1 + c;
        if (gy < 0 || gy >= jd->h || gx < 0 || gx >= jd->w) continue;
        const unsigned e = E[gmask(r, c)];
        if (!e) continue;
        const int cur = __ldcg(out + (int64_t)gy * jd->po + gx);
        bool need = false;
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int pr = r + nb_dy(8, n), pcc = c + nb_dx(8, n);
            if (pr < 1 || pr > TS || pcc < 1 || pcc > TS || !(e & (1u << n))) continue;
            if (ws_cand<PLAT>(V[gcell(pr, pcc)]) < cur) need = true;
        }
        if (need) hdr[H_FLAG + region(r) * 3 + region(c)] = 1;
    }
    __syncthreads();
    finish_tile(ka, jd, gt, tx, ty, hdr);
    pc.mark(hdr, 3);
    return true;
}

// =====================================================================
// kernels
// =====================================================================

template <int FAM>
__global__ void __launch_bounds__(FAM_NT[FAM], FAM_MINB[FAM]) persistent_kernel(const __grid_constant__ KArgs ka) {
    constexpr int NT = FAM_NT[FAM];
    extern __shared__ __align__(128) char smem[];
    int *hdr = (int *)smem;
    uint64_t *bar = (uint64_t *)(smem + 256);
    if (ld_volatile(&ka.ctl->done)) return;
    unsigned long long *cst = (unsigned long long *)(smem + HDR_STATS);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    if (threadIdx.x < 12) cst[threadIdx.x] = 0;
    __syncthreads();
    uint32_t phase = 0;
    unsigned long long t_wait = 0, t_visit = 0;
    while (true) {
        unsigned long long t0 = 0;
        if (threadIdx.x == 0) {
            t0 = globaltimer_ns();
            hdr[H_TILE] = tq_claim(ka.tq, ka.ctl, ka.timeout_ns);
            const unsigned long long t1 = globaltimer_ns();
            t_wait += t1 - t0;
            t0 = t1;
        }
        __syncthreads();
        const int t = hdr[H_TILE];
        if (t < 0) break;
        // waits inside one visit (its TMA boxes, the guard of its rounds) are
        // bounded from the visit's start: a visit takes micro- to
        // milliseconds, so only a defect reaches the bound; a long call made
        // of many visits does not
        const unsigned long long deadline = globaltimer_ns() + ka.timeout_ns;
        const JobDesc *jd = job_of(ka, t);
        bool ok = true;
        if (jd->op == OP_RECON) {
            if constexpr (FAM == FAM_RECON_U8 || FAM == FAM_MIXED) {
                if (jd->dtype == DT_U8)
                    ok = jd->conn == 8 ? recon_u8_visit<8, NT>(ka, jd, t, smem, phase, deadline)
                                       : recon_u8_visit<4, NT>(ka, jd, t, smem, phase, deadline);
            }
            if constexpr (FAM == FAM_RECON_I32 || FAM == FAM_MIXED) {
                if (jd->dtype == DT_I32)
                    ok = jd->conn == 8 ? recon_i32_visit<8, NT>(ka, jd, t, smem, phase, deadline)
                                       : recon_i32_visit<4, NT>(ka, jd, t, smem, phase, deadline);
            }
        } else {
            if constexpr (FAM == FAM_EDT || FAM == FAM_MIXED) {
                if (jd->op == OP_EDT) ok = edt_visit<NT>(ka, jd, t, smem, phase, deadline);
                else if (jd->op == OP_EDT_WIDE) ok = edt_wide_visit<NT, 8>(ka, jd, t, smem, phase, deadline);
            }
            if constexpr (FAM == FAM_GDT) {
                if (jd->op == OP_GDT) ok = gdt_visit<NT>(ka, jd, t, smem, phase, deadline);
            }
            if constexpr (FAM == FAM_WS) {
                if (jd->op == OP_WS_DIST) ok = ws_visit<NT, true>(ka, jd, t, smem, phase, deadline);
                else if (jd->op == OP_WS_LABEL) ok = ws_visit<NT, false>(ka, jd, t, smem, phase, deadline);
            }
        }
        if (!ok) break;  // timeout raised; the host reports it
        if (threadIdx.x == 0) {
            // the visit's pushes (ordered before by finish_tile's barrier)
            // are performed before its pending count goes
            __threadfence();
            atomicSub(ka.tq.pending, 1);
            t_visit += globaltimer_ns() - t0;
            // per-visit counters accumulate in shared memory; one flush per CTA
            cst[0] += 1;
            cst[1] += (unsigned)hdr[H_SEEDS];
            cst[2] += (unsigned)hdr[H_PUSH];
            cst[3] += (unsigned)hdr[H_SPILL];
            cst[4] += (unsigned)hdr[H_RESC];
            cst[5] += (unsigned)hdr[H_ROUNDS];
            for (int i = 0; i < 4; ++i) cst[6 + i] += (unsigned)hdr[H_PH + i];
            cst[10] += (unsigned)hdr[H_SETS];
            cst[11] += hdr[H_SRC + 4] != 0 ? 1u : 0u;  // the tile had been visited before
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&ka.ctl->wait_ns, t_wait);
        atomicAdd(&ka.ctl->visit_ns, t_visit);
        atomicAdd(&ka.ctl->tiles_processed, cst[0]);
        atomicAdd(&ka.ctl->seeds, cst[1]);
        atomicAdd(&ka.ctl->pushes, cst[2]);
        atomicAdd(&ka.ctl->spills, cst[3]);
        atomicAdd(&ka.ctl->rescans, cst[4]);
        atomicAdd(&ka.ctl->rounds, cst[5]);
        for (int i = 0; i < 4; ++i) atomicAdd(&ka.ctl->phase_ns[i], cst[6 + i]);
        atomicAdd(&ka.ctl->sweep_sets, cst[10]);
        atomicAdd(&ka.ctl->revisits, cst[11]);
    }
}

// Slot of tile t in the initial queue: colour class (x mod 2, y mod 2)
// first, so that tiles visited at the same time are never adjacent.
__device__ __forceinline__ int initial_slot(const JobDesc *jd, int t) {
    const int lt = t - jd->tile_base;
    const int x = lt % jd->tiles_x, y = lt / jd->tiles_x;
    const int a = x & 1, b = y & 1;
    const int nx = (jd->tiles_x - a + 1) >> 1;
    return jd->color_base[b * 2 + a] + (y >> 1) * nx + (x >> 1);
}

__global__ void fill_queue_kernel(const __grid_constant__ KArgs ka, int first) {
    if (!first && !ld_volatile(&ka.ctl->want_reset)) return;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)ka.tq.cap; i += stride) {
        if (i < ka.ntiles) {
            const int slot = initial_slot(job_of(ka, i), i);
            // timeout-path tests: slot 0 stays empty, so its claim waits out
            // the deadline and the launch ends with ST_TIMEOUT
            ka.tq.slots[slot] = (ka.test_empty_slot && slot == 0) ? -1 : i;
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

int family_threads(int fam) { return (fam >= 0 && fam < FAM_COUNT) ? FAM_NT[fam] : -1; }
int family_smem(int fam) { return (fam >= 0 && fam < FAM_COUNT) ? FAM_SMEM[fam] : -1; }

template <int FAM>
static cudaError_t occ(int *n) {
    cudaError_t e = cudaFuncSetAttribute(persistent_kernel<FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FAM_SMEM[FAM]);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, persistent_kernel<FAM>, FAM_NT[FAM], FAM_SMEM[FAM]);
}

cudaError_t family_occupancy(int fam, int *n) {
    switch (fam) {
        case FAM_RECON_U8: return occ<FAM_RECON_U8>(n);
        case FAM_RECON_I32: return occ<FAM_RECON_I32>(n);
        case FAM_EDT: return occ<FAM_EDT>(n);
        case FAM_MIXED: return occ<FAM_MIXED>(n);
        case FAM_GDT: return occ<FAM_GDT>(n);
        case FAM_WS: return occ<FAM_WS>(n);
        default: return cudaErrorInvalidValue;
    }
}

// Each launch helper first clears the calling thread's last-error slot: a
// status such as cudaErrorNotReady left there by an earlier query (e.g. an
// event poll) must not be mistaken for a failure of this launch.
cudaError_t launch_init(const KArgs &ka, int first_attempt, cudaStream_t s) {
    (void)cudaGetLastError();
    int blocks = (int)((ka.tq.cap + 255) / 256);
    blocks = blocks > 4096 ? 4096 : (blocks < 1 ? 1 : blocks);
    fill_queue_kernel<<<blocks, 256, 0, s>>>(ka, first_attempt);
    return cudaGetLastError();
}

template <int FAM>
static void launch_fam(const KArgs &ka, int grid, cudaStream_t s) {
    persistent_kernel<FAM><<<grid, FAM_NT[FAM], FAM_SMEM[FAM], s>>>(ka);
}

cudaError_t launch_persistent(const KArgs &ka, int fam, int grid, cudaStream_t s) {
    (void)cudaGetLastError();
    switch (fam) {
        case FAM_RECON_U8: launch_fam<FAM_RECON_U8>(ka, grid, s); break;
        case FAM_RECON_I32: launch_fam<FAM_RECON_I32>(ka, grid, s); break;
        case FAM_EDT: launch_fam<FAM_EDT>(ka, grid, s); break;
        case FAM_MIXED: launch_fam<FAM_MIXED>(ka, grid, s); break;
        case FAM_GDT: launch_fam<FAM_GDT>(ka, grid, s); break;
        case FAM_WS: launch_fam<FAM_WS>(ka, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_decide(const KArgs &ka, int final_step, cudaStream_t s) {
    (void)cudaGetLastError();
    decide_kernel<<<1, 1, 0, s>>>(ka, final_step);
    return cudaGetLastError();
}

cudaError_t launch_reset(const KArgs &ka, cudaStream_t s) { return launch_init(ka, 0, s); }

}  // namespace iwpp
