// iwpp_api.cu -- host side of the libiwpp C ABI (declared in include/iwpp.h):
// argument validation, the context and its device workspace, tile-size
// selection, and the launch sequence of the persistent tile-wavefront kernel.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/iwpp.h"
#include "iwpp_internal.h"
#include "iwpp_status.h"

using namespace iwpp;

struct iwpp_ctx {
    int device = 0;
    size_t budget = 0;
    int sm_count = 0;
    iwpp_options opt{};
    char err[256] = {0};
    void *ws = nullptr;        // workspace arena
    size_t ws_bytes = 0;
    void *aux = nullptr;       // planes of multi-step operations (watershed)
    size_t aux_bytes = 0;
    Control *ctl = nullptr;    // device control block (own allocation, persistent counters)
    Control *h_ctl = nullptr;  // pinned host copy
    uint64_t calls = 0;
    uint64_t tiles_initial = 0;
    uint64_t launches = 0;
    uint64_t kernel_ns = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending_events, free_events;
    int occupancy[FAM_COUNT] = {};  // blocks per SM per kernel family
    std::map<uint64_t, iwpp_options> tuned;   // autotuner results by workload key
    // submitted jobs (iwpp_submit): the context's own stream, a ring of
    // pinned status words (one per outstanding ticket) and the completion
    // event of every ticket not yet retired by iwpp_poll / iwpp_wait
    struct Ticket {
        cudaEvent_t ev = nullptr;
        int slot = -1;      // ring slot of its status word, -1 once moved to `status`
        int status = 0;     // ST_* bits, valid once slot == -1
    };
    cudaStream_t sub_stream = nullptr;
    int *h_sub_status = nullptr;              // kSubRing pinned ints
    std::vector<uint64_t> sub_slot_owner;     // ticket holding each ring slot (0 = free)
    std::map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
};

namespace {

int fail(iwpp_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof ctx->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(iwpp_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, IWPP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

size_t elem_size(int dtype) { return dtype == IWPP_U8 ? 1 : 4; }

int check_image(iwpp_ctx *ctx, const iwpp_image *im, const char *name) {
    if (!im) return fail(ctx, IWPP_EINVAL, "%s: null descriptor", name);
    if (im->h < 1 || im->w < 1) return fail(ctx, IWPP_EINVAL, "%s: shape %dx%d must be >= 1x1", name, im->h, im->w);
    if (im->pitch < im->w) return fail(ctx, IWPP_EINVAL, "%s: pitch %lld < width %d", name, (long long)im->pitch, im->w);
    if (im->dtype != IWPP_U8 && im->dtype != IWPP_I32) return fail(ctx, IWPP_EINVAL, "%s: dtype %d unsupported", name, im->dtype);
    if (!im->data) return fail(ctx, IWPP_EINVAL, "%s: null data pointer", name);
    if ((int64_t)im->h * im->pitch > ((int64_t)1 << 40)) return fail(ctx, IWPP_EINVAL, "%s: image too large", name);
    return IWPP_OK;
}

bool overlaps(const iwpp_image *a, const iwpp_image *b) {
    const char *a0 = (const char *)a->data, *b0 = (const char *)b->data;
    const char *a1 = a0 + ((int64_t)(a->h - 1) * a->pitch + a->w) * elem_size(a->dtype);
    const char *b1 = b0 + ((int64_t)(b->h - 1) * b->pitch + b->w) * elem_size(b->dtype);
    return a0 < b1 && b0 < a1;
}

// One persistent-kernel family per launch: a single-operation launch uses
// the specialised kernel with the smallest shared-memory footprint.
int pick_family(const std::vector<JobDesc> &jobs) {
    bool r8 = false, r32 = false, e = false;
    if (!jobs.empty() && jobs[0].op == OP_GDT) return FAM_GDT;  // geodesic launches hold only geodesic jobs
    if (!jobs.empty() && (jobs[0].op == OP_WS_DIST || jobs[0].op == OP_WS_LABEL)) return FAM_WS;
    for (const JobDesc &j : jobs) {
        if (j.op == OP_EDT || j.op == OP_EDT_WIDE) e = true;
        else if (j.dtype == DT_U8) r8 = true;
        else r32 = true;
    }
    if (e && !r8 && !r32) return FAM_EDT;
    if (r8 && !r32 && !e) return FAM_RECON_U8;
    if (r32 && !r8 && !e) return FAM_RECON_I32;
    return FAM_MIXED;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// TMA map of a 2-D image with the tile box (tile + halo, first column
// 16-byte aligned).  False when the image does not meet TMA's alignment
// rules (16-byte aligned base, row pitch a multiple of 16 bytes); the
// kernel then stages with plain loads.
bool make_map(CUtensorMap *m, const void *base, int dtype, int h, int w, int64_t pitch_elems, int box_w = 0,
              int box_h = 0) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const size_t es = dtype == DT_U8 ? 1 : 4;
    const uint64_t pitch_bytes = (uint64_t)pitch_elems * es;
    if (((uintptr_t)base & 15) || (pitch_bytes & 15) || pitch_bytes >= (1ull << 40)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {box_w ? (cuuint32_t)box_w : (dtype == DT_U8 ? 96u : 72u),
                         box_h ? (cuuint32_t)box_h : (cuuint32_t)(TILE + 2)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, dtype == DT_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_INT32, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void make_maps(JobDesc &d) {
    bool ok;
    if (d.op == OP_GDT) {  // mask, current result (sources are read directly)
        d.use_tma = make_map(&d.tm[0], d.a, DT_U8, d.h, d.w, d.pa) &&
                    make_map(&d.tm[2], d.out, DT_I32, d.h, d.w, d.po);
        return;
    }
    if (d.op == OP_WS_DIST || d.op == OP_WS_LABEL) {  // in-edge masks, values
        d.use_tma = make_map(&d.tm[0], d.a, DT_U8, d.h, d.w, d.pa) &&
                    make_map(&d.tm[2], d.out, DT_I32, d.h, d.w, d.po);
        return;
    }
    if (d.op == OP_EDT_WIDE) {  // the nearest indices with an 8-pixel halo: an 80 x 80 box
        d.use_tma = make_map(&d.tm[1], d.nearest, DT_I32, d.h, d.w, d.w, TILE + 16, TILE + 16) ? 1 : 0;
        return;
    }
    if (d.op == OP_RECON) {
        ok = make_map(&d.tm[0], d.a, d.dtype, d.h, d.w, d.pa) && make_map(&d.tm[1], d.b, d.dtype, d.h, d.w, d.pb) &&
             make_map(&d.tm[2], d.out, d.dtype, d.h, d.w, d.po);
    } else {
        ok = make_map(&d.tm[0], d.a, DT_U8, d.h, d.w, d.pa) && make_map(&d.tm[2], d.nearest, DT_I32, d.h, d.w, d.w);
    }
    d.use_tma = ok ? 1 : 0;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
size_t ws_alloc_size(const iwpp_ctx *ctx, size_t bytes);

int ensure_ws(iwpp_ctx *ctx, size_t bytes, cudaStream_t st) {
    if (bytes <= ctx->ws_bytes) return IWPP_OK;
    if (ctx->budget && bytes > ctx->budget)
        return fail(ctx, IWPP_ENOMEM, "workspace of %zu bytes exceeds the context budget of %zu", bytes, ctx->budget);
    if (ctx->ws) {
        CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        CK(cudaFree(ctx->ws), "cudaFree");
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    const size_t b = ws_alloc_size(ctx, bytes);
    cudaError_t e = cudaMalloc(&ctx->ws, b);
    if (e != cudaSuccess) {
        ctx->ws = nullptr;
        return fail(ctx, IWPP_ENOMEM, "cudaMalloc(%zu): %s", b, cudaGetErrorString(e));
    }
    ctx->ws_bytes = b;
    return IWPP_OK;
}

// Lays out the tile geometry of every job and the initial colour classes.
int64_t layout_jobs(std::vector<JobDesc> &jobs, int tile) {
    int64_t cls[4] = {0, 0, 0, 0};
    std::vector<int64_t> per(jobs.size() * 4);
    int64_t base = 0;
    for (size_t j = 0; j < jobs.size(); ++j) {
        JobDesc &d = jobs[j];
        d.tiles_x = (d.w + tile - 1) / tile;
        d.tiles_y = (d.h + tile - 1) / tile;
        d.tile_base = (int)base;
        base += (int64_t)d.tiles_x * d.tiles_y;
        for (int c = 0; c < 4; ++c) {
            const int a = c & 1, b = c >> 1;
            const int64_t n = (int64_t)((d.tiles_x - a + 1) / 2) * ((d.tiles_y - b + 1) / 2);
            per[j * 4 + c] = n;
            cls[c] += n;
        }
    }
    int64_t start[4];
    start[0] = 0;
    for (int c = 1; c < 4; ++c) start[c] = start[c - 1] + cls[c - 1];
    for (size_t j = 0; j < jobs.size(); ++j)
        for (int c = 0; c < 4; ++c) {
            jobs[j].color_base[c] = (int)start[c];
            start[c] += per[j * 4 + c];
        }
    return base;
}

// A launch sequence, prepared: tile layout, TMA maps, kernel family, grid,
// workspace layout and the kernel arguments (pointers bound to a workspace).
struct Prepared {
    KArgs ka;
    int fam = 0;
    int grid = 1;
    int64_t ntiles = 0;
    size_t ws_bytes = 0;
    size_t o_slots = 0, o_state = 0, o_visited = 0, o_cnt = 0, o_spill = 0, o_jobs = 0;
};

// Tile-queue slots per tile of a launch.  The shortest-path and watershed
// propagations follow paths that bend around obstacles and along optimal
// edges, so they visit a tile many more times than the reconstruction and
// the distance transform (6 and more times per tile on random fields, 23 in
// a 2048^2 serpentine maze): their queues take four times the option.
int queue_factor_of(int fam, const iwpp_options &opt) {
    return (fam == FAM_GDT || fam == FAM_WS) ? 4 * opt.queue_factor : opt.queue_factor;
}

// Byte offsets of a launch's workspace: tile-queue slots, tile states and
// visited flags, queue counters, per-CTA spill queues, the job table.
void layout_workspace(Prepared &P, int64_t cap64, size_t njobs, const iwpp_options &opt) {
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    P.o_slots = take((size_t)cap64 * 4);
    P.o_state = take((size_t)P.ntiles * 4);
    P.o_visited = take((size_t)P.ntiles * 4);
    P.o_cnt = take(16);
    P.o_spill = take((size_t)P.grid * 2 * std::max(1, opt.spill_cap) * sizeof(uint16_t));
    P.o_jobs = take(njobs > 1 ? njobs * sizeof(JobDesc) : 0);
    P.ws_bytes = off;
}

// The workspace bytes a launch sequence over `jobs` needs (no TMA encoding,
// no allocation): the same arithmetic as prepare().
int workspace_need(iwpp_ctx *ctx, std::vector<JobDesc> jobs, const iwpp_options &opt, size_t *bytes) {
    Prepared P;
    P.fam = pick_family(jobs);
    P.ntiles = layout_jobs(jobs, TILE);
    const int64_t cap64 = std::max<int64_t>(P.ntiles + 1, (int64_t)queue_factor_of(P.fam, opt) * P.ntiles);
    int &occ = ctx->occupancy[P.fam];
    if (occ == 0) CK(family_occupancy(P.fam, &occ), "occupancy query");
    const int bps = opt.blocks_per_sm > 0 ? std::min(opt.blocks_per_sm, occ) : occ;
    P.grid = (int)std::max<int64_t>(1, std::min<int64_t>(P.ntiles, (int64_t)bps * ctx->sm_count));
    layout_workspace(P, cap64, jobs.size(), opt);
    *bytes = P.ws_bytes;
    return IWPP_OK;
}

// The size ensure_ws() allocates for a request of `bytes`.
size_t ws_alloc_size(const iwpp_ctx *ctx, size_t bytes) {
    size_t b = align_up(bytes + bytes / 4, 1 << 20);
    if (ctx->budget && b > ctx->budget) b = bytes;
    return b;
}

int prepare(iwpp_ctx *ctx, std::vector<JobDesc> &jobs, const iwpp_options &opt, Prepared &P) {
    P.fam = pick_family(jobs);
    P.ntiles = layout_jobs(jobs, TILE);
    for (JobDesc &j : jobs) make_maps(j);
    if (P.ntiles <= 0 || P.ntiles > (int64_t)1 << 28)
        return fail(ctx, IWPP_EINVAL, "tile count %lld out of range", (long long)P.ntiles);
    const int64_t cap64 = std::max<int64_t>(P.ntiles + 1, (int64_t)queue_factor_of(P.fam, opt) * P.ntiles);
    if (cap64 > ((int64_t)1 << 31) - 1) return fail(ctx, IWPP_EINVAL, "tile queue too large");
    int &occ = ctx->occupancy[P.fam];
    if (occ == 0) {
        CK(family_occupancy(P.fam, &occ), "occupancy query");
        if (occ < 1) return fail(ctx, IWPP_ECUDA, "persistent kernel does not fit on an SM");
    }
    const int bps = opt.blocks_per_sm > 0 ? std::min(opt.blocks_per_sm, occ) : occ;
    P.grid = (int)std::max<int64_t>(1, std::min<int64_t>(P.ntiles, (int64_t)bps * ctx->sm_count));
    layout_workspace(P, cap64, jobs.size(), opt);
    KArgs &ka = P.ka;
    memset(&ka, 0, sizeof ka);
    ka.njobs = (int)jobs.size();
    ka.ntiles = (int)P.ntiles;
    ka.job0 = jobs[0];
    ka.tq.cap = (unsigned)cap64;
    ka.tq.ntiles = (int)P.ntiles;
    ka.spill_cap = std::max(0, opt.spill_cap);
    ka.sweeps = opt.sweeps;
    ka.revisit_sweep_min = opt.revisit_sweep_min;
    ka.edt_sweeps = opt.edt_sweeps;
    ka.edt_revisit_sweep_min = opt.edt_revisit_sweep_min;
    ka.revisit_sweeps = opt.revisit_sweeps < 0 ? opt.sweeps : opt.revisit_sweeps;
    ka.queue_mode = opt.queue_mode;
    ka.test_empty_slot = opt.test_empty_slot;
    ka.gdt_sweeps = opt.gdt_sweeps;
    ka.gdt_revisit_sweep_min = opt.gdt_revisit_sweep_min;
    ka.ws_sweeps = opt.ws_sweeps;
    ka.ws_revisit_sweep_min = opt.ws_revisit_sweep_min;
    for (int j = 0; j < 7; ++j) {  // window half-width j + 2 from distance (j + 1) * step on
        const int64_t t = (int64_t)(j + 1) * opt.edt_wide_step;
        ka.wide_u[j] = (int)std::min<int64_t>(t * t, INT32_MAX);
    }
    ka.timeout_ns = (unsigned long long)opt.timeout_ms * 1000000ull;
    return IWPP_OK;
}

void bind_workspace(Prepared &P, char *ws, Control *ctl) {
    KArgs &ka = P.ka;
    ka.jobs = ka.njobs > 1 ? (const JobDesc *)(ws + P.o_jobs) : nullptr;
    ka.tq.slots = (int *)(ws + P.o_slots);
    ka.tq.state = (int *)(ws + P.o_state);
    ka.tq.visited = (int *)(ws + P.o_visited);
    ka.tq.head = (unsigned *)(ws + P.o_cnt);
    ka.tq.tail = (unsigned *)(ws + P.o_cnt + 4);
    ka.tq.pending = (int *)(ws + P.o_cnt + 8);
    ka.ctl = ctl;
    ka.spill = (uint16_t *)(ws + P.o_spill);
}

// Enqueues the launch sequence: queue fill, persistent kernel, then
// `max_relaunch` device-side decide / refill / relaunch steps (no-ops when
// nothing overflowed) and the final decide that records the outcome.
// Kernel launches only: legal inside a stream capture.
int enqueue(iwpp_ctx *ctx, const Prepared &P, int max_relaunch, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    CK(launch_init(P.ka, 1, st), "launch fill_queue");
    if (e0) CK(cudaEventRecord(e0, st), "cudaEventRecord");
    CK(launch_persistent(P.ka, P.fam, P.grid, st), "launch persistent");
    for (int k = 0; k < max_relaunch; ++k) {
        CK(launch_decide(P.ka, 0, st), "launch decide");
        CK(launch_reset(P.ka, st), "launch reset");
        CK(launch_persistent(P.ka, P.fam, P.grid, st), "launch persistent");
    }
    if (e1) CK(cudaEventRecord(e1, st), "cudaEventRecord");
    CK(launch_decide(P.ka, 1, st), "launch decide");
    return IWPP_OK;
}

// The launch groups of a batch: all jobs together, or (batch_split) one
// group per operation family -- uint8 reconstruction, int32
// reconstruction, distance transform, shortest paths, watershed steps --
// in that order.
std::vector<std::vector<JobDesc>> launch_groups(const std::vector<JobDesc> &jobs, int split) {
    std::vector<std::vector<JobDesc>> g;
    if (!split) {
        g.push_back(jobs);
        return g;
    }
    std::vector<JobDesc> by[5];
    for (const JobDesc &j : jobs) {
        const int k = j.op == OP_RECON ? (j.dtype == DT_U8 ? 0 : 1)
                                       : ((j.op == OP_EDT || j.op == OP_EDT_WIDE) ? 2 : (j.op == OP_GDT ? 3 : 4));
        by[k].push_back(j);
    }
    for (auto &v : by)
        if (!v.empty()) g.push_back(v);
    return g;
}

int run_once(iwpp_ctx *ctx, std::vector<JobDesc> &jobs, cudaStream_t st, bool sync);

// Runs (or enqueues) the whole launch sequence for `jobs` on the context's
// workspace: one sequence per launch group, back to back on the stream
// (they share the status block; its error bits accumulate).  Distance
// transforms with IWPP_EDT_EXACT_PROPAGATION get their second, wide-window
// wavefront as a further launch sequence on the same stream.
int run(iwpp_ctx *ctx, std::vector<JobDesc> &jobs, cudaStream_t st, bool sync) {
    std::vector<JobDesc> wide;
    for (const JobDesc &j : jobs)
        if (j.op == OP_EDT && (j.flags & IWPP_EDT_EXACT_PROPAGATION)) {
            JobDesc w = j;
            w.op = OP_EDT_WIDE;
            wide.push_back(w);
        }
    if (wide.empty()) return run_once(ctx, jobs, st, sync);
    int rc = run_once(ctx, jobs, st, false);
    if (rc) return rc;
    rc = run_once(ctx, wide, st, sync);
    ctx->calls -= 1;  // the two wavefronts are one call
    return rc;
}

int run_once(iwpp_ctx *ctx, std::vector<JobDesc> &jobs, cudaStream_t st, bool sync) {
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<std::vector<JobDesc>> groups = launch_groups(jobs, ctx->opt.batch_split);
    if (groups.size() > 1) {
        std::vector<Prepared> Ps(groups.size());
        std::vector<size_t> offs(groups.size());
        size_t total = 0;
        for (size_t k = 0; k < groups.size(); ++k) {
            int rc = prepare(ctx, groups[k], ctx->opt, Ps[k]);
            if (rc) return rc;
            offs[k] = total;
            total += align_up(Ps[k].ws_bytes, 256);
        }
        int rc = ensure_ws(ctx, total, st);
        if (rc) return rc;
        for (size_t k = 0; k < groups.size(); ++k) {
            char *ws = (char *)ctx->ws + offs[k];
            bind_workspace(Ps[k], ws, ctx->ctl);
            if (groups[k].size() > 1)
                CK(cudaMemcpyAsync(ws + Ps[k].o_jobs, groups[k].data(), groups[k].size() * sizeof(JobDesc),
                                   cudaMemcpyHostToDevice, st),
                   "job table upload");
            if ((rc = enqueue(ctx, Ps[k], ctx->opt.max_relaunch, st, nullptr, nullptr))) return rc;
            ctx->launches += 3 + 3 * (uint64_t)ctx->opt.max_relaunch;
            ctx->tiles_initial += (uint64_t)Ps[k].ntiles;
        }
        ctx->calls += 1;
        if (!sync) return IWPP_OK;
        return iwpp_sync(ctx, st);
    }
    Prepared P;
    int rc = prepare(ctx, jobs, ctx->opt, P);
    if (rc) return rc;
    rc = ensure_ws(ctx, P.ws_bytes, st);
    if (rc) return rc;
    char *ws = (char *)ctx->ws;
    bind_workspace(P, ws, ctx->ctl);
    if (jobs.size() > 1)
        CK(cudaMemcpyAsync(ws + P.o_jobs, jobs.data(), jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, st),
           "job table upload");
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (ctx->opt.timing) {
        if (ctx->free_events.empty()) {
            CK(cudaEventCreate(&ev.first), "cudaEventCreate");
            CK(cudaEventCreate(&ev.second), "cudaEventCreate");
        } else {
            ev = ctx->free_events.back();
            ctx->free_events.pop_back();
        }
    }
    rc = enqueue(ctx, P, ctx->opt.max_relaunch, st, ev.first, ev.second);
    if (rc) return rc;
    if (ev.first) ctx->pending_events.push_back(ev);
    ctx->launches += 3 + 3 * (uint64_t)ctx->opt.max_relaunch;
    ctx->calls += 1;
    ctx->tiles_initial += (uint64_t)P.ntiles;
    if (!sync) return IWPP_OK;
    return iwpp_sync(ctx, st);
}

JobDesc recon_job(const iwpp_image *marker, const iwpp_image *mask, int conn, iwpp_image *out) {
    JobDesc d;
    memset(&d, 0, sizeof d);
    d.op = OP_RECON;
    d.dtype = marker->dtype == IWPP_U8 ? DT_U8 : DT_I32;
    d.conn = conn;
    d.h = marker->h;
    d.w = marker->w;
    d.a = marker->data;
    d.b = mask->data;
    d.out = out->data;
    d.pa = marker->pitch;
    d.pb = mask->pitch;
    d.po = out->pitch;
    return d;
}

int check_recon(iwpp_ctx *ctx, const iwpp_image *marker, const iwpp_image *mask, int conn, const iwpp_image *out) {
    int rc;
    if ((rc = check_image(ctx, marker, "marker")) || (rc = check_image(ctx, mask, "mask")) ||
        (rc = check_image(ctx, out, "out")))
        return rc;
    if (conn != 4 && conn != 8) return fail(ctx, IWPP_EINVAL, "conn must be 4 or 8, got %d", conn);
    if (marker->h != mask->h || marker->w != mask->w || out->h != mask->h || out->w != mask->w)
        return fail(ctx, IWPP_EINVAL, "marker, mask and out must have the same shape");
    if (marker->dtype != mask->dtype || out->dtype != mask->dtype)
        return fail(ctx, IWPP_EINVAL, "marker, mask and out must have the same dtype");
    if (overlaps(out, mask)) return fail(ctx, IWPP_EINVAL, "out must not alias the mask");
    if (out->data != marker->data && overlaps(out, marker))
        return fail(ctx, IWPP_EINVAL, "out may alias the marker only exactly (in place)");
    if (out->data == marker->data && out->pitch != marker->pitch)
        return fail(ctx, IWPP_EINVAL, "in-place reconstruction needs equal pitches");
    return IWPP_OK;
}

int check_edt(iwpp_ctx *ctx, const iwpp_image *bin, const int32_t *sq, const int32_t *nn, int flags) {
    int rc;
    if ((rc = check_image(ctx, bin, "binary"))) return rc;
    if (bin->dtype != IWPP_U8) return fail(ctx, IWPP_EINVAL, "binary image must be IWPP_U8");
    if (bin->h > 32768 || bin->w > 32768) return fail(ctx, IWPP_EINVAL, "distance transform limited to sides <= 32768");
    if (!sq || !nn) return fail(ctx, IWPP_EINVAL, "null output pointer");
    if (flags & ~3) return fail(ctx, IWPP_EINVAL, "unknown flags 0x%x", flags);
    if (sq == nn) return fail(ctx, IWPP_EINVAL, "sqdist and nearest must be distinct buffers");
    return IWPP_OK;
}

int check_gdt(iwpp_ctx *ctx, const iwpp_image *mask, const iwpp_image *seeds, const int32_t *dist) {
    int rc;
    if ((rc = check_image(ctx, mask, "mask")) || (rc = check_image(ctx, seeds, "seeds"))) return rc;
    if (mask->dtype != IWPP_U8 || seeds->dtype != IWPP_U8)
        return fail(ctx, IWPP_EINVAL, "geodesic distance: mask and seeds must be uint8");
    if (mask->h != seeds->h || mask->w != seeds->w)
        return fail(ctx, IWPP_EINVAL, "geodesic distance: mask and seeds must have the same shape");
    if (!dist) return fail(ctx, IWPP_EINVAL, "null output pointer");
    if ((int64_t)mask->h * mask->w >= ((int64_t)1 << 31))
        return fail(ctx, IWPP_EINVAL, "geodesic distance limited to h*w < 2^31");
    return IWPP_OK;
}

JobDesc gdt_job(const iwpp_image *mask, const iwpp_image *seeds, int32_t *dist) {
    JobDesc d;
    memset(&d, 0, sizeof d);
    d.op = OP_GDT;
    d.dtype = DT_U8;
    d.conn = 8;
    d.h = mask->h;
    d.w = mask->w;
    d.a = mask->data;
    d.b = seeds->data;
    d.out = dist;
    d.pa = mask->pitch;
    d.pb = seeds->pitch;
    d.po = mask->w;
    return d;
}

int ensure_aux(iwpp_ctx *ctx, size_t bytes, cudaStream_t st) {
    if (bytes <= ctx->aux_bytes) return IWPP_OK;
    if (ctx->budget && bytes > ctx->budget)
        return fail(ctx, IWPP_ENOMEM, "planes of %zu bytes exceed the context budget of %zu", bytes, ctx->budget);
    if (ctx->aux) {
        CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        CK(cudaFree(ctx->aux), "cudaFree");
        ctx->aux = nullptr;
        ctx->aux_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->aux, bytes);
    if (e != cudaSuccess) {
        ctx->aux = nullptr;
        return fail(ctx, IWPP_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    ctx->aux_bytes = bytes;
    return IWPP_OK;
}

int check_ws(iwpp_ctx *ctx, const iwpp_image *relief, const iwpp_image *markers, const int32_t *labels,
             const void *levels) {
    int rc;
    if ((rc = check_image(ctx, relief, "relief")) || (rc = check_image(ctx, markers, "markers"))) return rc;
    if (markers->dtype != IWPP_I32) return fail(ctx, IWPP_EINVAL, "watershed: markers must be int32");
    if (relief->h != markers->h || relief->w != markers->w)
        return fail(ctx, IWPP_EINVAL, "watershed: relief and markers must have the same shape");
    if (!labels) return fail(ctx, IWPP_EINVAL, "null output pointer");
    // plateau distances stay below h*w - 1 < WS_DINF, the not-reached value
    if ((int64_t)relief->h * relief->w >= ((int64_t)1 << 30))
        return fail(ctx, IWPP_EINVAL, "watershed limited to h*w < 2^30");
    iwpp_image lab{const_cast<int32_t *>(labels), relief->h, relief->w, relief->w, IWPP_I32};
    if (overlaps(&lab, relief) || overlaps(&lab, markers))
        return fail(ctx, IWPP_EINVAL, "labels must not alias the relief or the markers");
    if (levels) {
        iwpp_image lv{const_cast<void *>(levels), relief->h, relief->w, relief->w, relief->dtype};
        if (overlaps(&lv, relief) || overlaps(&lv, markers) || overlaps(&lv, &lab))
            return fail(ctx, IWPP_EINVAL, "levels must not alias the relief, the markers or the labels");
    }
    return IWPP_OK;
}

// A propagation step of the watershed: in-edge masks E, values V (both
// dense planes).
JobDesc ws_job(int op, int h, int w, const uint8_t *E, int32_t *V) {
    JobDesc d;
    memset(&d, 0, sizeof d);
    d.op = op;
    d.dtype = DT_U8;
    d.conn = 8;
    d.h = h;
    d.w = w;
    d.a = E;
    d.out = V;
    d.pa = w;
    d.po = w;
    return d;
}

JobDesc edt_job(const iwpp_image *bin, int32_t *sq, int32_t *nn, int flags) {
    JobDesc d;
    memset(&d, 0, sizeof d);
    d.op = OP_EDT;
    d.dtype = DT_U8;
    d.conn = 8;
    d.flags = flags;
    d.h = bin->h;
    d.w = bin->w;
    d.a = bin->data;
    d.pa = bin->pitch;
    d.sqdist = sq;
    d.nearest = nn;
    // division by the width through a multiply and a shift: with
    // l = ceil(log2 w) and m = floor(2^(32+l) / w) + 1, (n * m) >> (32 + l)
    // equals n / w for every n < 2^32 (m*w - 2^(32+l) lies in (0, w], so the
    // added fraction stays below 1/w); n < 2^31 keeps n * m below 2^64
    int l = 0;
    while ((1ll << l) < (long long)d.w) ++l;
    d.wdiv_m = (1ull << (32 + l)) / (unsigned long long)d.w + 1ull;
    d.wdiv_s = 32 + l;
    return d;
}

}  // namespace


// A prepared batch for repeated launches (see iwpp_plan_create).
struct iwpp_plan {
    iwpp_ctx *ctx = nullptr;
    std::vector<iwpp_job> src;   // the jobs as given (re-prepared per option set)
    std::vector<JobDesc> jobs;   // all prepared descriptors
    // launch groups (one, or one per operation family with batch_split):
    // descriptors (layout, TMA maps), prepared launch, workspace offset
    std::vector<std::vector<JobDesc>> gjobs;
    std::vector<Prepared> parts;
    std::vector<size_t> offs;
    int fam = 0;                 // the family of the whole batch (tuning key)
    iwpp_options opt{};
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t cap = nullptr;  // private stream used for graph capture
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t key = 0;
};

namespace {

void drop_graph(iwpp_plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

// Workload key for the autotuner cache: kernel family, log2 of the pixel
// count, log2 of the job count, SM count.
uint64_t plan_key(const iwpp_ctx *ctx, const std::vector<JobDesc> &jobs, int fam) {
    int64_t px = 0;
    for (const JobDesc &j : jobs) px += (int64_t)j.h * j.w;
    int lp = 0, lj = 0;
    while ((1ll << lp) < px) ++lp;
    while ((1ll << lj) < (int64_t)jobs.size()) ++lj;
    return ((uint64_t)fam << 48) | ((uint64_t)lp << 32) | ((uint64_t)lj << 16) | (uint64_t)ctx->sm_count;
}

int jobs_from(iwpp_ctx *ctx, int n, const iwpp_job *js, std::vector<JobDesc> &jobs);

// (Re)prepares the plan for option set `opt`: layout, workspace, job table.
int plan_prepare(iwpp_plan *p, const iwpp_options &opt) {
    iwpp_ctx *ctx = p->ctx;
    drop_graph(p);
    p->jobs.clear();
    int rc = jobs_from(ctx, (int)p->src.size(), p->src.data(), p->jobs);
    if (rc) return rc;
    p->fam = pick_family(p->jobs);
    p->gjobs = launch_groups(p->jobs, opt.batch_split);
    p->parts.assign(p->gjobs.size(), Prepared());
    p->offs.assign(p->gjobs.size(), 0);
    size_t total = 0;
    for (size_t k = 0; k < p->gjobs.size(); ++k) {
        if ((rc = prepare(ctx, p->gjobs[k], opt, p->parts[k]))) return rc;
        p->offs[k] = total;
        total += align_up(p->parts[k].ws_bytes, 256);
    }
    if (total > p->ws_bytes) {
        if (p->ws) {
            CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
            cudaFree(p->ws);
            p->ws = nullptr;
            p->ws_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&p->ws, total);
        if (e != cudaSuccess) return fail(ctx, IWPP_ENOMEM, "plan workspace: %s", cudaGetErrorString(e));
        p->ws_bytes = total;
    }
    for (size_t k = 0; k < p->gjobs.size(); ++k) {
        char *ws = (char *)p->ws + p->offs[k];
        bind_workspace(p->parts[k], ws, ctx->ctl);
        if (p->gjobs[k].size() > 1)
            CK(cudaMemcpy(ws + p->parts[k].o_jobs, p->gjobs[k].data(), p->gjobs[k].size() * sizeof(JobDesc),
                          cudaMemcpyHostToDevice),
               "job table upload");
    }
    p->opt = opt;
    p->key = plan_key(ctx, p->jobs, p->fam);
    return IWPP_OK;
}

}  // namespace

extern "C" {

int iwpp_version(void) { return 100; }

int iwpp_ctx_create(iwpp_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return IWPP_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return IWPP_ECUDA;
    if (device < 0 || device >= ndev) return IWPP_EINVAL;
    iwpp_ctx *ctx = new iwpp_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    ctx->opt.tile = 0;
    ctx->opt.blocks_per_sm = 0;
    ctx->opt.sweeps = 3;
    ctx->opt.queue_factor = 32;
    ctx->opt.spill_cap = 8192;
    ctx->opt.max_relaunch = 1;
    ctx->opt.timeout_ms = 10000;
    ctx->opt.revisit_sweep_min = 0;
    ctx->opt.edt_sweeps = 2;
    ctx->opt.edt_revisit_sweep_min = 64;
    ctx->opt.revisit_sweeps = -1;
    ctx->opt.gdt_sweeps = 8;
    ctx->opt.batch_split = 1;
    ctx->opt.ws_sweeps = 6;
    ctx->opt.ws_revisit_sweep_min = 0;
    ctx->opt.gdt_revisit_sweep_min = 4;
    ctx->opt.edt_wide_step = 12;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&ctx->ctl, sizeof(Control)) != cudaSuccess ||
        cudaMemset(ctx->ctl, 0, sizeof(Control)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ctl, sizeof(Control)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        if (ctx->ctl) cudaFree(ctx->ctl);
        if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
        delete ctx;
        return IWPP_ECUDA;
    }
    *out = ctx;
    return IWPP_OK;
}

int iwpp_ctx_destroy(iwpp_ctx *ctx) {
    if (!ctx) return IWPP_OK;
    cudaSetDevice(ctx->device);
    if (ctx->sub_stream) {
        cudaStreamSynchronize(ctx->sub_stream);
        cudaStreamDestroy(ctx->sub_stream);
    }
    for (auto &t : ctx->tickets)
        if (t.second.ev) cudaEventDestroy(t.second.ev);
    if (ctx->h_sub_status) cudaFreeHost(ctx->h_sub_status);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->ctl) cudaFree(ctx->ctl);
    for (auto &ev : ctx->pending_events) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
    for (auto &ev : ctx->free_events) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    delete ctx;
    return IWPP_OK;
}

const char *iwpp_last_error(const iwpp_ctx *ctx) { return ctx ? ctx->err : "null context"; }

int iwpp_get_options(const iwpp_ctx *ctx, iwpp_options *out) {
    if (!ctx || !out) return IWPP_EINVAL;
    *out = ctx->opt;
    return IWPP_OK;
}

int iwpp_set_options(iwpp_ctx *ctx, const iwpp_options *o) {
    if (!ctx || !o) return IWPP_EINVAL;
    if (o->tile != 0 && o->tile != TILE) return fail(ctx, IWPP_EINVAL, "tile must be 0 or %d (fixed)", TILE);
    if (o->blocks_per_sm < 0 || o->sweeps < 0 || o->sweeps > 64 || o->queue_factor < 1 || o->queue_factor > 4096 ||
        o->spill_cap < 0 || o->spill_cap > (1 << 20) || o->max_relaunch < 0 || o->max_relaunch > 64 ||
        o->timeout_ms < 1 || o->timeout_ms > 600000 || o->timing < 0 || o->timing > 1 ||
        o->revisit_sweep_min < 0 || o->edt_sweeps < 0 || o->edt_sweeps > 64 || o->edt_revisit_sweep_min < 0 ||
        o->revisit_sweeps < -1 || o->revisit_sweeps > 64 || o->queue_mode < 0 || o->queue_mode > 3 ||
        o->test_empty_slot < 0 || o->test_empty_slot > 1 || o->gdt_sweeps < 0 || o->gdt_sweeps > 64 ||
        o->batch_split < 0 || o->batch_split > 1 || o->ws_sweeps < 0 || o->ws_sweeps > 64 ||
        o->ws_revisit_sweep_min < 0 || o->gdt_revisit_sweep_min < 0 || o->edt_wide_step < 1 ||
        o->edt_wide_step > 65536)
        return fail(ctx, IWPP_EINVAL, "option out of range");
    ctx->opt = *o;
    return IWPP_OK;
}

int iwpp_recon_async(iwpp_ctx *ctx, const iwpp_image *marker, const iwpp_image *mask, int conn,
                     iwpp_image *out, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_recon(ctx, marker, mask, conn, out);
    if (rc) return rc;
    std::vector<JobDesc> jobs{recon_job(marker, mask, conn, out)};
    return run(ctx, jobs, (cudaStream_t)stream, false);
}

int iwpp_recon(iwpp_ctx *ctx, const iwpp_image *marker, const iwpp_image *mask, int conn, iwpp_image *out,
               void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_recon(ctx, marker, mask, conn, out);
    if (rc) return rc;
    std::vector<JobDesc> jobs{recon_job(marker, mask, conn, out)};
    return run(ctx, jobs, (cudaStream_t)stream, true);
}

int iwpp_edt_async(iwpp_ctx *ctx, const iwpp_image *binary, int32_t *sqdist, int32_t *nearest, int flags,
                   void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_edt(ctx, binary, sqdist, nearest, flags);
    if (rc) return rc;
    std::vector<JobDesc> jobs{edt_job(binary, sqdist, nearest, flags)};
    return run(ctx, jobs, (cudaStream_t)stream, false);
}

int iwpp_edt(iwpp_ctx *ctx, const iwpp_image *binary, int32_t *sqdist, int32_t *nearest, int flags, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_edt(ctx, binary, sqdist, nearest, flags);
    if (rc) return rc;
    std::vector<JobDesc> jobs{edt_job(binary, sqdist, nearest, flags)};
    return run(ctx, jobs, (cudaStream_t)stream, true);
}

int iwpp_geodesic(iwpp_ctx *ctx, const iwpp_image *mask, const iwpp_image *seeds, int32_t *dist, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_gdt(ctx, mask, seeds, dist);
    if (rc) return rc;
    std::vector<JobDesc> jobs{gdt_job(mask, seeds, dist)};
    return run(ctx, jobs, (cudaStream_t)stream, true);
}

int iwpp_geodesic_async(iwpp_ctx *ctx, const iwpp_image *mask, const iwpp_image *seeds, int32_t *dist,
                        void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_gdt(ctx, mask, seeds, dist);
    if (rc) return rc;
    std::vector<JobDesc> jobs{gdt_job(mask, seeds, dist)};
    return run(ctx, jobs, (cudaStream_t)stream, false);
}

int iwpp_watershed(iwpp_ctx *ctx, const iwpp_image *relief, const iwpp_image *markers, int32_t *labels,
                   void *levels, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_ws(ctx, relief, markers, labels, levels);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int h = relief->h, w = relief->w;
    const int dt = relief->dtype == IWPP_U8 ? DT_U8 : DT_I32;
    const size_t n = (size_t)h * w, es = dt == DT_U8 ? 1 : 4;
    const size_t oA = 0, oB = align_up(n * es, 256), oE = oB + align_up(n * es, 256), oD = oE + align_up(n, 256);
    if ((rc = ensure_aux(ctx, oD + align_up(n * 4, 256), st))) return rc;
    char *aux = (char *)ctx->aux;
    WsArgs a;
    a.relief = relief->data;
    a.markers = (const int32_t *)markers->data;
    a.pf = relief->pitch;
    a.pm = markers->pitch;
    a.h = h;
    a.w = w;
    a.dtype = dt;
    a.A = aux + oA;
    a.B = aux + oB;
    a.E = (uint8_t *)(aux + oE);
    a.D = (int32_t *)(aux + oD);
    a.labels = labels;
    a.levels = levels;
    // 1. flooding levels: reconstruction by dilation of the complements
    CK(launch_ws_complement(a, st), "watershed complement launch");
    iwpp_image A{a.A, h, w, w, relief->dtype}, B{a.B, h, w, w, relief->dtype};
    std::vector<JobDesc> j1{recon_job(&A, &B, 8, &A)};
    if ((rc = run(ctx, j1, st, false))) return rc;
    // 2. plateau distances
    CK(launch_ws_plateau_init(a, st), "watershed plateau init launch");
    std::vector<JobDesc> j2{ws_job(OP_WS_DIST, h, w, a.E, a.D)};
    if ((rc = run(ctx, j2, st, false))) return rc;
    // 3. labels
    CK(launch_ws_label_init(a, st), "watershed label init launch");
    std::vector<JobDesc> j3{ws_job(OP_WS_LABEL, h, w, a.E, labels)};
    if ((rc = run(ctx, j3, st, false))) return rc;
    CK(launch_ws_label_finish(a, st), "watershed label finish launch");
    ctx->launches += 4;
    ctx->calls -= 2;  // the three propagations are one call
    return iwpp_sync(ctx, st);
}

int iwpp_skiz(iwpp_ctx *ctx, const iwpp_image *mask, const iwpp_image *labels, int32_t *zones, uint8_t *skiz,
              int32_t *dist, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc;
    if ((rc = check_image(ctx, mask, "mask")) || (rc = check_image(ctx, labels, "labels"))) return rc;
    if (mask->dtype != IWPP_U8 || labels->dtype != IWPP_I32)
        return fail(ctx, IWPP_EINVAL, "skiz: mask must be uint8 and labels int32");
    if (mask->h != labels->h || mask->w != labels->w)
        return fail(ctx, IWPP_EINVAL, "skiz: mask and labels must have the same shape");
    if (!zones) return fail(ctx, IWPP_EINVAL, "null output pointer");
    if ((int64_t)mask->h * mask->w >= ((int64_t)1 << 31))
        return fail(ctx, IWPP_EINVAL, "skiz limited to h*w < 2^31");
    const int h = mask->h, w = mask->w;
    iwpp_image zi{zones, h, w, w, IWPP_I32};
    if (overlaps(&zi, mask) || overlaps(&zi, labels))
        return fail(ctx, IWPP_EINVAL, "zones must not alias the mask or the labels");
    if (dist) {
        iwpp_image di{dist, h, w, w, IWPP_I32};
        if (overlaps(&di, mask) || overlaps(&di, labels) || overlaps(&di, &zi))
            return fail(ctx, IWPP_EINVAL, "dist must not alias the inputs or zones");
    }
    if (skiz) {
        iwpp_image si{skiz, h, w, w, IWPP_U8};
        if (overlaps(&si, mask) || overlaps(&si, labels) || overlaps(&si, &zi))
            return fail(ctx, IWPP_EINVAL, "skiz must not alias the inputs or zones");
    }
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t n = (size_t)h * w;
    const size_t oS = 0, oE = align_up(n, 256), oN = oE + align_up(n, 256), oD = oN + align_up(n * 4, 256);
    if ((rc = ensure_aux(ctx, oD + (dist ? 0 : align_up(n * 4, 256)), st))) return rc;
    char *aux = (char *)ctx->aux;
    SkizArgs a;
    a.mask = (const uint8_t *)mask->data;
    a.labels = (const int32_t *)labels->data;
    a.pmask = mask->pitch;
    a.pl = labels->pitch;
    a.h = h;
    a.w = w;
    a.seeds = (uint8_t *)(aux + oS);
    a.E = (uint8_t *)(aux + oE);
    a.neg = (int32_t *)(aux + oN);
    a.dist = dist ? dist : (int32_t *)(aux + oD);
    a.zones = zones;
    a.skiz = skiz;
    // 1. least path costs from the sources
    CK(launch_skiz_prep(a, st), "skiz prep launch");
    iwpp_image seeds{a.seeds, h, w, w, IWPP_U8};
    std::vector<JobDesc> j1{gdt_job(mask, &seeds, a.dist)};
    if ((rc = run(ctx, j1, st, false))) return rc;
    // 2. least and greatest labels along the shortest-path edges, one launch
    CK(launch_skiz_label_init(a, st), "skiz label init launch");
    std::vector<JobDesc> j2{ws_job(OP_WS_LABEL, h, w, a.E, a.zones), ws_job(OP_WS_LABEL, h, w, a.E, a.neg)};
    if ((rc = run(ctx, j2, st, false))) return rc;
    CK(launch_skiz_finish(a, st), "skiz finish launch");
    ctx->launches += 3;
    ctx->calls -= 1;  // the two propagation launches are one call
    return iwpp_sync(ctx, st);
}

int iwpp_edt_exact(iwpp_ctx *ctx, const iwpp_image *binary, int32_t *sqdist, int32_t *nearest, int flags,
                   void *stream) {
    if (!ctx) return IWPP_EINVAL;
    int rc = check_edt(ctx, binary, sqdist, nearest, flags);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int h = binary->h, w = binary->w, nb = exact_bands(h);
    const size_t band_bytes = align_up((size_t)nb * w * sizeof(int32_t), 256);
    const size_t plane_bytes = align_up((size_t)h * w * sizeof(uint32_t), 256);
    if ((rc = ensure_ws(ctx, 4 * band_bytes + plane_bytes, st))) return rc;
    char *ws = (char *)ctx->ws;
    ExactArgs a;
    a.bin = (const uint8_t *)binary->data;
    a.pitch = binary->pitch;
    a.h = h;
    a.w = w;
    a.flags = flags;
    a.nb = nb;
    a.first = (int32_t *)ws;
    a.last = (int32_t *)(ws + band_bytes);
    a.above = (int32_t *)(ws + 2 * band_bytes);
    a.below = (int32_t *)(ws + 3 * band_bytes);
    a.G = (int32_t *)(ws + 4 * band_bytes);
    a.sqdist = sqdist;
    a.nearest = nearest;
    CK(launch_edt_exact(a, st), "exact distance transform launch");
    ctx->launches += 4;
    ctx->calls += 1;
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return IWPP_OK;
}

int iwpp_recon_batched(iwpp_ctx *ctx, int n, const iwpp_image *markers, const iwpp_image *masks, int conn,
                       iwpp_image *outs, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    if (n < 1 || !markers || !masks || !outs) return fail(ctx, IWPP_EINVAL, "batched: n >= 1 and arrays required");
    std::vector<JobDesc> jobs;
    jobs.reserve(n);
    for (int i = 0; i < n; ++i) {
        int rc = check_recon(ctx, markers + i, masks + i, conn, outs + i);
        if (rc) return rc;
        jobs.push_back(recon_job(markers + i, masks + i, conn, outs + i));
    }
    return run(ctx, jobs, (cudaStream_t)stream, true);
}

int iwpp_edt_batched(iwpp_ctx *ctx, int n, const iwpp_image *bins, int32_t *const *sqdists,
                     int32_t *const *nearests, int flags, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    if (n < 1 || !bins || !sqdists || !nearests) return fail(ctx, IWPP_EINVAL, "batched: n >= 1 and arrays required");
    std::vector<JobDesc> jobs;
    jobs.reserve(n);
    for (int i = 0; i < n; ++i) {
        int rc = check_edt(ctx, bins + i, sqdists[i], nearests[i], flags);
        if (rc) return rc;
        jobs.push_back(edt_job(bins + i, sqdists[i], nearests[i], flags));
    }
    return run(ctx, jobs, (cudaStream_t)stream, true);
}

}  // extern "C"

namespace {
int jobs_from(iwpp_ctx *ctx, int n, const iwpp_job *js, std::vector<JobDesc> &jobs) {
    if (n < 1 || !js) return fail(ctx, IWPP_EINVAL, "jobs: n >= 1 and an array required");
    jobs.reserve(n);
    for (int i = 0; i < n; ++i) {
        const iwpp_job &j = js[i];
        int rc;
        if (j.op == IWPP_OP_RECON) {
            if ((rc = check_recon(ctx, &j.a, &j.b, j.conn, &j.out))) return rc;
            jobs.push_back(recon_job(&j.a, &j.b, j.conn, const_cast<iwpp_image *>(&j.out)));
        } else if (j.op == IWPP_OP_EDT) {
            if ((rc = check_edt(ctx, &j.a, j.sqdist, j.nearest, j.flags))) return rc;
            jobs.push_back(edt_job(&j.a, j.sqdist, j.nearest, j.flags));
        } else {
            return fail(ctx, IWPP_EINVAL, "job %d: unknown op %d", i, j.op);
        }
    }
    return IWPP_OK;
}
}  // namespace

extern "C" {

int iwpp_run_jobs(iwpp_ctx *ctx, int n, const iwpp_job *js, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    std::vector<JobDesc> jobs;
    int rc = jobs_from(ctx, n, js, jobs);
    if (rc) return rc;
    return run(ctx, jobs, (cudaStream_t)stream, true);
}

int iwpp_run_jobs_async(iwpp_ctx *ctx, int n, const iwpp_job *js, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    std::vector<JobDesc> jobs;
    int rc = jobs_from(ctx, n, js, jobs);
    if (rc) return rc;
    return run(ctx, jobs, (cudaStream_t)stream, false);
}

}  // extern "C"

namespace {

constexpr int kSubRing = 256;  // outstanding tickets with a status word in the ring

int status_code(iwpp_ctx *ctx, int errors) {
    if (errors & ST_TIMEOUT) return fail(ctx, IWPP_ETIMEOUT, "a device-side wait saw no progress for %d ms",
                                         ctx->opt.timeout_ms);
    if (errors & ST_OVERFLOW) return fail(ctx, IWPP_EOVERFLOW, "tile queue overflowed after %d relaunches",
                                          ctx->opt.max_relaunch);
    return IWPP_OK;
}

// Waits for ticket t's event and keeps its status word on the host, so
// that its ring slot can serve another ticket.
int settle_ticket(iwpp_ctx *ctx, iwpp_ctx::Ticket &t) {
    if (t.slot < 0) return IWPP_OK;
    CK(cudaEventSynchronize(t.ev), "cudaEventSynchronize");
    t.status = ctx->h_sub_status[t.slot];
    ctx->sub_slot_owner[t.slot] = 0;
    t.slot = -1;
    return IWPP_OK;
}

// A free ring slot; when all are held, the oldest outstanding ticket is
// settled first.
int take_slot(iwpp_ctx *ctx, int *slot) {
    for (int i = 0; i < kSubRing; ++i)
        if (ctx->sub_slot_owner[i] == 0) {
            *slot = i;
            return IWPP_OK;
        }
    for (auto &kv : ctx->tickets)
        if (kv.second.slot >= 0) {
            const int s = kv.second.slot;
            int rc = settle_ticket(ctx, kv.second);
            if (rc) return rc;
            *slot = s;
            return IWPP_OK;
        }
    return fail(ctx, IWPP_ECUDA, "submit: no status slot");
}

int retire(iwpp_ctx *ctx, uint64_t ticket, int *status) {
    auto it = ctx->tickets.find(ticket);
    iwpp_ctx::Ticket t = it->second;
    ctx->tickets.erase(it);
    if (t.ev) cudaEventDestroy(t.ev);
    const int rc = status_code(ctx, t.status);
    if (status) *status = rc;
    return IWPP_OK;
}

}  // namespace

extern "C" {

int iwpp_submit(iwpp_ctx *ctx, const iwpp_job *job, uint64_t *ticket) {
    if (!ctx) return IWPP_EINVAL;
    if (!job || !ticket) return fail(ctx, IWPP_EINVAL, "submit: job and ticket required");
    *ticket = 0;
    std::vector<JobDesc> jobs;
    int rc = jobs_from(ctx, 1, job, jobs);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!ctx->sub_stream) {
        // a blocking stream: ordered with work on the legacy default stream
        CK(cudaStreamCreate(&ctx->sub_stream), "cudaStreamCreate");
        CK(cudaMallocHost(&ctx->h_sub_status, kSubRing * sizeof(int)), "cudaMallocHost");
        ctx->sub_slot_owner.assign(kSubRing, 0);
    }
    int slot = -1;
    if ((rc = take_slot(ctx, &slot))) return rc;
    cudaStream_t st = ctx->sub_stream;
    if ((rc = run(ctx, jobs, st, false))) return rc;
    // the job's outcome word goes to its own status slot, then the shared
    // word is cleared for the next job on the stream
    CK(cudaMemcpyAsync(ctx->h_sub_status + slot, &ctx->ctl->errors, sizeof(int), cudaMemcpyDeviceToHost, st),
       "status readback");
    CK(cudaMemsetAsync(&ctx->ctl->errors, 0, sizeof(int), st), "status reset");
    iwpp_ctx::Ticket t;
    CK(cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming), "cudaEventCreate");
    cudaError_t e = cudaEventRecord(t.ev, st);
    if (e != cudaSuccess) {
        cudaEventDestroy(t.ev);
        return cuda_fail(ctx, e, "cudaEventRecord");
    }
    t.slot = slot;
    const uint64_t id = ctx->next_ticket++;
    ctx->sub_slot_owner[slot] = id;
    ctx->tickets[id] = t;
    *ticket = id;
    return IWPP_OK;
}

int iwpp_poll(iwpp_ctx *ctx, uint64_t ticket, int *status) {
    if (!ctx) return IWPP_EINVAL;
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, IWPP_EINVAL, "poll: unknown or retired ticket %llu",
                                              (unsigned long long)ticket);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    iwpp_ctx::Ticket &t = it->second;
    if (t.slot >= 0) {
        const cudaError_t e = cudaEventQuery(t.ev);
        if (e == cudaErrorNotReady) {
            (void)cudaGetLastError();
            return 0;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventQuery");
        int rc = settle_ticket(ctx, t);
        if (rc) return rc;
    }
    int rc = retire(ctx, ticket, status);
    return rc ? rc : 1;
}

int iwpp_wait(iwpp_ctx *ctx, uint64_t ticket, int *status) {
    if (!ctx) return IWPP_EINVAL;
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, IWPP_EINVAL, "wait: unknown or retired ticket %llu",
                                              (unsigned long long)ticket);
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = settle_ticket(ctx, it->second);
    if (rc) return rc;
    return retire(ctx, ticket, status);
}

}  // extern "C"

namespace iwpp {

size_t ctx_device_bytes(const iwpp_ctx *ctx) {
    return ctx->ws_bytes + ctx->aux_bytes + sizeof(Control);
}

int ctx_device_bytes_after(iwpp_ctx *ctx, int n, const int *op, const int *dtype, const int *h, const int *w,
                           size_t *bytes) {
    std::vector<JobDesc> jobs(n);
    for (int i = 0; i < n; ++i) {
        memset(&jobs[i], 0, sizeof(JobDesc));
        jobs[i].op = op[i] == IWPP_OP_RECON ? OP_RECON : OP_EDT;
        jobs[i].dtype = dtype[i] == IWPP_I32 ? DT_I32 : DT_U8;
        jobs[i].h = h[i];
        jobs[i].w = w[i];
    }
    size_t need = 0;
    int rc;
    for (const std::vector<JobDesc> &g : launch_groups(jobs, ctx->opt.batch_split)) {
        size_t b = 0;
        if ((rc = workspace_need(ctx, g, ctx->opt, &b))) return rc;
        need += align_up(b, 256);
    }
    const size_t ws = need <= ctx->ws_bytes ? ctx->ws_bytes : ws_alloc_size(ctx, need);
    *bytes = ws + ctx->aux_bytes + sizeof(Control);
    return IWPP_OK;
}

int status_readback(iwpp_ctx *ctx, cudaStream_t st) {
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st), "status readback");
    return IWPP_OK;
}

int status_result(iwpp_ctx *ctx, cudaStream_t st) {
    const int errors = ctx->h_ctl->errors;
    if (errors) {
        CK(cudaMemsetAsync(&ctx->ctl->errors, 0, sizeof(int), st), "status reset");
        CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    }
    if (errors & ST_TIMEOUT) return fail(ctx, IWPP_ETIMEOUT, "a device-side wait exceeded %d ms", ctx->opt.timeout_ms);
    if (errors & ST_OVERFLOW)
        return fail(ctx, IWPP_EOVERFLOW, "tile queue overflowed after %d relaunches; raise queue_factor or max_relaunch",
                    ctx->opt.max_relaunch);
    return IWPP_OK;
}

}  // namespace iwpp

extern "C" {

int iwpp_sync(iwpp_ctx *ctx, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = iwpp::status_readback(ctx, st);
    if (rc) return rc;
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    for (auto &ev : ctx->pending_events) {
        float ms = 0.f;
        CK(cudaEventSynchronize(ev.second), "cudaEventSynchronize");
        CK(cudaEventElapsedTime(&ms, ev.first, ev.second), "cudaEventElapsedTime");
        ctx->kernel_ns += (uint64_t)((double)ms * 1e6);
        ctx->free_events.push_back(ev);
    }
    ctx->pending_events.clear();
    return iwpp::status_result(ctx, st);
}

int iwpp_stats(iwpp_ctx *ctx, iwpp_stats_t *out) {
    if (!ctx || !out) return IWPP_EINVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    Control c;
    CK(cudaMemcpy(&c, ctx->ctl, sizeof c, cudaMemcpyDeviceToHost), "stats readback");
    out->calls = ctx->calls;
    out->tiles_processed = c.tiles_processed;
    out->tiles_initial = ctx->tiles_initial;
    out->seeds = c.seeds;
    out->pushes = c.pushes;
    out->spills = c.spills;
    out->rescans = c.rescans;
    out->relaunches = c.relaunches;
    out->rounds = c.rounds;
    out->wait_ns = c.wait_ns;
    out->visit_ns = c.visit_ns;
    for (int i = 0; i < 4; ++i) out->phase_ns[i] = c.phase_ns[i];
    out->kernel_launches = ctx->launches;
    out->kernel_ns = ctx->kernel_ns;
    out->sweep_sets = c.sweep_sets;
    out->revisits = c.revisits;
    return IWPP_OK;
}

int iwpp_stats_reset(iwpp_ctx *ctx) {
    if (!ctx) return IWPP_EINVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    Control c;
    CK(cudaMemcpy(&c, ctx->ctl, sizeof c, cudaMemcpyDeviceToHost), "stats readback");
    c.tiles_processed = c.seeds = c.pushes = c.spills = c.rescans = c.relaunches = c.rounds = 0;
    c.wait_ns = c.visit_ns = 0;
    for (int i = 0; i < 4; ++i) c.phase_ns[i] = 0;
    c.sweep_sets = c.revisits = 0;
    CK(cudaMemcpy(ctx->ctl, &c, sizeof c, cudaMemcpyHostToDevice), "stats reset");
    ctx->calls = 0;
    ctx->tiles_initial = 0;
    ctx->launches = 0;
    ctx->kernel_ns = 0;
    return IWPP_OK;
}

int iwpp_plan_create(iwpp_ctx *ctx, int n, const iwpp_job *jobs, iwpp_plan **out) {
    if (!ctx || !out) return IWPP_EINVAL;
    *out = nullptr;
    if (n < 1 || !jobs) return fail(ctx, IWPP_EINVAL, "plan: n >= 1 and a job array required");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    iwpp_plan *p = new iwpp_plan();
    p->ctx = ctx;
    p->src.assign(jobs, jobs + n);
    // a tuned option set for this kind of workload, if the autotuner ran
    iwpp_options opt = ctx->opt;
    {
        std::vector<JobDesc> tmp;
        if (jobs_from(ctx, n, jobs, tmp) == IWPP_OK) {
            const uint64_t key = plan_key(ctx, tmp, pick_family(tmp));
            auto it = ctx->tuned.find(key);
            if (it != ctx->tuned.end()) opt = it->second;
        }
    }
    int rc = plan_prepare(p, opt);
    if (rc == IWPP_OK && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
        rc = fail(ctx, IWPP_ECUDA, "plan: stream creation failed");
    if (rc) {
        iwpp_plan_destroy(p);
        return rc;
    }
    *out = p;
    return IWPP_OK;
}

int iwpp_plan_launch(iwpp_plan *p, void *stream) {
    if (!p) return IWPP_EINVAL;
    iwpp_ctx *ctx = p->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    for (const Prepared &P : p->parts) {
        int rc = enqueue(ctx, P, p->opt.max_relaunch, (cudaStream_t)stream, nullptr, nullptr);
        if (rc) return rc;
        ctx->launches += 3 + 3 * (uint64_t)p->opt.max_relaunch;
        ctx->tiles_initial += (uint64_t)P.ntiles;
    }
    ctx->calls += 1;
    return IWPP_OK;
}

int iwpp_plan_launch_graph(iwpp_plan *p, void *stream) {
    if (!p) return IWPP_EINVAL;
    iwpp_ctx *ctx = p->ctx;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if (!p->exec) {
        CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        int rc = IWPP_OK;
        for (const Prepared &P : p->parts)
            if (rc == IWPP_OK) rc = enqueue(ctx, P, p->opt.max_relaunch, p->cap, nullptr, nullptr);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        p->graph = g;
        CK(cudaGraphInstantiate(&p->exec, p->graph, 0), "cudaGraphInstantiate");
    }
    CK(cudaGraphLaunch(p->exec, (cudaStream_t)stream), "cudaGraphLaunch");
    for (const Prepared &P : p->parts) {
        ctx->launches += 3 + 3 * (uint64_t)p->opt.max_relaunch;
        ctx->tiles_initial += (uint64_t)P.ntiles;
    }
    ctx->calls += 1;
    return IWPP_OK;
}

int iwpp_plan_autotune(iwpp_plan *p, void *stream, int reps, iwpp_options *best) {
    if (!p || reps < 1) return IWPP_EINVAL;
    iwpp_ctx *ctx = p->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    CK(cudaEventCreate(&e1), "cudaEventCreate");
    const iwpp_options base = p->opt;
    iwpp_options best_opt = base;
    float best_ms = 1e30f;
    int rc = IWPP_OK;
    const int occ = ctx->occupancy[p->fam];
    // sweep candidates per operation; a mixed plan pairs them up
    const int sweeps_c[3] = {2, 3, 4};
    const int revisit_c[2] = {0, 32};
    const int edt_sweeps_c[3] = {1, 2, 3};
    const int edt_revisit_c[2] = {16, 64};
    const int fam = p->fam;
    const int bps_c[2] = {0, occ > 2 ? occ - 1 : 0};
    // a batch of several operation families: one mixed launch, or one
    // launch per family (then all CTAs per SM: occupancy differs per part)
    const int nsplit = launch_groups(p->jobs, 1).size() > 1 ? 2 : 1;
    for (int sp = 0; sp < nsplit && rc == IWPP_OK; ++sp)
    for (int a = 0; a < 3 && rc == IWPP_OK; ++a)
        for (int b = 0; b < 2 && rc == IWPP_OK; ++b)
            for (int c = 0; c < 2 && rc == IWPP_OK; ++c) {
                if (c == 1 && (bps_c[1] == 0 || sp == 1)) continue;
                iwpp_options o = base;
                o.batch_split = sp;
                if (fam != FAM_EDT) {
                    o.sweeps = sweeps_c[a];
                    o.revisit_sweep_min = revisit_c[b];
                }
                if (fam == FAM_EDT || fam == FAM_MIXED) {
                    o.edt_sweeps = edt_sweeps_c[a];
                    o.edt_revisit_sweep_min = edt_revisit_c[b];
                }
                o.blocks_per_sm = bps_c[c];
                if ((rc = plan_prepare(p, o))) break;
                if ((rc = iwpp_plan_launch(p, st))) break;  // warm-up
                if ((rc = iwpp_sync(ctx, st))) break;
                CK(cudaEventRecord(e0, st), "cudaEventRecord");
                for (int r = 0; r < reps && rc == IWPP_OK; ++r) rc = iwpp_plan_launch(p, st);
                CK(cudaEventRecord(e1, st), "cudaEventRecord");
                if (rc || (rc = iwpp_sync(ctx, st))) break;
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
                if (ms < best_ms) {
                    best_ms = ms;
                    best_opt = o;
                }
            }
    // second stage, from the best option set: the capacities of the tile
    // queue (slots per tile) and of each CTA's spill queue.  Too few slots
    // cost a relaunch, too many cost memory; the spill queue trades global
    // memory against in-tile rescans.
    const int qf_c[3] = {8, 16, 32};
    const int sc_c[2] = {1024, 8192};
    const iwpp_options stage1 = best_opt;
    for (int a = 0; a < 3 && rc == IWPP_OK; ++a)
        for (int b = 0; b < 2 && rc == IWPP_OK; ++b) {
            iwpp_options o = stage1;
            o.queue_factor = qf_c[a];
            o.spill_cap = sc_c[b];
            if (o.queue_factor == stage1.queue_factor && o.spill_cap == stage1.spill_cap) continue;
            if ((rc = plan_prepare(p, o))) break;
            if ((rc = iwpp_plan_launch(p, st))) break;  // warm-up
            if ((rc = iwpp_sync(ctx, st))) break;
            CK(cudaEventRecord(e0, st), "cudaEventRecord");
            for (int r = 0; r < reps && rc == IWPP_OK; ++r) rc = iwpp_plan_launch(p, st);
            CK(cudaEventRecord(e1, st), "cudaEventRecord");
            if (rc || (rc = iwpp_sync(ctx, st))) break;
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            if (ms < best_ms) {
                best_ms = ms;
                best_opt = o;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        plan_prepare(p, base);
        return rc;
    }
    rc = plan_prepare(p, best_opt);
    if (rc) return rc;
    ctx->tuned[p->key] = best_opt;
    if (best) *best = best_opt;
    return IWPP_OK;
}

int iwpp_plan_destroy(iwpp_plan *p) {
    if (!p) return IWPP_OK;
    cudaSetDevice(p->ctx->device);
    drop_graph(p);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->ws) {
        cudaDeviceSynchronize();
        cudaFree(p->ws);
    }
    delete p;
    return IWPP_OK;
}

}  // extern "C"

