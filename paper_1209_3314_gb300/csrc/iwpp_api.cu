// iwpp_api.cu -- host side of the libiwpp C ABI (declared in include/iwpp.h):
// argument validation, the context and its device workspace, tile-size
// selection, and the launch sequence of the persistent tile-wavefront kernel.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/iwpp.h"
#include "iwpp_internal.h"

using namespace iwpp;

struct iwpp_ctx {
    int device = 0;
    size_t budget = 0;
    int sm_count = 0;
    iwpp_options opt{};
    char err[256] = {0};
    void *ws = nullptr;        // workspace arena
    size_t ws_bytes = 0;
    Control *ctl = nullptr;    // device control block (own allocation, persistent counters)
    Control *h_ctl = nullptr;  // pinned host copy
    uint64_t calls = 0;
    uint64_t tiles_initial = 0;
    uint64_t launches = 0;
    uint64_t kernel_ns = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending_events, free_events;
    int occupancy[FAM_COUNT] = {0, 0, 0, 0};  // blocks per SM per kernel family
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
    for (const JobDesc &j : jobs) {
        if (j.op == OP_EDT) e = true;
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
bool make_map(CUtensorMap *m, const void *base, int dtype, int h, int w, int64_t pitch_elems) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const size_t es = dtype == DT_U8 ? 1 : 4;
    const uint64_t pitch_bytes = (uint64_t)pitch_elems * es;
    if (((uintptr_t)base & 15) || (pitch_bytes & 15) || pitch_bytes >= (1ull << 40)) return false;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[1] = {pitch_bytes};
    cuuint32_t box[2] = {dtype == DT_U8 ? 96u : 72u, (cuuint32_t)(TILE + 2)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, dtype == DT_U8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_INT32, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void make_maps(JobDesc &d) {
    bool ok;
    if (d.op == OP_RECON) {
        ok = make_map(&d.tm[0], d.a, d.dtype, d.h, d.w, d.pa) && make_map(&d.tm[1], d.b, d.dtype, d.h, d.w, d.pb) &&
             make_map(&d.tm[2], d.out, d.dtype, d.h, d.w, d.po);
    } else {
        ok = make_map(&d.tm[0], d.a, DT_U8, d.h, d.w, d.pa) && make_map(&d.tm[2], d.nearest, DT_I32, d.h, d.w, d.w);
    }
    d.use_tma = ok ? 1 : 0;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

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
    size_t b = align_up(bytes + bytes / 4, 1 << 20);
    if (ctx->budget && b > ctx->budget) b = bytes;
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

// Runs (or enqueues) the whole launch sequence for `jobs`.
int run(iwpp_ctx *ctx, std::vector<JobDesc> &jobs, cudaStream_t st, bool sync) {
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int tile = TILE;
    const int fam = pick_family(jobs);
    const int64_t ntiles = layout_jobs(jobs, tile);
    for (JobDesc &j : jobs) make_maps(j);
    if (ntiles <= 0 || ntiles > (int64_t)1 << 28) return fail(ctx, IWPP_EINVAL, "tile count %lld out of range", (long long)ntiles);
    const int64_t cap64 = std::max<int64_t>(ntiles + 1, (int64_t)ctx->opt.queue_factor * ntiles);
    if (cap64 > ((int64_t)1 << 31) - 1) return fail(ctx, IWPP_EINVAL, "tile queue too large");

    int &occ = ctx->occupancy[fam];
    if (occ == 0) {
        CK(family_occupancy(fam, &occ), "occupancy query");
        if (occ < 1) return fail(ctx, IWPP_ECUDA, "persistent kernel does not fit on an SM");
    }
    int bps = ctx->opt.blocks_per_sm > 0 ? std::min(ctx->opt.blocks_per_sm, occ) : occ;
    int64_t grid64 = std::min<int64_t>(ntiles, (int64_t)bps * ctx->sm_count);
    const int grid = (int)std::max<int64_t>(1, grid64);

    // workspace layout
    const size_t n_slots = (size_t)cap64;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_slots = take(n_slots * 4);
    const size_t o_state = take((size_t)ntiles * 4);
    const size_t o_visited = take((size_t)ntiles * 4);
    const size_t o_cnt = take(16);
    const size_t o_spill = take((size_t)grid * 2 * std::max(1, ctx->opt.spill_cap) * sizeof(uint16_t));
    const size_t o_jobs = take(jobs.size() > 1 ? jobs.size() * sizeof(JobDesc) : 0);
    int rc = ensure_ws(ctx, off, st);
    if (rc) return rc;
    char *ws = (char *)ctx->ws;

    KArgs ka;
    memset(&ka, 0, sizeof ka);
    ka.njobs = (int)jobs.size();
    ka.ntiles = (int)ntiles;
    ka.job0 = jobs[0];
    ka.jobs = jobs.size() > 1 ? (const JobDesc *)(ws + o_jobs) : nullptr;
    ka.tq.slots = (int *)(ws + o_slots);
    ka.tq.state = (int *)(ws + o_state);
    ka.tq.visited = (int *)(ws + o_visited);
    ka.tq.head = (unsigned *)(ws + o_cnt);
    ka.tq.tail = (unsigned *)(ws + o_cnt + 4);
    ka.tq.pending = (int *)(ws + o_cnt + 8);
    ka.tq.cap = (unsigned)cap64;
    ka.tq.ntiles = (int)ntiles;
    ka.ctl = ctx->ctl;
    ka.spill = (uint16_t *)(ws + o_spill);
    ka.spill_cap = std::max(0, ctx->opt.spill_cap);
    ka.sweeps = ctx->opt.sweeps;
    ka.revisit_sweep_min = ctx->opt.revisit_sweep_min;
    ka.timeout_ns = (unsigned long long)ctx->opt.timeout_ms * 1000000ull;

    if (jobs.size() > 1)
        CK(cudaMemcpyAsync(ws + o_jobs, jobs.data(), jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, st),
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
    CK(launch_init(ka, 1, st), "launch fill_queue");
    if (ev.first) CK(cudaEventRecord(ev.first, st), "cudaEventRecord");
    CK(launch_persistent(ka, fam, grid, st), "launch persistent");
    for (int k = 0; k < ctx->opt.max_relaunch; ++k) {
        CK(launch_decide(ka, 0, st), "launch decide");
        CK(launch_reset(ka, st), "launch reset");
        CK(launch_persistent(ka, fam, grid, st), "launch persistent");
    }
    if (ev.second) {
        CK(cudaEventRecord(ev.second, st), "cudaEventRecord");
        ctx->pending_events.push_back(ev);
    }
    CK(launch_decide(ka, 1, st), "launch decide");
    ctx->launches += 3 + 3 * (uint64_t)ctx->opt.max_relaunch;
    ctx->calls += 1;
    ctx->tiles_initial += (uint64_t)ntiles;
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
    if (flags & ~1) return fail(ctx, IWPP_EINVAL, "unknown flags 0x%x", flags);
    if (sq == nn) return fail(ctx, IWPP_EINVAL, "sqdist and nearest must be distinct buffers");
    return IWPP_OK;
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
    return d;
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
    ctx->opt.sweeps = 2;
    ctx->opt.queue_factor = 32;
    ctx->opt.spill_cap = 8192;
    ctx->opt.max_relaunch = 1;
    ctx->opt.timeout_ms = 10000;
    ctx->opt.revisit_sweep_min = 0;
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
    if (ctx->ws) cudaFree(ctx->ws);
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
    if (o->tile != 0 && o->tile != TILE) return fail(ctx, IWPP_EINVAL, "tile must be 0 (auto) or %d", TILE);
    if (o->blocks_per_sm < 0 || o->sweeps < 0 || o->sweeps > 64 || o->queue_factor < 1 || o->queue_factor > 4096 ||
        o->spill_cap < 0 || o->spill_cap > (1 << 20) || o->max_relaunch < 0 || o->max_relaunch > 64 ||
        o->timeout_ms < 1 || o->timeout_ms > 600000 || o->timing < 0 || o->timing > 1 ||
        o->revisit_sweep_min < 0)
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

static int jobs_from(iwpp_ctx *ctx, int n, const iwpp_job *js, std::vector<JobDesc> &jobs) {
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

int iwpp_sync(iwpp_ctx *ctx, void *stream) {
    if (!ctx) return IWPP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st), "status readback");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    for (auto &ev : ctx->pending_events) {
        float ms = 0.f;
        CK(cudaEventSynchronize(ev.second), "cudaEventSynchronize");
        CK(cudaEventElapsedTime(&ms, ev.first, ev.second), "cudaEventElapsedTime");
        ctx->kernel_ns += (uint64_t)((double)ms * 1e6);
        ctx->free_events.push_back(ev);
    }
    ctx->pending_events.clear();
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
    out->kernel_launches = ctx->launches;
    out->kernel_ns = ctx->kernel_ns;
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
    CK(cudaMemcpy(ctx->ctl, &c, sizeof c, cudaMemcpyHostToDevice), "stats reset");
    ctx->calls = 0;
    ctx->tiles_initial = 0;
    ctx->launches = 0;
    ctx->kernel_ns = 0;
    return IWPP_OK;
}

}  // extern "C"
