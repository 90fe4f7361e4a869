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
    int occupancy[2] = {0, 0};  // blocks per SM for tile 32 / 64
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

int pick_tile(const iwpp_ctx *ctx, const std::vector<JobDesc> &jobs) {
    if (ctx->opt.tile) return ctx->opt.tile;
    // autotuned rule: small images need more tiles than SMs, large ones
    // amortise the halo better with the bigger tile
    int64_t px = 0;
    for (const JobDesc &j : jobs) px += (int64_t)j.h * j.w;
    return px <= (int64_t)1536 * 1536 ? 32 : 64;
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
    const int tile = pick_tile(ctx, jobs);
    if (tile != 32 && tile != 64) return fail(ctx, IWPP_EINVAL, "tile %d unsupported", tile);
    const int64_t ntiles = layout_jobs(jobs, tile);
    if (ntiles <= 0 || ntiles > (int64_t)1 << 28) return fail(ctx, IWPP_EINVAL, "tile count %lld out of range", (long long)ntiles);
    const int64_t cap64 = std::max<int64_t>(ntiles + 1, (int64_t)ctx->opt.queue_factor * ntiles);
    if (cap64 > ((int64_t)1 << 31) - 1) return fail(ctx, IWPP_EINVAL, "tile queue too large");

    int &occ = ctx->occupancy[tile == 32 ? 0 : 1];
    if (occ == 0) {
        int r = max_blocks_per_sm(tile, &occ);
        if (r != 0) return cuda_fail(ctx, (cudaError_t)r, "occupancy query");
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
    const size_t o_spill = take((size_t)grid * 2 * std::max(1, ctx->opt.spill_cap) * 4);
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
    ka.spill = (int *)(ws + o_spill);
    ka.spill_cap = std::max(0, ctx->opt.spill_cap);
    ka.sweeps = ctx->opt.sweeps;
    ka.timeout_ns = (unsigned long long)ctx->opt.timeout_ms * 1000000ull;

    if (jobs.size() > 1)
        CK(cudaMemcpyAsync(ws + o_jobs, jobs.data(), jobs.size() * sizeof(JobDesc), cudaMemcpyHostToDevice, st),
           "job table upload");
    CK(launch_init(ka, 1, st), "launch fill_queue");
    CK(launch_persistent(ka, tile, grid, st), "launch persistent");
    for (int k = 0; k < ctx->opt.max_relaunch; ++k) {
        CK(launch_decide(ka, 0, st), "launch decide");
        CK(launch_reset(ka, st), "launch reset");
        CK(launch_persistent(ka, tile, grid, st), "launch persistent");
    }
    CK(launch_decide(ka, 1, st), "launch decide");
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
    ctx->opt.sweeps = 1;
    ctx->opt.queue_factor = 32;
    ctx->opt.spill_cap = 4096;
    ctx->opt.max_relaunch = 1;
    ctx->opt.timeout_ms = 10000;
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
    if (o->tile != 0 && o->tile != 32 && o->tile != 64) return fail(ctx, IWPP_EINVAL, "tile must be 0, 32 or 64");
    if (o->blocks_per_sm < 0 || o->sweeps < 0 || o->sweeps > 64 || o->queue_factor < 1 || o->queue_factor > 4096 ||
        o->spill_cap < 0 || o->spill_cap > (1 << 24) || o->max_relaunch < 0 || o->max_relaunch > 64 ||
        o->timeout_ms < 1 || o->timeout_ms > 600000)
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
    return IWPP_OK;
}

int iwpp_stats_reset(iwpp_ctx *ctx) {
    if (!ctx) return IWPP_EINVAL;
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    Control c;
    CK(cudaMemcpy(&c, ctx->ctl, sizeof c, cudaMemcpyDeviceToHost), "stats readback");
    c.tiles_processed = c.seeds = c.pushes = c.spills = c.rescans = c.relaunches = 0;
    CK(cudaMemcpy(ctx->ctl, &c, sizeof c, cudaMemcpyHostToDevice), "stats reset");
    ctx->calls = 0;
    ctx->tiles_initial = 0;
    return IWPP_OK;
}

}  // extern "C"
