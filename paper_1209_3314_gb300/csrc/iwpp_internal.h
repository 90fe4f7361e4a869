// iwpp_internal.h -- types shared by the kernels (iwpp_kernels.cu) and the
// host side of the C ABI (iwpp_api.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "iwpp_device.cuh"

namespace iwpp {

// OP_WS_DIST / OP_WS_LABEL: the plateau-distance and label propagations of
// the watershed from markers (min-propagations along per-pixel in-edge masks)
// OP_EDT_WIDE: the distance transform's second wavefront with the wide window
enum : int { OP_RECON = 0, OP_EDT = 1, OP_GDT = 2, OP_WS_DIST = 3, OP_WS_LABEL = 4, OP_EDT_WIDE = 5 };
enum : int { DT_U8 = 0, DT_I32 = 1 };

// kernel families (one persistent-kernel instantiation each)
enum : int { FAM_RECON_U8 = 0, FAM_RECON_I32 = 1, FAM_EDT = 2, FAM_MIXED = 3, FAM_GDT = 4, FAM_WS = 5, FAM_COUNT = 6 };

constexpr int TILE = 64;  // tile side in pixels

// The 8-neighbour order of the kernels: neighbour k of p is p + (nb8_dy(k),
// nb8_dx(k)) = (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1); 7 - k
// is the mirror of k.  Bit k of a watershed in-edge mask says that
// neighbour k may lower the pixel.
__host__ __device__ constexpr int nb8_dy(int k) { return k < 3 ? -1 : (k < 5 ? 0 : 1); }
__host__ __device__ constexpr int nb8_dx(int k) {
    return (k == 0 || k == 3 || k == 5) ? -1 : ((k == 2 || k == 4 || k == 7) ? 1 : 0);
}
constexpr int WS_DINF = 0x3FFFFFFF;  // plateau distance of a pixel not reached (yet)

// One image job inside a launch.  Tiles of job j have global ids
// [tile_base, tile_base + tiles_x * tiles_y).
struct alignas(64) JobDesc {
    CUtensorMap tm[3];   // TMA maps: a, b, out/nearest (valid when use_tma); the
                         // wide-window pass keeps its nearest box map in tm[1]
    int op, dtype, conn, flags;
    int h, w, tiles_x, tiles_y;
    int tile_base;
    int use_tma;
    int color_base[4];   // first initial-queue slot of each tile colour class
    const void *a;       // recon: marker      edt: binary
    const void *b;       // recon: mask
    void *out;           // recon: result
    int32_t *sqdist;     // edt outputs (dense, pitch w)
    int32_t *nearest;
    int64_t pa, pb, po;  // pitches in elements
    // n / w for 0 <= n < 2^31 as (n * wdiv_m) >> wdiv_s (distance transform:
    // linear feature index -> row)
    unsigned long long wdiv_m;
    int wdiv_s;
};

struct alignas(64) KArgs {
    JobDesc job0;         // the job when njobs == 1
    const JobDesc *jobs;  // device array when njobs > 1
    int njobs;
    int ntiles;
    TileQueue tq;
    Control *ctl;
    uint16_t *spill;      // per CTA: 2 * spill_cap entries
    int spill_cap;
    int sweeps;           // raster + anti-raster sweep sets per bulk visit
    int revisit_sweep_min;  // later visits sweep when more halo seeds than this
    int edt_sweeps;       // the same two settings for the distance transform
    int edt_revisit_sweep_min;
    int revisit_sweeps;   // reconstruction: sweep sets on a later visit
    int queue_mode;       // queue ablation: bit 0 per-thread atomics, bit 1 global-only
    int test_empty_slot;  // timeout-path tests: initial queue slot 0 left unfilled
    int gdt_sweeps;       // shortest paths: sweep sets per bulk visit
    int gdt_revisit_sweep_min;  // and their later visits' sweep threshold
    int ws_sweeps;        // watershed propagations: sweep sets per bulk visit
    int ws_revisit_sweep_min;  // and their later visits' sweep threshold
    int wide_u[7];        // wide-window distance transform: the window's half-width is 1 + the
                          // number of these squared-distance thresholds a pixel reaches (1..8)
    unsigned long long timeout_ns;
};

// Exact separable distance transform (iwpp_edt_exact.cu).
struct ExactArgs {
    const uint8_t *bin;
    int64_t pitch;        // binary image pitch in bytes
    int h, w, flags, nb;  // nb: bands of the column pass
    int32_t *first, *last, *above, *below;  // nb x w band summaries
    int32_t *G;           // h x w scratch: row of the nearest feature in the pixel's column
    int32_t *sqdist, *nearest;
};
int exact_bands(int h);
cudaError_t launch_edt_exact(const ExactArgs &a, cudaStream_t s);

// Watershed from markers, per-pixel steps (iwpp_watershed.cu).  Planes are
// dense (pitch w): A and B of the relief's type, E uint8, D and labels int32.
struct WsArgs {
    const void *relief;   // u8 or i32, pitch `pf` elements
    const int32_t *markers;
    int64_t pf, pm;       // pitches in elements
    int h, w, dtype;      // DT_U8 / DT_I32
    void *A, *B;          // complemented marker / mask; A holds the complemented levels after the reconstruction
    uint8_t *E;           // in-edge masks
    int32_t *D;           // plateau distances
    int32_t *labels;
    void *levels;         // optional flooding-level output (relief's type)
};
cudaError_t launch_ws_complement(const WsArgs &a, cudaStream_t s);
cudaError_t launch_ws_plateau_init(const WsArgs &a, cudaStream_t s);
cudaError_t launch_ws_label_init(const WsArgs &a, cudaStream_t s);
cudaError_t launch_ws_label_finish(const WsArgs &a, cudaStream_t s);

// Influence zones / SKIZ, per-pixel steps (iwpp_skiz.cu).  Planes are dense
// (pitch w).
struct SkizArgs {
    const uint8_t *mask;    // free where != 0, pitch `pmask`
    const int32_t *labels;  // sources where free and != 0, pitch `pl`
    int64_t pmask, pl;
    int h, w;
    uint8_t *seeds;         // labels != 0
    int32_t *dist;          // shortest-path distances (INT_MAX: obstacle / unreached)
    uint8_t *E;             // in-edge masks
    int32_t *zones;         // least label (INT_MAX while none)
    int32_t *neg;           // least negated label
    uint8_t *skiz;          // optional
};
cudaError_t launch_skiz_prep(const SkizArgs &a, cudaStream_t s);
cudaError_t launch_skiz_label_init(const SkizArgs &a, cudaStream_t s);
cudaError_t launch_skiz_finish(const SkizArgs &a, cudaStream_t s);

}  // namespace iwpp

struct iwpp_ctx;

namespace iwpp {

// Device memory a context holds (workspace, planes, control block), now and
// after it has run one batch of n reconstruction / distance-transform jobs
// of the given ops (IWPP_OP_*), dtypes (IWPP_U8 / IWPP_I32) and shapes --
// which may grow its workspace (iwpp_api.cu; the server's admission counts
// it).
size_t ctx_device_bytes(const iwpp_ctx *ctx);
int ctx_device_bytes_after(iwpp_ctx *ctx, int n, const int *op, const int *dtype, const int *h, const int *w,
                           size_t *bytes);

// Launch helpers implemented in iwpp_kernels.cu.
int family_threads(int fam);
int family_smem(int fam);
cudaError_t family_occupancy(int fam, int *blocks_per_sm);
cudaError_t launch_init(const KArgs &ka, int first_attempt, cudaStream_t s);
cudaError_t launch_persistent(const KArgs &ka, int fam, int grid, cudaStream_t s);
cudaError_t launch_decide(const KArgs &ka, int final_step, cudaStream_t s);
cudaError_t launch_reset(const KArgs &ka, cudaStream_t s);

}  // namespace iwpp
