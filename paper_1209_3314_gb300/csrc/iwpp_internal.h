// iwpp_internal.h -- types shared by the kernels (iwpp_kernels.cu) and the
// host side of the C ABI (iwpp_api.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "iwpp_device.cuh"

namespace iwpp {

enum : int { OP_RECON = 0, OP_EDT = 1 };
enum : int { DT_U8 = 0, DT_I32 = 1 };

// One image job inside a launch.  Tiles of job j have global ids
// [tile_base, tile_base + tiles_x * tiles_y).
struct JobDesc {
    int op, dtype, conn, flags;
    int h, w, tiles_x, tiles_y;
    int tile_base;
    int color_base[4];   // first initial-queue slot of each tile colour class
    const void *a;       // recon: marker      edt: binary
    const void *b;       // recon: mask
    void *out;           // recon: result
    int32_t *sqdist;     // edt outputs (dense, pitch w)
    int32_t *nearest;
    int64_t pa, pb, po;  // pitches in elements
};

struct KArgs {
    const JobDesc *jobs;  // device array (njobs > 1) ...
    JobDesc job0;         // ... or this copy when njobs == 1
    int njobs;
    int ntiles;
    TileQueue tq;
    Control *ctl;
    int *spill;           // per CTA: 2 * spill_cap ints
    int spill_cap;
    int sweeps;
    unsigned long long timeout_ns;
};

// Launch helpers implemented in iwpp_kernels.cu.
int smem_bytes(int tile);
int max_blocks_per_sm(int tile, int *out);
cudaError_t launch_init(const KArgs &ka, int first_attempt, cudaStream_t s);
cudaError_t launch_persistent(const KArgs &ka, int tile, int grid, cudaStream_t s);
cudaError_t launch_decide(const KArgs &ka, int final_step, cudaStream_t s);
cudaError_t launch_reset(const KArgs &ka, cudaStream_t s);

}  // namespace iwpp
