// iwpp_noalloc.cu -- iwpp_recon_u8_noalloc(): uint8 reconstruction for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code running inside another
// allocator's or a framework's memory accounting (a caching allocator that
// owns the whole device budget, where a side allocation would go unseen or
// fail), and real-time paths that forbid allocation after start-up because
// cudaMalloc can block and synchronise the device.  The regular entry
// points take their workspace (tile queue, tile states, spill queues,
// status block) from a context, and creating or growing a context
// allocates.  This entry point instead uses one statically sized scratch
// array compiled into the library (file scope, __device__), so it needs no
// context and performs no allocation of its own.
//
// Properties a caller must know:
//   * the scratch array (IWPP_NOALLOC_SCRATCH_BYTES) occupies device memory
//     on every GPU that loads the library, from load until process exit;
//   * every call uses the same array and it keeps the last call's contents
//     (each call clears its status block and refills its queue first): two
//     calls whose GPU work overlaps (different streams, or different host
//     threads on one device) race and corrupt each other's results -- order
//     them on one stream;
//   * the first call on a device resolves the array's device address with
//     cudaGetSymbolAddress;
//   * images larger than the array supports are rejected with IWPP_EINVAL
//     (no more than IWPP_NOALLOC_MAX_TILES tiles of 64x64 pixels);
//   * the call is synchronous: it returns after the work on `stream` has
//     finished and its outcome word has been read back.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/iwpp.h"
#include "iwpp_internal.h"

using namespace iwpp;

namespace {

constexpr int kMaxTiles = IWPP_NOALLOC_MAX_TILES;     // 16384^2 pixels in 64x64 tiles
constexpr int kQueueFactor = 16;                      // tile-queue slots per tile
constexpr int kMaxGrid = 2048;                        // persistent CTAs at most
constexpr int kSpillCap = 512;                        // spill entries per CTA and buffer
constexpr int kMaxRelaunch = 4;

// byte layout of the scratch array
constexpr size_t kCtl = 0;                                            // Control
constexpr size_t kCnt = 256;                                          // head, tail, pending
constexpr size_t kState = 512;                                        // int[kMaxTiles]
constexpr size_t kVisited = kState + sizeof(int) * kMaxTiles;         // int[kMaxTiles]
constexpr size_t kSlots = kVisited + sizeof(int) * kMaxTiles;         // int[kQueueFactor*kMaxTiles]
constexpr size_t kSpill = kSlots + sizeof(int) * kQueueFactor * (size_t)kMaxTiles;  // u16[kMaxGrid*2*kSpillCap]
constexpr size_t kEnd = kSpill + sizeof(uint16_t) * 2 * kSpillCap * (size_t)kMaxGrid;
static_assert(kEnd <= IWPP_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");
static_assert(sizeof(Control) <= kCnt - kCtl, "Control block");

// The scratch: one copy per device, alive while the library is loaded.
static __device__ __align__(256) unsigned char g_scratch[IWPP_NOALLOC_SCRATCH_BYTES];

struct DeviceSlot {
    unsigned char *base = nullptr;  // device address of g_scratch on this device
    int sm_count = 0;
    int occupancy = 0;
};

std::mutex g_mutex;
DeviceSlot g_slots[64];

// Resolves (once per device, with that device current) the scratch address
// and the launch geometry.  Returns a CUDA error code.
cudaError_t setup_device(int dev, DeviceSlot **out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSlot &s = g_slots[dev];
    if (!s.base) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&s.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = family_occupancy(FAM_RECON_U8, &s.occupancy);
        if (e != cudaSuccess) return e;
        if (s.occupancy < 1) return cudaErrorInvalidConfiguration;
        s.base = (unsigned char *)p;
    }
    *out = &s;
    return cudaSuccess;
}

}  // namespace

extern "C" int iwpp_recon_u8_noalloc(const uint8_t *marker, int64_t marker_pitch, const uint8_t *mask,
                                     int64_t mask_pitch, uint8_t *out, int64_t out_pitch, int h, int w,
                                     int conn, void *stream) {
    if (!marker || !mask || !out || h < 1 || w < 1 || (conn != 4 && conn != 8)) return IWPP_EINVAL;
    if (marker_pitch < w || mask_pitch < w || out_pitch < w) return IWPP_EINVAL;
    const int64_t tiles_x = (w + TILE - 1) / TILE, tiles_y = (h + TILE - 1) / TILE;
    if (tiles_x * tiles_y > kMaxTiles) return IWPP_EINVAL;  // beyond the scratch array
    // byte ranges [first, last) of the three images: out may be the marker
    // exactly (in place) but must not touch the mask at all
    const uint8_t *out_end = out + (int64_t)(h - 1) * out_pitch + w;
    const uint8_t *mask_end = mask + (int64_t)(h - 1) * mask_pitch + w;
    const uint8_t *marker_end = marker + (int64_t)(h - 1) * marker_pitch + w;
    if (out < mask_end && mask < out_end) return IWPP_EINVAL;
    if (out != marker && out < marker_end && marker < out_end) return IWPP_EINVAL;
    if (out == marker && out_pitch != marker_pitch) return IWPP_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return IWPP_ECUDA;
    DeviceSlot *slot = nullptr;
    if (setup_device(dev, &slot) != cudaSuccess) return IWPP_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;

    // the job: one uint8 reconstruction, plain (non-TMA) staging
    KArgs ka;
    memset(&ka, 0, sizeof ka);
    JobDesc &d = ka.job0;
    d.op = OP_RECON;
    d.dtype = DT_U8;
    d.conn = conn;
    d.h = h;
    d.w = w;
    d.tiles_x = (int)tiles_x;
    d.tiles_y = (int)tiles_y;
    d.tile_base = 0;
    d.use_tma = 0;
    d.a = marker;
    d.b = mask;
    d.out = out;
    d.pa = marker_pitch;
    d.pb = mask_pitch;
    d.po = out_pitch;
    int64_t start = 0;
    for (int c = 0; c < 4; ++c) {  // first slot of each tile colour class
        const int a = c & 1, b = c >> 1;
        d.color_base[c] = (int)start;
        start += ((tiles_x - a + 1) / 2) * ((tiles_y - b + 1) / 2);
    }
    const int ntiles = (int)(tiles_x * tiles_y);
    unsigned char *base = slot->base;
    ka.njobs = 1;
    ka.ntiles = ntiles;
    ka.tq.slots = (int *)(base + kSlots);
    ka.tq.head = (unsigned *)(base + kCnt);
    ka.tq.tail = (unsigned *)(base + kCnt + 4);
    ka.tq.pending = (int *)(base + kCnt + 8);
    ka.tq.state = (int *)(base + kState);
    ka.tq.visited = (int *)(base + kVisited);
    ka.tq.cap = (unsigned)(kQueueFactor * ntiles);
    ka.tq.ntiles = ntiles;
    ka.ctl = (Control *)(base + kCtl);
    ka.spill = (uint16_t *)(base + kSpill);
    ka.spill_cap = kSpillCap;
    ka.sweeps = 3;
    ka.revisit_sweeps = 3;
    ka.revisit_sweep_min = 0;
    // a device-side wait gives up after 10 s without progress (a long call
    // that keeps making progress is not cut off)
    ka.timeout_ns = 10000000000ull;
    int grid = slot->occupancy * slot->sm_count;
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid > ntiles) grid = ntiles;

    // The array keeps the previous call's contents: the status block must
    // start at zero; the fill kernel initialises the queue, states and flags.
    if (cudaMemsetAsync(base + kCtl, 0, sizeof(Control), st) != cudaSuccess) return IWPP_ECUDA;
    if (launch_init(ka, 1, st) != cudaSuccess) return IWPP_ECUDA;
    if (launch_persistent(ka, FAM_RECON_U8, grid, st) != cudaSuccess) return IWPP_ECUDA;
    for (int k = 0; k < kMaxRelaunch; ++k) {
        if (launch_decide(ka, 0, st) != cudaSuccess || launch_reset(ka, st) != cudaSuccess ||
            launch_persistent(ka, FAM_RECON_U8, grid, st) != cudaSuccess)
            return IWPP_ECUDA;
    }
    if (launch_decide(ka, 1, st) != cudaSuccess) return IWPP_ECUDA;

    // synchronous: read the outcome word of this call
    int errors = 0;
    if (cudaMemcpyAsync(&errors, base + kCtl + offsetof(Control, errors), sizeof(int), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return IWPP_ECUDA;
    if (errors & ST_TIMEOUT) return IWPP_ETIMEOUT;
    if (errors & ST_OVERFLOW) return IWPP_EOVERFLOW;
    return IWPP_OK;
}
