// iwpp_device.cuh -- device-side building blocks shared by the
// reconstruction and distance-transform kernels of libiwpp:
//
//   * the tile work queue that drives the persistent kernels (the tile-level
//     form of the wavefront loop of Algorithm 1 / Algorithm 4: a tile is
//     re-queued whenever a neighbour can still propagate into it);
//   * the pixel queue used inside one tile: per-warp staging queues filled
//     by warp-aggregated ballot/popc (the "per-thread queue" level of
//     Section 3.2, one level per warp here), a per-block shared-memory queue
//     (BQ) and a per-CTA global spill queue (GBQ) with drop-and-rescan on
//     overflow (Section 3.2: excess items are dropped and the propagation is
//     restarted from the partial result, which yields the same result);
//   * bounded waits (every spin has a deadline on %globaltimer).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace iwpp {

// ---------------------------------------------------------------- status

enum : int {
    ST_OVERFLOW = 1,  // a tile could not be queued: relaunch needed
    ST_TIMEOUT = 2,   // a bounded wait gave up
};

// Device-resident control block of one launch sequence.
struct Control {
    int status;             // ST_* bits of the current attempt
    int sticky;             // ST_* bits accumulated over attempts (timeouts)
    int done;               // 1 once an attempt finished (or failed for good)
    int want_reset;         // set by the decide step: refill the tile queue
    int errors;             // ST_* outcomes of finished calls since the last host sync
    int pad_[3];
    unsigned long long tiles_processed;
    unsigned long long seeds;
    unsigned long long pushes;
    unsigned long long spills;
    unsigned long long rescans;
    unsigned long long relaunches;
    unsigned long long rounds;
    unsigned long long wait_ns;   // summed time CTAs waited for a tile
    unsigned long long visit_ns;  // summed time CTAs spent visiting tiles
    unsigned long long phase_ns[4];  // visit phases: stage, sweep+seed, queue, store+border
    unsigned long long sweep_sets;   // sweep sets run, summed over visits
    unsigned long long revisits;     // visits of tiles visited before
};

// Tile queue: a linear array of `cap` slots filled once each.  Tickets
// (head) and reservations (tail) only grow; a launch can process at most
// `cap` tile visits, after which enqueues fail, ST_OVERFLOW is raised and
// the host-enqueued relaunch starts again from the current (partial,
// still valid) result with every tile queued.
//
// Each tile has a state word so that no two CTAs ever visit the same tile
// at once (a second visit could store values computed from older data over
// newer ones):
//   IDLE -> QUEUED        a neighbour asks for a visit (slot reserved)
//   QUEUED -> BUSY        a CTA claims the slot
//   BUSY -> BUSY_DIRTY    a neighbour asks for a visit during the visit
//   BUSY -> IDLE          visit finished, nobody asked
//   BUSY_DIRTY -> QUEUED  visit finished, re-queued (new slot)
enum : int { TS_IDLE = 0, TS_QUEUED = 1, TS_BUSY = 2, TS_BUSY_DIRTY = 3 };

struct TileQueue {
    int *slots;             // cap entries, -1 until written
    unsigned int *head;     // next ticket
    unsigned int *tail;     // next reservation
    int *pending;           // tiles queued or being visited
    int *state;             // per tile: TS_* above
    int *visited;           // per tile: 1 once its result was stored
    unsigned int cap;
    int ntiles;
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile(const int *p) {
    return *(const volatile int *)p;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Claims the next tile (called by ONE thread).  Returns the tile id, or -1
// when the whole launch is finished (nothing queued or in process), the
// ticket lies beyond the queue capacity, or the wait saw no progress for
// `timeout_ns` (then ST_TIMEOUT is raised).  The bound is on a wait without
// progress, not on the work: while other CTAs finish visits or queue tiles
// (the pending count or the reservation counter moves), the wait goes on.
__device__ inline int tq_claim(const TileQueue &q, Control *ctl, unsigned long long timeout_ns) {
    unsigned int h = atomicAdd(q.head, 1u);
    if (h >= q.cap) return -1;
    unsigned int ns = 32;
    unsigned long long last = globaltimer_ns();
    int seen_pending = ld_volatile(q.pending);
    unsigned int seen_tail = *(volatile unsigned int *)q.tail;
    while (true) {
        int t = ld_acquire(q.slots + h);
        if (t >= 0) {
            atomicExch(q.state + t, TS_BUSY);
            __threadfence();
            return t;
        }
        const int pend = ld_volatile(q.pending);
        if (pend == 0) return -1;
        const unsigned int tail = *(volatile unsigned int *)q.tail;
        const unsigned long long now = globaltimer_ns();
        if (pend != seen_pending || tail != seen_tail) {
            seen_pending = pend;
            seen_tail = tail;
            last = now;
        } else if (now - last > timeout_ns) {
            atomicOr(&ctl->status, ST_TIMEOUT);
            atomicOr(&ctl->sticky, ST_TIMEOUT);
            return -1;
        }
        __nanosleep(ns);
        if (ns < 1024) ns *= 2;
    }
}

// Reserves a slot for tile t, whose state the caller has just set to
// TS_QUEUED.  On overflow the tile goes back to TS_IDLE (the relaunch
// queues every tile again).
__device__ inline void tq_enqueue(const TileQueue &q, Control *ctl, int t) {
    atomicAdd(q.pending, 1);
    unsigned int r = atomicAdd(q.tail, 1u);
    if (r < q.cap) {
        st_release(q.slots + r, t);
    } else {
        atomicExch(q.state + t, TS_IDLE);
        atomicOr(&ctl->status, ST_OVERFLOW);
        atomicSub(q.pending, 1);
    }
}

// Asks for a visit of tile t (called by one thread, after a __threadfence
// that publishes the caller's stores).
__device__ inline void tq_push(const TileQueue &q, Control *ctl, int t) {
    int s = ld_volatile(q.state + t);
    while (true) {
        if (s == TS_QUEUED || s == TS_BUSY_DIRTY) return;
        const int want = (s == TS_IDLE) ? TS_QUEUED : TS_BUSY_DIRTY;
        const int old = atomicCAS(q.state + t, s, want);
        if (old == s) {
            if (want == TS_QUEUED) tq_enqueue(q, ctl, t);
            return;
        }
        s = old;
    }
}

// Ends the visit of tile t (one thread, after the tile's stores and its
// neighbour pushes); re-queues it if a neighbour asked meanwhile.
__device__ inline void tq_finish(const TileQueue &q, Control *ctl, int t) {
    __threadfence();
    const int old = atomicCAS(q.state + t, TS_BUSY, TS_IDLE);
    if (old == TS_BUSY_DIRTY) {
        atomicExch(q.state + t, TS_QUEUED);
        tq_enqueue(q, ctl, t);
    }
}

}  // namespace iwpp
