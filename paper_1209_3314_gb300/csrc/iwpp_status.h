// iwpp_status.h -- the status readback of a context, in two halves for
// callers that order it on a stream themselves (the request server).
#pragma once

#include <cuda_runtime.h>

#include "../../include/iwpp.h"

namespace iwpp {

// Enqueues on `st` the copy of the context's status block to its pinned
// host copy.  A caller that orders it after a batch's own work reads the
// batch's status without a later device-to-host copy, which would queue
// behind other streams' transfers.
int status_readback(iwpp_ctx *ctx, cudaStream_t st);

// The status of the work the last readback followed: call once `st` has
// passed that copy (e.g. after an event recorded behind it completed).
// Clears recorded device errors (a short synchronous reset on `st`).
int status_result(iwpp_ctx *ctx, cudaStream_t st);

}  // namespace iwpp
