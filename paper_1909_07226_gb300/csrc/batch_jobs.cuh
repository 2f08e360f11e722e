// Job table of the batched form: the geometry and device buffers of one job
// (one plan), read by the persistent batch kernels through (job, subgrid) work
// items, and on the host the arguments of the tensor-core kernels' per-job launches.
#pragma once

#include <cuda_runtime.h>

#include "idg_internal.h"

namespace idg {

struct JobDev {
    Geometry g;
    const float4 *vis;
    float4 *vis_out;
    const uint8_t *flags;
    const float4 *aterms;
    const float *taper;
    float4 *grid;
};

// sets the shared-memory size of the fused tensor-core kernels the batches launch (once,
// before any graph capture)
cudaError_t prepare_tcw_batch_kernels();
cudaError_t prepare_gridder_tcw_batch();
cudaError_t prepare_sep_batch_kernels();
cudaError_t prepare_gridder_sep_batch();

}  // namespace idg
