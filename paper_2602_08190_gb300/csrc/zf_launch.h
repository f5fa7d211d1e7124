// zf_launch.h -- host-side launch descriptions of the decode kernels.
#pragma once
#include <cuda_runtime.h>

#include "zf_internal.h"

namespace zf {

// Words of one decode stream's work queue: [0] next job, [1] CTAs done,
// [2, 2 + kAffinitySms) blocks taken from each SM's range (string-dictionary
// launches), zero between launches.
constexpr uint32_t kAffinitySms = 256;
constexpr uint32_t kQueueWords = 2 + kAffinitySms + 6;

struct TileLaunch {
    const ZfDevChunk* chunks;   // device descriptors of this launch
    uint32_t nchunks;
    uint32_t ntiles;            // warp jobs
    int scheme, dtype;          // -1, -1 for the batched work-queue kernel
    uint32_t tile_rows;         // rows per warp job
    uint32_t threads;
    uint32_t ctas_per_sm;       // 0 = occupancy limit
    uint32_t smem;              // dynamic shared memory: threads/32 slices of equal size
    int num_sms;
    uint32_t* err;
    uint32_t* queue;            // kQueueWords zeroed words owned by the launching stream
};

uint32_t warp_smem_bytes(int scheme, int dtype, uint32_t bmax);
cudaError_t launch_tiles(const TileLaunch& L, cudaStream_t s);
cudaError_t launch_lz(const ZfDevChunk* chunks, uint32_t n, uint32_t* err, int num_sms, cudaStream_t s);
// ANS chunks: njobs warp jobs of up to 32 streams (chunk descriptors carry tile0 in jobs).
cudaError_t launch_ans(const ZfDevChunk* chunks, uint32_t nchunks, uint32_t njobs, uint32_t* err, cudaStream_t s);

}  // namespace zf
