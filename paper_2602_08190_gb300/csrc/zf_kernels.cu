// zf_kernels.cu -- decode kernels and their launchers.
//
//   tiles_kernel<SCHEME, DT, THREADS>  one (scheme, dtype) per launch; a
//       persistent grid strides over the tiles of all chunks in the launch.
//   tiles_kernel<-1, -1, THREADS>     the batched kernel: tiles of chunks of
//       any scheme and dtype, handed out by an atomic work queue; the last
//       CTA to finish resets the queue so the launch can be replayed from a
//       CUDA graph.
// The LZ77 kernel (Non-Parallel pattern) is in zf_lz.cu.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "zf_device.cuh"
#include "zf_launch.h"
#include "zf_strdict.cuh"

namespace {

struct LaunchArgs {
    const ZfDevChunk* chunks;
    uint32_t nchunks;
    uint32_t njobs;        // warp jobs in the launch
    uint32_t job_rows;     // rows of one warp job (a multiple of 1024)
    uint32_t warp_smem;    // bytes of shared memory per warp
    uint32_t* err;
    uint32_t* queue;       // [0] next job, [1] CTAs done, [2 + s] blocks taken near SM s (zf::kQueueWords)
    uint32_t nsm;          // SMs of the device (string-dictionary launches: SM ranges, at most kAffinitySms)
};

// The block of a string-dictionary launch this CTA decodes.  The launch's
// blocks are cut into one contiguous range per SM, and a CTA first takes the
// next untaken block of the range of the SM it runs on, then of the ranges
// after it: consecutive blocks decode tokens of the same chunk, so the CTAs
// sharing an SM read one chunk's dictionary and keep it in that SM's L1.
// Every CTA gets a block and every block is taken once: there are as many
// blocks as CTAs, and a CTA that finds every range taken would leave fewer
// takers than blocks.  Each range counter is raised at most once per CTA, so
// the search ends after at most nsm atomics.
__device__ uint32_t claim_near_sm(uint32_t* q, uint32_t nsm) {
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const uint32_t nblk = gridDim.x, per = (nblk + nsm - 1) / nsm;
    const uint32_t s0 = smid % nsm;
    for (uint32_t i = 0; i < nsm; i++) {
        const uint32_t s = s0 + i < nsm ? s0 + i : s0 + i - nsm;
        const uint64_t lo64 = (uint64_t)s * per;
        if (lo64 >= nblk) continue;
        const uint32_t lo = (uint32_t)lo64, cnt = min(per, nblk - lo);
        if (*reinterpret_cast<volatile uint32_t*>(q + 2 + s) >= cnt) continue;
        const uint32_t j = atomicAdd(q + 2 + s, 1u);
        if (j < cnt) return lo + j;
    }
    return blockIdx.x;   // not reached (see above)
}

__device__ __forceinline__ uint32_t find_chunk(const ZfDevChunk* ch, uint32_t n, uint32_t job) {
    uint32_t a = 0, z = n;
    while (z - a > 1) {
        uint32_t mid = (a + z) >> 1;
        if (__ldg(&ch[mid].tile0) <= job) a = mid;
        else z = mid;
    }
    return a;
}

// WS: 256-bit stores (single-scheme kernels only).
template <int SCHEME, int DT, bool WS>
__device__ __forceinline__ void decode_one(const ZfDevChunk& c, const zfd::Hdr& h, uint32_t r0, uint32_t nrows,
                                           uint32_t* wsm, uint32_t* err) {
    if constexpr (DT == ZF_I32 || DT == ZF_I64) {
        using T = typename std::conditional<DT == ZF_I64, int64_t, int32_t>::type;
        if constexpr (SCHEME == ZF_FOR_BP || SCHEME == ZF_DICT_BP || SCHEME == ZF_RAW)
            zfd::fp_job<T, SCHEME>(c, h, r0, nrows, wsm, err);
        else if constexpr (SCHEME == ZF_DELTA_BP)
            zfd::delta_job<T, WS>(c, h, r0, nrows, wsm, err, c.bmax);
        else if constexpr (SCHEME == ZF_RLE)
            zfd::rle_job<T, WS>(c, h, r0, nrows, wsm, err);
    } else if constexpr (DT == ZF_F64) {
        // doubles travel as their 64-bit patterns
        if constexpr (SCHEME == ZF_RAW || SCHEME == ZF_FLOAT2INT) zfd::fp_job<int64_t, SCHEME>(c, h, r0, nrows, wsm, err);
    } else if constexpr (DT == ZF_BYTES && SCHEME == ZF_STRDICT) {
        zfd::strdict_job(c, h, r0, nrows, wsm, err);   // r0, nrows count tokens
    } else if constexpr (DT == ZF_BYTES && SCHEME == ZF_RAW) {
        // raw bytes: 16-byte copies
        const uint32_t lane = threadIdx.x & 31;
        const uint8_t* src = c.blob + h.off[0] + r0;
        uint8_t* dst = c.dst + r0;
        for (uint32_t i0 = lane * 16; i0 < nrows; i0 += 512) {
            if (i0 + 16 <= nrows) reinterpret_cast<uint4*>(dst + i0)[0] = zfd::ldg16(src + i0);
            else
                for (uint32_t i = i0; i < nrows; i++) dst[i] = src[i];
        }
    }
}

__device__ __forceinline__ void decode_mixed(const ZfDevChunk& c, const zfd::Hdr& h, uint32_t r0, uint32_t nrows,
                                             uint32_t* wsm, uint32_t* err) {
    switch (c.scheme * 4 + c.dtype) {
#define ZF_CASE(S, D) \
    case S * 4 + D: decode_one<S, D, true>(c, h, r0, nrows, wsm, err); break;
        ZF_CASE(ZF_RAW, ZF_I32) ZF_CASE(ZF_RAW, ZF_I64) ZF_CASE(ZF_RAW, ZF_BYTES)
        ZF_CASE(ZF_FOR_BP, ZF_I32) ZF_CASE(ZF_FOR_BP, ZF_I64)
        ZF_CASE(ZF_DICT_BP, ZF_I32) ZF_CASE(ZF_DICT_BP, ZF_I64)
        ZF_CASE(ZF_DELTA_BP, ZF_I32) ZF_CASE(ZF_DELTA_BP, ZF_I64)
        ZF_CASE(ZF_RLE, ZF_I32) ZF_CASE(ZF_RLE, ZF_I64)
        ZF_CASE(ZF_RAW, ZF_F64) ZF_CASE(ZF_FLOAT2INT, ZF_F64) ZF_CASE(ZF_STRDICT, ZF_BYTES)
#undef ZF_CASE
    default:
        if ((threadIdx.x & 31) == 0) zfd::report(err, ZF_EINVAL, c.chunk_id);
    }
}

// One warp job of a chunk: job_rows consecutive rows (the last job of a
// chunk may be shorter).
template <int SCHEME, int DT>
__device__ __forceinline__ void run_job(const LaunchArgs& a, uint32_t job, uint32_t* wsm) {
    const uint32_t k = find_chunk(a.chunks, a.nchunks, job);
    const ZfDevChunk c = a.chunks[k];
    zfd::Hdr h;
    zfd::load_hdr(c.blob, h);
    const uint32_t r0 = (job - c.tile0) * a.job_rows;
    const uint32_t sz = (c.dtype == ZF_I64 || c.dtype == ZF_F64) ? 8 : c.dtype == ZF_I32 ? 4 : 1;
    if (h.rows != c.rows || r0 >= c.rows || (uint64_t)c.rows * sz > c.dst_cap) {
        if ((threadIdx.x & 31) == 0) zfd::report(a.err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t nrows = min(a.job_rows, c.rows - r0);
    if constexpr (SCHEME < 0) decode_mixed(c, h, r0, nrows, wsm, a.err);
    else decode_one<SCHEME, DT, true>(c, h, r0, nrows, wsm, a.err);
}

// Specialized launches (one scheme and dtype): one warp job per warp, as
// many CTAs as jobs need.  The batched launch (SCHEME < 0) is persistent: its
// CTAs pop one job per warp from a work queue that the last CTA resets, so
// the launch can be replayed from a CUDA graph.
// At least 32 resident warps per SM: registers are capped at 64 per thread.
template <int SCHEME, int DT, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) tiles_kernel(LaunchArgs a) {
    extern __shared__ uint4 smem4[];
    constexpr uint32_t NW = THREADS / 32;
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t* wsm = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(smem4) + warp * a.warp_smem);
    if constexpr (SCHEME == ZF_STRDICT) {
        __shared__ uint32_t s_blk;
        if (threadIdx.x == 0) s_blk = a.queue ? claim_near_sm(a.queue, a.nsm) : blockIdx.x;
        __syncthreads();
        const uint32_t job = s_blk * NW + warp;
        if (job < a.njobs) run_job<SCHEME, DT>(a, job, wsm);
        if (a.queue) {
            // the last CTA to finish clears the range counters for the next launch on this queue
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                if (atomicAdd(&a.queue[1], 1u) == gridDim.x - 1) {
                    for (uint32_t s = 0; s < a.nsm; s++) a.queue[2 + s] = 0;
                    a.queue[1] = 0;
                    __threadfence();
                }
            }
        }
    } else if constexpr (SCHEME >= 0) {
        const uint32_t job = blockIdx.x * NW + warp;
        if (job < a.njobs) run_job<SCHEME, DT>(a, job, wsm);
    } else {
        __shared__ uint32_t s_job;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) s_job = atomicAdd(&a.queue[0], NW);
            __syncthreads();
            const uint32_t base = s_job;
            if (base >= a.njobs) break;
            if (base + warp < a.njobs) run_job<SCHEME, DT>(a, base + warp, wsm);
        }
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&a.queue[1], 1u) == gridDim.x - 1) {
                a.queue[0] = 0;
                a.queue[1] = 0;
                __threadfence();
            }
        }
    }
}

// ---------------------------------------------------------------- launch table
typedef void (*KernelFn)(LaunchArgs);

template <int THREADS>
KernelFn pick(int scheme, int dtype) {
    switch (scheme * 4 + dtype) {
#define ZF_K(S, D) \
    case S * 4 + D: return tiles_kernel<S, D, THREADS>;
        ZF_K(ZF_RAW, ZF_I32) ZF_K(ZF_RAW, ZF_I64) ZF_K(ZF_RAW, ZF_BYTES)
        ZF_K(ZF_FOR_BP, ZF_I32) ZF_K(ZF_FOR_BP, ZF_I64)
        ZF_K(ZF_DICT_BP, ZF_I32) ZF_K(ZF_DICT_BP, ZF_I64)
        ZF_K(ZF_DELTA_BP, ZF_I32) ZF_K(ZF_DELTA_BP, ZF_I64)
        ZF_K(ZF_RLE, ZF_I32) ZF_K(ZF_RLE, ZF_I64)
        ZF_K(ZF_RAW, ZF_F64) ZF_K(ZF_FLOAT2INT, ZF_F64) ZF_K(ZF_STRDICT, ZF_BYTES)
#undef ZF_K
    }
    if (scheme < 0) return tiles_kernel<-1, -1, THREADS>;
    return nullptr;
}

struct OccKey {
    KernelFn fn;
    uint32_t smem, threads;
    bool operator==(const OccKey& o) const { return fn == o.fn && smem == o.smem && threads == o.threads; }
};
struct OccHash {
    size_t operator()(const OccKey& k) const {
        return std::hash<void*>()((void*)k.fn) ^ (k.smem * 2654435761u) ^ (k.threads * 40503u);
    }
};
std::mutex g_occ_mu;
std::unordered_map<OccKey, int, OccHash> g_occ;
std::unordered_map<void*, bool> g_attr_set;

}  // namespace

namespace zf {

uint32_t warp_smem_bytes(int scheme, int dtype, uint32_t bmax) {
    return zfd::warp_smem(scheme, (dtype == ZF_I64 || dtype == ZF_F64) ? 8 : dtype == ZF_I32 ? 4 : 1, bmax);
}

cudaError_t launch_tiles(const TileLaunch& L, cudaStream_t s) {
    KernelFn fn = nullptr;
    switch (L.threads) {
    case 128: fn = pick<128>(L.scheme, L.dtype); break;
    case 256: fn = pick<256>(L.scheme, L.dtype); break;
    case 512: fn = pick<512>(L.scheme, L.dtype); break;
    default: return cudaErrorInvalidValue;
    }
    if (!fn) return cudaErrorInvalidValue;
    int per_sm = (int)L.ctas_per_sm;
    {
        std::lock_guard<std::mutex> g(g_occ_mu);
        if (!g_attr_set.count((void*)fn)) {
            // allow the largest dynamic shared memory any launch of this kernel may ask for
            int dev = 0, optin = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 optin - (int)(2 * 1024));
            if (e != cudaSuccess) return e;
            g_attr_set[(void*)fn] = true;
        }
        OccKey key{fn, L.smem, L.threads};
        auto it = g_occ.find(key);
        if (it == g_occ.end()) {
            int occ = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, (int)L.threads, L.smem);
            if (e != cudaSuccess) return e;
            it = g_occ.emplace(key, occ).first;
        }
        if (per_sm <= 0 || per_sm > it->second) per_sm = it->second;
    }
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    const uint32_t nw = L.threads / 32;
    uint64_t grid = ((uint64_t)L.ntiles + nw - 1) / nw;               // one job per warp
    if (L.scheme < 0) {                                                // persistent work-queue launch
        uint64_t resident = (uint64_t)per_sm * (uint64_t)L.num_sms;
        if (grid > resident) grid = resident;
    }
    if (grid == 0) return cudaSuccess;
    const bool affinity = L.scheme == ZF_STRDICT && L.num_sms > 0 && L.num_sms <= (int)kAffinitySms;
    LaunchArgs a{L.chunks, L.nchunks, L.ntiles, L.tile_rows, L.smem / nw, L.err,
                 (L.scheme < 0 || affinity) ? L.queue : nullptr, (uint32_t)L.num_sms};
    fn<<<(unsigned)grid, L.threads, L.smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace zf
