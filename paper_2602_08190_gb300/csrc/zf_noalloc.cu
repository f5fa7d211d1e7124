// zf_noalloc.cu -- zf_decompress_device_noalloc: decode a compressed integer
// or float64 column that is already in device memory without allocating
// anything.
//
// Who needs it: code that must not call cudaMalloc (or any allocator) after
// start-up -- for example a query engine that reserved all device memory up
// front, a process whose memory budget is fixed by another runtime, or code
// running inside a library call that may not grow the device heap.  Such a
// caller passes its own input and output buffers; the only other memory the
// decode needs (chunk descriptors, the work-queue counters and the error
// word) lives in the fixed-size device array below, which every GPU that
// loads the library holds until the process exits.
//
// The array is shared by all calls on a device and keeps the last call's
// contents; each call rewrites what it needs (descriptors, counters, error
// word) before the decode reads it.  Calls that overlap on the GPU -- from
// several host threads or streams at once on the same device -- race on the
// array; serialize them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "zf_device.cuh"

namespace {

constexpr uint32_t kCtrlBytes = 256;
constexpr uint32_t kNoallocMaxChunks = 4096;
constexpr uint32_t kNoallocScratchBytes = kCtrlBytes + kNoallocMaxChunks * sizeof(ZfDevChunk);  // 262,400 B
constexpr uint32_t kThreads = 256;
constexpr uint32_t kTileRows = 1024 * (kThreads / 32);
constexpr int kMaxDevices = 64;

// Control block: [0] chunks, [1] tiles, [2] queue next, [3] CTAs done,
// [4] error bits, [5] first failing chunk.  Descriptors follow at kCtrlBytes.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];   // device address of g_noalloc_scratch per device (set once)
bool g_attr_set[kMaxDevices];        // shared-memory attribute of noalloc_decode set on the device

// Structural checks of one chunk blob on the device (the host path makes the
// same checks before a column is accepted).
__device__ bool chunk_ok(const uint8_t* c, uint64_t len, int scheme, int dtype, uint32_t rows) {
    if (len < 64 || (len & 15) || ((uintptr_t)c & 15)) return false;
    const uint32_t* w = reinterpret_cast<const uint32_t*>(c);
    if (w[0] != zf::kChunkMagic || c[4] != scheme || c[5] != dtype || w[2] != rows) return false;
    const uint32_t b = c[6], n_aux = w[3];
    const uint32_t* off = w + 6;
    const uint32_t* ln = w + 9;
    const int nsec = (scheme == ZF_RLE || scheme == ZF_FLOAT2INT) ? 3
                     : (scheme == ZF_DICT_BP || scheme == ZF_DELTA_BP) ? 2 : 1;
    for (int s = 0; s < nsec; s++)
        if (off[s] < 64 || (off[s] & 15) || (uint64_t)off[s] + ln[s] > len) return false;
    const uint32_t sz = dtype == ZF_I32 ? 4 : 8, wd = 8 * sz;
    switch (scheme) {
    case ZF_RAW: return ln[0] == (uint64_t)rows * sz;
    case ZF_FOR_BP: return b <= wd && ln[0] == ((uint64_t)rows * b + 7) / 8;
    case ZF_DICT_BP: {
        uint32_t bits = 0;
        for (uint32_t x = n_aux ? n_aux - 1 : 0; x; x >>= 1) bits++;
        return n_aux <= zf::kMaxDict && (!rows || n_aux) && ln[0] == (uint64_t)n_aux * sz && b == bits &&
               ln[1] == ((uint64_t)rows * b + 7) / 8;
    }
    case ZF_DELTA_BP: {
        const uint32_t nb = (rows + zf::kDeltaBlock - 1) / zf::kDeltaBlock;
        if (n_aux != nb || ln[0] != (uint64_t)nb * zf::kDeltaEntry) return false;
        for (uint32_t k = 0; k < nb; k++) {
            const uint8_t* e = c + off[0] + (uint64_t)k * zf::kDeltaEntry;
            const uint32_t po = *reinterpret_cast<const uint32_t*>(e + 16), bk = e[20];
            const uint32_t mk = min(zf::kDeltaBlock, rows - k * zf::kDeltaBlock);
            if (bk > wd || (po & 15) || (uint64_t)po + ((((uint64_t)mk * bk + 7) / 8 + 15) & ~15ull) > ln[1])
                return false;
        }
        return true;
    }
    case ZF_RLE:
        return n_aux <= rows && (!rows || n_aux) && ln[0] == (uint64_t)n_aux * sz && ln[1] == 4ull * n_aux &&
               ln[2] == 8ull * ((rows + zf::kRleDirRows - 1) / zf::kRleDirRows);
    case ZF_FLOAT2INT: {
        if (b > 64 || c[48] > zf::kF2IMaxExp || n_aux > rows || ln[0] != ((uint64_t)rows * b + 7) / 8 ||
            ln[1] != 4ull * n_aux || ln[2] != 8ull * n_aux)
            return false;
        return true;   // the order of the exception rows is checked by the whole CTA
    }
    }
    return false;
}

// One CTA: check every chunk of the column and write its descriptor into the
// scratch array, then the tile counts and a reset work queue and error word.
__global__ void noalloc_setup(const uint8_t* col, uint64_t col_bytes, uint8_t* out, uint64_t out_bytes,
                              uint32_t nch, int scheme, int dtype, uint64_t n_rows, uint32_t chunk_rows) {
    uint32_t* ctrl = reinterpret_cast<uint32_t*>(g_noalloc_scratch);
    ZfDevChunk* desc = reinterpret_cast<ZfDevChunk*>(g_noalloc_scratch + kCtrlBytes);
    __shared__ uint32_t s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const uint32_t sz = dtype == ZF_I32 ? 4 : 8;
    uint64_t expect_end = 64 + 32ull * nch;
    for (uint32_t k = threadIdx.x; k < nch; k += blockDim.x) {
        const uint8_t* d = col + 64 + 32ull * k;
        const uint64_t off = *reinterpret_cast<const uint64_t*>(d);
        const uint64_t len = *reinterpret_cast<const uint64_t*>(d + 8);
        const uint64_t row0 = *reinterpret_cast<const uint64_t*>(d + 16);
        const uint32_t rows = *reinterpret_cast<const uint32_t*>(d + 24);
        bool ok = off >= expect_end && off <= col_bytes && len <= col_bytes - off &&
                  row0 == (uint64_t)k * chunk_rows && rows == (uint32_t)min((uint64_t)chunk_rows, n_rows - row0) &&
                  chunk_ok(col + off, len, scheme, dtype, rows);
        ZfDevChunk dc{};
        dc.blob = col + off;
        dc.dst = out + row0 * sz;
        dc.dst_cap = out_bytes - row0 * sz;
        dc.rows = rows;
        dc.ntiles = (rows + kTileRows - 1) / kTileRows;
        dc.blob_bytes = (uint32_t)len;
        dc.chunk_id = k;
        dc.scheme = (uint8_t)scheme;
        dc.dtype = (uint8_t)dtype;
        desc[k] = dc;
        if (!ok) atomicOr(&s_bad, 1u);
    }
    __syncthreads();
    if (scheme == ZF_FLOAT2INT && !s_bad) {
        // Float2Int exception rows strictly increasing and inside the chunk
        // (the decoder's search over them relies on the order); the CTA's
        // threads share each chunk's rows
        bool bad = false;
        for (uint32_t k = 0; k < nch; k++) {
            const uint8_t* cb = col + *reinterpret_cast<const uint64_t*>(col + 64 + 32ull * k);
            const uint32_t* w = reinterpret_cast<const uint32_t*>(cb);
            const uint32_t rows = w[2], n_aux = w[3];
            const uint32_t* er = reinterpret_cast<const uint32_t*>(cb + w[7]);   // section 1
            for (uint32_t j = threadIdx.x; j < n_aux; j += blockDim.x)
                bad |= er[j] >= rows || (j && er[j] <= er[j - 1]);
        }
        if (bad) atomicOr(&s_bad, 1u);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // chunks must follow each other: each starts where the previous ends
        uint32_t tiles = 0;
        uint64_t pos = expect_end;
        for (uint32_t k = 0; k < nch; k++) {
            const uint8_t* d = col + 64 + 32ull * k;
            const uint64_t off = *reinterpret_cast<const uint64_t*>(d);
            if (off != pos) s_bad = 1;
            pos = off + *reinterpret_cast<const uint64_t*>(d + 8);
            desc[k].tile0 = tiles;
            tiles += desc[k].ntiles;
        }
        ctrl[0] = nch;
        ctrl[1] = s_bad ? 0 : tiles;
        ctrl[2] = 0;
        ctrl[3] = 0;
        ctrl[4] = s_bad ? (1u << ZF_ECORRUPT) : 0u;
        ctrl[5] = 0xFFFFFFFFu;
        __threadfence();
    }
}

__device__ __noinline__ void noalloc_tile(const ZfDevChunk& c, const zfd::Hdr& h, uint32_t r0, uint32_t nr,
                                          uint32_t* wsm, uint32_t* err) {
    switch (c.scheme * 4 + c.dtype) {
    case ZF_RAW * 4 + ZF_I32: zfd::fp_warp<int32_t, ZF_RAW>(c, h, r0, nr, wsm, err); break;
    case ZF_RAW * 4 + ZF_I64: zfd::fp_warp<int64_t, ZF_RAW>(c, h, r0, nr, wsm, err); break;
    case ZF_FOR_BP * 4 + ZF_I32: zfd::fp_warp<int32_t, ZF_FOR_BP>(c, h, r0, nr, wsm, err); break;
    case ZF_FOR_BP * 4 + ZF_I64: zfd::fp_warp<int64_t, ZF_FOR_BP>(c, h, r0, nr, wsm, err); break;
    case ZF_DICT_BP * 4 + ZF_I32: zfd::fp_warp<int32_t, ZF_DICT_BP>(c, h, r0, nr, wsm, err); break;
    case ZF_DICT_BP * 4 + ZF_I64: zfd::fp_warp<int64_t, ZF_DICT_BP>(c, h, r0, nr, wsm, err); break;
    case ZF_DELTA_BP * 4 + ZF_I32: zfd::delta_warp<int32_t>(c, h, r0, nr, wsm, err); break;
    case ZF_DELTA_BP * 4 + ZF_I64: zfd::delta_warp<int64_t>(c, h, r0, nr, wsm, err); break;
    case ZF_RLE * 4 + ZF_I32: zfd::rle_warp<int32_t>(c, h, r0, nr, wsm, err); break;
    case ZF_RLE * 4 + ZF_I64: zfd::rle_warp<int64_t>(c, h, r0, nr, wsm, err); break;
    // doubles travel as their 64-bit patterns
    case ZF_RAW * 4 + ZF_F64: zfd::fp_warp<int64_t, ZF_RAW>(c, h, r0, nr, wsm, err); break;
    case ZF_FLOAT2INT * 4 + ZF_F64: zfd::fp_warp<int64_t, ZF_FLOAT2INT>(c, h, r0, nr, wsm, err); break;
    default:
        if ((threadIdx.x & 31) == 0) zfd::report(err, ZF_EINVAL, c.chunk_id);
    }
}

// Persistent decode: CTAs pop tiles from the queue in the scratch array; the
// last CTA to finish resets the queue.
__global__ void __launch_bounds__(kThreads, 2) noalloc_decode(uint32_t warp_smem) {
    extern __shared__ uint4 smem4[];
    __shared__ uint32_t s_tile;
    uint32_t* ctrl = reinterpret_cast<uint32_t*>(g_noalloc_scratch);
    const ZfDevChunk* desc = reinterpret_cast<const ZfDevChunk*>(g_noalloc_scratch + kCtrlBytes);
    uint32_t* err = ctrl + 4;
    const uint32_t nch = ctrl[0], ntiles = ctrl[1];
    const uint32_t warp = threadIdx.x >> 5;
    uint32_t* wsm = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(smem4) + warp * warp_smem);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctrl[2], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        uint32_t a = 0, z = nch;
        while (z - a > 1) {
            const uint32_t mid = (a + z) >> 1;
            if (desc[mid].tile0 <= tile) a = mid;
            else z = mid;
        }
        const ZfDevChunk c = desc[a];
        zfd::Hdr h;
        zfd::load_hdr(c.blob, h);
        const uint32_t rc = (tile - c.tile0) * kTileRows;
        const uint32_t sz = c.dtype == ZF_I32 ? 4 : 8;
        if (h.rows != c.rows || rc >= c.rows || (uint64_t)c.rows * sz > c.dst_cap) {
            if (threadIdx.x == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
            continue;
        }
        const uint32_t r0 = rc + warp * zfd::kWarpRows;
        if (r0 < c.rows) noalloc_tile(c, h, r0, min(zfd::kWarpRows, c.rows - r0), wsm, err);
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctrl[3], 1u) == gridDim.x - 1) {
            ctrl[2] = 0;
            ctrl[3] = 0;
            __threadfence();
        }
    }
}

}  // namespace

extern "C" zf_status zf_decompress_device_noalloc(const void* d_column, uint64_t column_bytes, void* d_out,
                                                  uint64_t out_bytes, void* stream) {
    if (!d_column || column_bytes < 64 || ((uintptr_t)d_column & 15) || ((uintptr_t)d_out & 15))
        return ZF_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ZF_ECUDA;
    void* scratch = nullptr;
    {
        // first call on this device: look up the array's device address (the
        // host-side name of the array is not a device address)
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return ZF_ECUDA;
            }
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // column header, read on the caller's stream so it follows the caller's writes
    unsigned char hdr[64];
    if (cudaMemcpyAsync(hdr, d_column, 64, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ZF_ECUDA;
    uint32_t magic, nch, chunk_rows;
    uint16_t ver;
    uint64_t n_rows, total;
    memcpy(&magic, hdr, 4);
    memcpy(&ver, hdr + 4, 2);
    const int scheme = hdr[6], dtype = hdr[7];
    memcpy(&nch, hdr + 8, 4);
    memcpy(&chunk_rows, hdr + 12, 4);
    memcpy(&n_rows, hdr + 16, 8);
    memcpy(&total, hdr + 32, 8);
    if (magic != zf::kColMagic || ver != 1) return ZF_ECORRUPT;
    if (dtype != ZF_I32 && dtype != ZF_I64 && dtype != ZF_F64) return ZF_EUNSUPPORTED;
    if (scheme == ZF_ANS) return ZF_EUNSUPPORTED;   // decoded by its own kernel on the regular paths
    const bool scheme_ok = dtype == ZF_F64 ? (scheme == ZF_RAW || scheme == ZF_FLOAT2INT)
                                           : (scheme >= ZF_RAW && scheme <= ZF_RLE);
    if (!scheme_ok || chunk_rows == 0 || chunk_rows % 1024 || chunk_rows > (1u << 30) || n_rows > (1ull << 48))
        return ZF_ECORRUPT;
    if (nch > kNoallocMaxChunks) return ZF_EINVAL;  // above the fixed scratch size
    if ((uint64_t)nch != (n_rows + chunk_rows - 1) / chunk_rows || total > column_bytes ||
        64 + 32ull * nch > total)
        return ZF_ECORRUPT;
    const uint32_t sz = dtype == ZF_I32 ? 4 : 8;
    if (n_rows * sz > out_bytes) return ZF_EINVAL;
    if (n_rows == 0) return ZF_OK;
    noalloc_setup<<<1, 256, 0, s>>>((const uint8_t*)d_column, total, (uint8_t*)d_out, out_bytes, nch, scheme,
                                    dtype, n_rows, chunk_rows);
    if (cudaGetLastError() != cudaSuccess) return ZF_ECUDA;
    // widest per-warp slice any chunk of this dtype may need (bit widths are not read on the host)
    auto slice = [](uint32_t vb) {
        uint32_t w = zfd::warp_smem(ZF_FOR_BP, vb, 8 * vb);
        w = w > zfd::warp_smem(ZF_RLE, vb, 0) ? w : zfd::warp_smem(ZF_RLE, vb, 0);
        return (w + 15) & ~15u;
    };
    const uint32_t ws = slice(sz);
    const uint32_t smem = ws * (kThreads / 32);
    {
        // once per device, allow the largest launch of any value size (8-byte values need the most)
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_attr_set[dev]) {
            if (cudaFuncSetAttribute(noalloc_decode, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(slice(8) * (kThreads / 32))) != cudaSuccess) {
                cudaGetLastError();
                return ZF_ECUDA;
            }
            g_attr_set[dev] = true;
        }
    }
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_decode, kThreads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
        return ZF_ECUDA;
    noalloc_decode<<<per_sm * sms, kThreads, smem, s>>>(ws);
    if (cudaGetLastError() != cudaSuccess) return ZF_ECUDA;
    uint32_t e[2] = {0, 0};
    if (cudaMemcpyAsync(e, (const uint8_t*)scratch + 16, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ZF_ECUDA;
    if (e[0] & (1u << ZF_ECORRUPT)) return ZF_ECORRUPT;
    if (e[0]) return ZF_EINVAL;
    return ZF_OK;
}
