// zf_internal.h -- library-internal layout constants, host objects and the
// device chunk descriptor.  The container format itself is described in zf.h.
#pragma once
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/zf.h"

#include <cuda_runtime_api.h>

namespace zf {

// Entry points make their context's device current; this puts the caller's
// current device back when the entry point returns.
struct KeepDevice {
    int dev = -1;
    KeepDevice() {
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            dev = -1;
        }
    }
    ~KeepDevice() {
        int cur = -1;
        if (dev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != dev) cudaSetDevice(dev);
    }
    KeepDevice(const KeepDevice&) = delete;
    KeepDevice& operator=(const KeepDevice&) = delete;
};

constexpr uint32_t kColMagic = 0x4C4F435Au;    // 'ZCOL'
constexpr uint32_t kChunkMagic = 0x4B48435Au;  // 'ZCHK'
constexpr uint32_t kColHeader = 64;
constexpr uint32_t kDirEntry = 32;
constexpr uint32_t kChunkHeader = 64;
constexpr uint32_t kDeltaBlock = 1024;         // rows per delta block
constexpr uint32_t kRleDirRows = 1024;         // rows per RLE directory entry
constexpr uint32_t kDeltaEntry = 24;           // bytes per delta block entry
constexpr uint32_t kLzBlock = 65536;           // bytes per LZ77 block
constexpr uint32_t kLzMinMatch = 4;
constexpr uint32_t kLzMaxOffset = 65535;
constexpr uint32_t kMaxDict = 65536;
constexpr uint32_t kMaxTileRows = 16384;   // rows per warp job (16 warp tiles)
constexpr uint32_t kStrTokenMax = 64;          // bytes of one string-dictionary token at most
constexpr uint32_t kStrDictMax = 65536;        // string-dictionary entries at most
constexpr uint32_t kStrTile = 1024;            // tokens per tile-start entry
constexpr uint32_t kStrChunkMax = 1u << 26;    // bytes of one string-dictionary chunk at most
constexpr uint32_t kAnsMaxSymbols = 256;       // ANS: distinct values of a chunk at most
constexpr uint32_t kAnsScale = 12;             // ANS: frequencies sum to M = 2^12
constexpr uint32_t kAnsM = 1u << kAnsScale;
constexpr uint32_t kAnsL = 1u << 23;           // ANS: states stay in [L, 256 L)
constexpr uint32_t kAnsStream = 512;           // ANS: rows per independent stream unless the plan names others
constexpr uint32_t kAnsLogMin = 5, kAnsLogMax = 12;   // ANS: rows per stream = 2^k, k in 5..12 (header byte 48)
constexpr uint32_t kAnsStreamsPerJob = 32;     // ANS: one stream per lane of a warp job
constexpr uint32_t kAnsJobsPerCta = 4;         // ANS: a CTA's warps take jobs of one chunk (padded to a multiple)

inline uint64_t align16(uint64_t x) { return (x + 15) & ~uint64_t(15); }
inline uint32_t bits_of(uint64_t x) { return x ? 64u - (uint32_t)__builtin_clzll(x) : 0u; }
inline uint32_t dtype_size(int dt) { return (dt == ZF_I64 || dt == ZF_F64) ? 8u : dt == ZF_I32 ? 4u : 1u; }
constexpr int kF2IMaxExp = 18;                 // Float2Int decimal exponents 0..18
inline uint64_t packed_bytes(uint64_t n, uint32_t b) { return (n * b + 7) / 8; }

// Host-side description of one chunk of one part of a compressed column.
struct ChunkInfo {
    uint64_t off;     // blob offset from the start of the serialized buffer
    uint64_t bytes;   // blob length
    uint64_t row0;    // first row within its part
    uint32_t rows;
    uint8_t scheme, dtype, part;
    uint8_t bmax;     // widest bit width in the chunk (FOR/DICT: b; DELTA: widest block)
    uint32_t units = 0;   // string dictionary: tokens of the chunk; ANS: streams
};

struct PartInfo {
    uint64_t off = 0, len = 0;   // byte range of the part in the serialized buffer
    int scheme = 0, dtype = 0;
    uint64_t n_rows = 0;
    uint32_t chunk_rows = 0;
    uint32_t first_chunk = 0, n_chunks = 0;  // range in zf_compressed::chunks
};

}  // namespace zf

struct zf_compressed {
    uint8_t* host = nullptr;     // serialized bytes (pinned when `pinned`)
    uint64_t len = 0;
    bool pinned = false;
    int nparts = 0;
    zf::PartInfo parts[2];
    std::vector<zf::ChunkInfo> chunks;
    uint64_t raw_bytes = 0;
};

// Device descriptor of one chunk inside one launch (64 bytes).
struct ZfDevChunk {
    const uint8_t* blob;     // device address of the chunk blob
    uint8_t* dst;            // device address of the chunk's row 0 in the output
    uint64_t dst_cap;        // writable bytes at dst
    uint32_t rows;
    uint32_t tile0;          // first warp job of this chunk within the launch
    uint32_t ntiles;         // warp jobs of this chunk
    uint32_t blob_bytes;
    uint32_t chunk_id;       // index reported with a decode error
    uint8_t scheme, dtype;
    uint8_t bmax;            // widest bit width of the chunk (sizes the staging buffers)
    uint8_t pad1;
    uint32_t pad2[4];
};
static_assert(sizeof(ZfDevChunk) == 64, "descriptor layout");

namespace zf {
// host encoder / parser (zf_host.cpp)
zf_status encode_column(const zf_plan_t& plan, const zf_column& col, zf_compressed** out, std::string* why);
zf_status parse_serialized(zf_compressed* c, std::string* why);
void free_compressed(zf_compressed* c);
uint32_t tiles_of(const ChunkInfo& ch, uint32_t tile_rows);
// Johnson's rule for a two-machine flow shop (zf_plan.cpp): the order of n
// jobs with times copy[i] on the first machine and dec[i] on the second.
void johnson_sequence(const double* copy, const double* dec, uint32_t n, uint32_t* order);
}  // namespace zf
