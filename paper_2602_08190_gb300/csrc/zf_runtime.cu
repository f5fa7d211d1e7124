// zf_runtime.cu -- the C ABI: contexts, the pinned-host chunk pipeline
// (Section 3.3) and device-resident decode.
//
// Pipeline of zf_transfer_decompress: columns are put in Johnson's-rule order
// (johnson_order), and their chunks are cut into stages of about
// kcfg.stage_bytes compressed bytes, the last three stages smaller (1/8, 1/4,
// 1/2) so little decode is left after the last copy.  Stage s is copied by
// cudaMemcpyAsync on the copy stream into staging slot s % nslots, after the
// decode of the stage that last used the slot has finished (event
// slot_free); decode stream s % nslots waits for the copy (event
// slot_copied) and decodes the stage into the caller's buffers.  Copies of
// stage s+1.. run while stage s decodes, and the decodes of different stages
// may run at once (stages are independent): a launch too small to fill the
// GPU -- an LZ77 stage has one warp per 64 KiB block -- overlaps the next.
// The compute stream joins every decode stream at the end.  All descriptors
// of a call are built on the host and copied once, ahead of the first stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "zf_internal.h"
#include "zf_launch.h"

namespace {
constexpr uint32_t kMaxSlots = 8;
}

struct zf_resident {
    uint8_t* d = nullptr;
    uint64_t len = 0;
    int device = 0;
    int nparts = 0;
    zf::PartInfo parts[2];
    std::vector<zf::ChunkInfo> chunks;
    uint64_t raw_bytes = 0;
};

struct zf_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t copy = nullptr, compute = nullptr;
    cudaStream_t lane[kMaxSlots] = {};  // decode stream of each staging slot
    bool own_copy = false, own_compute = false;
    uint32_t nslots = 8;
    uint64_t slot_req = 0;
    uint8_t* slots[kMaxSlots] = {};
    uint64_t slot_cap = 0;
    cudaEvent_t ev_copied[kMaxSlots] = {}, ev_free[kMaxSlots] = {};
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;
    uint32_t* d_err = nullptr;     // [s * kQueueWords, (s + 1) * kQueueWords): work queue of decode stream s
    // The decoders' error word, [0] status bits and [1] first failing chunk, in
    // mapped pinned host memory: the host resets it before a call and reads it
    // after the call's last event, and the kernels write it only when a stream
    // is malformed -- no memset or read-back rides on the streams.
    uint32_t* h_err = nullptr;
    uint32_t* d_errw = nullptr;    // the device address of h_err
    ZfDevChunk* d_desc = nullptr;
    ZfDevChunk* h_desc = nullptr;  // pinned
    size_t desc_cap = 0;
    std::vector<ZfDevChunk> resident_cache;   // descriptors last uploaded for resident decode
    zf_kcfg kcfg{0, 0, 0, 64u << 20, 0};
    // Geometry found by zf_tune per (scheme, dtype, bit-width bucket), used
    // by launches of that class while the context's tile_rows / threads are 0.
    struct Tuned {
        uint32_t tile_rows = 0, threads = 0;
        float gbs = 0;                 // measured decode rate at that geometry (plain GB/s), 0 = none
    } tuned[ZF_NSCHEMES][4][4];
    float link_gbs = 0;               // measured host-to-device rate of the call's pieces (zf_measure_copy), 0 = none
    uint64_t tuned_gen = 0;
    uint64_t slots_gen = 0;        // bumped whenever the staging slots are reallocated
    // CUDA graph of the last transfer (ZF_KCFG_GRAPH) and what it was built for
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<uint64_t> graph_key;
    ZfDevChunk* g_d_desc = nullptr;
    ZfDevChunk* g_h_desc = nullptr;   // pinned, read by the graph's descriptor copy
    size_t g_desc_cap = 0;
    zf_stats graph_stats{};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    zf_mlp* selector = nullptr;       // learned selector (not owned) and its feature scaling
    float sel_mean[32] = {0}, sel_std[32] = {0};
    bool sel_scaled = false;          // standardize with sel_mean / sel_std (else the network's own scaling)
    bool busy = false;
    zf_status host_err = ZF_OK;
    std::string last_error;
    zf_stats st{};
};

namespace {

zf_status cuda_fail(zf_ctx* ctx, cudaError_t e, const char* what) {
    if (ctx) ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return ZF_ECUDA;
}

#define ZF_CU(ctx, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// tile_rows and threads stay 0 ("auto") here and are resolved per launch
// group (group_geometry); a zero stage size takes 64 MiB.
zf_kcfg effective_kcfg(const zf_ctx* ctx) {
    zf_kcfg k = ctx->kcfg;
    if (!k.stage_bytes) k.stage_bytes = 64u << 20;
    return k;
}

uint32_t width_bucket(uint32_t bmax) { return bmax <= 8 ? 0u : bmax <= 16 ? 1u : bmax <= 32 ? 2u : 3u; }

// The geometry of one launch: the context's tile_rows / threads where set,
// else the tuned entry of the launch's (scheme, dtype, widest bit width)
// class, else the built-in values: 128 threads, warp jobs of two 1024-row
// tiles for delta and four for the others (the fastest, or within 1% of it,
// for delta and RLE columns of 1M-row chunks in a full search on GB300).
struct Geometry {
    uint32_t tile_rows, threads;
};
Geometry group_geometry(const zf_ctx* ctx, const zf_kcfg& k, int scheme, int dtype, uint32_t bmax) {
    Geometry g{k.tile_rows, k.threads};
    if (scheme >= 0 && scheme < ZF_NSCHEMES && dtype >= 0 && dtype < 4) {
        const auto& t = ctx->tuned[scheme][dtype][width_bucket(bmax)];
        if (!g.tile_rows) g.tile_rows = t.tile_rows;
        if (!g.threads) g.threads = t.threads;
    }
    if (!g.tile_rows) g.tile_rows = scheme == ZF_DELTA_BP ? 2048u : 4096u;
    if (!g.threads) g.threads = 128;
    return g;
}

bool kcfg_valid(const zf_kcfg& k) {
    return (k.tile_rows == 0 || (k.tile_rows % 1024 == 0 && k.tile_rows >= 1024 && k.tile_rows <= zf::kMaxTileRows)) &&
           (k.threads == 0 || k.threads == 128 || k.threads == 256 || k.threads == 512) && k.ctas_per_sm <= 64;
}

// One decode unit of a call: a chunk with its host source, device output and part.
struct Work {
    const uint8_t* host;      // serialized bytes (transfer) or null (resident)
    const uint8_t* dev;       // device address of the chunk blob (slot or resident copy)
    const zf::ChunkInfo* ch;
    uint8_t* dst;
    uint64_t cap;
    uint32_t id;
};

// Build the output mapping for the columns of one call.
template <class Col>
zf_status map_outputs(zf_ctx* ctx, const Col* const* cols, uint32_t ncols, void* const* d_out,
                      const uint64_t* d_out_bytes, std::vector<Work>& work, uint64_t* raw, uint64_t* comp,
                      const uint8_t* (*hostp)(const Col*), const uint8_t* (*devp)(const Col*)) {
    uint32_t o = 0;
    uint32_t id = 0;
    for (uint32_t c = 0; c < ncols; c++) {
        const Col* col = cols[c];
        if (!col) {
            ctx->last_error = "null column";
            return ZF_EINVAL;
        }
        for (int p = 0; p < col->nparts; p++, o++) {
            const zf::PartInfo& pi = col->parts[p];
            uint8_t* out = (uint8_t*)d_out[o];
            uint64_t need = pi.n_rows * zf::dtype_size(pi.dtype);
            if (need && (!out || d_out_bytes[o] < need || ((uintptr_t)out & 15))) {
                ctx->last_error = "output buffer missing, too small or not 16-byte aligned";
                return ZF_EINVAL;
            }
            for (uint32_t k = 0; k < pi.n_chunks; k++) {
                const zf::ChunkInfo& ch = col->chunks[pi.first_chunk + k];
                uint64_t off = ch.row0 * zf::dtype_size(pi.dtype);
                const uint8_t* dv = devp(col);
                work.push_back({hostp(col), dv ? dv + ch.off : nullptr, &ch, out + off, d_out_bytes[o] - off, id++});
                *comp += ch.bytes;
            }
            *raw += need;
        }
    }
    return ZF_OK;
}

const uint8_t* host_of(const zf_compressed* c) { return c->host; }
const uint8_t* nodev_of(const zf_compressed*) { return nullptr; }
const uint8_t* nohost_of(const zf_resident*) { return nullptr; }
const uint8_t* dev_of(const zf_resident* r) { return r->d; }

zf_status ensure_desc(zf_ctx* ctx, size_t n) {
    if (n <= ctx->desc_cap) return ZF_OK;
    size_t cap = std::max<size_t>(n, 2 * ctx->desc_cap);
    if (ctx->d_desc) cudaFree(ctx->d_desc);
    if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
    ctx->d_desc = nullptr;
    ctx->h_desc = nullptr;
    ctx->desc_cap = 0;
    ctx->resident_cache.clear();
    if (cudaMalloc(&ctx->d_desc, cap * sizeof(ZfDevChunk)) != cudaSuccess ||
        cudaHostAlloc(&ctx->h_desc, cap * sizeof(ZfDevChunk), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        ctx->last_error = "descriptor buffers";
        return ZF_ENOMEM;
    }
    ctx->desc_cap = cap;
    return ZF_OK;
}

zf_status ensure_slots(zf_ctx* ctx, uint64_t bytes) {
    if (bytes <= ctx->slot_cap) return ZF_OK;
    for (uint32_t s = 0; s < kMaxSlots; s++)
        if (ctx->slots[s]) {
            cudaFree(ctx->slots[s]);
            ctx->slots[s] = nullptr;
        }
    ctx->slot_cap = 0;
    for (uint32_t s = 0; s < ctx->nslots; s++)
        if (cudaMalloc(&ctx->slots[s], bytes) != cudaSuccess) {
            cudaGetLastError();
            ctx->last_error = "staging slots";
            return ZF_ENOMEM;
        }
    ctx->slot_cap = bytes;
    ctx->slots_gen++;
    return ZF_OK;
}

// A group of chunks decoded by one launch.
struct Group {
    int scheme, dtype;   // (-1, -1): batched work-queue kernel; (LZ77, BYTES): LZ kernel
    uint32_t first, count, ntiles;
    uint32_t warp_smem;  // widest per-warp shared memory of the group's chunks
    uint32_t tile_rows;  // rows of a warp job in this launch
    uint32_t threads;    // threads per CTA of this launch
};

// Append descriptors of works[b, e) to `desc`, grouped for launching.
void build_groups(const zf_ctx* ctx, const std::vector<Work>& w, size_t b, size_t e, const zf_kcfg& k,
                  std::vector<ZfDevChunk>& desc, std::vector<Group>& groups) {
    const bool batched = k.flags & ZF_KCFG_BATCHED;
    std::vector<std::pair<int, int>> keys;
    for (size_t i = b; i < e; i++) {
        int s = w[i].ch->scheme, d = w[i].ch->dtype;
        if (s == ZF_LZ77) {
            d = ZF_BYTES;
        } else if (s == ZF_ANS) {
            // ANS streams have their own kernel, batched or not
        } else if (batched) {
            s = -1;
            d = -1;
        }
        if (std::find(keys.begin(), keys.end(), std::make_pair(s, d)) == keys.end()) keys.push_back({s, d});
    }
    for (auto& key : keys) {
        uint32_t bmax = 0;   // widest bit width of the group: its geometry class
        for (size_t i = b; i < e; i++)
            if (w[i].ch->scheme == key.first && w[i].ch->dtype == key.second) bmax = std::max<uint32_t>(bmax, w[i].ch->bmax);
        const Geometry geo = group_geometry(ctx, k, key.first, key.second, bmax);
        Group g{key.first, key.second, (uint32_t)desc.size(), 0, 0, 16, geo.tile_rows, geo.threads};
        for (size_t i = b; i < e; i++) {
            int s = w[i].ch->scheme, d = w[i].ch->dtype;
            bool lz = s == ZF_LZ77, own = lz || s == ZF_ANS;   // chunks with a kernel of their own
            bool match = lz ? key.first == ZF_LZ77
                            : (key.first < 0 ? true : (key.first == s && key.second == d));
            if (!match || (key.first < 0 && own)) continue;
            ZfDevChunk dc{};
            dc.blob = w[i].dev;
            dc.dst = w[i].dst;
            dc.dst_cap = w[i].cap;
            dc.rows = w[i].ch->rows;
            dc.tile0 = g.ntiles;
            dc.ntiles = zf::tiles_of(*w[i].ch, g.tile_rows);
            dc.blob_bytes = (uint32_t)w[i].ch->bytes;
            dc.chunk_id = w[i].id;
            dc.scheme = (uint8_t)s;
            dc.dtype = (uint8_t)d;
            dc.bmax = w[i].ch->bmax;
            g.ntiles += dc.ntiles;
            g.warp_smem = std::max(g.warp_smem, zf::warp_smem_bytes(s, d, w[i].ch->bmax));
            desc.push_back(dc);
            g.count++;
        }
        if (g.count) groups.push_back(g);
    }
}

zf_status launch_groups(zf_ctx* ctx, const std::vector<Group>& groups, const ZfDevChunk* d_desc, const zf_kcfg& k,
                        cudaStream_t stream, uint32_t* queue) {
    for (const Group& g : groups) {
        const ZfDevChunk* dchunks = d_desc + g.first;
        cudaError_t e;
        if (g.scheme == ZF_LZ77) {
            e = zf::launch_lz(dchunks, g.count, ctx->d_errw, ctx->num_sms, stream);
        } else if (g.scheme == ZF_ANS) {
            e = zf::launch_ans(dchunks, g.count, g.ntiles, ctx->d_errw, stream);
        } else {
            uint32_t smem = ((g.warp_smem + 15) & ~15u) * (g.threads / 32);
            zf::TileLaunch L{dchunks, g.count, g.ntiles, g.scheme, g.dtype, g.tile_rows, g.threads,
                             k.ctas_per_sm, smem, ctx->num_sms, ctx->d_errw, queue};
            e = zf::launch_tiles(L, stream);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "decode launch");
        ctx->st.n_launches++;
    }
    return ZF_OK;
}

// Nominal decode rates (GB/s of plain output per scheme on GB300), used for
// Johnson's rule when no rate of the class has been measured.
double nominal_decode_gbs(int scheme) {
    switch (scheme) {
    case ZF_LZ77: return 300;
    case ZF_RLE: return 3500;
    case ZF_DELTA_BP: case ZF_DICT_BP: return 5000;
    case ZF_FLOAT2INT: return 1500;
    case ZF_STRDICT: return 1000;
    case ZF_ANS: return 500;
    default: return 6000;
    }
}

// Johnson's rule for the two-machine flow shop of Section 3.3 (copy, then
// decode) over the columns of a call: a job is a column (its chunks are
// contiguous in one host buffer and stay in order, so they still leave in
// few copies).  A job's copy time is its compressed bytes over the host link
// rate measured by zf_measure_copy (200 GB/s if none was measured), its
// decode time the plain bytes of each chunk over the rate zf_tune measured
// for the chunk's (scheme, dtype, bit-width bucket) class (a nominal rate if
// none).  With ZF_KCFG_KEEP_ORDER the caller's order stays.
void johnson_order(const zf_ctx* ctx, std::vector<Work>& work) {
    std::vector<std::pair<size_t, size_t>> span;
    std::vector<double> copy, dec;
    const double link = ctx->link_gbs > 0 ? ctx->link_gbs : 200.0;
    for (size_t i = 0; i < work.size();) {
        size_t j = i;
        double cp = 0, dc = 0;
        while (j < work.size() && work[j].host == work[i].host) {
            const zf::ChunkInfo& c = *work[j].ch;
            const double plain = (double)c.rows * zf::dtype_size(c.dtype);
            double rate = 0;
            if (c.scheme < ZF_NSCHEMES && c.dtype < 4) rate = ctx->tuned[c.scheme][c.dtype][width_bucket(c.bmax)].gbs;
            if (!(rate > 0)) rate = nominal_decode_gbs(c.scheme);
            cp += (double)c.bytes / link;
            dc += plain / rate;
            j++;
        }
        span.push_back({i, j});
        copy.push_back(cp);
        dec.push_back(dc);
        i = j;
    }
    if (span.size() < 2) return;
    std::vector<uint32_t> order(span.size());
    zf::johnson_sequence(copy.data(), dec.data(), (uint32_t)span.size(), order.data());
    std::vector<Work> out;
    out.reserve(work.size());
    for (uint32_t k : order) out.insert(out.end(), work.begin() + span[k].first, work.begin() + span[k].second);
    work.swap(out);
}

// Stages and copy pieces of a transfer.  Stages: consecutive chunks up to
// stage_bytes of compressed bytes, cut from the end so that the last stages
// are small (1/8, 1/4, 1/2 of stage_bytes): the decode left after the last
// copy is short.  (Cutting the first stages the same way measured slower:
// while decode outruns the link the copy engine is busy from the start
// anyway, and small copies run below the link rate.)  Copy plan: runs of
// chunks contiguous in one host buffer
// become one copy, started at a 128-byte aligned host address (on GB300 an
// H2D copy from an address that is not runs about 15% slower): up to 112
// bytes before the run (never before its buffer) come along, and the run
// lands that far into the slot, so chunk blobs stay 16-byte aligned there.
struct Piece { const uint8_t* src; uint64_t bytes; uint64_t slot_off; };
struct StagePlan {
    std::vector<std::pair<size_t, size_t>> stages;
    std::vector<std::vector<Piece>> pieces;
    std::vector<uint64_t> dev_off;   // offset of each work item's blob in its stage's slot
    uint64_t slot_need = 16;
};
void plan_stages(const std::vector<Work>& work, uint64_t stage_bytes, StagePlan& P) {
    uint64_t max_stage = 0;
    for (size_t j = work.size(), n = 0; j > 0; n++) {
        const uint64_t cap = n < 3 ? std::min<uint64_t>(stage_bytes, std::max<uint64_t>(stage_bytes >> (3 - n), 1u << 20))
                                   : stage_bytes;
        size_t i = j;
        uint64_t bytes = 0;
        while (i > 0 && (i == j || bytes + work[i - 1].ch->bytes <= cap)) bytes += work[--i].ch->bytes;
        P.stages.push_back({i, j});
        max_stage = std::max(max_stage, bytes);
        j = i;
    }
    std::reverse(P.stages.begin(), P.stages.end());
    P.pieces.assign(P.stages.size(), {});
    P.dev_off.assign(work.size(), 0);
    P.slot_need = std::max<uint64_t>(max_stage, 16);
    for (size_t s = 0; s < P.stages.size(); s++) {
        auto [b, e] = P.stages[s];
        uint64_t pos = 0;
        for (size_t i = b; i < e;) {
            size_t j = i + 1;
            while (j < e && work[j].host == work[i].host && work[j].ch->off == work[j - 1].ch->off + work[j - 1].ch->bytes) j++;
            const uint8_t* src = work[i].host + work[i].ch->off;
            const uint64_t lead = std::min<uint64_t>(reinterpret_cast<uintptr_t>(src) & 127, work[i].ch->off);
            const uint64_t bytes = work[j - 1].ch->off + work[j - 1].ch->bytes - work[i].ch->off;
            P.pieces[s].push_back({src - lead, bytes + lead, pos});
            for (size_t q = i; q < j; q++) P.dev_off[q] = pos + lead + (work[q].ch->off - work[i].ch->off);
            pos += (bytes + lead + 15) & ~15ull;
            i = j;
        }
        P.slot_need = std::max(P.slot_need, pos);
    }
}

zf_status begin_call(zf_ctx* ctx) {
    if (ctx->busy) {
        ctx->last_error = "previous call not synced";
        return ZF_EBUSY;
    }
    ZF_CU(ctx, cudaSetDevice(ctx->device));
    ctx->st = zf_stats{};
    ctx->host_err = ZF_OK;
    // the previous call has finished (zf_sync), so no kernel writes the word now
    reinterpret_cast<volatile uint32_t*>(ctx->h_err)[0] = 0;
    reinterpret_cast<volatile uint32_t*>(ctx->h_err)[1] = 0xFFFFFFFFu;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    return ZF_OK;
}

zf_status finish_enqueue(zf_ctx* ctx) {
    ZF_CU(ctx, cudaEventRecord(ctx->ev_t1, ctx->compute));
    ctx->busy = true;
    return ZF_OK;
}

}  // namespace

extern "C" {

zf_status zf_ctx_create(int device, void* copy_stream, void* compute_stream, zf_ctx** out) {
    zf::KeepDevice keep_device;
    if (!out) return ZF_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ZF_ECUDA;
    }
    zf_ctx* ctx = new (std::nothrow) zf_ctx();
    if (!ctx) return ZF_ENOMEM;
    ctx->device = device;
    auto fail = [&](zf_status s) {
        zf_ctx_destroy(ctx);
        return s;
    };
    if (cudaSetDevice(device) != cudaSuccess) return fail(ZF_ECUDA);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (copy_stream) ctx->copy = (cudaStream_t)copy_stream;
    else if (cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking) == cudaSuccess) ctx->own_copy = true;
    else return fail(ZF_ECUDA);
    if (compute_stream) ctx->compute = (cudaStream_t)compute_stream;
    else if (cudaStreamCreateWithFlags(&ctx->compute, cudaStreamNonBlocking) == cudaSuccess) ctx->own_compute = true;
    else return fail(ZF_ECUDA);
    for (uint32_t s = 0; s < kMaxSlots; s++)
        if (cudaEventCreateWithFlags(&ctx->ev_copied[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_free[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ctx->lane[s], cudaStreamNonBlocking) != cudaSuccess)
            return fail(ZF_ECUDA);
    if (cudaEventCreate(&ctx->ev_t0) != cudaSuccess || cudaEventCreate(&ctx->ev_t1) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(ZF_ECUDA);
    if (cudaMalloc(&ctx->d_err, 4 * zf::kQueueWords * kMaxSlots) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, 4 * zf::kQueueWords * kMaxSlots) != cudaSuccess)
        return fail(ZF_ENOMEM);
    if (cudaHostAlloc(&ctx->h_err, 64, cudaHostAllocMapped) != cudaSuccess) return fail(ZF_ENOMEM);
    memset(ctx->h_err, 0, 64);
    ctx->h_err[1] = 0xFFFFFFFFu;
    if (cudaHostGetDevicePointer((void**)&ctx->d_errw, ctx->h_err, 0) != cudaSuccess) return fail(ZF_ECUDA);
    *out = ctx;
    return ZF_OK;
}

zf_status zf_ctx_destroy(zf_ctx* ctx) {
    zf::KeepDevice keep_device;
    if (!ctx) return ZF_OK;
    cudaSetDevice(ctx->device);
    if (ctx->compute) cudaStreamSynchronize(ctx->compute);
    if (ctx->copy) cudaStreamSynchronize(ctx->copy);
    for (uint32_t s = 0; s < kMaxSlots; s++)
        if (ctx->lane[s]) cudaStreamSynchronize(ctx->lane[s]);
    for (uint32_t s = 0; s < kMaxSlots; s++) {
        if (ctx->lane[s]) cudaStreamDestroy(ctx->lane[s]);
        if (ctx->slots[s]) cudaFree(ctx->slots[s]);
        if (ctx->ev_copied[s]) cudaEventDestroy(ctx->ev_copied[s]);
        if (ctx->ev_free[s]) cudaEventDestroy(ctx->ev_free[s]);
    }
    if (ctx->ev_t0) cudaEventDestroy(ctx->ev_t0);
    if (ctx->ev_t1) cudaEventDestroy(ctx->ev_t1);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->g_d_desc) cudaFree(ctx->g_d_desc);
    if (ctx->g_h_desc) cudaFreeHost(ctx->g_h_desc);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->d_desc) cudaFree(ctx->d_desc);
    if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
    if (ctx->own_copy) cudaStreamDestroy(ctx->copy);
    if (ctx->own_compute) cudaStreamDestroy(ctx->compute);
    delete ctx;
    return ZF_OK;
}

const char* zf_last_error(const zf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

zf_status zf_ctx_set_kcfg(zf_ctx* ctx, const zf_kcfg* k) {
    if (!ctx || !k) return ZF_EINVAL;
    zf_kcfg n = *k;
    if (!n.stage_bytes) n.stage_bytes = 64u << 20;
    if (!kcfg_valid(n)) {
        ctx->last_error = "invalid kernel geometry";
        return ZF_EINVAL;
    }
    ctx->kcfg = n;
    return ZF_OK;
}

zf_status zf_ctx_set_ring(zf_ctx* ctx, uint32_t slots, uint64_t slot_bytes) {
    zf::KeepDevice keep_device;
    if (!ctx || slots < 2 || slots > kMaxSlots) return ZF_EINVAL;
    if (ctx->busy) return ZF_EBUSY;
    cudaSetDevice(ctx->device);
    for (uint32_t s = 0; s < kMaxSlots; s++)
        if (ctx->slots[s]) {
            cudaFree(ctx->slots[s]);
            ctx->slots[s] = nullptr;
        }
    ctx->slot_cap = 0;
    ctx->nslots = slots;
    ctx->slot_req = slot_bytes;
    return ZF_OK;
}

zf_status zf_compress_host(const zf_plan_t* plan, const zf_column* col, zf_compressed** out) {
    if (!plan || !col || !out) return ZF_EINVAL;
    *out = nullptr;
    std::string why;
    return zf::encode_column(*plan, *col, out, &why);
}

zf_status zf_compressed_info(const zf_compressed* c, uint64_t* raw, uint64_t* comp, uint32_t* nch) {
    if (!c) return ZF_EINVAL;
    if (raw) *raw = c->raw_bytes;
    if (comp) *comp = c->len;
    if (nch) *nch = (uint32_t)c->chunks.size();
    return ZF_OK;
}

zf_status zf_compressed_free(zf_compressed* c) {
    zf::free_compressed(c);
    return ZF_OK;
}

zf_status zf_compressed_bytes(const zf_compressed* c, const uint8_t** data, uint64_t* len) {
    if (!c || !data || !len) return ZF_EINVAL;
    *data = c->host;
    *len = c->len;
    return ZF_OK;
}

zf_status zf_compressed_from_bytes(const uint8_t* data, uint64_t len, zf_compressed** out) {
    if (!data || !out || len < zf::kColHeader) return ZF_EINVAL;
    *out = nullptr;
    auto* c = new (std::nothrow) zf_compressed();
    if (!c) return ZF_ENOMEM;
    int ndev = 0;
    void* p = nullptr;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
        if (cudaHostAlloc(&p, len, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return ZF_ENOMEM;
        }
        c->pinned = true;
    } else {
        cudaGetLastError();
        p = malloc(len);
        if (!p) {
            delete c;
            return ZF_ENOMEM;
        }
    }
    c->host = (uint8_t*)p;
    c->len = len;
    memcpy(c->host, data, len);
    std::string why;
    zf_status st = zf::parse_serialized(c, &why);
    if (st) {
        zf::free_compressed(c);
        return st;
    }
    *out = c;
    return ZF_OK;
}

zf_status zf_transfer_decompress(zf_ctx* ctx, const zf_compressed* const* cols, uint32_t ncols,
                                 void* const* d_out, const uint64_t* d_out_bytes) {
    zf::KeepDevice keep_device;
    if (!ctx || (ncols && (!cols || !d_out || !d_out_bytes))) return ZF_EINVAL;
    zf_status st = begin_call(ctx);
    if (st) return st;
    const zf_kcfg k = effective_kcfg(ctx);
    const bool use_graph = (k.flags & ZF_KCFG_GRAPH) != 0;
    std::vector<uint64_t> key;
    uint32_t nout = 0;
    if (use_graph) {
        // everything the captured work depends on
        for (uint32_t c = 0; c < ncols; c++) {
            if (!cols[c]) return ZF_EINVAL;
            key.push_back((uint64_t)(uintptr_t)cols[c]);
            key.push_back((uint64_t)(uintptr_t)cols[c]->host);
            key.push_back(cols[c]->len);
            nout += (uint32_t)cols[c]->nparts;
        }
        for (uint32_t o = 0; o < nout; o++) {
            key.push_back((uint64_t)(uintptr_t)d_out[o]);
            key.push_back(d_out_bytes[o]);
        }
        uint32_t link_bits;
        memcpy(&link_bits, &ctx->link_gbs, 4);   // the column order depends on the measured rates
        key.insert(key.end(), {k.tile_rows, k.threads, k.ctas_per_sm, k.stage_bytes, k.flags, ctx->tuned_gen, link_bits,
                               ctx->nslots, ctx->slot_req, ctx->slots_gen});
        if (ctx->graph_exec && key == ctx->graph_key) {
            ZF_CU(ctx, cudaEventRecord(ctx->ev_t0, ctx->copy));
            ZF_CU(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->copy));
            ZF_CU(ctx, cudaEventRecord(ctx->ev_t1, ctx->copy));
            ctx->st = ctx->graph_stats;
            ctx->busy = true;
            return ZF_OK;
        }
    }
    std::vector<Work> work;
    uint64_t raw = 0, comp = 0;
    st = map_outputs<zf_compressed>(ctx, cols, ncols, d_out, d_out_bytes, work, &raw, &comp, host_of, nodev_of);
    if (st) return st;
    if (!(k.flags & ZF_KCFG_KEEP_ORDER)) johnson_order(ctx, work);
    StagePlan P;
    plan_stages(work, k.stage_bytes, P);
    const auto& stages = P.stages;
    const auto& pieces = P.pieces;
    st = ensure_slots(ctx, std::max(P.slot_need, ctx->slot_req));
    if (st) return st;
    if (use_graph) key.back() = ctx->slots_gen;
    for (size_t s = 0; s < stages.size(); s++)
        for (size_t q = stages[s].first; q < stages[s].second; q++) work[q].dev = ctx->slots[s % ctx->nslots] + P.dev_off[q];
    std::vector<ZfDevChunk> desc;
    std::vector<std::vector<Group>> groups(stages.size());
    for (size_t s = 0; s < stages.size(); s++) build_groups(ctx, work, stages[s].first, stages[s].second, k, desc, groups[s]);
    const size_t nd = std::max<size_t>(desc.size(), 1);
    ZfDevChunk* d_desc;
    ZfDevChunk* h_desc;
    if (use_graph) {
        // the graph keeps its own descriptor buffers: other calls reuse the context's
        if (nd > ctx->g_desc_cap) {
            if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
            if (ctx->graph) cudaGraphDestroy(ctx->graph);
            ctx->graph_exec = nullptr;
            ctx->graph = nullptr;
            ctx->graph_key.clear();
            if (ctx->g_d_desc) cudaFree(ctx->g_d_desc);
            if (ctx->g_h_desc) cudaFreeHost(ctx->g_h_desc);
            ctx->g_d_desc = nullptr;
            ctx->g_h_desc = nullptr;
            ctx->g_desc_cap = 0;
            if (cudaMalloc(&ctx->g_d_desc, nd * sizeof(ZfDevChunk)) != cudaSuccess ||
                cudaHostAlloc(&ctx->g_h_desc, nd * sizeof(ZfDevChunk), cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                ctx->last_error = "graph descriptor buffers";
                return ZF_ENOMEM;
            }
            ctx->g_desc_cap = nd;
        }
        d_desc = ctx->g_d_desc;
        h_desc = ctx->g_h_desc;
    } else {
        st = ensure_desc(ctx, nd);
        if (st) return st;
        ctx->resident_cache.clear();
        d_desc = ctx->d_desc;
        h_desc = ctx->h_desc;
    }
    if (!desc.empty()) memcpy(h_desc, desc.data(), desc.size() * sizeof(ZfDevChunk));
    if (use_graph) {
        // capture the whole call (both streams) into a graph, then launch it
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        if (ctx->graph) cudaGraphDestroy(ctx->graph);
        ctx->graph_exec = nullptr;
        ctx->graph = nullptr;
        ctx->graph_key.clear();
        ZF_CU(ctx, cudaStreamBeginCapture(ctx->copy, cudaStreamCaptureModeRelaxed));
        ZF_CU(ctx, cudaEventRecord(ctx->ev_fork, ctx->copy));
        ZF_CU(ctx, cudaStreamWaitEvent(ctx->compute, ctx->ev_fork, 0));
    } else {
        ZF_CU(ctx, cudaEventRecord(ctx->ev_t0, ctx->copy));
    }
    auto abort_capture = [&](zf_status s2) {
        if (use_graph) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(ctx->copy, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
        cudaStreamSynchronize(ctx->copy);
        cudaStreamSynchronize(ctx->compute);
        for (uint32_t q = 0; q < ctx->nslots; q++) cudaStreamSynchronize(ctx->lane[q]);
        return s2;
    };
#define ZF_CAP(call)                                                          \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return abort_capture(cuda_fail(ctx, e_, #call)); \
    } while (0)
    // the error word and the descriptors go first on the copy stream: an H2D
    // copy on another stream can queue behind the stage copies on the same
    // copy engine and hold every decode back
    if (!desc.empty())
        ZF_CAP(cudaMemcpyAsync(d_desc, h_desc, desc.size() * sizeof(ZfDevChunk), cudaMemcpyHostToDevice, ctx->copy));
    if (stages.empty()) ZF_CAP(cudaEventRecord(ctx->ev_copied[0], ctx->copy));
    if (stages.empty()) ZF_CAP(cudaStreamWaitEvent(ctx->compute, ctx->ev_copied[0], 0));
    for (size_t s = 0; s < stages.size(); s++) {
        uint32_t slot = (uint32_t)(s % ctx->nslots);
        if (s >= ctx->nslots) ZF_CAP(cudaStreamWaitEvent(ctx->copy, ctx->ev_free[slot], 0));
        for (const Piece& p : pieces[s])
            ZF_CAP(cudaMemcpyAsync(ctx->slots[slot] + p.slot_off, p.src, p.bytes, cudaMemcpyHostToDevice, ctx->copy));
        ZF_CAP(cudaEventRecord(ctx->ev_copied[slot], ctx->copy));
        ZF_CAP(cudaStreamWaitEvent(ctx->lane[slot], ctx->ev_copied[slot], 0));
        st = launch_groups(ctx, groups[s], d_desc, k, ctx->lane[slot], ctx->d_err + zf::kQueueWords * slot);
        if (st) return abort_capture(st);
        ZF_CAP(cudaEventRecord(ctx->ev_free[slot], ctx->lane[slot]));
    }
    for (size_t q = 0; q < std::min<size_t>(ctx->nslots, stages.size()); q++)
        ZF_CAP(cudaStreamWaitEvent(ctx->compute, ctx->ev_free[q], 0));
#undef ZF_CAP
    ctx->st.raw_bytes = raw;
    ctx->st.comp_bytes = comp;
    ctx->st.n_chunks = (uint32_t)work.size();
    ctx->st.n_stages = (uint32_t)stages.size();
    if (!use_graph) {
        ZF_CU(ctx, cudaEventRecord(ctx->ev_t1, ctx->compute));
        ctx->busy = true;
        return ZF_OK;
    }
    cudaError_t e = cudaEventRecord(ctx->ev_join, ctx->compute);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy, ctx->ev_join, 0);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(ctx->copy, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, e != cudaSuccess ? e : e2, "graph capture");
    }
    e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        ctx->graph_exec = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    ctx->graph = g;
    ctx->graph_key = key;
    ctx->graph_stats = ctx->st;
    ZF_CU(ctx, cudaEventRecord(ctx->ev_t0, ctx->copy));
    ZF_CU(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->copy));
    ZF_CU(ctx, cudaEventRecord(ctx->ev_t1, ctx->copy));
    ctx->busy = true;
    return ZF_OK;
}

zf_status zf_sync(zf_ctx* ctx, zf_stats* stats) {
    zf::KeepDevice keep_device;
    if (!ctx) return ZF_EINVAL;
    if (!ctx->busy) {
        if (stats) *stats = ctx->st;
        return ctx->host_err;
    }
    cudaSetDevice(ctx->device);
    ctx->busy = false;
    cudaError_t e = cudaEventSynchronize(ctx->ev_t1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "zf_sync");
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev_t0, ctx->ev_t1);
    ctx->st.total_ms = ms;
    const uint32_t bits = reinterpret_cast<volatile uint32_t*>(ctx->h_err)[0];
    const uint32_t bad_chunk = reinterpret_cast<volatile uint32_t*>(ctx->h_err)[1];
    ctx->st.device_error = bits;
    if (stats) *stats = ctx->st;
    if (bits) {
        ctx->last_error = "device decoder reported an error in chunk " + std::to_string(bad_chunk);
        if (bits & (1u << ZF_ECORRUPT)) return ZF_ECORRUPT;
        if (bits & (1u << ZF_ETIMEOUT)) return ZF_ETIMEOUT;
        return ZF_EINVAL;
    }
    return ZF_OK;
}

zf_status zf_measure_copy(zf_ctx* ctx, const zf_compressed* const* cols, uint32_t ncols, uint32_t reps, float* ms) {
    zf::KeepDevice keep_device;
    if (!ctx || !ms || !ncols || !cols) return ZF_EINVAL;
    if (ctx->busy) return ZF_EBUSY;
    ZF_CU(ctx, cudaSetDevice(ctx->device));
    if (!reps) reps = 5;
    std::vector<Work> work;
    uint64_t comp = 0;
    for (uint32_t c = 0; c < ncols; c++) {
        if (!cols[c]) return ZF_EINVAL;
        for (const zf::ChunkInfo& ch : cols[c]->chunks) {
            work.push_back({cols[c]->host, nullptr, &ch, nullptr, 0, 0});
            comp += ch.bytes;
        }
    }
    const zf_kcfg k = effective_kcfg(ctx);
    if (!(k.flags & ZF_KCFG_KEEP_ORDER)) johnson_order(ctx, work);
    StagePlan P;
    plan_stages(work, k.stage_bytes, P);
    zf_status st = ensure_slots(ctx, std::max(P.slot_need, ctx->slot_req));
    if (st) return st;
    float best = 3.0e38f;
    for (uint32_t r = 0; r < reps + 1; r++) {
        ZF_CU(ctx, cudaEventRecord(ctx->ev_t0, ctx->copy));
        for (size_t s = 0; s < P.stages.size(); s++)
            for (const Piece& p : P.pieces[s])
                ZF_CU(ctx, cudaMemcpyAsync(ctx->slots[s % ctx->nslots] + p.slot_off, p.src, p.bytes,
                                           cudaMemcpyHostToDevice, ctx->copy));
        ZF_CU(ctx, cudaEventRecord(ctx->ev_t1, ctx->copy));
        ZF_CU(ctx, cudaEventSynchronize(ctx->ev_t1));
        float t = 0;
        ZF_CU(ctx, cudaEventElapsedTime(&t, ctx->ev_t0, ctx->ev_t1));
        if (r) best = std::min(best, t);
    }
    *ms = best;
    if (best > 0) ctx->link_gbs = (float)((double)comp / (best * 1e6));
    return ZF_OK;
}

zf_status zf_upload(zf_ctx* ctx, const zf_compressed* c, zf_resident** out) {
    zf::KeepDevice keep_device;
    if (!ctx || !c || !out) return ZF_EINVAL;
    *out = nullptr;
    if (ctx->busy) return ZF_EBUSY;
    ZF_CU(ctx, cudaSetDevice(ctx->device));
    auto* r = new (std::nothrow) zf_resident();
    if (!r) return ZF_ENOMEM;
    if (cudaMalloc(&r->d, std::max<uint64_t>(c->len, 16)) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        ctx->last_error = "device memory for a resident column";
        return ZF_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(r->d, c->host, c->len, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(r->d);
        delete r;
        return cuda_fail(ctx, e, "zf_upload copy");
    }
    r->len = c->len;
    r->device = ctx->device;
    r->nparts = c->nparts;
    r->parts[0] = c->parts[0];
    r->parts[1] = c->parts[1];
    r->chunks = c->chunks;
    r->raw_bytes = c->raw_bytes;
    *out = r;
    return ZF_OK;
}

zf_status zf_resident_free(zf_resident* r) {
    zf::KeepDevice keep_device;
    if (!r) return ZF_OK;
    cudaSetDevice(r->device);
    if (r->d) cudaFree(r->d);
    delete r;
    return ZF_OK;
}

zf_status zf_decompress_resident(zf_ctx* ctx, const zf_resident* const* cols, uint32_t ncols,
                                 void* const* d_out, const uint64_t* d_out_bytes) {
    zf::KeepDevice keep_device;
    if (!ctx || (ncols && (!cols || !d_out || !d_out_bytes))) return ZF_EINVAL;
    zf_status st = begin_call(ctx);
    if (st) return st;
    const zf_kcfg k = effective_kcfg(ctx);
    std::vector<Work> work;
    uint64_t raw = 0, comp = 0;
    st = map_outputs<zf_resident>(ctx, cols, ncols, d_out, d_out_bytes, work, &raw, &comp, nohost_of, dev_of);
    if (st) return st;
    std::vector<ZfDevChunk> desc;
    std::vector<Group> groups;
    build_groups(ctx, work, 0, work.size(), k, desc, groups);
    ZF_CU(ctx, cudaEventRecord(ctx->ev_t0, ctx->compute));
    bool same = desc.size() == ctx->resident_cache.size() &&
                (desc.empty() || memcmp(desc.data(), ctx->resident_cache.data(), desc.size() * sizeof(ZfDevChunk)) == 0);
    if (!same) {
        st = ensure_desc(ctx, std::max<size_t>(desc.size(), 1));
        if (st) return st;
        if (!desc.empty()) {
            memcpy(ctx->h_desc, desc.data(), desc.size() * sizeof(ZfDevChunk));
            ZF_CU(ctx, cudaMemcpyAsync(ctx->d_desc, ctx->h_desc, desc.size() * sizeof(ZfDevChunk),
                                       cudaMemcpyHostToDevice, ctx->compute));
        }
        ctx->resident_cache = desc;
    }
    if (groups.size() <= 1) {
        st = launch_groups(ctx, groups, ctx->d_desc, k, ctx->compute, ctx->d_err);
    } else {
        // one launch per (scheme, dtype) group, each on its own decode stream,
        // so a launch's tail overlaps the next launch's start
        ZF_CU(ctx, cudaEventRecord(ctx->ev_fork, ctx->compute));
        const size_t nl = std::min<size_t>(groups.size(), ctx->nslots);
        for (size_t q = 0; q < nl; q++) ZF_CU(ctx, cudaStreamWaitEvent(ctx->lane[q], ctx->ev_fork, 0));
        for (size_t gi = 0; gi < groups.size() && st == ZF_OK; gi++) {
            const size_t q = gi % nl;
            st = launch_groups(ctx, std::vector<Group>{groups[gi]}, ctx->d_desc, k, ctx->lane[q],
                               ctx->d_err + zf::kQueueWords * q);
        }
        for (size_t q = 0; q < nl; q++) {
            ZF_CU(ctx, cudaEventRecord(ctx->ev_free[q], ctx->lane[q]));
            ZF_CU(ctx, cudaStreamWaitEvent(ctx->compute, ctx->ev_free[q], 0));
        }
    }
    if (st) {
        cudaStreamSynchronize(ctx->compute);
        for (uint32_t q = 0; q < ctx->nslots; q++) cudaStreamSynchronize(ctx->lane[q]);
        return st;
    }
    ctx->st.raw_bytes = raw;
    ctx->st.comp_bytes = comp;
    ctx->st.n_chunks = (uint32_t)work.size();
    ctx->st.n_stages = 1;
    return finish_enqueue(ctx);
}

}  // extern "C"

namespace zf {
int heuristic_scheme(const zf_column& col, uint32_t chunk_rows);
}

namespace {
// Selector classes: label = scheme * 2 + size; size 0 = 4 MiB, 1 = 32 MiB of
// uncompressed bytes per chunk (string columns keep 64 KiB LZ77 blocks).
uint32_t class_chunk_rows(const zf_column& col, int label) {
    if (col.dtype == ZF_BYTES) return zf::kLzBlock;
    const uint64_t bytes = (label & 1) ? (32ull << 20) : (4ull << 20);
    const uint64_t rows = bytes / zf::dtype_size(col.dtype) / 1024 * 1024;
    return (uint32_t)std::max<uint64_t>(rows, 1024);
}

void class_mask(const zf_column& col, uint8_t* mask) {
    for (int k = 0; k < ZF_MLP_CLASSES; k++) {
        const int scheme = k / 2;
        mask[k] = col.dtype == ZF_BYTES ? (scheme == ZF_RAW || scheme == ZF_LZ77) : (scheme != ZF_LZ77);
    }
}
}  // namespace

// Median end-to-end time (transfer + decode, zf_sync's total_ms) of every
// selector class on this column; classes that do not apply get -1.
extern "C" zf_status zf_measure_classes(zf_ctx* ctx, const zf_column* col, uint32_t reps, float* ms) {
    zf::KeepDevice keep_device;
    if (!ctx || !col || !ms) return ZF_EINVAL;
    if (ctx->busy) return ZF_EBUSY;
    if (!reps) reps = 3;
    uint8_t mask[ZF_MLP_CLASSES];
    class_mask(*col, mask);
    uint64_t outs[2] = {0, 0};
    void* dbuf[2] = {nullptr, nullptr};
    if (col->dtype == ZF_BYTES) {
        outs[0] = std::max<uint64_t>((uint64_t)(uint32_t)col->offsets[col->n], 16);
        outs[1] = 4 * (col->n + 1);
    } else {
        outs[0] = std::max<uint64_t>(col->n * zf::dtype_size(col->dtype), 16);
    }
    cudaSetDevice(ctx->device);
    for (int o = 0; o < 2; o++)
        if (outs[o] && cudaMalloc(&dbuf[o], outs[o]) != cudaSuccess) {
            cudaGetLastError();
            for (void* q : dbuf)
                if (q) cudaFree(q);
            return ZF_ENOMEM;
        }
    zf_status result = ZF_OK;
    for (int k = 0; k < ZF_MLP_CLASSES && !result; k++) {
        ms[k] = -1.0f;
        if (!mask[k]) continue;
        zf_plan_t p{};
        p.scheme = k / 2;
        p.chunk_rows = class_chunk_rows(*col, k);
        p.offsets_scheme = ZF_DELTA_BP;
        p.label = k;
        zf_compressed* c = nullptr;
        std::string why;
        zf_status st = zf::encode_column(p, *col, &c, &why);
        if (st == ZF_EINVAL) continue;          // the scheme does not fit (dictionary too large)
        if (st) {
            result = st;
            break;
        }
        std::vector<float> t;
        for (uint32_t r = 0; r < reps + 1 && !result; r++) {
            const zf_compressed* cc = c;
            st = zf_transfer_decompress(ctx, &cc, 1, dbuf, outs);
            if (!st) {
                zf_stats sts;
                st = zf_sync(ctx, &sts);
                if (r) t.push_back(sts.total_ms);
            }
            if (st) result = st;
        }
        zf::free_compressed(c);
        if (!result) {
            std::sort(t.begin(), t.end());
            ms[k] = t[t.size() / 2];
        }
    }
    for (void* q : dbuf)
        if (q) cudaFree(q);
    return result;
}

// The chunk-size dimension of the search: the column encoded with each
// candidate chunk size, then timed through the whole transfer + decode.
extern "C" zf_status zf_tune_chunk_rows(zf_ctx* ctx, const zf_column* col, int32_t scheme, const uint32_t* chunk_rows,
                                        uint32_t n, uint32_t reps, float* ms, uint32_t* best) {
    zf::KeepDevice keep_device;
    if (!ctx || !col || !chunk_rows || !n || !ms || scheme < 0 || scheme >= ZF_NSCHEMES) return ZF_EINVAL;
    if (ctx->busy) return ZF_EBUSY;
    if (!reps) reps = 3;
    uint64_t outs[2] = {0, 0};
    void* dbuf[2] = {nullptr, nullptr};
    if (col->dtype == ZF_BYTES) {
        if (!col->offsets) return ZF_EINVAL;
        outs[0] = std::max<uint64_t>((uint64_t)(uint32_t)col->offsets[col->n], 16);
        outs[1] = 4 * (col->n + 1);
    } else {
        outs[0] = std::max<uint64_t>(col->n * zf::dtype_size(col->dtype), 16);
    }
    cudaSetDevice(ctx->device);
    for (int o = 0; o < 2; o++)
        if (outs[o] && cudaMalloc(&dbuf[o], outs[o]) != cudaSuccess) {
            cudaGetLastError();
            for (void* q : dbuf)
                if (q) cudaFree(q);
            return ZF_ENOMEM;
        }
    zf_status result = ZF_OK;
    int32_t bi = -1;
    for (uint32_t i = 0; i < n && !result; i++) {
        ms[i] = -1.0f;
        zf_plan_t p{};
        p.scheme = scheme;
        p.chunk_rows = chunk_rows[i];
        p.offsets_scheme = ZF_DELTA_BP;
        p.label = -1;
        zf_compressed* c = nullptr;
        std::string why;
        zf_status st = zf::encode_column(p, *col, &c, &why);
        if (st == ZF_EINVAL) continue;          // the scheme or the size does not fit this column
        if (st) {
            result = st;
            break;
        }
        std::vector<float> t;
        for (uint32_t r = 0; r < reps + 1 && !result; r++) {
            const zf_compressed* cc = c;
            st = zf_transfer_decompress(ctx, &cc, 1, dbuf, outs);
            if (!st) {
                zf_stats sts;
                st = zf_sync(ctx, &sts);
                if (r) t.push_back(sts.total_ms);
            }
            if (st) result = st;
        }
        zf::free_compressed(c);
        if (!result) {
            std::sort(t.begin(), t.end());
            ms[i] = t[t.size() / 2];
            if (bi < 0 || ms[i] < ms[bi]) bi = (int32_t)i;
        }
    }
    for (void* q : dbuf)
        if (q) cudaFree(q);
    if (!result && bi < 0) result = ZF_EINVAL;
    if (!result && best) *best = (uint32_t)bi;
    return result;
}

extern "C" zf_status zf_ctx_set_selector(zf_ctx* ctx, zf_mlp* net, const float* mean, const float* std_) {
    if (!ctx || (!mean) != (!std_)) return ZF_EINVAL;
    ctx->selector = net;
    ctx->sel_scaled = net && mean;
    if (ctx->sel_scaled) {
        memcpy(ctx->sel_mean, mean, sizeof(ctx->sel_mean));
        memcpy(ctx->sel_std, std_, sizeof(ctx->sel_std));
    }
    return ZF_OK;
}

extern "C" zf_status zf_plan(zf_ctx* ctx, const zf_column* col, const zf_plan_opts* opts, zf_plan_t* out) {
    if (!col || !out) return ZF_EINVAL;
    if (col->dtype != ZF_I32 && col->dtype != ZF_I64 && col->dtype != ZF_BYTES && col->dtype != ZF_F64) return ZF_EINVAL;
    zf_plan_opts o{-1, 0, 0, -1, 0};
    if (opts) o = *opts;
    if (col->dtype == ZF_F64 && o.scheme < 0) o.selector = 0;   // the selector's classes cover integer and byte columns
    zf_plan_t p{};
    p.label = -1;
    p.offsets_scheme = o.offsets_scheme < 0 ? ZF_DELTA_BP : o.offsets_scheme;
    p.ans_stream_rows = o.ans_stream_rows;
    p.chunk_rows = col->dtype == ZF_BYTES ? zf::kLzBlock : (o.chunk_rows ? o.chunk_rows : (1u << 20));
    if (col->dtype != ZF_BYTES && (p.chunk_rows % 1024 || p.chunk_rows > (1u << 30))) {
        if (ctx) ctx->last_error = "chunk_rows must be a multiple of 1024 and at most 2^30";
        return ZF_EINVAL;
    }
    p.kcfg = ctx ? ctx->kcfg : zf_kcfg{0, 0, 0, 64u << 20, 0};
    if (o.scheme >= 0) {
        if (o.scheme >= ZF_NSCHEMES) return ZF_EINVAL;
        p.scheme = o.scheme;
        if (p.scheme == ZF_STRDICT && col->dtype == ZF_BYTES) {
            // string-dictionary chunks: o.chunk_rows bytes (a multiple of 64 KiB), else 4 MiB
            p.chunk_rows = o.chunk_rows ? o.chunk_rows : (4u << 20);
            if (p.chunk_rows % zf::kLzBlock || p.chunk_rows > zf::kStrChunkMax) {
                if (ctx) ctx->last_error = "string-dictionary chunks are a multiple of 65536 bytes, at most 2^26";
                return ZF_EINVAL;
            }
        }
    } else if (o.selector == 0) {
        p.scheme = zf::heuristic_scheme(*col, p.chunk_rows);
    } else if (o.selector == 1) {
        if (!ctx || !ctx->selector) {
            if (ctx) ctx->last_error = "no learned selector attached (zf_ctx_set_selector)";
            return ZF_EUNSUPPORTED;
        }
        float f[32];
        zf_status st = zf_column_features(col, f);
        if (st) return st;
        if (ctx->sel_scaled)
            for (int i = 0; i < 32; i++) f[i] = (f[i] - ctx->sel_mean[i]) / (ctx->sel_std[i] > 0 ? ctx->sel_std[i] : 1.0f);
        uint8_t mask[ZF_MLP_CLASSES];
        class_mask(*col, mask);
        int32_t label = -1;
        st = zf_mlp_predict(ctx->selector, f, mask, 1, &label);
        if (st) return st;
        if (label < 0) return ZF_EINVAL;
        p.label = label;
        p.scheme = label / 2;
        p.chunk_rows = class_chunk_rows(*col, label);
    } else if (o.selector == 2) {
        if (!ctx) return ZF_EINVAL;
        float ms[ZF_MLP_CLASSES];
        zf_status st = zf_measure_classes(ctx, col, 3, ms);
        if (st) return st;
        int best = -1;
        for (int k = 0; k < ZF_MLP_CLASSES; k++)
            if (ms[k] >= 0 && (best < 0 || ms[k] < ms[best])) best = k;
        if (best < 0) return ZF_EINVAL;
        p.label = best;
        p.scheme = best / 2;
        p.chunk_rows = class_chunk_rows(*col, best);
        p.predicted_ms = ms[best];
    } else {
        return ZF_EINVAL;
    }
    *out = p;
    return ZF_OK;
}

// ---------------------------------------------------------------- exhaustive autotuner
namespace {
const uint32_t kTuneTileRows[] = {1024, 2048, 4096, 8192, 16384};
const uint32_t kTuneThreads[] = {128, 256, 512};
const uint32_t kTuneStageMiB[] = {4, 8, 16, 32, 64};
}  // namespace

extern "C" zf_status zf_tune(zf_ctx* ctx, const zf_compressed* const* cols, uint32_t ncols, void* const* d_out,
                             const uint64_t* d_out_bytes, int32_t transfer, uint32_t reps, zf_tune_point* points,
                             uint32_t max_points, uint32_t* n_points, zf_kcfg* best) {
    zf::KeepDevice keep_device;
    if (!ctx || !cols || !ncols || !d_out || !d_out_bytes || !n_points) return ZF_EINVAL;
    if (ctx->busy) return ZF_EBUSY;
    if (reps == 0) reps = 3;
    const zf_kcfg saved = ctx->kcfg;
    std::vector<zf_resident*> res;
    auto cleanup = [&](zf_status s) {
        for (zf_resident* r : res) zf_resident_free(r);
        if (s != ZF_OK) ctx->kcfg = saved;
        return s;
    };
    if (!transfer) {
        for (uint32_t c = 0; c < ncols; c++) {
            zf_resident* r = nullptr;
            zf_status s = zf_upload(ctx, cols[c], &r);
            if (s) return cleanup(s);
            res.push_back(r);
        }
    }
    const uint32_t nstage = transfer ? (uint32_t)(sizeof(kTuneStageMiB) / sizeof(kTuneStageMiB[0])) : 1;
    const uint32_t ngraph = transfer ? 2u : 1u;
    uint32_t n = 0;
    float best_ms = 3.0e38f;
    zf_kcfg best_k = saved;
    for (uint32_t gi = 0; gi < ngraph; gi++)
    for (uint32_t si = 0; si < nstage; si++)
        for (uint32_t tr : kTuneTileRows)
            for (uint32_t th : kTuneThreads) {
                zf_kcfg k = saved;
                k.tile_rows = tr;
                k.threads = th;
                k.flags = (saved.flags & ~ZF_KCFG_GRAPH) | (gi ? ZF_KCFG_GRAPH : 0u);
                k.stage_bytes = transfer ? (kTuneStageMiB[si] << 20) : (saved.stage_bytes ? saved.stage_bytes : 64u << 20);
                ctx->kcfg = k;
                std::vector<float> ms;
                for (uint32_t rep = 0; rep < reps + 1; rep++) {   // first run warms up (and captures a graph)
                    const auto t0 = std::chrono::steady_clock::now();
                    zf_status s = transfer ? zf_transfer_decompress(ctx, cols, ncols, d_out, d_out_bytes)
                                           : zf_decompress_resident(ctx, res.data(), ncols, d_out, d_out_bytes);
                    if (s) return cleanup(s);
                    zf_stats stt;
                    s = zf_sync(ctx, &stt);
                    if (s) return cleanup(s);
                    // a transfer is timed as its caller sees it, on the host clock around the call
                    // and zf_sync (graph replay costs the host less but each stage more on the device);
                    // a resident decode by the device events
                    const float wall = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
                    if (rep) ms.push_back(transfer ? wall : stt.total_ms);
                }
                std::sort(ms.begin(), ms.end());
                const float med = ms[ms.size() / 2];
                if (points && n < max_points) points[n] = zf_tune_point{k, med};
                n++;
                if (med < best_ms) {
                    best_ms = med;
                    best_k = k;
                }
            }
    best_k.flags = (saved.flags & ~ZF_KCFG_GRAPH) | (transfer ? (best_k.flags & ZF_KCFG_GRAPH) : (saved.flags & ZF_KCFG_GRAPH));
    // Columns of one (scheme, dtype, bit-width bucket) class: the result is
    // kept for that class and the context's geometry stays automatic, so
    // later calls give every class its own; otherwise the context takes it.
    // (a string column's int32 offsets are its second part: the class is
    // that of its bytes, whose decode dominates)
    int cs = -1, cd = -1, cb = -1;
    bool one = true;
    for (uint32_t c = 0; c < ncols && one; c++)
        for (const zf::ChunkInfo& ch : cols[c]->chunks) {
            if (ch.part != 0) continue;
            const int b = (int)width_bucket(ch.bmax);
            if (cs >= 0 && (ch.scheme != cs || ch.dtype != cd || b != cb)) {
                one = false;
                break;
            }
            cs = ch.scheme;
            cd = ch.dtype;
            cb = b;
        }
    if (one && cs >= 0) {
        ctx->tuned[cs][cd][cb].tile_rows = best_k.tile_rows;
        ctx->tuned[cs][cd][cb].threads = best_k.threads;
        if (!transfer && best_ms > 0) {
            uint64_t raw = 0;
            for (uint32_t c = 0; c < ncols; c++) raw += cols[c]->raw_bytes;
            ctx->tuned[cs][cd][cb].gbs = (float)((double)raw / (best_ms * 1e6));
        }
        ctx->tuned_gen++;
        ctx->kcfg = saved;
        if (transfer) {
            ctx->kcfg.stage_bytes = best_k.stage_bytes;
            ctx->kcfg.flags = best_k.flags;
        }
    } else {
        ctx->kcfg = best_k;
    }
    *n_points = n;
    if (best) *best = best_k;
    return cleanup(ZF_OK);
}

extern "C" zf_status zf_ctx_rates(const zf_ctx* ctx, int32_t scheme, int32_t dtype, uint32_t bmax, float* decode_gbs,
                                  float* link_gbs) {
    if (!ctx || scheme < 0 || scheme >= ZF_NSCHEMES || dtype < 0 || dtype > ZF_F64 || bmax > 64) return ZF_EINVAL;
    if (decode_gbs) decode_gbs[0] = ctx->tuned[scheme][dtype][width_bucket(bmax)].gbs;
    if (link_gbs) link_gbs[0] = ctx->link_gbs;
    return ZF_OK;
}

extern "C" zf_status zf_ctx_tuned_geometry(const zf_ctx* ctx, int32_t scheme, int32_t dtype, uint32_t bmax,
                                           zf_kcfg* out) {
    if (!ctx || !out || scheme < 0 || scheme >= ZF_NSCHEMES || dtype < 0 || dtype > ZF_F64 || bmax > 64)
        return ZF_EINVAL;
    const zf_kcfg k = effective_kcfg(ctx);
    const Geometry g = group_geometry(ctx, k, scheme, dtype, bmax);
    *out = k;
    out->tile_rows = g.tile_rows;
    out->threads = g.threads;
    return ZF_OK;
}
