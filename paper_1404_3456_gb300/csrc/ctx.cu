// ctx.cu -- context, workspace, status handling, the pack step and the
// order-preserving compaction used by several steps.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <utility>

#include "block.cuh"
#include "common.cuh"

namespace dnasa {

int fail(dnasa_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

int cuda_fail(dnasa_ctx *ctx, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    if (e == cudaErrorMemoryAllocation) return fail(ctx, DNASA_OOM, msg);
    return fail(ctx, DNASA_CUDA_ERROR, msg);
}

cudaError_t smem_attr_fn(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void *, int>> done;   // (kernel, device) pairs configured
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({fn, dev})) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.insert({fn, dev});
    return e;
}

int ws_reserve(dnasa_ctx *ctx, size_t bytes, cudaStream_t s) {
    if (bytes <= ctx->ws_size) return DNASA_OK;
    if (ctx->ws_cap && bytes > ctx->ws_cap)
        return fail(ctx, DNASA_OOM, "workspace of " + std::to_string(bytes) +
                                        " bytes exceeds the context cap of " +
                                        std::to_string(ctx->ws_cap));
    if (ctx->ws) {
        cudaStreamSynchronize(s);
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_size = 0;
    }
    size_t want = bytes + bytes / 8 + (1u << 20);
    if (ctx->ws_cap) want = std::min(want, ctx->ws_cap);
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return fail(ctx, DNASA_OOM, "workspace cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    ctx->ws_size = want;
    return DNASA_OK;
}

bool is_device_ptr(dnasa_ctx *ctx, const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return at.device == ctx->device;
    return false;
}

int check_device_status(dnasa_ctx *ctx, cudaStream_t s, const char *where) {
    // the error word has its own pinned slot (63) so that a caller's readback
    // into the low slots, enqueued just before, is not overwritten
    uint32_t *slot = reinterpret_cast<uint32_t *>(ctx->pinned + 63);
    DNASA_CUDA(ctx, cudaMemcpyAsync(slot, &ctx->ctrl->err, sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, s));
    DNASA_CUDA(ctx, cudaStreamSynchronize(s));
    uint32_t err = *(volatile uint32_t *)slot;
    if (err == 0) return DNASA_OK;
    DNASA_CUDA(ctx, cudaMemsetAsync(&ctx->ctrl->err, 0, sizeof(uint32_t), s));
    DNASA_CUDA(ctx, cudaStreamSynchronize(s));
    std::string w(where);
    if (err & DERR_TIMEOUT) return fail(ctx, DNASA_DEVICE_TIMEOUT, w + ": a bounded device wait gave up");
    if (err & DERR_ALPHABET) return fail(ctx, DNASA_BAD_ALPHABET, w + ": byte outside A/C/G/T/'$'");
    if (err & DERR_EMPTY_READ) return fail(ctx, DNASA_BAD_ALPHABET, w + ": empty fragment or text not '$'-terminated");
    return fail(ctx, DNASA_CUDA_ERROR, w + ": device index check failed");
}

// ------------------------------------------------------------------ profiling
static cudaEvent_t ev_get(dnasa_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

LaunchScope::LaunchScope(dnasa_ctx *c, int kind, cudaStream_t st, double bytes) : ctx(c), s(st) {
    ++ctx->launches;
    if (!ctx->prof_on) return;
    ProfRec r;
    r.kind = kind;
    r.bytes = bytes;
    r.a = ev_get(ctx);
    r.b = ev_get(ctx);
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    idx = (int)ctx->prof.size();
    ctx->prof.push_back(r);
}

LaunchScope::~LaunchScope() {
    if (idx >= 0) cudaEventRecord(ctx->prof[idx].b, s);
}

// ------------------------------------------------------------------ small scans

// Exclusive scan of a[0..n) in place by one block; a[n] (if store_total) = sum.
__global__ void __launch_bounds__(1024) k_scan_small(int64_t *a, int64_t n, int64_t *total) {
    __shared__ int64_t tmp[33];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < n ? a[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_sum<1024>(v, tmp, &tot);
        if (i < n) a[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// ------------------------------------------------------------------ compaction
constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 16;
constexpr int kCompactTile = kCompactThreads * kCompactItems;

__global__ void __launch_bounds__(kCompactThreads) k_flag_count(const uint8_t *__restrict__ flags,
                                                                int64_t n, int64_t *tile_counts) {
    __shared__ int64_t tmp[9];
    int64_t base = (int64_t)blockIdx.x * kCompactTile;
    int64_t c = 0;
    for (int i = 0; i < kCompactItems; ++i) {
        int64_t idx = base + (int64_t)i * kCompactThreads + threadIdx.x;
        if (idx < n && flags[idx]) ++c;
    }
    int64_t tot;
    block_exclusive_sum<kCompactThreads>(c, tmp, &tot);
    if (threadIdx.x == 0) tile_counts[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kCompactThreads) k_flag_scatter(const uint8_t *__restrict__ flags,
                                                                  int64_t n,
                                                                  const int64_t *tile_prefix,
                                                                  uint32_t *__restrict__ out) {
    __shared__ int64_t tmp[9];
    int64_t base = (int64_t)blockIdx.x * kCompactTile + (int64_t)threadIdx.x * kCompactItems;
    int64_t c = 0;
    uint32_t bits = 0;
    for (int i = 0; i < kCompactItems; ++i) {
        int64_t idx = base + i;
        if (idx < n && flags[idx]) { ++c; bits |= 1u << i; }
    }
    int64_t tot;
    int64_t ex = block_exclusive_sum<kCompactThreads>(c, tmp, &tot);
    int64_t o = tile_prefix[blockIdx.x] + ex;
    for (int i = 0; i < kCompactItems; ++i)
        if (bits >> i & 1u) out[o++] = (uint32_t)(base + i);
}

size_t compact_scratch_bytes(int64_t n) {
    return (((size_t)ceil_div(n, kCompactTile) + 1) * sizeof(int64_t) + 255) & ~size_t(255);
}

int compact_flags(dnasa_ctx *ctx, Arena &a, const uint8_t *flags, int64_t n, uint32_t *out,
                  unsigned long long *d_count, cudaStream_t s) {
    if (n <= 0) {
        DNASA_CUDA(ctx, cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), s));
        return DNASA_OK;
    }
    int tiles = ceil_div(n, kCompactTile);
    int64_t *tc = a.take<int64_t>((size_t)tiles + 1);
    if (!tc) return fail(ctx, DNASA_OOM, "compaction scratch");
    {
        LaunchScope ls_(ctx, PK_OTHER, s, (double)n);
        k_flag_count<<<tiles, kCompactThreads, 0, s>>>(flags, n, tc);
    }
    {
        LaunchScope ls_(ctx, PK_OTHER, s, 0);
        k_scan_small<<<1, 1024, 0, s>>>(tc, tiles, (int64_t *)d_count);
    }
    {
        LaunchScope ls_(ctx, PK_OTHER, s, (double)n);
        k_flag_scatter<<<tiles, kCompactThreads, 0, s>>>(flags, n, tc, out);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}

// ------------------------------------------------------------------ pack
constexpr int kPackThreads = 256;
constexpr int kPackChunk = 32;                         // bytes per thread
constexpr int kPackTile = kPackThreads * kPackChunk;   // 8192 bytes

__device__ __forceinline__ int code_of(uint8_t c) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        case '$': return 4;
        default: return -1;
    }
}

__global__ void __launch_bounds__(kPackThreads) k_pack_count(const uint8_t *__restrict__ text,
                                                             int64_t N, int64_t *tile_counts,
                                                             uint32_t *err) {
    __shared__ int64_t tmp[9];
    int64_t base = (int64_t)blockIdx.x * kPackTile + (int64_t)threadIdx.x * kPackChunk;
    int64_t c = 0;
    uint32_t bad = 0;
    for (int i = 0; i < kPackChunk; ++i) {
        int64_t p = base + i;
        if (p >= N) break;
        int k = code_of(text[p]);
        if (k < 0) bad |= DERR_ALPHABET;
        if (k == 4) {
            ++c;
            if (p == 0 || text[p - 1] == '$') bad |= DERR_EMPTY_READ;
        }
        if (p == N - 1 && k != 4) bad |= DERR_EMPTY_READ;
    }
    if (bad) atomicOr(err, bad);
    int64_t tot;
    block_exclusive_sum<kPackThreads>(c, tmp, &tot);
    if (threadIdx.x == 0) tile_counts[blockIdx.x] = tot;
}

// Writes toff entries and one 2-bit code byte per base (base coordinate order).
__global__ void __launch_bounds__(kPackThreads) k_pack_emit(const uint8_t *__restrict__ text,
                                                            int64_t N, const int64_t *tile_prefix,
                                                            int64_t *__restrict__ toff,
                                                            int64_t toff_cap,
                                                            uint8_t *__restrict__ codes) {
    __shared__ int64_t tmp[9];
    int64_t base = (int64_t)blockIdx.x * kPackTile + (int64_t)threadIdx.x * kPackChunk;
    int64_t c = 0;
    for (int i = 0; i < kPackChunk; ++i) {
        int64_t p = base + i;
        if (p < N && text[p] == '$') ++c;
    }
    int64_t tot;
    int64_t r = tile_prefix[blockIdx.x] + block_exclusive_sum<kPackThreads>(c, tmp, &tot);
    for (int i = 0; i < kPackChunk; ++i) {
        int64_t p = base + i;
        if (p >= N) break;
        uint8_t ch = text[p];
        int k = code_of(ch);
        if (k == 4) {
            if (r + 1 < toff_cap) toff[r + 1] = p + 1;
            ++r;
        } else {
            codes[p - r] = (uint8_t)(k < 0 ? 0 : k);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && toff_cap > 0) toff[0] = 0;
}

__global__ void k_pack_words(const uint8_t *__restrict__ codes, const int64_t *n_dollars,
                             int64_t N, int64_t nwords, uint64_t *__restrict__ packed) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    int64_t B = N - *n_dollars;   // bases
    uint64_t x = 0;
    int64_t b0 = w * 32;
    for (int i = 0; i < 32; ++i) {
        int64_t b = b0 + i;
        uint64_t code = b < B ? (uint64_t)(codes[b] & 3u) : 0ull;
        x |= code << (62 - 2 * i);
    }
    packed[w] = x;
}

int pack_impl(dnasa_ctx *ctx, const uint8_t *text, int64_t N, uint64_t *packed, int64_t *toff,
              int64_t toff_cap, int64_t *n_reads, cudaStream_t s) {
    PhaseRange nvtx_("dnasa.pack");
    int tiles = ceil_div(N, kPackTile);
    size_t need = ((size_t)(tiles + 1) * 8 + 255) / 256 * 256 + (size_t)N + 4096;
    DNASA_TRY(ws_reserve(ctx, need, s));
    Arena a = ws_arena(ctx);
    int64_t *tc = a.take<int64_t>((size_t)tiles + 1);
    uint8_t *codes = a.take<uint8_t>((size_t)N + 64);
    unsigned long long *cnt = &ctx->ctrl->count[CNT_DOLLARS];
    {
        LaunchScope ls_(ctx, PK_PACK, s, (double)N);
        k_pack_count<<<tiles, kPackThreads, 0, s>>>(text, N, tc, &ctx->ctrl->err);
    }
    {
        LaunchScope ls_(ctx, PK_OTHER, s, 0);
        k_scan_small<<<1, 1024, 0, s>>>(tc, tiles, (int64_t *)cnt);
    }
    {
        LaunchScope ls_(ctx, PK_PACK, s, 2.0 * N);
        k_pack_emit<<<tiles, kPackThreads, 0, s>>>(text, N, tc, toff, toff_cap, codes);
    }
    int64_t nwords = dnasa_packed_words(N);
    {
        LaunchScope ls_(ctx, PK_PACK, s, 1.25 * N);
        k_pack_words<<<ceil_div(nwords, 256), 256, 0, s>>>(codes, (const int64_t *)cnt, N, nwords,
                                                          packed);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt, 8, cudaMemcpyDeviceToHost, s));
    DNASA_TRY(check_device_status(ctx, s, "dnasa_pack"));
    int64_t nr = (int64_t)ctx->pinned[0];
    *n_reads = nr;
    if (nr + 1 > toff_cap)
        return fail(ctx, DNASA_CAPACITY, "toff needs n_reads + 1 = " + std::to_string(nr + 1) + " entries");
    return DNASA_OK;
}

}  // namespace dnasa

using namespace dnasa;

extern "C" {

int64_t dnasa_packed_words(int64_t N) { return N <= 0 ? 2 : (N + 31) / 32 + 2; }

int dnasa_create(int device, size_t workspace_cap, dnasa_ctx **out) {
    if (!out) return DNASA_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DNASA_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return DNASA_CUDA_ERROR;
    dnasa_ctx *ctx = new dnasa_ctx();
    ctx->device = device;
    ctx->ws_cap = workspace_cap;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->ctrl, sizeof(DevCtrl)) != cudaSuccess ||
        cudaMemset(ctx->ctrl, 0, sizeof(DevCtrl)) != cudaSuccess ||
        cudaMallocHost(&ctx->pinned, 64 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        dnasa_destroy(ctx);
        return DNASA_OOM;
    }
    *out = ctx;
    return DNASA_OK;
}

void dnasa_destroy(dnasa_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->sa_graph && ctx->sa_graph_free) ctx->sa_graph_free(ctx->sa_graph);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->lb_buf) cudaFree(ctx->lb_buf);
    if (ctx->ctrl) cudaFree(ctx->ctrl);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    for (auto &r : ctx->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
}

const char *dnasa_last_error(dnasa_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

int dnasa_sync_status(dnasa_ctx *ctx, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    return check_device_status(ctx, (cudaStream_t)stream, "dnasa_sync_status");
}

int dnasa_profile(dnasa_ctx *ctx, int enable) {
    if (!ctx) return DNASA_INVALID_ARG;
    for (auto &r : ctx->prof) {
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof.clear();
    ctx->prof_on = enable != 0;
    return DNASA_OK;
}

int dnasa_profile_read(dnasa_ctx *ctx, dnasa_prof_entry *out, int max_entries, int *n_out) {
    if (!ctx || !out || !n_out || max_entries < 0) return DNASA_INVALID_ARG;
    dnasa_prof_entry agg[PK_COUNT];
    for (int k = 0; k < PK_COUNT; ++k) agg[k] = dnasa_prof_entry{k, 0, 0.0, 0.0};
    for (auto &r : ctx->prof) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "dnasa_profile_read");
        agg[r.kind].launches += 1;
        agg[r.kind].ms += ms;
        agg[r.kind].bytes += r.bytes;
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof.clear();
    int n = 0;
    for (int k = 0; k < PK_COUNT && n < max_entries; ++k)
        if (agg[k].launches) out[n++] = agg[k];
    *n_out = n;
    return DNASA_OK;
}

uint64_t dnasa_launch_count(dnasa_ctx *ctx) { return ctx ? ctx->launches : 0; }

int dnasa_get_trace(dnasa_ctx *ctx, dnasa_trace *out) {
    if (!ctx || !out) return DNASA_INVALID_ARG;
    *out = ctx->trace;
    return DNASA_OK;
}

int dnasa_pack(dnasa_ctx *ctx, const uint8_t *text, int64_t N, uint64_t *packed, int64_t *toff,
               int64_t toff_cap, int64_t *n_reads, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (N <= 0 || N >= (int64_t(1) << 31) || !n_reads || toff_cap < 1)
        return fail(ctx, DNASA_INVALID_ARG, "dnasa_pack: bad size or null pointer");
    if (!is_device_ptr(ctx, text) || !is_device_ptr(ctx, packed) || !is_device_ptr(ctx, toff))
        return fail(ctx, DNASA_INVALID_ARG, "dnasa_pack: text, packed and toff must be device pointers");
    cudaSetDevice(ctx->device);
    return pack_impl(ctx, text, N, packed, toff, toff_cap, n_reads, (cudaStream_t)stream);
}

}  // extern "C"
