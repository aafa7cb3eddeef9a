// capi.cu -- the extern "C" entry points of the suffix-array path
// (sa_build, lcp_build, overlap_search, assemble): argument checks, then the
// stream-ordered pipeline.  Intermediate buffers of assemble() come from the
// stream-ordered allocator; each step's scratch comes from the context
// workspace.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace dnasa {

int layout_impl(dnasa_ctx *ctx, const TextDesc &t, int64_t max_reads_per_inst,
                const dnasa_edge *edges, int64_t ne, const uint8_t *contained, uint8_t *contigs,
                int64_t cap, int64_t *contig_off, int64_t off_cap, int64_t *inst_contig_off,
                int64_t *n_contigs, int64_t *needed, cudaStream_t s);

namespace {

int check_text_args(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                    int64_t N, const char *who) {
    if (N <= 0 || N >= (int64_t(1) << 31) || n_reads < 1 || n_reads > N)
        return fail(ctx, DNASA_INVALID_ARG, std::string(who) + ": need 1 <= n_reads <= N < 2^31");
    if (!is_device_ptr(ctx, packed) || !is_device_ptr(ctx, toff))
        return fail(ctx, DNASA_INVALID_ARG, std::string(who) + ": packed and toff must be device pointers");
    return DNASA_OK;
}

TextDesc one_instance(const uint64_t *packed, const int64_t *toff, int64_t n_reads, int64_t N) {
    TextDesc t;
    t.packed = packed;
    t.toff = toff;
    t.n_reads = n_reads;
    t.N = N;
    t.inst_toff = nullptr;
    t.inst_roff = nullptr;
    t.n_inst = 1;
    t.fid = nullptr;
    return t;
}

// SA in the caller's width: int32 writes straight into the caller's buffer,
// int64 goes through a uint32 stage then widens.
struct SaView {
    const uint32_t *sa32 = nullptr;
    uint32_t *owned = nullptr;
};

__global__ void k_narrow(const int64_t *__restrict__ a, int64_t n, uint32_t *__restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (uint32_t)a[i];
}

// A uint32 view of a caller SA (narrowing an int64 SA into a temporary).
int sa_view(dnasa_ctx *ctx, const void *sa, int idx_width, int64_t N, DevBuf &tmp, cudaStream_t s,
            const uint32_t **out) {
    if (idx_width == DNASA_I32) {
        *out = (const uint32_t *)sa;
        return DNASA_OK;
    }
    DNASA_TRY(dev_alloc(ctx, tmp, (size_t)N * 4, s));
    int grid = (int)std::min<int64_t>(ceil_div(N, 256), (int64_t)ctx->num_sms * 16);
    {
        LaunchScope ls_(ctx, PK_OTHER, s, 12.0 * N);
        k_narrow<<<std::max(grid, 1), 256, 0, s>>>((const int64_t *)sa, N, (uint32_t *)tmp.p);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    *out = (const uint32_t *)tmp.p;
    return DNASA_OK;
}

// inst_roff[i] = the fragment that starts at text offset inst_toff[i] (flags an
// instance boundary that is not a fragment start).
__global__ void k_inst_roff(const int64_t *__restrict__ toff, int64_t n_reads,
                            const int64_t *__restrict__ inst_toff, int32_t n_inst,
                            int64_t *__restrict__ inst_roff, uint32_t *err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n_inst;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t x = inst_toff[i];
        int64_t lo = 0, hi = n_reads + 1;     // first r with toff[r] >= x
        while (lo < hi) {
            int64_t m = (lo + hi) >> 1;
            if (toff[m] < x) lo = m + 1; else hi = m;
        }
        if (lo > n_reads || toff[lo] != x) atomicOr(err, DERR_BOUNDS);
        inst_roff[i] = lo;
    }
}

// SA slots of instance i are [inst_toff[i], inst_toff[i+1]); rewrite positions
// in the instance's own coordinates.
__global__ void k_localize(uint32_t *__restrict__ sa, int64_t N, const int64_t *__restrict__ inst_toff,
                           int32_t n_inst) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = upper_index(inst_toff, 0, n_inst, j);
        sa[j] = (uint32_t)((int64_t)sa[j] - __ldg(inst_toff + i));
    }
}

}  // namespace

int dev_alloc(dnasa_ctx *ctx, DevBuf &b, size_t bytes, cudaStream_t s) {
    b.s = s;
    cudaError_t e = cudaMallocAsync(&b.p, std::max<size_t>(bytes, 256), s);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return cuda_fail(ctx, e, "cudaMallocAsync");
    }
    return DNASA_OK;
}

// Device copies of the instance offsets (text and fragment), with checks.
int make_instances(dnasa_ctx *ctx, const int64_t *toff, int64_t n_reads, int64_t N,
                   const int64_t *inst_toff_host, int32_t n_inst, DevBuf &inst_toff, DevBuf &inst_roff,
                   int64_t *max_reads, cudaStream_t s) {
    if (inst_toff_host[0] != 0 || inst_toff_host[n_inst] != N)
        return fail(ctx, DNASA_INVALID_ARG, "batched: inst_off must start at 0 and end at N");
    for (int i = 0; i < n_inst; ++i)
        if (inst_toff_host[i + 1] <= inst_toff_host[i])
            return fail(ctx, DNASA_INVALID_ARG, "batched: inst_off must increase strictly");
    DNASA_TRY(dev_alloc(ctx, inst_toff, (size_t)(n_inst + 1) * 8, s));
    DNASA_TRY(dev_alloc(ctx, inst_roff, (size_t)(n_inst + 1) * 8, s));
    DNASA_CUDA(ctx, cudaMemcpyAsync(inst_toff.p, inst_toff_host, (size_t)(n_inst + 1) * 8,
                                    cudaMemcpyHostToDevice, s));
    {
        LaunchScope ls_(ctx, PK_OTHER, s, 0.0);
        k_inst_roff<<<ceil_div(n_inst + 1, 256), 256, 0, s>>>(toff, n_reads, (const int64_t *)inst_toff.p,
                                                             n_inst, (int64_t *)inst_roff.p, &ctx->ctrl->err);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    std::vector<int64_t> roff((size_t)n_inst + 1);
    DNASA_CUDA(ctx, cudaMemcpyAsync(roff.data(), inst_roff.p, (size_t)(n_inst + 1) * 8,
                                    cudaMemcpyDeviceToHost, s));
    int rc = check_device_status(ctx, s, "batched");
    if (rc != DNASA_OK) return fail(ctx, DNASA_INVALID_ARG, "batched: an instance does not start at a fragment");
    *max_reads = 0;
    for (int i = 0; i < n_inst; ++i) *max_reads = std::max(*max_reads, roff[i + 1] - roff[i]);
    return DNASA_OK;
}

// Whole pipeline on a text already on the device, possibly several instances.
int assemble_impl(dnasa_ctx *ctx, const uint8_t *text, int64_t N, const int64_t *inst_toff_host,
                  int32_t n_inst, int32_t min_overlap, uint8_t *contigs, int64_t cap,
                  int64_t *contig_off, int64_t off_cap, int64_t *inst_contig_off, int64_t *n_contigs,
                  int64_t *needed, const dnasa_opts *opts, cudaStream_t s) {
    DevBuf packed, toff, sa, lcp, contained, edges, inst_toff, inst_roff, fid, isa;
    const int64_t toff_cap = N / 2 + 2;
    DNASA_TRY(dev_alloc(ctx, packed, (size_t)dnasa_packed_words(N) * 8, s));
    DNASA_TRY(dev_alloc(ctx, toff, (size_t)toff_cap * 8, s));
    int64_t n_reads = 0;
    DNASA_TRY(pack_impl(ctx, text, N, (uint64_t *)packed.p, (int64_t *)toff.p, toff_cap, &n_reads, s));
    TextDesc t = one_instance((const uint64_t *)packed.p, (const int64_t *)toff.p, n_reads, N);
    int64_t max_reads = n_reads;
    if (n_inst > 1) {
        DNASA_TRY(make_instances(ctx, (const int64_t *)toff.p, n_reads, N, inst_toff_host, n_inst,
                                 inst_toff, inst_roff, &max_reads, s));
        t.inst_toff = (const int64_t *)inst_toff.p;
        t.inst_roff = (const int64_t *)inst_roff.p;
        t.n_inst = n_inst;
    }
    DNASA_TRY(dev_alloc(ctx, sa, (size_t)N * 4, s));
    DNASA_TRY(dev_alloc(ctx, lcp, (size_t)N * 4, s));
    DNASA_TRY(dev_alloc(ctx, contained, (size_t)n_reads, s));
    DNASA_TRY(dev_alloc(ctx, isa, (size_t)N * 4, s));
    if (n_reads > 1) {   // fragment of every position: one load instead of a binary search
        DNASA_TRY(dev_alloc(ctx, fid, (size_t)N * 4, s));
        DNASA_TRY(fragment_ids(ctx, t, (uint32_t *)fid.p, s));
        t.fid = (const uint32_t *)fid.p;
    }
    DNASA_TRY(sa_build_u32(ctx, t, (uint32_t *)sa.p, opts, s, (uint32_t *)isa.p));
    DNASA_TRY(lcp_build_impl(ctx, t, (const uint32_t *)sa.p, (int32_t *)lcp.p, s,
                             (const uint32_t *)isa.p));
    int64_t ecap = std::max<int64_t>(8 * n_reads, 1024), ne = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (edges.p) { cudaFreeAsync(edges.p, s); edges.p = nullptr; }
        DNASA_TRY(dev_alloc(ctx, edges, (size_t)ecap * sizeof(dnasa_edge), s));
        int rc = overlap_impl(ctx, t, (const uint32_t *)sa.p, (const int32_t *)lcp.p, min_overlap,
                              (dnasa_edge *)edges.p, ecap, &ne, (uint8_t *)contained.p, s,
                              (const uint32_t *)isa.p);
        if (rc == DNASA_CAPACITY && attempt == 0) { ecap = ne + 16; continue; }
        DNASA_TRY(rc);
        break;
    }
    return layout_impl(ctx, t, max_reads, (const dnasa_edge *)edges.p, ne,
                       (const uint8_t *)contained.p, contigs, cap, contig_off, off_cap,
                       inst_contig_off, n_contigs, needed, s);
}

}  // namespace dnasa

using namespace dnasa;

namespace {

int check_sa_opts(dnasa_ctx *ctx, const dnasa_opts *opts, const char *who) {
    if (!opts) return DNASA_OK;
    auto bad = [&](const char *what) { return fail(ctx, DNASA_INVALID_ARG, std::string(who) + ": " + what); };
    if (opts->tile_items != 0 && opts->tile_items != 2048 && opts->tile_items != 3840 && opts->tile_items != 5120)
        return bad("tile_items must be 0, 2048, 3840 or 5120");
    if (opts->reserved0 != 0) return bad("reserved0 must be 0");
    if (opts->lookback != 0 && opts->lookback != 1 && opts->lookback != 8) return bad("lookback must be 0, 1 or 8");
    if (opts->seg_max != 0 && (opts->seg_max < 8 || opts->seg_max > 12288))
        return bad("seg_max must be 0 or in [8, 12288]");
    if (opts->pack_position != 0 && opts->pack_position != -1) return bad("pack_position must be 0 or -1");
    if (opts->builder != 0 && opts->builder != 1) return bad("builder must be 0 (doubling) or 1 (DC3)");
    if (opts->rounds_on_host != 0 && opts->rounds_on_host != 1) return bad("rounds_on_host must be 0 or 1");
    return DNASA_OK;
}

}  // namespace

extern "C" {

int sa_build(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
             int64_t N, void *sa, int idx_width, const dnasa_opts *opts, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    DNASA_TRY(check_text_args(ctx, packed, toff, n_reads, N, "sa_build"));
    if (idx_width != DNASA_I32 && idx_width != DNASA_I64)
        return fail(ctx, DNASA_INVALID_ARG, "sa_build: idx_width must be DNASA_I32 or DNASA_I64");
    if (!is_device_ptr(ctx, sa)) return fail(ctx, DNASA_INVALID_ARG, "sa_build: sa must be a device pointer");
    DNASA_TRY(check_sa_opts(ctx, opts, "sa_build"));
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    TextDesc t = one_instance(packed, toff, n_reads, N);
    if (idx_width == DNASA_I32) return sa_build_u32(ctx, t, (uint32_t *)sa, opts, s);
    DevBuf tmp;
    DNASA_TRY(dev_alloc(ctx, tmp, (size_t)N * 4, s));
    DNASA_TRY(sa_build_u32(ctx, t, (uint32_t *)tmp.p, opts, s));
    return widen_u32_to_i64(ctx, (const uint32_t *)tmp.p, N, (int64_t *)sa, s);
}

int sa_lcp_build(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                 int64_t N, void *sa, int idx_width, int32_t *lcp, const dnasa_opts *opts, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (!is_device_ptr(ctx, lcp)) return fail(ctx, DNASA_INVALID_ARG, "sa_lcp_build: lcp must be a device pointer");
    if (opts && opts->builder == 1) {   // DC3 has no initial keys to read LCPs from
        DNASA_TRY(sa_build(ctx, packed, toff, n_reads, N, sa, idx_width, opts, stream));
        return lcp_build(ctx, packed, toff, n_reads, N, sa, idx_width, lcp, stream);
    }
    // the same argument checks as sa_build, then the build writing round 0's LCPs
    DNASA_TRY(check_text_args(ctx, packed, toff, n_reads, N, "sa_lcp_build"));
    if (idx_width != DNASA_I32 && idx_width != DNASA_I64)
        return fail(ctx, DNASA_INVALID_ARG, "sa_lcp_build: idx_width must be DNASA_I32 or DNASA_I64");
    if (!is_device_ptr(ctx, sa)) return fail(ctx, DNASA_INVALID_ARG, "sa_lcp_build: sa must be a device pointer");
    DNASA_TRY(check_sa_opts(ctx, opts, "sa_lcp_build"));
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const TextDesc t = one_instance(packed, toff, n_reads, N);
    if (idx_width == DNASA_I32) return sa_build_u32(ctx, t, (uint32_t *)sa, opts, s, nullptr, lcp);
    DevBuf tmp;
    DNASA_TRY(dev_alloc(ctx, tmp, (size_t)N * 4, s));
    DNASA_TRY(sa_build_u32(ctx, t, (uint32_t *)tmp.p, opts, s, nullptr, lcp));
    return widen_u32_to_i64(ctx, (const uint32_t *)tmp.p, N, (int64_t *)sa, s);
}

int lcp_build(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
              int64_t N, const void *sa, int idx_width, int32_t *lcp, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    DNASA_TRY(check_text_args(ctx, packed, toff, n_reads, N, "lcp_build"));
    if (idx_width != DNASA_I32 && idx_width != DNASA_I64)
        return fail(ctx, DNASA_INVALID_ARG, "lcp_build: bad idx_width");
    if (!is_device_ptr(ctx, sa) || !is_device_ptr(ctx, lcp))
        return fail(ctx, DNASA_INVALID_ARG, "lcp_build: sa and lcp must be device pointers");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf tmp;
    const uint32_t *sa32;
    DNASA_TRY(sa_view(ctx, sa, idx_width, N, tmp, s, &sa32));
    return lcp_build_impl(ctx, one_instance(packed, toff, n_reads, N), sa32, lcp, s);
}

int overlap_search(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                   int64_t N, const void *sa, const int32_t *lcp, int idx_width,
                   int32_t min_overlap, dnasa_edge *edges, int64_t cap, int64_t *n_edges,
                   uint8_t *contained, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    DNASA_TRY(check_text_args(ctx, packed, toff, n_reads, N, "overlap_search"));
    if (idx_width != DNASA_I32 && idx_width != DNASA_I64)
        return fail(ctx, DNASA_INVALID_ARG, "overlap_search: bad idx_width");
    if (min_overlap < 1 || !n_edges || cap < 0)
        return fail(ctx, DNASA_INVALID_ARG, "overlap_search: min_overlap >= 1, n_edges and cap >= 0 required");
    if (!is_device_ptr(ctx, sa) || !is_device_ptr(ctx, lcp) || !is_device_ptr(ctx, contained) ||
        (cap > 0 && !is_device_ptr(ctx, edges)))
        return fail(ctx, DNASA_INVALID_ARG, "overlap_search: sa, lcp, edges, contained must be device pointers");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf tmp;
    const uint32_t *sa32;
    DNASA_TRY(sa_view(ctx, sa, idx_width, N, tmp, s, &sa32));
    return overlap_impl(ctx, one_instance(packed, toff, n_reads, N), sa32, lcp, min_overlap, edges,
                        cap, n_edges, contained, s);
}

int assemble(dnasa_ctx *ctx, const uint8_t *text, int64_t N, int32_t min_overlap,
             uint8_t *contigs, int64_t cap, int64_t *contig_off, int64_t off_cap,
             int64_t *n_contigs, int64_t *needed, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (N <= 0 || N >= (int64_t(1) << 31) || min_overlap < 1 || !n_contigs || !needed ||
        cap < 0 || off_cap < 1)
        return fail(ctx, DNASA_INVALID_ARG, "assemble: bad size, min_overlap or null output");
    if (!is_device_ptr(ctx, text) || !is_device_ptr(ctx, contig_off) ||
        (cap > 0 && !is_device_ptr(ctx, contigs)))
        return fail(ctx, DNASA_INVALID_ARG, "assemble: text, contigs and contig_off must be device pointers");
    cudaSetDevice(ctx->device);
    return assemble_impl(ctx, text, N, nullptr, 1, min_overlap, contigs, cap, contig_off, off_cap,
                         nullptr, n_contigs, needed, nullptr, (cudaStream_t)stream);
}

int sa_build_batched(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                     int64_t N, const int64_t *inst_off, int32_t n_inst, int32_t *sa,
                     const dnasa_opts *opts, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    DNASA_TRY(check_text_args(ctx, packed, toff, n_reads, N, "sa_build_batched"));
    if (n_inst < 1 || !inst_off) return fail(ctx, DNASA_INVALID_ARG, "sa_build_batched: n_inst >= 1 and inst_off required");
    if (!is_device_ptr(ctx, sa)) return fail(ctx, DNASA_INVALID_ARG, "sa_build_batched: sa must be a device pointer");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    TextDesc t = one_instance(packed, toff, n_reads, N);
    DevBuf inst_toff, inst_roff;
    if (n_inst > 1) {
        int64_t max_reads;
        DNASA_TRY(make_instances(ctx, toff, n_reads, N, inst_off, n_inst, inst_toff, inst_roff, &max_reads, s));
        t.inst_toff = (const int64_t *)inst_toff.p;
        t.inst_roff = (const int64_t *)inst_roff.p;
        t.n_inst = n_inst;
    }
    DNASA_TRY(sa_build_u32(ctx, t, (uint32_t *)sa, opts, s));
    if (n_inst > 1) {
        int grid = (int)std::min<int64_t>(ceil_div(N, 256), (int64_t)ctx->num_sms * 16);
        LaunchScope ls_(ctx, PK_OTHER, s, 8.0 * N);
        k_localize<<<std::max(grid, 1), 256, 0, s>>>((uint32_t *)sa, N, t.inst_toff, n_inst);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}

int assemble_batched(dnasa_ctx *ctx, const uint8_t *texts, const int64_t *inst_off, int32_t n_inst,
                     int32_t min_overlap, const dnasa_opts *opts, uint8_t *contigs, int64_t cap,
                     int64_t *contig_off, int64_t off_cap, int64_t *inst_contig_off,
                     int64_t *n_contigs, int64_t *needed, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (n_inst < 1 || !inst_off) return fail(ctx, DNASA_INVALID_ARG, "assemble_batched: n_inst >= 1 and inst_off required");
    const int64_t N = inst_off[n_inst];
    if (N <= 0 || N >= (int64_t(1) << 31) || min_overlap < 1 || !n_contigs || !needed || cap < 0 ||
        off_cap < 1)
        return fail(ctx, DNASA_INVALID_ARG, "assemble_batched: bad size, min_overlap or null output");
    if (!is_device_ptr(ctx, texts) || !is_device_ptr(ctx, contig_off) ||
        (cap > 0 && !is_device_ptr(ctx, contigs)) ||
        (inst_contig_off && !is_device_ptr(ctx, inst_contig_off)))
        return fail(ctx, DNASA_INVALID_ARG, "assemble_batched: texts, contigs, contig_off and "
                                            "inst_contig_off must be device pointers");
    cudaSetDevice(ctx->device);
    return assemble_impl(ctx, texts, N, inst_off, n_inst, min_overlap, contigs, cap, contig_off,
                         off_cap, inst_contig_off, n_contigs, needed, opts, (cudaStream_t)stream);
}

int dnasa_autotune(dnasa_ctx *ctx, const uint64_t *packed, const int64_t *toff, int64_t n_reads,
                   int64_t N, const int64_t *inst_off, int32_t n_inst, const char *cache_path,
                   dnasa_opts *best, double *best_ms, void *stream) {
    if (!ctx || !best) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    DNASA_TRY(check_text_args(ctx, packed, toff, n_reads, N, "dnasa_autotune"));
    if (n_inst < 1 || (n_inst > 1 && !inst_off))
        return fail(ctx, DNASA_INVALID_ARG, "dnasa_autotune: n_inst >= 1 (and inst_off when > 1)");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaDeviceProp prop;
    DNASA_CUDA(ctx, cudaGetDeviceProperties(&prop, ctx->device));
    char key[320];
    snprintf(key, sizeof key, "%s|n%d|i%d", prop.name, bits_for((uint64_t)N),
             bits_for((uint64_t)n_inst));
    if (cache_path) {   // one line per key: key \t tile \t finish \t lookback \t ms
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof line, f)) {
                char *tab = strchr(line, '\t');
                if (!tab || (size_t)(tab - line) != strlen(key) || strncmp(line, key, strlen(key))) continue;
                int tile, lb, sm;
                long long fin;
                double ms;
                if (sscanf(tab + 1, "%d\t%lld\t%d\t%d\t%lf", &tile, &fin, &lb, &sm, &ms) == 5) {
                    *best = dnasa_opts{};
                    best->tile_items = tile;
                    best->finish_threshold = fin;
                    best->lookback = lb;
                    best->seg_max = sm;
                    if (best_ms) *best_ms = ms;
                    fclose(f);
                    return DNASA_OK;
                }
            }
            fclose(f);
        }
    }
    TextDesc t = one_instance(packed, toff, n_reads, N);
    DevBuf inst_toff, inst_roff, sa;
    if (n_inst > 1) {
        int64_t max_reads;
        DNASA_TRY(make_instances(ctx, toff, n_reads, N, inst_off, n_inst, inst_toff, inst_roff, &max_reads, s));
        t.inst_toff = (const int64_t *)inst_toff.p;
        t.inst_roff = (const int64_t *)inst_roff.p;
        t.n_inst = n_inst;
    }
    DNASA_TRY(dev_alloc(ctx, sa, (size_t)N * 4, s));
    cudaEvent_t e0, e1;
    DNASA_CUDA(ctx, cudaEventCreate(&e0));
    DNASA_CUDA(ctx, cudaEventCreate(&e1));
    dnasa_opts warm{};
    int rc = sa_build_u32(ctx, t, (uint32_t *)sa.p, &warm, s);   // also sizes the workspace
    auto time_once = [&](const dnasa_opts &o, float *ms) -> int {
        cudaEventRecord(e0, s);
        int r = sa_build_u32(ctx, t, (uint32_t *)sa.p, &o, s);
        cudaEventRecord(e1, s);
        if (r != DNASA_OK) return r;
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(ms, e0, e1);
        return DNASA_OK;
    };
    // every candidate once, then the four fastest three more times each: the
    // choice is the best median of three, not one noisy sample
    struct Cand { dnasa_opts o; float ms; };
    std::vector<Cand> cands;
    const int tiles[3] = {2048, 3840, 5120};
    const int64_t fins[4] = {-1, std::max<int64_t>(N / 64, 1), std::max<int64_t>(N / 8, 1), N};
    const int segs[3] = {256, 2048, 12288};
    for (int ti = 0; ti < 3 && rc == DNASA_OK; ++ti) {
        for (int fi = 0; fi < 4 * 3 && rc == DNASA_OK; ++fi) {
            dnasa_opts o{};
            o.tile_items = tiles[ti];
            o.finish_threshold = fins[fi % 4];
            o.seg_max = segs[fi / 4];
            o.lookback = 8;
            float ms = 0.f;
            rc = time_once(o, &ms);
            if (rc == DNASA_OK) cands.push_back({o, ms});
        }
    }
    std::sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.ms < b.ms; });
    double bms = 1e30;
    dnasa_opts bopt{};
    for (size_t c = 0; c < std::min<size_t>(cands.size(), 4) && rc == DNASA_OK; ++c) {
        float r3[3];
        for (int k = 0; k < 3 && rc == DNASA_OK; ++k) rc = time_once(cands[c].o, &r3[k]);
        if (rc != DNASA_OK) break;
        std::sort(r3, r3 + 3);
        if (r3[1] < bms) {
            bms = r3[1];
            bopt = cands[c].o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    DNASA_TRY(rc);
    *best = bopt;
    if (best_ms) *best_ms = bms;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s\t%d\t%lld\t%d\t%d\t%.4f\n", key, bopt.tile_items,
                    (long long)bopt.finish_threshold, bopt.lookback, bopt.seg_max, bms);
            fclose(f);
        }
    }
    return DNASA_OK;
}

}  // extern "C"

