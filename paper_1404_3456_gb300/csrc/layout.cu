// layout.cu -- greedy layout of the overlap graph and spelling of contigs.
//
// Sec. III turns the fragments into a weighted directed graph (Fig. 3) whose
// maximal path spells the reconstructed sequence, and concatenates the chosen
// fragments into RS.  The choice here is greedy: edges between non-contained
// fragments in order of (L desc, j asc, k asc) -- a radix sort -- and (j, k) is
// taken when j has no successor yet, k no predecessor yet, and they lie on
// different chains (union-find).  This acceptance is sequential by definition,
// so one thread runs it per instance (instances run in parallel); spelling the
// contigs is parallel, one warp per fragment.
#include <algorithm>

#include "common.cuh"

namespace dnasa {

namespace {

__device__ __forceinline__ int64_t frag_len(const int64_t *__restrict__ toff, int64_t r) {
    return __ldg(toff + r + 1) - 1 - __ldg(toff + r);
}

__device__ __forceinline__ int64_t inst_of_read(const TextDesc &t, int64_t r) {
    return t.n_inst > 1 ? upper_index(t.inst_roff, 0, t.n_inst, r) : 0;
}

__device__ __forceinline__ int64_t inst_r0(const TextDesc &t, int64_t inst) {
    return t.n_inst > 1 ? __ldg(t.inst_roff + inst) : 0;
}

__global__ void k_edge_filter(const dnasa_edge *__restrict__ edges, int64_t ne,
                              const uint8_t *__restrict__ contained, uint8_t *__restrict__ flags) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
         e += (int64_t)gridDim.x * blockDim.x) {
        dnasa_edge ed = edges[e];
        flags[e] = !contained[ed.j] && !contained[ed.k];
    }
}

// key = [instance | lmask - L | j local | k local]
__global__ void k_edge_keys(TextDesc t, const dnasa_edge *__restrict__ edges,
                            const uint32_t *__restrict__ idx, const unsigned long long *d_count,
                            int kbl, int lb, unsigned long long *__restrict__ keys) {
    const int64_t n = (int64_t)*d_count;
    const unsigned long long lmask = (1ull << lb) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        dnasa_edge ed = edges[idx[e]];
        int64_t inst = inst_of_read(t, ed.j);
        int64_t r0 = inst_r0(t, inst);
        keys[e] = ((unsigned long long)inst << (lb + 2 * kbl)) |
                  ((lmask - (unsigned long long)ed.L) << (2 * kbl)) |
                  ((unsigned long long)(ed.j - r0) << kbl) | (unsigned long long)(ed.k - r0);
    }
}

struct LayoutArrays {
    int32_t *succ, *succL, *pred, *parent, *skip, *chead;
    int64_t *out_off;            // per fragment: byte offset inside its instance, or -1
    int64_t *inst_bytes, *inst_contigs;
};

__device__ int32_t uf_find(int32_t *parent, int32_t x) {
    while (parent[x] != x) {
        int32_t g = parent[parent[x]];
        parent[x] = g;
        x = g;
    }
    return x;
}

// One CTA per instance.  The acceptance is sequential (each decision depends on
// the ones before), so one thread makes it, but against successor /
// predecessor / union-find arrays in shared memory (instances of up to
// kGreedyMaxReads fragments; larger ones use the global arrays), with the
// instance's sorted edges staged into shared memory in chunks by the whole CTA.
constexpr int kGreedyMaxReads = 4096;
constexpr int kGreedyChunk = 2048;
constexpr int kGreedyThreads = 128;
constexpr size_t kGreedySmem = (size_t)kGreedyMaxReads * 4 * 4 + (size_t)kGreedyChunk * 8;

__global__ void __launch_bounds__(kGreedyThreads) k_greedy(TextDesc t,
                                                          const unsigned long long *__restrict__ keys,
                                                          int64_t ne, int kbl, int lb,
                                                          const uint8_t *__restrict__ contained,
                                                          LayoutArrays A) {
    extern __shared__ __align__(16) unsigned char gsm[];
    unsigned long long *ebuf = reinterpret_cast<unsigned long long *>(gsm);
    int32_t *s_succ = reinterpret_cast<int32_t *>(ebuf + kGreedyChunk);
    int32_t *s_pred = s_succ + kGreedyMaxReads;
    int32_t *s_succL = s_pred + kGreedyMaxReads;
    int32_t *s_parent = s_succL + kGreedyMaxReads;
    __shared__ int64_t s_range[2];
    const unsigned long long lmask = (1ull << lb) - 1ull;
    const unsigned long long kmask = (1ull << kbl) - 1ull;
    const int shift = lb + 2 * kbl;
    for (int64_t inst = blockIdx.x; inst < t.n_inst; inst += gridDim.x) {
        const int64_t r0 = inst_r0(t, inst);
        const int64_t r1 = t.n_inst > 1 ? __ldg(t.inst_roff + inst + 1) : t.n_reads;
        const int64_t nr = r1 - r0;
        const bool fast = nr <= kGreedyMaxReads;
        int32_t *succ = fast ? s_succ : A.succ + r0;       // indexed by local fragment number
        int32_t *pred = fast ? s_pred : A.pred + r0;
        int32_t *succL = fast ? s_succL : A.succL + r0;
        int32_t *parent = fast ? s_parent : A.parent + r0;
        for (int64_t i = threadIdx.x; i < nr; i += kGreedyThreads) {
            succ[i] = -1; pred[i] = -1; succL[i] = 0; parent[i] = (int32_t)i;
            A.out_off[r0 + i] = -1; A.skip[r0 + i] = 0; A.chead[r0 + i] = -1;
        }
        if (threadIdx.x == 0) {   // this instance's edges: keys whose instance field == inst
            const unsigned long long kinst = (unsigned long long)inst;
            int64_t lo = 0, hi = ne;
            while (lo < hi) {
                int64_t m = (lo + hi) >> 1;
                if ((keys[m] >> shift) < kinst) lo = m + 1; else hi = m;
            }
            int64_t e = lo;
            hi = ne;
            while (e < hi) {
                int64_t m = (e + hi) >> 1;
                if ((keys[m] >> shift) <= kinst) e = m + 1; else hi = m;
            }
            s_range[0] = lo;
            s_range[1] = e;
        }
        __syncthreads();
        const int64_t e0 = s_range[0], e1 = s_range[1];
        for (int64_t c0 = e0; c0 < e1; c0 += kGreedyChunk) {
            const int len = (int)min((int64_t)kGreedyChunk, e1 - c0);
            for (int i = threadIdx.x; i < len; i += kGreedyThreads) ebuf[i] = keys[c0 + i];
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int i = 0; i < len; ++i) {
                    const unsigned long long key = ebuf[i];
                    const int32_t L = (int32_t)(lmask - ((key >> (2 * kbl)) & lmask));
                    const int32_t j = (int32_t)((key >> kbl) & kmask);
                    const int32_t k = (int32_t)(key & kmask);
                    if (succ[j] != -1 || pred[k] != -1) continue;
                    const int32_t a = uf_find(parent, j), b = uf_find(parent, k);
                    if (a == b) continue;
                    succ[j] = k; succL[j] = L; pred[k] = j; parent[a] = b;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {   // chains in ascending head order: output offsets
            int64_t bytes = 0, nc = 0;
            for (int64_t r = 0; r < nr; ++r) {
                if (contained[r0 + r] || pred[r] != -1) continue;
                A.chead[r0 + r] = (int32_t)nc;
                int64_t cur = r;
                int32_t sk = 0;
                for (;;) {
                    A.out_off[r0 + cur] = bytes;
                    A.skip[r0 + cur] = sk;
                    bytes += frag_len(t.toff, r0 + cur) - sk;
                    if (succ[cur] == -1) break;
                    sk = succL[cur];
                    cur = succ[cur];
                }
                ++nc;
            }
            A.inst_bytes[inst] = bytes;
            A.inst_contigs[inst] = nc;
        }
        __syncthreads();
    }
}

__global__ void k_contig_off(TextDesc t, LayoutArrays A, const int64_t *__restrict__ byte_base,
                             const int64_t *__restrict__ contig_base, int64_t *__restrict__ contig_off,
                             int64_t *__restrict__ inst_contig_off, const int64_t *total_bytes,
                             const int64_t *total_contigs) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < t.n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = A.chead[r];
        if (c < 0) continue;
        int64_t inst = inst_of_read(t, r);
        contig_off[contig_base[inst] + c] = byte_base[inst] + A.out_off[r];
    }
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) contig_off[*total_contigs] = *total_bytes;
    if (inst_contig_off) {
        for (int64_t i = tid; i <= t.n_inst; i += (int64_t)gridDim.x * blockDim.x)
            inst_contig_off[i] = i < t.n_inst ? contig_base[i] : *total_contigs;
    }
}

__global__ void k_spell(TextDesc t, LayoutArrays A, const int64_t *__restrict__ byte_base,
                        uint8_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < t.n_reads;
         r += nwarps) {
        int64_t o = A.out_off[r];
        if (o < 0) continue;
        int64_t inst = inst_of_read(t, r);
        int64_t dst = byte_base[inst] + o;
        int64_t len = frag_len(t.toff, r);
        int64_t sk = A.skip[r];
        uint64_t b0 = (uint64_t)(__ldg(t.toff + r) - r);
        for (int64_t x = sk + lane; x < len; x += 32) {
            uint64_t b = b0 + (uint64_t)x;
            uint32_t code = (uint32_t)(__ldg(t.packed + (b >> 5)) >> (62 - 2 * (b & 31))) & 3u;
            out[dst + x - sk] = "ACGT"[code];
        }
    }
}

__global__ void k_scan_two(int64_t *a, int64_t *b, int64_t n, int64_t *ta, int64_t *tb) {
    // exclusive scans of a and b (n small: one thread each; instances are few thousand)
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int64_t i = 0; i < n; ++i) { int64_t v = a[i]; a[i] = run; run += v; }
        *ta = run;
    } else if (threadIdx.x == 32) {
        int64_t run = 0;
        for (int64_t i = 0; i < n; ++i) { int64_t v = b[i]; b[i] = run; run += v; }
        *tb = run;
    }
}

__global__ void k_max_len(TextDesc t, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < t.n_reads;
         r += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)frag_len(t.toff, r));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

inline int grid_for(dnasa_ctx *ctx, int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), threads),
                                                      (int64_t)ctx->num_sms * 16));
}

}  // namespace

// max_reads_per_inst: largest fragment count of one instance (host known).
int layout_impl(dnasa_ctx *ctx, const TextDesc &t, int64_t max_reads_per_inst,
                const dnasa_edge *edges, int64_t ne, const uint8_t *contained, uint8_t *contigs,
                int64_t cap, int64_t *contig_off, int64_t off_cap, int64_t *inst_contig_off,
                int64_t *n_contigs, int64_t *needed, cudaStream_t s) {
    PhaseRange nvtx_("dnasa.layout");
    const int64_t nr = t.n_reads;
    const int kbl = bits_for((uint64_t)std::max<int64_t>(max_reads_per_inst - 1, 1));
    const int ib = t.n_inst > 1 ? bits_for((uint64_t)(t.n_inst - 1)) : 0;
    // an overlap L is shorter than the longest fragment
    unsigned long long *cnt = ctx->ctrl->count;
    DNASA_CUDA(ctx, cudaMemsetAsync(cnt + CNT_TMP, 0, 8, s));
    {
        LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
        k_max_len<<<grid_for(ctx, nr), 256, 0, s>>>(t, cnt + CNT_TMP);
    }
    DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_TMP, 8, cudaMemcpyDeviceToHost, s));
    DNASA_TRY(check_device_status(ctx, s, "assemble/layout"));
    const int lb = bits_for((uint64_t)ctx->pinned[0]);
    if (ib + lb + 2 * kbl > 64)
        return fail(ctx, DNASA_INVALID_ARG, "layout: instance/fragment counts too large for a 64-bit key");
    const int tile = radix_tile_default();
    size_t need = 0;
    auto add = [&](size_t bytes) { need += (bytes + 255) & ~size_t(255); };
    const int64_t nemax = std::max<int64_t>(ne, 1);
    add((size_t)nemax);                     // flags
    add((size_t)nemax * 4);                 // idx
    add((size_t)nemax * 8); add((size_t)nemax * 8);   // keys x2
    add(compact_scratch_bytes(nemax));
    add(radix_scratch_bytes(nemax, 64, tile));
    for (int i = 0; i < 6; ++i) add((size_t)nr * 4);
    add((size_t)nr * 8);
    for (int i = 0; i < 2; ++i) add((size_t)(t.n_inst + 1) * 8);
    add(64);
    DNASA_TRY(ws_reserve(ctx, need + 8192, s));
    Arena a = ws_arena(ctx);
    uint8_t *flags = a.take<uint8_t>((size_t)nemax);
    uint32_t *idx = a.take<uint32_t>((size_t)nemax);
    unsigned long long *keys[2] = {a.take<unsigned long long>((size_t)nemax),
                                   a.take<unsigned long long>((size_t)nemax)};
    LayoutArrays A;
    A.succ = a.take<int32_t>((size_t)nr); A.succL = a.take<int32_t>((size_t)nr);
    A.pred = a.take<int32_t>((size_t)nr); A.parent = a.take<int32_t>((size_t)nr);
    A.skip = a.take<int32_t>((size_t)nr); A.chead = a.take<int32_t>((size_t)nr);
    A.out_off = a.take<int64_t>((size_t)nr);
    A.inst_bytes = a.take<int64_t>((size_t)t.n_inst + 1);
    A.inst_contigs = a.take<int64_t>((size_t)t.n_inst + 1);
    int64_t *totals = a.take<int64_t>(8);
    RadixScratch rs = radix_scratch_take(a, nemax, 64, tile);
    if (!rs.hist || !totals) return fail(ctx, DNASA_OOM, "layout workspace");

    int64_t nsel = 0;
    int which = 0;
    if (ne > 0) {
        {
            LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
            k_edge_filter<<<grid_for(ctx, ne), 256, 0, s>>>(edges, ne, contained, flags);
        }
        DNASA_TRY(compact_flags(ctx, a, flags, ne, idx, cnt + CNT_TMP, s));
        {
            LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
            k_edge_keys<<<grid_for(ctx, ne), 256, 0, s>>>(t, edges, idx, cnt + CNT_TMP, kbl, lb, keys[0]);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_TMP, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "assemble/layout"));
        nsel = (int64_t)ctx->pinned[0];
        if (nsel > 0) {
            uint32_t *nov[2] = {nullptr, nullptr};
            DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs, keys, nov, nsel, nullptr,
                                                           ib + lb + 2 * kbl, false, tile, &which, s));
        }
    }
    DNASA_CUDA(ctx, smem_attr(k_greedy, kGreedySmem));   // once per (kernel, device)
    {
        LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
        int g = (int)std::min<int64_t>(t.n_inst, (int64_t)ctx->num_sms * 8);
        k_greedy<<<std::max(g, 1), kGreedyThreads, kGreedySmem, s>>>(t, keys[which], nsel, kbl, lb,
                                                                    contained, A);
    }
    {
        LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
        k_scan_two<<<1, 64, 0, s>>>(A.inst_bytes, A.inst_contigs, t.n_inst, totals, totals + 1);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, totals, 16, cudaMemcpyDeviceToHost, s));
    DNASA_TRY(check_device_status(ctx, s, "assemble/layout"));
    const int64_t tb = (int64_t)ctx->pinned[0], tc = (int64_t)ctx->pinned[1];
    *needed = tb;
    *n_contigs = tc;
    if (tb > cap || tc + 1 > off_cap)
        return fail(ctx, DNASA_CAPACITY, "assemble: contigs need " + std::to_string(tb) + " bytes and " +
                                             std::to_string(tc + 1) + " offsets");
    {
        LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
        k_contig_off<<<grid_for(ctx, nr), 256, 0, s>>>(t, A, A.inst_bytes, A.inst_contigs, contig_off,
                                                      inst_contig_off, totals, totals + 1);
    }
    {
        LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
        k_spell<<<grid_for(ctx, nr * 32), 256, 0, s>>>(t, A, A.inst_bytes, contigs);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    return check_device_status(ctx, s, "assemble/layout");
}

}  // namespace dnasa
