// dc3.cu -- suffix array by the difference-cover (skew, DC3) algorithm of
// Kaerkkaeinen and Sanders, the construction the paper's GPU kernel is named
// after (Sec. IV, "cudaDC3RS"), with its radix sorts on the onesweep passes of
// radix.cu.
//
// One level on a string s[0..n) over [1, K] (three zeros appended):
//   1. the sample: the positions i mod 3 != 0 (plus position n when n mod 3 == 1),
//      radix sorted by their triples (s[i], s[i+1], s[i+2]);
//   2. each sample position named by the rank of its triple; if two triples are
//      equal, the names, mod-1 positions first then mod-2, form the string of the
//      next level, whose suffix array orders the sample;
//   3. the mod-0 positions: ordered by (s[i], rank of i+1) -- the order of the
//      mod-1 sample positions, then a stable radix pass on s[i];
//   4. the two ordered lists merged: a mod-0 suffix against a mod-1 one compares
//      (s[i], rank of i+1); against a mod-2 one (s[i], s[i+1], rank of i+2) --
//      the ranks those comparisons need are always sample ranks.
// The merge is a merge path: each thread finds where its run of outputs starts
// by binary search on its diagonal, then merges its run sequentially.
//
// Level 0 is the fragment text with every '$' its own symbol, ordered by
// position and smaller than A < C < G < T ('$' of fragment r -> r + 1, base b ->
// n_reads + 1 + b), so the suffix order is exactly the one sa_build produces.
#include <algorithm>
#include <cstring>
#include <vector>

#include "block.cuh"
#include "common.cuh"

namespace dnasa {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kMergeRun = 64;   // outputs per thread of the merge (one diagonal search per run)

inline int grid_for(dnasa_ctx *ctx, int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), threads),
                                                      (int64_t)ctx->num_sms * 16));
}

// Level-0 symbols from the packed text: the '$' of fragment r -> r + 1, base b
// -> n_reads + 1 + b; three zeros after the end.
__global__ void k_dc3_symbols(TextDesc t, uint32_t *__restrict__ s) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < t.N + 3;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= t.N) { s[i] = 0u; continue; }
        const int64_t r = frag_of(t, i);
        if (i == __ldg(t.toff + r + 1) - 1) {
            s[i] = (uint32_t)r + 1u;
        } else {
            const uint64_t b = (uint64_t)(i - r);
            const uint32_t code = (uint32_t)(__ldg(t.packed + (b >> 5)) >> (62 - 2 * (b & 31))) & 3u;
            s[i] = (uint32_t)t.n_reads + 1u + code;
        }
    }
}

// isa[sa[j]] = j
__global__ void k_dc3_inverse(const uint32_t *__restrict__ sa, int64_t n, uint32_t *__restrict__ isa) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        isa[sa[j]] = (uint32_t)j;
}

__device__ __forceinline__ uint32_t sample_pos(int64_t t, int64_t n0) {
    return t < n0 ? (uint32_t)(3 * t + 1) : (uint32_t)(3 * (t - n0) + 2);
}

// Keys for one pass of the triple sort: the whole triple when it fits a word
// (sh = bits per symbol, c = -1), else symbol s[i + c] of the sample position
// already in vals (c = 2, 1, 0 in turn).
__global__ void k_dc3_keys(const uint32_t *__restrict__ s, int64_t n02, int64_t n0, int sh, int c,
                           const uint32_t *__restrict__ pos_in, unsigned long long *__restrict__ keys,
                           uint32_t *__restrict__ vals) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n02;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = pos_in ? pos_in[t] : sample_pos(t, n0);
        if (c < 0)
            keys[t] = ((unsigned long long)s[i] << (2 * sh)) | ((unsigned long long)s[i + 1] << sh) |
                      (unsigned long long)s[i + 2];
        else
            keys[t] = (unsigned long long)s[i + c];
        vals[t] = i;
    }
}

// flag[j] = 1 when the triple of sorted sample position P[j] differs from P[j-1]'s.
__global__ void k_dc3_newname(const uint32_t *__restrict__ s, const uint32_t *__restrict__ P, int64_t n02,
                              uint32_t *__restrict__ flag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n02;
         j += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f = 1u;
        if (j > 0) {
            const uint32_t a = P[j - 1], b = P[j];
            f = (s[a] != s[b] || s[a + 1] != s[b + 1] || s[a + 2] != s[b + 2]) ? 1u : 0u;
        }
        flag[j] = f;
    }
}

// Tile sums of x, for the inclusive scan.
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const uint32_t *__restrict__ x, int64_t n,
                                                           uint64_t *__restrict__ sums) {
    __shared__ uint64_t tmp[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint64_t v = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t i = base + threadIdx.x + q * kScanThreads;
        if (i < n) v += x[i];
    }
    uint64_t tot;
    block_exclusive_sum<kScanThreads>(v, tmp, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of the tile sums (one block, loops over the tiles).
__global__ void __launch_bounds__(1024) k_scan_sums(uint64_t *__restrict__ sums, int64_t tiles) {
    __shared__ uint64_t tmp[1024 / 32 + 1];
    uint64_t run = 0;
    for (int64_t b0 = 0; b0 < tiles; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const uint64_t v = i < tiles ? sums[i] : 0ull;
        uint64_t tot;
        const uint64_t ex = block_exclusive_sum<1024>(v, tmp, &tot);
        if (i < tiles) sums[i] = run + ex;
        run += tot;
    }
}

// Inclusive scan within each tile plus the tile's offset; x scanned in place.
__global__ void __launch_bounds__(kScanThreads) k_tile_apply(uint32_t *__restrict__ x, int64_t n,
                                                            const uint64_t *__restrict__ sums) {
    __shared__ uint64_t tmp[kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint64_t local = 0;
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t i = base + q;
        v[q] = i < n ? x[i] : 0u;
        local += v[q];
    }
    uint64_t tot;
    uint64_t run = block_exclusive_sum<kScanThreads>(local, tmp, &tot) + sums[blockIdx.x];
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t i = base + q;
        run += v[q];
        if (i < n) x[i] = (uint32_t)run;
    }
}

// s12[index of sample position P[j]] = name[j]  (mod-1 positions first).
__global__ void k_dc3_s12(const uint32_t *__restrict__ P, const uint32_t *__restrict__ name, int64_t n02,
                          int64_t n0, uint32_t *__restrict__ s12) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n02;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = P[j];
        const int64_t idx = (i % 3u == 1u) ? (int64_t)(i / 3u) : (int64_t)(i / 3u) + n0;
        s12[idx] = name[j];
    }
    if (blockIdx.x == 0 && threadIdx.x < 3) s12[n02 + threadIdx.x] = 0u;
}

// Unique names: SA12[name - 1] = t.
__global__ void k_dc3_direct(const uint32_t *__restrict__ s12, int64_t n02, uint32_t *__restrict__ SA12) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n02;
         t += (int64_t)gridDim.x * blockDim.x)
        SA12[s12[t] - 1u] = (uint32_t)t;
}

// Ranks from the next level's suffix array: s12[SA12[j]] = j + 1.
__global__ void k_dc3_ranks(const uint32_t *__restrict__ SA12, int64_t n02, uint32_t *__restrict__ s12) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n02;
         j += (int64_t)gridDim.x * blockDim.x)
        s12[SA12[j]] = (uint32_t)(j + 1);
}

// The mod-0 positions in the order of their mod-1 successors: 3 * SA12[t] for
// SA12[t] < n0, written in order (keys for the stable pass on s[i]).
__global__ void k_dc3_flag0(const uint32_t *__restrict__ SA12, int64_t n02, int64_t n0,
                            uint8_t *__restrict__ flags) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n02;
         t += (int64_t)gridDim.x * blockDim.x)
        flags[t] = SA12[t] < (uint32_t)n0 ? 1 : 0;
}

__global__ void k_dc3_keys0(const uint32_t *__restrict__ s, const uint32_t *__restrict__ SA12,
                            const uint32_t *__restrict__ idx, const unsigned long long *__restrict__ cnt,
                            unsigned long long *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t m = (int64_t)*cnt;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < m;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = 3u * SA12[idx[p]];
        keys[p] = s[i];
        vals[p] = i;
    }
}

struct MergeArgs {
    const uint32_t *s, *s12, *SA0, *SA12;
    int64_t n0, n02, m0, m12;    // m12 = sample entries after the skipped dummy
    int64_t skip;                // 1 when SA12[0] is the dummy (n mod 3 == 1)
    uint32_t *SA;
    int64_t n;
};

// Position of the suffix at entry t of the sample order.
__device__ __forceinline__ uint32_t pos12(const MergeArgs &M, int64_t t) {
    const uint32_t v = M.SA12[t + M.skip];
    return v < (uint32_t)M.n0 ? 3u * v + 1u : 3u * (v - (uint32_t)M.n0) + 2u;
}

// Is the sample suffix at entry t smaller than the mod-0 suffix at entry p?
__device__ __forceinline__ bool sample_less(const MergeArgs &M, int64_t t, int64_t p) {
    const uint32_t v = M.SA12[t + M.skip];
    const uint32_t j = M.SA0[p];
    if (v < (uint32_t)M.n0) {   // mod 1: (s[i], rank(i+1)) against (s[j], rank(j+1))
        const uint32_t i = 3u * v + 1u;
        const uint32_t a0 = M.s[i], b0 = M.s[j];
        if (a0 != b0) return a0 < b0;
        return M.s12[v + M.n0] < M.s12[j / 3u];
    }
    const uint32_t i = 3u * (v - (uint32_t)M.n0) + 2u;   // mod 2: one more symbol, rank(i+2)
    const uint32_t a0 = M.s[i], b0 = M.s[j];
    if (a0 != b0) return a0 < b0;
    const uint32_t a1 = M.s[i + 1], b1 = M.s[j + 1];
    if (a1 != b1) return a1 < b1;
    return M.s12[v - (uint32_t)M.n0 + 1u] < M.s12[j / 3u + (uint32_t)M.n0];
}

// Merge path: thread k writes outputs [k * run, (k + 1) * run).  Among the first
// d outputs, a come from the mod-0 list: the largest a with the mod-0 entry a - 1
// smaller than the sample entry d - a.
__global__ void k_dc3_merge(MergeArgs M) {
    const int64_t total = M.m0 + M.m12;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k * kMergeRun < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = k * kMergeRun;
        int64_t lo = max((int64_t)0, d - M.m12), hi = min(d, M.m0);
        while (lo < hi) {
            const int64_t a = (lo + hi + 1) >> 1;   // is mod-0 entry a-1 before sample entry d-a?
            if (!sample_less(M, d - a, a - 1)) lo = a; else hi = a - 1;
        }
        int64_t a = lo, b = d - lo;
        const int64_t e = min(total, d + kMergeRun);
        for (int64_t o = d; o < e; ++o) {
            bool take0;
            if (a >= M.m0) take0 = false;
            else if (b >= M.m12) take0 = true;
            else take0 = !sample_less(M, b, a);
            M.SA[o] = take0 ? M.SA0[a++] : pos12(M, b++);
        }
    }
}

// s = n + 3 symbols in [1, K] (three zeros after), SA = n entries.
int dc3_level(dnasa_ctx *ctx, const uint32_t *s, int64_t n, uint64_t K, uint32_t *SA, cudaStream_t st,
              int depth, int *max_depth) {
    *max_depth = std::max(*max_depth, depth);
    if (depth > 60) return fail(ctx, DNASA_CUDA_ERROR, "dc3: recursion did not end");
    if (n == 1) {
        DNASA_CUDA(ctx, cudaMemsetAsync(SA, 0, 4, st));
        return DNASA_OK;
    }
    const int64_t n0 = (n + 2) / 3, n1 = (n + 1) / 3, n2 = n / 3, n02 = n0 + n2;
    const int tile = radix_tile_default();
    DevBuf kb0, kb1, vb0, vb1, s12b, SA12b, flagb, hist, scanb, SA0b, idxb;
    DNASA_TRY(dev_alloc(ctx, kb0, (size_t)n02 * 8, st));
    DNASA_TRY(dev_alloc(ctx, kb1, (size_t)n02 * 8, st));
    DNASA_TRY(dev_alloc(ctx, vb0, (size_t)n02 * 4, st));
    DNASA_TRY(dev_alloc(ctx, vb1, (size_t)n02 * 4, st));
    DNASA_TRY(dev_alloc(ctx, hist, 8 * 256 * 4 + 256, st));
    RadixScratch rs;
    rs.hist = (uint32_t *)hist.p;
    unsigned long long *keys[2] = {(unsigned long long *)kb0.p, (unsigned long long *)kb1.p};
    uint32_t *vals[2] = {(uint32_t *)vb0.p, (uint32_t *)vb1.p};
    const int sh = bits_for(K);
    int cur = 0;
    // ---- 1. sample positions sorted by their triples
    if (3 * sh <= 64) {
        {
            LaunchScope ls_(ctx, PK_INIT, st, 24.0 * n02);
            k_dc3_keys<<<grid_for(ctx, n02), 256, 0, st>>>(s, n02, n0, sh, -1, nullptr, keys[0], vals[0]);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs, keys, vals, n02, nullptr, 3 * sh, false, tile,
                                                       &cur, st));
    } else {
        for (int c = 2; c >= 0; --c) {   // least significant symbol first, each pass stable
            uint32_t *in = c == 2 ? nullptr : vals[cur];
            unsigned long long *kk[2] = {keys[0], keys[1]};
            uint32_t *vv[2] = {vals[cur ^ 1], vals[cur]};
            {
                LaunchScope ls_(ctx, PK_INIT, st, 16.0 * n02);
                k_dc3_keys<<<grid_for(ctx, n02), 256, 0, st>>>(s, n02, n0, sh, c, in, kk[0], vv[0]);
            }
            DNASA_CUDA(ctx, cudaGetLastError());
            int w = 0;
            DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs, kk, vv, n02, nullptr, sh, false, tile, &w, st));
            cur = (vv[w] == vals[0]) ? 0 : 1;
        }
    }
    const uint32_t *P = vals[cur];
    // ---- 2. names, then the sample order (recursion when names repeat)
    uint32_t *name = vals[cur ^ 1];
    const int64_t tiles = ceil_div(n02, kScanTile);
    DNASA_TRY(dev_alloc(ctx, scanb, (size_t)(tiles + 1) * 8, st));
    {
        LaunchScope ls_(ctx, PK_RERANK, st, 20.0 * n02);
        k_dc3_newname<<<grid_for(ctx, n02), 256, 0, st>>>(s, P, n02, name);
    }
    {
        LaunchScope ls_(ctx, PK_RERANK, st, 8.0 * n02);
        k_tile_sums<<<(int)tiles, kScanThreads, 0, st>>>(name, n02, (uint64_t *)scanb.p);
        k_scan_sums<<<1, 1024, 0, st>>>((uint64_t *)scanb.p, tiles);
        k_tile_apply<<<(int)tiles, kScanThreads, 0, st>>>(name, n02, (const uint64_t *)scanb.p);
    }
    DNASA_TRY(dev_alloc(ctx, s12b, (size_t)(n02 + 3) * 4, st));
    DNASA_TRY(dev_alloc(ctx, SA12b, (size_t)(n02 + 3) * 4, st));
    uint32_t *s12 = (uint32_t *)s12b.p, *SA12 = (uint32_t *)SA12b.p;
    {
        LaunchScope ls_(ctx, PK_RERANK, st, 12.0 * n02);
        k_dc3_s12<<<grid_for(ctx, n02), 256, 0, st>>>(P, name, n02, n0, s12);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    uint32_t names = 0;
    DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, name + n02 - 1, 4, cudaMemcpyDeviceToHost, st));
    DNASA_TRY(check_device_status(ctx, st, "dc3"));
    names = *(volatile uint32_t *)ctx->pinned;
    if ((int64_t)names < n02) {
        DNASA_TRY(dc3_level(ctx, s12, n02, names, SA12, st, depth + 1, max_depth));
        LaunchScope ls_(ctx, PK_APPLY, st, 8.0 * n02);
        k_dc3_ranks<<<grid_for(ctx, n02), 256, 0, st>>>(SA12, n02, s12);
    } else {
        LaunchScope ls_(ctx, PK_APPLY, st, 8.0 * n02);
        k_dc3_direct<<<grid_for(ctx, n02), 256, 0, st>>>(s12, n02, SA12);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    // ---- 3. mod-0 positions: in the order of their successors, then by s[i]
    DNASA_TRY(dev_alloc(ctx, flagb, (size_t)n02, st));
    DNASA_TRY(dev_alloc(ctx, idxb, (size_t)n02 * 4, st));
    {
        LaunchScope ls_(ctx, PK_GATHER, st, 5.0 * n02);
        k_dc3_flag0<<<grid_for(ctx, n02), 256, 0, st>>>(SA12, n02, n0, (uint8_t *)flagb.p);
    }
    DNASA_TRY(ws_reserve(ctx, compact_scratch_bytes(n02) + 4096, st));
    {
        Arena a = ws_arena(ctx);
        DNASA_TRY(compact_flags(ctx, a, (const uint8_t *)flagb.p, n02, (uint32_t *)idxb.p,
                                ctx->ctrl->count + CNT_TMP, st));
    }
    {
        LaunchScope ls_(ctx, PK_GATHER, st, 20.0 * n0);
        k_dc3_keys0<<<grid_for(ctx, n0), 256, 0, st>>>(s, SA12, (const uint32_t *)idxb.p,
                                                       ctx->ctrl->count + CNT_TMP, keys[0], vals[0]);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    int w0 = 0;
    DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs, keys, vals, n0, nullptr, sh, false, tile, &w0, st));
    const uint32_t *SA0 = vals[w0];
    // ---- 4. merge
    MergeArgs M;
    M.s = s;
    M.s12 = s12;
    M.SA0 = SA0;
    M.SA12 = SA12;
    M.n0 = n0;
    M.n02 = n02;
    M.skip = n0 > n1 ? 1 : 0;
    M.m0 = n0;
    M.m12 = n02 - M.skip;
    M.SA = SA;
    M.n = n;
    {
        LaunchScope ls_(ctx, PK_SEGSORT, st, 16.0 * n);
        k_dc3_merge<<<grid_for(ctx, ceil_div(n, kMergeRun), 128), 128, 0, st>>>(M);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    (void)n2;
    return DNASA_OK;
}

}  // namespace

// x[i] = x[0] + ... + x[i] in place (n uint32 values, sums below 2^32).
int scan_inclusive_u32(dnasa_ctx *ctx, uint32_t *x, int64_t n, cudaStream_t st) {
    if (n <= 0) return DNASA_OK;
    const int64_t tiles = ceil_div(n, kScanTile);
    DevBuf sums;
    DNASA_TRY(dev_alloc(ctx, sums, (size_t)(tiles + 1) * 8, st));
    LaunchScope ls_(ctx, PK_OTHER, st, 8.0 * n);
    k_tile_sums<<<(int)tiles, kScanThreads, 0, st>>>(x, n, (uint64_t *)sums.p);
    k_scan_sums<<<1, 1024, 0, st>>>((uint64_t *)sums.p, tiles);
    k_tile_apply<<<(int)tiles, kScanThreads, 0, st>>>(x, n, (const uint64_t *)sums.p);
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}

// Suffix array of the packed text by DC3 (one instance); isa_out (may be null)
// receives the inverse.
int sa_build_dc3(dnasa_ctx *ctx, const TextDesc &t, uint32_t *sa32, cudaStream_t st, uint32_t *isa_out) {
    PhaseRange nvtx_("dnasa.sa_dc3");
    const int64_t N = t.N;
    if (t.n_inst > 1) return fail(ctx, DNASA_INVALID_ARG, "sa_build: the DC3 builder takes one instance");
    DevBuf sb;
    DNASA_TRY(dev_alloc(ctx, sb, (size_t)(N + 3) * 4, st));
    {
        LaunchScope ls_(ctx, PK_INIT, st, 4.0 * N);
        k_dc3_symbols<<<grid_for(ctx, N + 3), 256, 0, st>>>(t, (uint32_t *)sb.p);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    int depth = 0;
    DNASA_TRY(dc3_level(ctx, (const uint32_t *)sb.p, N, (uint64_t)t.n_reads + 4, sa32, st, 0, &depth));
    if (isa_out) {
        LaunchScope ls_(ctx, PK_OTHER, st, 8.0 * N);
        k_dc3_inverse<<<grid_for(ctx, N), 256, 0, st>>>(sa32, N, isa_out);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    dnasa_trace &tr = ctx->trace;
    memset(&tr, 0, sizeof(tr));
    tr.rounds = depth;   // recursion levels below the text
    tr.h0 = 1;
    return check_device_status(ctx, st, "dc3");
}

}  // namespace dnasa
