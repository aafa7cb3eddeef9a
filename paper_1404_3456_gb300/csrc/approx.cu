// approx.cu -- overlaps under the paper's DEFINITION (Sec. III): fragments
// read on either strand, with a rate mu of errors.
//
// The definition asks that every fragment A lie within mu * |A| of a piece of
// the result, read as A or as its reverse complement.  Here errors are
// substitutions (Hamming distance) and the overlap relation follows: oriented
// fragments a, b (2r = fragment r, 2r + 1 = its reverse complement when both
// strands are indexed) overlap by L when the last L bases of a and the first L
// of b differ in at most floor(L * mu) places; the largest such L per ordered
// pair is kept (min_overlap <= L < both lengths).
//
// Search (Sec. IV: the suffix array answers prefix queries; here it also finds
// the exact pieces an approximate overlap must contain):
//   1. the text of oriented fragments (each fragment, then its reverse
//      complement), packed, with its suffix array and LCP;
//   2. seed length s = the shortest exact run that every admissible overlap
//      must contain: L bases with at most e mismatches hold a run of at least
//      ceil((L - e) / (e + 1)) equal bases (pigeonhole), minimised over L;
//   3. every pair of suffixes in one LCP interval of depth >= s whose exact
//      match cannot be extended to the left (the run starts at a fragment start
//      or right after a mismatch) names a diagonal (a, b, d): b starting d
//      bases into a; candidates radix sorted and made unique;
//   4. each diagonal verified with XOR + population count over packed words
//      (a base differs when either of its two bits differs), up to the allowed
//      count; accepted overlaps radix sorted by (a, b, L desc), the first per
//      pair kept.
// Every admissible overlap contains such a left-maximal run of length >= s on
// its diagonal, so the set equals the definition's; the work for a repeat
// family of g copies is g^2 pairs per shared position.
#include <algorithm>

#include "common.cuh"

namespace dnasa {

namespace {

__device__ __forceinline__ int64_t alen(const int64_t *__restrict__ toff, int64_t r) {
    return __ldg(toff + r + 1) - 1 - __ldg(toff + r);
}

__device__ __forceinline__ uint8_t comp_base(uint8_t c) {
    return c == 'A' ? 'T' : c == 'C' ? 'G' : c == 'G' ? 'C' : 'A';
}

// One warp per fragment r: the fragment, '$', its reverse complement, '$',
// at 2 * toff[r] of the oriented text.
__global__ void k_orient(const uint8_t *__restrict__ text, const int64_t *__restrict__ toff,
                         int64_t nr, uint8_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nr; r += nw) {
        const int64_t a = __ldg(toff + r), len = alen(toff, r);
        uint8_t *o = out + 2 * a;
        for (int64_t i = lane; i < len; i += 32) {
            const uint8_t c = text[a + i];
            o[i] = c;
            o[len + 1 + (len - 1 - i)] = comp_base(c);
        }
        if (lane == 0) {
            o[len] = '$';
            o[2 * len + 1] = '$';
        }
    }
}

struct SeedArgs {
    const uint32_t *sa, *fid;
    const int32_t *lcp;
    const int64_t *toff;
    const uint64_t *packed;
    int64_t N;
    int s;               // seed length
    int rc;              // 1: oriented fragments 2r, 2r+1 share fragment r
    int kb, db;          // bits of an oriented fragment index and of a diagonal
    unsigned long long *cand;
    unsigned long long cap;
    unsigned long long *count;
};

// Base i (0..3) of the packed text at base coordinate b.
__device__ __forceinline__ uint32_t base_at(const uint64_t *__restrict__ packed, uint64_t b) {
    return (uint32_t)(__ldg(packed + (b >> 5)) >> (62 - 2 * (b & 31))) & 3u;
}

// The diagonals named by the left-maximal pairs (j, j'), j' > j, of the LCP
// interval (depth >= s) that starts below slot j.
template <typename F>
__device__ __forceinline__ void seed_pairs(const SeedArgs &A, int64_t j, F emit) {
    if (j + 1 >= A.N || __ldg(A.lcp + j + 1) < A.s) return;
    const int64_t p = A.sa[j];
    const int64_t a = __ldg(A.fid + p);
    const int64_t op = p - __ldg(A.toff + a);
    const uint32_t left_p = op > 0 ? base_at(A.packed, (uint64_t)(p - 1 - a)) : 4u;
    for (int64_t jj = j + 1; jj < A.N && __ldg(A.lcp + jj) >= A.s; ++jj) {
        const int64_t q = A.sa[jj];
        const int64_t b = __ldg(A.fid + q);
        if ((A.rc ? (a >> 1) : a) == (A.rc ? (b >> 1) : b)) continue;   // same fragment
        const int64_t oq = q - __ldg(A.toff + b);
        if (op > 0 && oq > 0 && base_at(A.packed, (uint64_t)(q - 1 - b)) == left_p) continue;
        if (op > oq) emit(a, b, op - oq);        // b starts op - oq bases into a
        else if (oq > op) emit(b, a, oq - op);
    }
}

__global__ void __launch_bounds__(256) k_seeds(SeedArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < A.N; base += stride) {
        const int64_t j = base + lane;
        uint32_t c = 0;
        if (j < A.N) seed_pairs(A, j, [&](int64_t, int64_t, int64_t) { ++c; });
        uint32_t inc = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        unsigned long long at = 0;
        if (lane == 31 && inc) at = atomicAdd(A.count, (unsigned long long)inc);
        at = __shfl_sync(0xffffffffu, at, 31) + (inc - c);
        if (c) {
            seed_pairs(A, j, [&](int64_t x, int64_t y, int64_t d) {
                if (at < A.cap)
                    A.cand[at] = ((unsigned long long)x << (A.kb + A.db)) |
                                 ((unsigned long long)y << A.db) | (unsigned long long)d;
                ++at;
            });
        }
    }
}

__global__ void k_first_of_run(const unsigned long long *__restrict__ keys, int64_t n, int shift,
                               uint8_t *__restrict__ flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = i == 0 || (keys[i] >> shift) != (keys[i - 1] >> shift);
}

struct VerifyArgs {
    const unsigned long long *cand;
    const uint32_t *idx;
    const unsigned long long *n_unique;
    const int64_t *toff;
    const uint64_t *packed;
    int32_t lmin, mu_num, mu_den;
    int kb, db, lb;
    unsigned long long *acc;     // (a << (kb + lb)) | (b << lb) | (lmask - L)
    uint32_t *acc_mm;
    unsigned long long *n_acc;
};

// Mismatching bases between the L bases at base coordinates x and y, counting
// at most until `stop` is passed.
__device__ __forceinline__ int64_t mismatches(const uint64_t *__restrict__ packed, uint64_t x, uint64_t y,
                                              int64_t L, int64_t stop) {
    int64_t mm = 0;
    for (int64_t i = 0; i < L && mm <= stop; i += 32) {
        uint64_t d = bases32(packed, x + i) ^ bases32(packed, y + i);
        d = (d | (d >> 1)) & 0x5555555555555555ull;          // one bit per differing base
        if (L - i < 32) d &= ~0ull << (2 * (32 - (L - i)));   // bases past the overlap
        mm += __popcll(d);
    }
    return mm;
}

__global__ void k_verify(VerifyArgs V) {
    const int64_t n = (int64_t)*V.n_unique;
    const unsigned long long dmask = (1ull << V.db) - 1ull, kmask = (1ull << V.kb) - 1ull;
    const unsigned long long lmask = (1ull << V.lb) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = V.cand[V.idx[e]];
        const int64_t a = (int64_t)(key >> (V.kb + V.db)), b = (int64_t)((key >> V.db) & kmask);
        const int64_t d = (int64_t)(key & dmask);
        const int64_t la = alen(V.toff, a), lb = alen(V.toff, b);
        const int64_t L = la - d;
        if (L < V.lmin || L >= lb || d < 1) continue;
        const int64_t allow = L * (int64_t)V.mu_num / V.mu_den;
        const int64_t mm = mismatches(V.packed, (uint64_t)(__ldg(V.toff + a) - a + d),
                                      (uint64_t)(__ldg(V.toff + b) - b), L, allow);
        if (mm > allow) continue;
        const unsigned long long at = atomicAdd(V.n_acc, 1ull);
        V.acc[at] = ((unsigned long long)a << (V.kb + V.lb)) | ((unsigned long long)b << V.lb) |
                    (lmask - (unsigned long long)L);
        V.acc_mm[at] = (uint32_t)mm;
    }
}

__global__ void k_emit_aedges(const unsigned long long *__restrict__ acc, const uint32_t *__restrict__ mm,
                              const uint32_t *__restrict__ idx, const unsigned long long *n_edges, int kb,
                              int lb, dnasa_aedge *__restrict__ out, int64_t cap) {
    const int64_t n = (int64_t)*n_edges;
    const unsigned long long lmask = (1ull << lb) - 1ull, kmask = (1ull << kb) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n && e < cap;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[e];
        const unsigned long long k = acc[i];
        dnasa_aedge ed;
        ed.a = (int32_t)(k >> (kb + lb));
        ed.b = (int32_t)((k >> lb) & kmask);
        ed.L = (int32_t)(lmask - (k & lmask));
        ed.mismatches = (int32_t)mm[i];
        out[e] = ed;
    }
}

__global__ void k_amax_len(const int64_t *__restrict__ toff, int64_t nr, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)alen(toff, r));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

inline int grid_for(dnasa_ctx *ctx, int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), threads),
                                                      (int64_t)ctx->num_sms * 16));
}

}  // namespace

// Shortest exact run every admissible overlap of length L in [lmin, max_len)
// contains: with e = floor(L * num / den) allowed mismatches, ceil((L - e) / (e + 1)).
int approx_seed_length(int64_t lmin, int64_t max_len, int32_t num, int32_t den) {
    int64_t s = INT32_MAX;
    for (int64_t L = lmin; L < max_len; ++L) {
        const int64_t e = L * num / den;
        const int64_t run = L / (e + 1);   // = ceil((L - e) / (e + 1))
        s = std::min(s, run);
    }
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, INT32_MAX));
}

int overlap_approx_impl(dnasa_ctx *ctx, const uint8_t *text, int64_t N, int32_t lmin, int32_t mu_num,
                        int32_t mu_den, int rc, dnasa_aedge *edges, int64_t cap, int64_t *n_edges,
                        int64_t *n_oriented, cudaStream_t s) {
    PhaseRange nvtx_("dnasa.overlap_approx");
    // ---- oriented text: each fragment followed by its reverse complement
    DevBuf packed0, toff0, text2, packed, toff, sa, isa, lcp, fid;
    const int64_t toff_cap = N / 2 + 2;
    int64_t nr = 0;
    const uint8_t *T = text;
    int64_t N2 = N;
    if (rc) {
        DNASA_TRY(dev_alloc(ctx, packed0, (size_t)dnasa_packed_words(N) * 8, s));
        DNASA_TRY(dev_alloc(ctx, toff0, (size_t)toff_cap * 8, s));
        DNASA_TRY(pack_impl(ctx, text, N, (uint64_t *)packed0.p, (int64_t *)toff0.p, toff_cap, &nr, s));
        N2 = 2 * N;
        if (N2 >= (int64_t(1) << 31)) return fail(ctx, DNASA_INVALID_ARG, "overlap_search_approx: text too large");
        DNASA_TRY(dev_alloc(ctx, text2, (size_t)N2, s));
        {
            LaunchScope ls_(ctx, PK_PACK, s, 3.0 * N);
            k_orient<<<grid_for(ctx, 32 * nr), 256, 0, s>>>(text, (const int64_t *)toff0.p, nr,
                                                           (uint8_t *)text2.p);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        T = (const uint8_t *)text2.p;
    }
    const int64_t toff2_cap = N2 / 2 + 2;
    DNASA_TRY(dev_alloc(ctx, packed, (size_t)dnasa_packed_words(N2) * 8, s));
    DNASA_TRY(dev_alloc(ctx, toff, (size_t)toff2_cap * 8, s));
    int64_t m = 0;
    DNASA_TRY(pack_impl(ctx, T, N2, (uint64_t *)packed.p, (int64_t *)toff.p, toff2_cap, &m, s));
    *n_oriented = m;
    TextDesc t;
    t.packed = (const uint64_t *)packed.p;
    t.toff = (const int64_t *)toff.p;
    t.n_reads = m;
    t.N = N2;
    t.inst_toff = nullptr;
    t.inst_roff = nullptr;
    t.n_inst = 1;
    t.fid = nullptr;
    DNASA_TRY(dev_alloc(ctx, fid, (size_t)N2 * 4, s));
    DNASA_TRY(fragment_ids(ctx, t, (uint32_t *)fid.p, s));
    t.fid = (const uint32_t *)fid.p;
    DNASA_TRY(dev_alloc(ctx, sa, (size_t)N2 * 4, s));
    DNASA_TRY(dev_alloc(ctx, isa, (size_t)N2 * 4, s));
    DNASA_TRY(dev_alloc(ctx, lcp, (size_t)N2 * 4, s));
    DNASA_TRY(sa_build_u32(ctx, t, (uint32_t *)sa.p, nullptr, s, (uint32_t *)isa.p));
    DNASA_TRY(lcp_build_impl(ctx, t, (const uint32_t *)sa.p, (int32_t *)lcp.p, s, (const uint32_t *)isa.p));

    unsigned long long *cnt = ctx->ctrl->count;
    DNASA_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 8, s));
    {
        LaunchScope ls_(ctx, PK_OVERLAP, s, 8.0 * m);
        k_amax_len<<<grid_for(ctx, m), 256, 0, s>>>(t.toff, m, cnt + CNT_TMP);
    }
    DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_TMP, 8, cudaMemcpyDeviceToHost, s));
    DNASA_TRY(check_device_status(ctx, s, "overlap_search_approx"));
    const int64_t max_len = (int64_t)ctx->pinned[0];
    const int kb = bits_for((uint64_t)std::max<int64_t>(m - 1, 1));
    const int db = bits_for((uint64_t)std::max<int64_t>(max_len, 1));
    const int lb = db;
    if (2 * kb + db > 64)
        return fail(ctx, DNASA_INVALID_ARG, "overlap_search_approx: fragments too many or too long");
    *n_edges = 0;
    if (max_len <= lmin) return DNASA_OK;   // no fragment can overlap by min_overlap
    const int seed = approx_seed_length(lmin, max_len, mu_num, mu_den);
    const int tile = radix_tile_default();

    int64_t ccap = std::max<int64_t>(8 * m, 1 << 16);
    for (int attempt = 0; attempt < 2; ++attempt) {
        size_t need = 0;
        auto add = [&](size_t bytes) { need += (bytes + 255) & ~size_t(255); };
        add((size_t)ccap * 8); add((size_t)ccap * 8);     // candidates x2
        add((size_t)ccap); add((size_t)ccap * 4);         // first-of-run flags, unique index
        add((size_t)ccap * 8); add((size_t)ccap * 8);     // accepted keys x2
        add((size_t)ccap * 4); add((size_t)ccap * 4);     // accepted mismatch counts x2
        add((size_t)ccap); add((size_t)ccap * 4);         // flags, index of the accepted
        add(compact_scratch_bytes(ccap) * 2);
        add(radix_scratch_bytes(ccap, 64, tile) * 2);
        DNASA_TRY(ws_reserve(ctx, need + 16384, s));
        Arena a = ws_arena(ctx);
        unsigned long long *ck[2] = {a.take<unsigned long long>((size_t)ccap),
                                     a.take<unsigned long long>((size_t)ccap)};
        uint8_t *flags = a.take<uint8_t>((size_t)ccap);
        uint32_t *uidx = a.take<uint32_t>((size_t)ccap);
        unsigned long long *ak[2] = {a.take<unsigned long long>((size_t)ccap),
                                     a.take<unsigned long long>((size_t)ccap)};
        uint32_t *am[2] = {a.take<uint32_t>((size_t)ccap), a.take<uint32_t>((size_t)ccap)};
        uint8_t *aflags = a.take<uint8_t>((size_t)ccap);
        uint32_t *aidx = a.take<uint32_t>((size_t)ccap);
        RadixScratch rs1 = radix_scratch_take(a, ccap, 64, tile);
        RadixScratch rs2 = radix_scratch_take(a, ccap, 64, tile);
        if (!rs2.hist) return fail(ctx, DNASA_OOM, "overlap_search_approx workspace");
        DNASA_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 8, s));
        SeedArgs A;
        A.sa = (const uint32_t *)sa.p;
        A.fid = t.fid;
        A.lcp = (const int32_t *)lcp.p;
        A.toff = t.toff;
        A.packed = t.packed;
        A.N = N2;
        A.s = seed;
        A.rc = rc;
        A.kb = kb;
        A.db = db;
        A.cand = ck[0];
        A.cap = (unsigned long long)ccap;
        A.count = cnt + CNT_CAND;
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 8.0 * N2);
            k_seeds<<<grid_for(ctx, N2), 256, 0, s>>>(A);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_CAND, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "overlap_search_approx"));
        const int64_t nc = (int64_t)ctx->pinned[0];
        if (nc > ccap) {
            if (attempt == 1) return fail(ctx, DNASA_CUDA_ERROR, "overlap_search_approx: seed count changed");
            ccap = nc + nc / 8 + 1024;
            continue;
        }
        if (nc == 0) return DNASA_OK;
        int w1 = 0;
        uint32_t *nov[2] = {nullptr, nullptr};
        DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs1, ck, nov, nc, nullptr, 2 * kb + db, false,
                                                       tile, &w1, s));
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 9.0 * nc);
            k_first_of_run<<<grid_for(ctx, nc), 256, 0, s>>>(ck[w1], nc, 0, flags);
        }
        Arena rest = a;
        DNASA_TRY(compact_flags(ctx, rest, flags, nc, uidx, cnt + CNT_TMP, s));
        VerifyArgs V;
        V.cand = ck[w1];
        V.idx = uidx;
        V.n_unique = cnt + CNT_TMP;
        V.toff = t.toff;
        V.packed = t.packed;
        V.lmin = lmin;
        V.mu_num = mu_num;
        V.mu_den = mu_den;
        V.kb = kb;
        V.db = db;
        V.lb = lb;
        V.acc = ak[0];
        V.acc_mm = am[0];
        V.n_acc = cnt + CNT_EDGES;
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 16.0 * nc);
            k_verify<<<grid_for(ctx, nc), 256, 0, s>>>(V);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_EDGES, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "overlap_search_approx"));
        const int64_t na = (int64_t)ctx->pinned[0];
        if (na == 0) return DNASA_OK;
        int w2 = 0;
        DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs2, ak, am, na, nullptr, 2 * kb + lb, false,
                                                       tile, &w2, s));
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 9.0 * na);
            k_first_of_run<<<grid_for(ctx, na), 256, 0, s>>>(ak[w2], na, lb, aflags);
        }
        Arena rest2 = a;
        DNASA_TRY(compact_flags(ctx, rest2, aflags, na, aidx, cnt + CNT_EDGES + 1, s));
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 28.0 * na);
            k_emit_aedges<<<grid_for(ctx, na), 256, 0, s>>>(ak[w2], am[w2], aidx, cnt + CNT_EDGES + 1, kb,
                                                           lb, edges, cap);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_EDGES + 1, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "overlap_search_approx"));
        *n_edges = (int64_t)ctx->pinned[0];
        if (*n_edges > cap)
            return fail(ctx, DNASA_CAPACITY, "overlap_search_approx: " + std::to_string(*n_edges) +
                                                 " edges exceed cap " + std::to_string(cap));
        return DNASA_OK;
    }
    return DNASA_OK;
}

}  // namespace dnasa

using namespace dnasa;

extern "C" int overlap_search_approx(dnasa_ctx *ctx, const uint8_t *text, int64_t N, int32_t min_overlap,
                                     int32_t mu_num, int32_t mu_den, int32_t both_strands,
                                     dnasa_aedge *edges, int64_t cap, int64_t *n_edges,
                                     int64_t *n_oriented, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (N <= 0 || N >= (int64_t(1) << 31) || min_overlap < 1 || mu_num < 0 || mu_den < 1 ||
        mu_num >= mu_den || cap < 0 || !n_edges || !n_oriented || (both_strands != 0 && both_strands != 1))
        return fail(ctx, DNASA_INVALID_ARG, "overlap_search_approx: bad size, min_overlap, mu or output");
    if (!is_device_ptr(ctx, text) || (cap > 0 && !is_device_ptr(ctx, edges)))
        return fail(ctx, DNASA_INVALID_ARG, "overlap_search_approx: text and edges must be device pointers");
    cudaSetDevice(ctx->device);
    return overlap_approx_impl(ctx, text, N, min_overlap, mu_num, mu_den, both_strands, edges, cap, n_edges,
                               n_oriented, (cudaStream_t)stream);
}
