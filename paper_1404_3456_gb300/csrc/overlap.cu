// overlap.cu -- suffix-array driven overlap search and containment.
//
// Sec. III reconstructs the sequence from "fir" relations: fragment D_k is a
// prefix of another fragment, or the remainder of a cut fragment is the
// prefix of the next one -- i.e. a suffix of one fragment equals a prefix of
// another.  Sec. IV answers these questions (is X the beginning of some fragment?) by
// searching the suffix array.  Here every suffix X = r_j[o..] (o >= 1,
// |X| >= min_overlap) is a query:
//   * R = the fragment-start suffixes in SA order (a subsequence of the SA),
//     with LCP_R[k] = common prefix of R[k-1] and R[k];
//   * the fragments having X as a prefix are exactly the fragment starts that
//     follow X's own SA slot within X's LCP interval (X ends in its '$', which
//     sorts before any base); the first candidate's index in R is the number of
//     fragment starts at smaller SA slots (Sec. IV's binary search of X among
//     the fragments, answered for every slot at once by one prefix count over
//     the SA), checked by one direct packed-word comparison, and the rest are
//     read off LCP_R while it stays >= |X|.
// Candidates (j, k, L) are radix sorted by (j, k, L desc) and reduced to the
// largest L per ordered pair.  Containment of fragment k: some other suffix
// shares all |r_k| bases with r_k's start suffix (the SA neighbour just before
// it, or a later neighbour that is not an identical fragment of larger index).
#include <algorithm>

#include "common.cuh"

namespace dnasa {

namespace {

__device__ __forceinline__ int64_t frag_len(const int64_t *__restrict__ toff, int64_t r) {
    return __ldg(toff + r + 1) - 1 - __ldg(toff + r);
}

// Equal bases at the start of base coordinates ba and bb, at most maxlen.
__device__ __forceinline__ int64_t common_bases(const uint64_t *__restrict__ packed, uint64_t ba,
                                                uint64_t bb, int64_t maxlen) {
    int64_t h = 0;
    while (h < maxlen) {
        uint64_t d = bases32(packed, ba + h) ^ bases32(packed, bb + h);
        if (d) return min(h + (int64_t)(__clzll((long long)d) >> 1), maxlen);
        h += 32;
    }
    return maxlen;
}

__global__ void k_isa(const uint32_t *__restrict__ sa, int64_t N, uint32_t *__restrict__ isa) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x)
        isa[sa[j]] = (uint32_t)j;
}

__global__ void k_read_keys(TextDesc t, const uint32_t *__restrict__ isa, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ val, unsigned long long *maxlen) {
    unsigned long long m = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < t.n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        key[r] = isa[__ldg(t.toff + r)];
        val[r] = (uint32_t)r;
        m = max(m, (unsigned long long)frag_len(t.toff, r));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxlen, m);
}

__device__ __forceinline__ int64_t inst_of_read(const TextDesc &t, int64_t r) {
    return t.n_inst > 1 ? upper_index(t.inst_roff, 0, t.n_inst, r) : 0;
}

__global__ void k_lcp_r(TextDesc t, const uint32_t *__restrict__ R, int32_t *__restrict__ lcpr) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < t.n_reads;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (k == 0) { lcpr[0] = 0; continue; }
        int64_t a = R[k - 1], b = R[k];
        if (t.n_inst > 1 && inst_of_read(t, a) != inst_of_read(t, b)) { lcpr[k] = 0; continue; }
        int64_t m = min(frag_len(t.toff, a), frag_len(t.toff, b));
        lcpr[k] = (int32_t)common_bases(t.packed, (uint64_t)(__ldg(t.toff + a) - a),
                                        (uint64_t)(__ldg(t.toff + b) - b), m);
    }
}

// flag[s] = 1 when the suffix at SA slot s starts a fragment (then scanned).
__global__ void k_startflag(TextDesc t, const uint32_t *__restrict__ sa, uint32_t *__restrict__ flag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < t.N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = sa[j];
        flag[j] = p == __ldg(t.toff + frag_of(t, p)) ? 1u : 0u;
    }
}

struct QueryArgs {
    const uint32_t *isa, *Rslot, *R;
    const uint32_t *nstart;           // [N]: fragment-start suffixes at SA slots <= s
    const int32_t *lcpr;
    const uint2 *rrange;              // per fragment: its instance's range in R (batches)
    int32_t lmin;
    int kb, lb;                       // bits of k and of L in a candidate key
    unsigned long long *cand;
    unsigned long long cap;
    unsigned long long *count;
};

// X = r_j[q - toff[j] ..]: the first fragment start at or after X's own SA slot
// within X's instance (binary search of the slot among R's slots), checked by
// one packed-word comparison.  Returns false when q is no query or the first
// candidate does not start with X.
struct QueryHit {
    int j, L, lo, ri1;
};
__device__ __forceinline__ bool query_locate(const TextDesc &t, const QueryArgs &a, int64_t q,
                                             QueryHit &h) {
    const int64_t j = frag_of(t, q);
    const int64_t start = __ldg(t.toff + j);
    const int64_t o = q - start;
    const int64_t L = __ldg(t.toff + j + 1) - 1 - q;   // bases of X = r_j[o..]
    if (o < 1 || L < a.lmin) return false;
    const uint32_t s = a.isa[q];
    const int ri1 = a.rrange ? (int)__ldg(a.rrange + j).y : (int)t.n_reads;
    // first fragment start after X's slot = the fragment starts at smaller slots
    // (X itself is no fragment start: o >= 1); instances occupy consecutive slots
    const int lo = (int)__ldg(a.nstart + s);
    if (lo >= ri1) return false;
    const int64_t k = __ldg(a.R + lo);
    if (frag_len(t.toff, k) < L) return false;
    if (common_bases(t.packed, (uint64_t)(q - j), (uint64_t)(__ldg(t.toff + k) - k), L) < L)
        return false;
    h.j = (int)j;
    h.L = (int)L;
    h.lo = lo;
    h.ri1 = ri1;
    return true;
}

// The fragment starts that have X as a prefix: R[lo] and its successors while
// LCP_R stays >= |X|; emit(k) for each proper overlap (j, k, |X|).
template <typename F>
__device__ __forceinline__ void query_walk(const TextDesc &t, const QueryArgs &a, const QueryHit &h,
                                           F emit) {
    for (int kk = h.lo; kk < h.ri1; ++kk) {
        if (kk > h.lo && __ldg(a.lcpr + kk) < h.L) break;
        const int64_t k = __ldg(a.R + kk);
        if (k != h.j && h.L < frag_len(t.toff, k)) emit(k);
    }
}

// One thread per text position.  Each warp counts its overlaps, claims room
// with one atomic, then walks again from the located start to write them.
__global__ void __launch_bounds__(256) k_query(TextDesc t, QueryArgs a) {
    const unsigned long long lmask = (1ull << a.lb) - 1ull;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; b < t.N; b += stride) {
        const int64_t q = b + lane;
        uint32_t c = 0;
        QueryHit h;
        const bool hit = q < t.N && query_locate(t, a, q, h);
        if (hit) query_walk(t, a, h, [&](int64_t) { ++c; });
        uint32_t inc = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        unsigned long long base = 0;
        if (lane == 31 && inc) base = atomicAdd(a.count, (unsigned long long)inc);
        base = __shfl_sync(0xffffffffu, base, 31) + (inc - c);
        if (c) {
            query_walk(t, a, h, [&](int64_t k) {
                unsigned long long key = ((unsigned long long)h.j << (a.kb + a.lb)) |
                                         ((unsigned long long)k << a.lb) |
                                         (lmask - (unsigned long long)h.L);
                if (base < a.cap) a.cand[base] = key;
                ++base;
            });
        }
    }
}

// Per fragment: the range of R that holds its instance's fragment starts.
__global__ void k_read_range(TextDesc t, uint2 *__restrict__ rrange) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < t.n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t inst = inst_of_read(t, r);
        rrange[r] = make_uint2((uint32_t)__ldg(t.inst_roff + inst), (uint32_t)__ldg(t.inst_roff + inst + 1));
    }
}

__global__ void k_unique_flags(const unsigned long long *__restrict__ keys, int64_t n, int lb,
                               uint8_t *__restrict__ flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0) || ((keys[i] >> lb) != (keys[i - 1] >> lb));
}

__global__ void k_emit_edges(const unsigned long long *__restrict__ keys,
                             const uint32_t *__restrict__ idx, const unsigned long long *d_count,
                             int kb, int lb, dnasa_edge *__restrict__ edges, int64_t cap) {
    const int64_t n = (int64_t)*d_count;
    const unsigned long long lmask = (1ull << lb) - 1ull;
    const unsigned long long kmask = (1ull << kb) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n && e < cap;
         e += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = keys[idx[e]];
        dnasa_edge ed;
        ed.j = (int32_t)(key >> (kb + lb));
        ed.k = (int32_t)((key >> lb) & kmask);
        ed.L = (int32_t)(lmask - (key & lmask));
        edges[e] = ed;
    }
}

__global__ void k_contained(TextDesc t, const uint32_t *__restrict__ sa,
                            const uint32_t *__restrict__ isa, const int32_t *__restrict__ lcp,
                            uint8_t *__restrict__ contained) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < t.n_reads;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t len = frag_len(t.toff, k);
        int64_t s = isa[__ldg(t.toff + k)];
        int64_t is0 = 0, is1 = t.N;
        if (t.n_inst > 1) {
            int64_t inst = inst_of_read(t, k);
            is0 = __ldg(t.inst_toff + inst);
            is1 = __ldg(t.inst_toff + inst + 1);
        }
        uint8_t c = 0;
        if (s > is0 && lcp[s] >= len) {
            c = 1;
        } else {
            for (int64_t u = s + 1; u < is1 && lcp[u] >= len; ++u) {
                int64_t p = sa[u];
                int64_t rp = frag_of(t, p);
                if (p != __ldg(t.toff + rp) || frag_len(t.toff, rp) > len) { c = 1; break; }
            }
        }
        contained[k] = c;
    }
}

inline int grid_for(dnasa_ctx *ctx, int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), threads),
                                                      (int64_t)ctx->num_sms * 16));
}

}  // namespace

int overlap_impl(dnasa_ctx *ctx, const TextDesc &t, const uint32_t *sa32, const int32_t *lcp,
                 int32_t min_overlap, dnasa_edge *edges, int64_t cap, int64_t *n_edges,
                 uint8_t *contained, cudaStream_t s, const uint32_t *isa_in) {
    PhaseRange nvtx_("dnasa.overlap");
    const int64_t N = t.N, nr = t.n_reads;
    const int kb = bits_for((uint64_t)std::max<int64_t>(nr - 1, 1));
    const int tile = radix_tile_default();

    // ---- phase 1: ISA, R, LCP_R (fixed-size workspace)
    size_t need = 0;
    auto add = [&](size_t bytes) { need += (bytes + 255) & ~size_t(255); };
    add((size_t)N * 4);                              // isa
    add((size_t)N * 4);                              // fragment starts per SA slot (scanned)
    for (int i = 0; i < 4; ++i) add((size_t)nr * 4); // R keys/vals x2
    add((size_t)nr * 4);                             // lcp_r
    if (t.n_inst > 1) add((size_t)nr * 8);           // per-fragment instance range in R
    add(radix_scratch_bytes(nr, 64, tile));
    int64_t cand_cap = std::max<int64_t>(4 * nr, 1 << 16);
    auto cand_bytes = [&](int64_t cc) {
        return 2 * (((size_t)cc * 8 + 255) & ~size_t(255)) + (((size_t)cc + 255) & ~size_t(255)) +
               (((size_t)cc * 4 + 255) & ~size_t(255)) + compact_scratch_bytes(cc) +
               radix_scratch_bytes(cc, 64, tile);
    };
    DNASA_TRY(ws_reserve(ctx, need + cand_bytes(cand_cap) + 8192, s));

    unsigned long long *cnt = ctx->ctrl->count;
    for (int attempt = 0; attempt < 2; ++attempt) {
        Arena a = ws_arena(ctx);
        uint32_t *isa_ws = a.take<uint32_t>((size_t)N);
        uint32_t *nstart = a.take<uint32_t>((size_t)N);
        const uint32_t *isa = isa_in ? isa_in : isa_ws;
        uint32_t *rk[2] = {a.take<uint32_t>((size_t)nr), a.take<uint32_t>((size_t)nr)};
        uint32_t *rv[2] = {a.take<uint32_t>((size_t)nr), a.take<uint32_t>((size_t)nr)};
        int32_t *lcpr = a.take<int32_t>((size_t)nr);
        uint2 *rrange = t.n_inst > 1 ? a.take<uint2>((size_t)nr) : nullptr;
        RadixScratch rs = radix_scratch_take(a, nr, 64, tile);
        unsigned long long *ck[2] = {a.take<unsigned long long>((size_t)cand_cap),
                                     a.take<unsigned long long>((size_t)cand_cap)};
        uint8_t *flags = a.take<uint8_t>((size_t)cand_cap);
        uint32_t *cidx = a.take<uint32_t>((size_t)cand_cap);
        RadixScratch rs2 = radix_scratch_take(a, cand_cap, 64, tile);
        if (!rs2.hist) return fail(ctx, DNASA_OOM, "overlap_search workspace");

        DNASA_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 8, s));
        if (!isa_in) {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 8.0 * N);   // read sa[j], write isa[sa[j]]
            k_isa<<<grid_for(ctx, N), 256, 0, s>>>(sa32, N, isa_ws);
        }
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 24.0 * nr);   // toff, isa, key and value
            k_read_keys<<<grid_for(ctx, nr), 256, 0, s>>>(t, isa, rk[0], rv[0], cnt + CNT_TMP);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        int which;
        DNASA_TRY(radix_sort_pairs<uint32_t>(ctx, rs, rk, rv, nr, nullptr,
                                             bits_for((uint64_t)(N - 1)), false, tile, &which, s));
        const uint32_t *Rslot = rk[which], *R = rv[which];
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 24.0 * nr);   // R, two starts, LCP_R
            k_lcp_r<<<grid_for(ctx, nr), 256, 0, s>>>(t, R, lcpr);
        }
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_TMP, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "overlap_search"));
        const int64_t maxlen = (int64_t)ctx->pinned[0];
        const int lb = bits_for((uint64_t)maxlen);
        if (2 * kb + lb > 64)
            return fail(ctx, DNASA_INVALID_ARG, "overlap_search: fragments too many or too long "
                                                "for a 64-bit edge key");
        if (rrange) {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 24.0 * nr);
            k_read_range<<<grid_for(ctx, nr), 256, 0, s>>>(t, rrange);
        }
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 8.0 * N);
            k_startflag<<<grid_for(ctx, N), 256, 0, s>>>(t, sa32, nstart);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_TRY(scan_inclusive_u32(ctx, nstart, N, s));
        QueryArgs qa;
        qa.isa = isa; qa.Rslot = Rslot; qa.R = R; qa.lcpr = lcpr; qa.rrange = rrange; qa.nstart = nstart;
        qa.lmin = min_overlap;
        qa.kb = kb; qa.lb = lb; qa.cand = ck[0]; qa.cap = (unsigned long long)cand_cap;
        qa.count = cnt + CNT_CAND;
        {
            // per position: isa[q] (and its fragment id), one packed word
            LaunchScope ls_(ctx, PK_OVERLAP, s, (t.fid ? 8.25 : 4.25) * N);
            k_query<<<grid_for(ctx, N), 256, 0, s>>>(t, qa);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_CAND, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "overlap_search"));
        const int64_t ncand = (int64_t)ctx->pinned[0];
        if (ncand > cand_cap) {
            if (attempt == 1) return fail(ctx, DNASA_CUDA_ERROR, "overlap_search: candidate count changed");
            cand_cap = ncand + ncand / 8 + 1024;
            DNASA_TRY(ws_reserve(ctx, need + cand_bytes(cand_cap) + 8192, s));
            continue;
        }
        // ---- phase 2: sort candidates, keep the max L per (j, k), emit in (j, k) order
        int which2 = 0;
        if (ncand > 0) {
            uint32_t *nov[2] = {nullptr, nullptr};
            DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs2, ck, nov, ncand, nullptr,
                                                           2 * kb + lb, false, tile, &which2, s));
            {
                LaunchScope ls_(ctx, PK_OVERLAP, s, 9.0 * ncand);
                k_unique_flags<<<grid_for(ctx, ncand), 256, 0, s>>>(ck[which2], ncand, lb, flags);
            }
            DNASA_TRY(compact_flags(ctx, a, flags, ncand, cidx, cnt + CNT_EDGES, s));
            {
                LaunchScope ls_(ctx, PK_OVERLAP, s, 20.0 * ncand);
                k_emit_edges<<<grid_for(ctx, ncand), 256, 0, s>>>(ck[which2], cidx, cnt + CNT_EDGES, kb,
                                                                 lb, edges, cap);
            }
            DNASA_CUDA(ctx, cudaGetLastError());
        }
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 24.0 * nr);
            k_contained<<<grid_for(ctx, nr), 256, 0, s>>>(t, sa32, isa, lcp, contained);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_EDGES, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "overlap_search"));
        const int64_t ne = ncand > 0 ? (int64_t)ctx->pinned[0] : 0;
        *n_edges = ne;
        if (ne > cap)
            return fail(ctx, DNASA_CAPACITY, "overlap_search: " + std::to_string(ne) +
                                                 " edges exceed cap " + std::to_string(cap));
        return DNASA_OK;
    }
    return DNASA_OK;
}

}  // namespace dnasa
