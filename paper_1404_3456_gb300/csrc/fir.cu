// fir.cu -- Sec. III reconstruction of a sequence cut by two shotguns, from
// "fir" relations found in the suffix array, with back-tracking (Figs. 5-8).
//
// The fragments are the pieces of two cuttings of one sequence (Fig. 2), all
// break positions different (Fig. 4).  Both cuttings start at the beginning, so
// the first piece of one is a prefix of the first piece of the other (a "fir"
// pair).  Cutting the shorter from the longer leaves a remainder X; the next
// piece of the other cutting starts where X starts, so it is a prefix of X or X
// is a prefix of it, and the process repeats on what is left (Figs. 5-6).  When
// a choice leads nowhere the search backs up (Figs. 7-8).
//
// Sec. IV's point is that the relation "some fragment is a prefix of X, or X is
// a prefix of some fragment" is answered by a binary search in the suffix array.
// Here it is answered for every suffix X of every fragment at once, in one
// parallel pass over the text, before the search:
//   * R = the fragment starts in SA order with LCP_R (common prefix of
//     consecutive entries), per instance;
//   * for X at text position x: its place among R's slots (the number of
//     fragment starts at smaller slots, from one prefix count over the SA --
//     Sec. IV's binary search answered for every slot at once); walking
//     forward while the common prefix with X stays >= |X| gives the
//     fragments X is a prefix of (or equal to); walking backward, a fragment c
//     whose common prefix with X is all of c is a prefix of X;
//   * the (x, c) pairs are radix sorted, so the candidates of each x are a run
//     in ascending fragment order.
// Then one thread per instance runs the depth-first search over these runs:
// start pairs (k ascending, then the prefix fragment ascending), at each
// remainder the unused candidates in ascending index, equal-length matches only
// as the last fragment, a step bound after which the search gives up.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace dnasa {

namespace {

__device__ __forceinline__ int64_t flen(const int64_t *__restrict__ toff, int64_t r) {
    return __ldg(toff + r + 1) - 1 - __ldg(toff + r);
}

// Equal bases at the start of base coordinates ba and bb, at most maxlen.
__device__ __forceinline__ int64_t same_bases(const uint64_t *__restrict__ packed, uint64_t ba,
                                              uint64_t bb, int64_t maxlen) {
    int64_t h = 0;
    while (h < maxlen) {
        const uint64_t d = bases32(packed, ba + h) ^ bases32(packed, bb + h);
        if (d) return min(h + (int64_t)(__clzll((long long)d) >> 1), maxlen);
        h += 32;
    }
    return maxlen;
}

__device__ __forceinline__ int64_t inst_of_frag(const TextDesc &t, int64_t r) {
    return t.n_inst > 1 ? upper_index(t.inst_roff, 0, t.n_inst, r) : 0;
}

// R keys: SA slot of each fragment start (sorted next), value = fragment; also
// the shortest fragment.
__global__ void k_fir_rkeys(TextDesc t, const uint32_t *__restrict__ isa, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ val, unsigned long long *minlen) {
    unsigned long long m = ~0ull;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < t.n_reads;
         r += (int64_t)gridDim.x * blockDim.x) {
        key[r] = isa[__ldg(t.toff + r)];
        val[r] = (uint32_t)r;
        m = min(m, (unsigned long long)flen(t.toff, r));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(minlen, m);
}

// LCP_R[i] = common prefix of fragments R[i-1] and R[i] (0 across instances);
// rrange[r] = the range of R holding fragment r's instance.
__global__ void k_fir_lcpr(TextDesc t, const uint32_t *__restrict__ R, int32_t *__restrict__ lcpr,
                           uint2 *__restrict__ rrange) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < t.n_reads;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (t.n_inst > 1) {
            const int64_t inst = inst_of_frag(t, i);
            rrange[i] = make_uint2((uint32_t)__ldg(t.inst_roff + inst),
                                   (uint32_t)__ldg(t.inst_roff + inst + 1));
        } else {
            rrange[i] = make_uint2(0u, (uint32_t)t.n_reads);
        }
        if (i == 0) { lcpr[0] = 0; continue; }
        const int64_t a = R[i - 1], b = R[i];
        if (t.n_inst > 1 && inst_of_frag(t, a) != inst_of_frag(t, b)) { lcpr[i] = 0; continue; }
        const int64_t m = min(flen(t.toff, a), flen(t.toff, b));
        lcpr[i] = (int32_t)same_bases(t.packed, (uint64_t)(__ldg(t.toff + a) - a),
                                      (uint64_t)(__ldg(t.toff + b) - b), m);
    }
}

// flag[s] = 1 when the suffix at SA slot s starts a fragment (then scanned).
__global__ void k_fir_startflag(TextDesc t, const uint32_t *__restrict__ sa, uint32_t *__restrict__ flag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < t.N;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = sa[j];
        flag[j] = p == __ldg(t.toff + frag_of(t, p)) ? 1u : 0u;
    }
}

struct FirIndex {
    const uint32_t *isa, *Rslot, *R;
    const uint32_t *nstart;               // [N]: fragment-start suffixes at SA slots <= s
    const int32_t *lcpr;
    const uint2 *rrange;
    int64_t minlen;
    int kb;                               // bits of a fragment index in a pair key
    unsigned long long *pairs;            // (x << kb) | c
    unsigned long long cap;
    unsigned long long *count;
};

// Every fragment c in fir relation with X = suffix at text position x (inside
// fragment k): X a prefix of c or equal to it (forward walk in R from X's slot),
// c a proper prefix of X (backward walk).  emit(c) for each.
template <typename F>
__device__ __forceinline__ void fir_candidates(const TextDesc &t, const FirIndex &fi, int64_t x,
                                               F emit) {
    const int64_t k = frag_of(t, x);
    const int64_t o = x - __ldg(t.toff + k);
    const int64_t l = flen(t.toff, k) - o;          // |X|
    if (l <= 0) return;                             // x is a '$'
    const uint32_t s = fi.isa[x];
    const uint2 rg = __ldg(fi.rrange + k);
    // first fragment start at or after X's slot: the fragment starts at smaller
    // slots, counted once for every slot (instances occupy consecutive slots, so
    // this index lies in the instance's range of R)
    const bool self = o == 0;                       // X is itself a fragment
    const int lo = (int)__ldg(fi.nstart + s) - (self ? 1 : 0);
    const uint64_t bx = (uint64_t)(x - k);          // base coordinate of X
    // forward: fragments having X as a prefix (|c| >= l)
    {
        int64_t h = -1;                             // common prefix of X with R[i]
        for (int i = self ? lo + 1 : lo; i < (int)rg.y; ++i) {
            const int64_t c = __ldg(fi.R + i);
            if (h < 0)
                h = self ? min((int64_t)__ldg(fi.lcpr + i), l)
                         : same_bases(t.packed, bx, (uint64_t)(__ldg(t.toff + c) - c), l);
            else
                h = min(h, (int64_t)__ldg(fi.lcpr + i));
            if (h < l) break;
            emit(c);
        }
    }
    // backward: fragments c before X in SA order with common prefix == |c|
    // (c a proper prefix of X, or c equal to X at a smaller position)
    {
        int64_t h = -1;
        for (int i = lo - 1; i >= (int)rg.x; --i) {
            const int64_t c = __ldg(fi.R + i);
            const int64_t lc = flen(t.toff, c);
            if (h < 0)
                h = self ? min((int64_t)__ldg(fi.lcpr + lo), l)
                         : same_bases(t.packed, bx, (uint64_t)(__ldg(t.toff + c) - c), min(l, lc));
            else
                h = min(h, (int64_t)__ldg(fi.lcpr + i + 1));
            if (h < fi.minlen || h == 0) break;     // no shorter common prefix can be a fragment
            if (h == lc && lc <= l) emit(c);
        }
    }
}

// One thread per text position; each warp claims room for its pairs with one
// atomic, then walks again to write them.
__global__ void __launch_bounds__(256) k_fir_query(TextDesc t, FirIndex fi) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; b < t.N; b += stride) {
        const int64_t x = b + lane;
        uint32_t c = 0;
        if (x < t.N) fir_candidates(t, fi, x, [&](int64_t) { ++c; });
        uint32_t inc = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        unsigned long long base = 0;
        if (lane == 31 && inc) base = atomicAdd(fi.count, (unsigned long long)inc);
        base = __shfl_sync(0xffffffffu, base, 31) + (inc - c);
        if (c) {
            fir_candidates(t, fi, x, [&](int64_t cc) {
                if (base < fi.cap) fi.pairs[base] = ((unsigned long long)x << fi.kb) | (unsigned long long)cc;
                ++base;
            });
        }
    }
}

// One fir relation as a move of the search: from the remainder at position x,
// place fragment c; the next remainder starts at text position nx, adv bases
// further in the result.  kind 0: c inside the remainder (c a proper prefix of
// it: the remainder continues in the same fragment past |c|); 1: the remainder
// inside c (the remainder continues in c past |X|); 2: c equal to the
// remainder (allowed only as the last fragment; the result ends adv bases on).
struct FirMove {
    uint32_t c, nx, adv, kind;
};

struct FirState {
    const FirMove *moves;                 // one per pair, in pair order (x, then c ascending)
    const uint32_t *xoff;                 // [N + 1]: moves of position x are [xoff[x], xoff[x+1])
    int64_t npairs;
    int64_t max_steps;
    uint8_t *used;                        // [n_reads]
    uint4 *frames;                        // [n_reads]: (x, index of the placed move + 1, result offset of x)
    int64_t *start;                       // [n_reads] output: offset in the instance's result
    int32_t *status;                      // [n_inst] 0 solved, 1 none, 2 gave up
    int64_t *steps;                       // [n_inst]
    int64_t *rs_len;                      // [n_inst]
};

// The move of every (x, c) pair: the lengths that decide it are read once here,
// so that a step of the search is a few dependent loads.
__global__ void k_fir_moves(TextDesc t, const unsigned long long *__restrict__ pairs, int64_t np, int kb,
                            FirMove *__restrict__ moves) {
    const unsigned long long cmask = (1ull << kb) - 1ull;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = (int64_t)(pairs[p] >> kb), c = (int64_t)(pairs[p] & cmask);
        const int64_t k = frag_of(t, x);
        const int64_t l = flen(t.toff, k) - (x - __ldg(t.toff + k));   // |X|
        const int64_t lc = flen(t.toff, c);
        FirMove m;
        m.c = (uint32_t)c;
        if (lc < l) { m.kind = 0u; m.nx = (uint32_t)(x + lc); m.adv = (uint32_t)lc; }
        else if (lc > l) { m.kind = 1u; m.nx = (uint32_t)(__ldg(t.toff + c) + l); m.adv = (uint32_t)l; }
        else { m.kind = 2u; m.nx = 0u; m.adv = (uint32_t)l; }
        moves[p] = m;
    }
}

// xoff[x] = first pair of position x (pairs sorted by x): each pair that starts a
// run of its position fills the offsets of the positions since the previous run.
__global__ void k_fir_xoff(const unsigned long long *__restrict__ pairs, int64_t np, int kb, int64_t N,
                           uint32_t *__restrict__ xoff) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = p < np ? (int64_t)(pairs[p] >> kb) : N;
        const int64_t xp = p > 0 ? (int64_t)(pairs[p - 1] >> kb) : -1;
        if (p < np && x == xp) continue;
        for (int64_t y = xp + 1; y <= x; ++y) xoff[y] = (uint32_t)p;
    }
}

// Depth-first search of one instance (one thread per instance).  Frame f holds
// the remainder's text position x, 1 + the index of the move placed from it (0:
// none yet), and the remainder's offset in the result.  Fragment indices of an
// instance are the contiguous range [r0, r1).
__global__ void k_fir_dfs(TextDesc t, FirState S) {
    const int64_t inst = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= t.n_inst) return;
    const int64_t r0 = t.n_inst > 1 ? __ldg(t.inst_roff + inst) : 0;
    const int64_t r1 = t.n_inst > 1 ? __ldg(t.inst_roff + inst + 1) : t.n_reads;
    const int64_t n = r1 - r0;
    for (int64_t r = r0; r < r1; ++r) { S.used[r] = 0; S.start[r] = -1; }
    uint4 *F = S.frames + r0;
    int64_t steps = 0;
    int status = 1;
    int64_t rs_len = 0;
    bool done = false;
    for (int64_t k = r0; k < r1 && !done && status != 2; ++k) {
        const uint64_t xk = (uint64_t)__ldg(t.toff + k);
        const int64_t pe = (int64_t)__ldg(S.xoff + xk + 1);
        for (int64_t pi = (int64_t)__ldg(S.xoff + xk); pi < pe && !done && status != 2; ++pi) {
            const FirMove st = S.moves[pi];
            if (st.kind != 0u) continue;            // start pairs: proper prefixes of d_k
            const int64_t i = (int64_t)st.c;
            if (++steps > S.max_steps) { status = 2; break; }
            S.used[i] = S.used[k] = 1;
            S.start[i] = S.start[k] = 0;
            int64_t top = 0;
            F[0] = make_uint4(st.nx, 0u, st.adv, 0u);
            while (top >= 0 && !done) {
                const uint4 f = F[top];
                int64_t from;
                if (f.y) {                          // back from the child: undo its fragment
                    const int64_t prev = (int64_t)f.y - 1;
                    const int64_t c = (int64_t)S.moves[prev].c;
                    S.used[c] = 0;
                    S.start[c] = -1;
                    from = prev + 1;
                    F[top].y = 0u;
                } else {
                    from = (int64_t)__ldg(S.xoff + f.x);
                }
                const int64_t nused = 2 + top;
                const int64_t to = (int64_t)__ldg(S.xoff + f.x + 1);
                int64_t pick = -1;
                FirMove m;
                for (int64_t p = from; p < to; ++p) {
                    m = S.moves[p];
                    if (S.used[m.c]) continue;
                    if (m.kind == 2u && nused + 1 != n) continue;   // equal: only as the last one
                    pick = p;
                    break;
                }
                if (pick < 0) { --top; continue; }  // no fir fragment: back-track
                if (++steps > S.max_steps) { status = 2; break; }
                S.used[m.c] = 1;
                S.start[m.c] = (int64_t)f.z;
                F[top].y = (uint32_t)(pick + 1);
                if (m.kind == 2u) {                 // both cuttings end here
                    done = true;
                    status = 0;
                    rs_len = (int64_t)f.z + (int64_t)m.adv;
                    break;
                }
                ++top;
                F[top] = make_uint4(m.nx, 0u, f.z + m.adv, 0u);
            }
            if (!done)
                for (int64_t r = r0; r < r1; ++r) { S.used[r] = 0; S.start[r] = -1; }
        }
    }
    if (status != 0)
        for (int64_t r = r0; r < r1; ++r) S.start[r] = -1;
    S.status[inst] = status;
    S.steps[inst] = steps;
    S.rs_len[inst] = status == 0 ? rs_len : 0;
}

// rs_off = exclusive scan of rs_len (one thread: instances are few thousand)
__global__ void k_fir_scan(const int64_t *__restrict__ rs_len, int64_t n, int64_t *__restrict__ rs_off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t run = 0;
    for (int64_t i = 0; i < n; ++i) { rs_off[i] = run; run += rs_len[i]; }
    rs_off[n] = run;
}

// Every placed fragment writes its bases at its offset (the two cuttings cover
// each base twice with the same value).  One warp per fragment.
__global__ void k_fir_spell(TextDesc t, const uint8_t *__restrict__ text, const int64_t *__restrict__ start,
                            const int64_t *__restrict__ rs_off, const int32_t *__restrict__ status,
                            uint8_t *__restrict__ rs, int64_t cap) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < t.n_reads; r += nw) {
        const int64_t inst = inst_of_frag(t, r);
        if (status[inst] != 0) continue;
        const int64_t st = start[r];
        const int64_t len = flen(t.toff, r);
        const int64_t a = __ldg(t.toff + r);
        const int64_t dst = rs_off[inst] + st;
        for (int64_t i = lane; i < len; i += 32)
            if (dst + i < cap) rs[dst + i] = text[a + i];
    }
}

inline int grid_for(dnasa_ctx *ctx, int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(std::max<int64_t>(n, 1), threads),
                                                      (int64_t)ctx->num_sms * 16));
}

}  // namespace

// Whole fir reconstruction of n_inst instances (text on the device).
int fir_impl(dnasa_ctx *ctx, const uint8_t *text, int64_t N, const int64_t *inst_toff_host,
             int32_t n_inst, int64_t max_steps, int64_t *frag_start, int64_t frag_cap, uint8_t *rs,
             int64_t rs_cap, int64_t *rs_off, int32_t *status, int64_t *steps, int64_t *rs_total,
             int64_t *n_frags, cudaStream_t s) {
    PhaseRange nvtx_("dnasa.fir");
    DevBuf packed, toff, sa, isa, fid, inst_toff, inst_roff, rs_len;
    const int64_t toff_cap = N / 2 + 2;
    DNASA_TRY(dev_alloc(ctx, packed, (size_t)dnasa_packed_words(N) * 8, s));
    DNASA_TRY(dev_alloc(ctx, toff, (size_t)toff_cap * 8, s));
    int64_t nr = 0;
    DNASA_TRY(pack_impl(ctx, text, N, (uint64_t *)packed.p, (int64_t *)toff.p, toff_cap, &nr, s));
    *n_frags = nr;
    if (nr > frag_cap)
        return fail(ctx, DNASA_CAPACITY, "fir_reconstruct: " + std::to_string(nr) +
                                             " fragments exceed frag_cap " + std::to_string(frag_cap));
    if (nr >= (int64_t(1) << 31)) return fail(ctx, DNASA_INVALID_ARG, "fir_reconstruct: too many fragments");
    TextDesc t;
    t.packed = (const uint64_t *)packed.p;
    t.toff = (const int64_t *)toff.p;
    t.n_reads = nr;
    t.N = N;
    t.inst_toff = nullptr;
    t.inst_roff = nullptr;
    t.n_inst = 1;
    t.fid = nullptr;
    if (n_inst > 1) {
        int64_t max_reads;
        DNASA_TRY(make_instances(ctx, t.toff, nr, N, inst_toff_host, n_inst, inst_toff, inst_roff,
                                 &max_reads, s));
        t.inst_toff = (const int64_t *)inst_toff.p;
        t.inst_roff = (const int64_t *)inst_roff.p;
        t.n_inst = n_inst;
    }
    DNASA_TRY(dev_alloc(ctx, sa, (size_t)N * 4, s));
    DNASA_TRY(dev_alloc(ctx, isa, (size_t)N * 4, s));
    DNASA_TRY(dev_alloc(ctx, rs_len, (size_t)n_inst * 8, s));
    if (nr > 1) {
        DNASA_TRY(dev_alloc(ctx, fid, (size_t)N * 4, s));
        DNASA_TRY(fragment_ids(ctx, t, (uint32_t *)fid.p, s));
        t.fid = (const uint32_t *)fid.p;
    }
    DNASA_TRY(sa_build_u32(ctx, t, (uint32_t *)sa.p, nullptr, s, (uint32_t *)isa.p));
    {   // the SA itself is needed no further: it becomes the count of fragment starts per slot
        LaunchScope ls_(ctx, PK_OVERLAP, s, 8.0 * N);
        k_fir_startflag<<<grid_for(ctx, N), 256, 0, s>>>(t, (const uint32_t *)sa.p, (uint32_t *)sa.p);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    DNASA_TRY(scan_inclusive_u32(ctx, (uint32_t *)sa.p, N, s));

    // ---- R, LCP_R, then the fir pairs of every text position
    const int tile = radix_tile_default();
    const int kb = bits_for((uint64_t)std::max<int64_t>(nr - 1, 1));
    const int xb = bits_for((uint64_t)(N - 1));
    if (kb + xb > 64) return fail(ctx, DNASA_INVALID_ARG, "fir_reconstruct: text too large for pair keys");
    int64_t cap = std::max<int64_t>(4 * nr, 1 << 16);
    unsigned long long *cnt = ctx->ctrl->count;
    for (int attempt = 0; attempt < 2; ++attempt) {
        size_t need = 0;
        auto add = [&](size_t bytes) { need += (bytes + 255) & ~size_t(255); };
        for (int i = 0; i < 4; ++i) add((size_t)nr * 4);   // R keys/values x2
        add((size_t)nr * 4);                               // LCP_R
        add((size_t)nr * 8);                               // R range per fragment
        add(radix_scratch_bytes(nr, 32, tile));
        add((size_t)cap * 8); add((size_t)cap * 8);        // pairs x2
        add(radix_scratch_bytes(cap, 64, tile));
        add((size_t)nr); add((size_t)nr * 16);             // used flags, frames
        DNASA_TRY(ws_reserve(ctx, need + 8192, s));
        Arena a = ws_arena(ctx);
        uint32_t *rk[2] = {a.take<uint32_t>((size_t)nr), a.take<uint32_t>((size_t)nr)};
        uint32_t *rv[2] = {a.take<uint32_t>((size_t)nr), a.take<uint32_t>((size_t)nr)};
        int32_t *lcpr = a.take<int32_t>((size_t)nr);
        uint2 *rrange = a.take<uint2>((size_t)nr);
        RadixScratch rs1 = radix_scratch_take(a, nr, 32, tile);
        unsigned long long *pk[2] = {a.take<unsigned long long>((size_t)cap),
                                     a.take<unsigned long long>((size_t)cap)};
        RadixScratch rs2 = radix_scratch_take(a, cap, 64, tile);
        uint8_t *used = a.take<uint8_t>((size_t)nr);
        uint4 *frames = a.take<uint4>((size_t)nr);
        if (!frames) return fail(ctx, DNASA_OOM, "fir_reconstruct workspace");
        DNASA_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 8, s));
        DNASA_CUDA(ctx, cudaMemsetAsync(cnt + CNT_TMP, 0xff, 8, s));   // running minimum
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 24.0 * nr);
            k_fir_rkeys<<<grid_for(ctx, nr), 256, 0, s>>>(t, (const uint32_t *)isa.p, rk[0], rv[0],
                                                         cnt + CNT_TMP);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        int which;
        DNASA_TRY(radix_sort_pairs<uint32_t>(ctx, rs1, rk, rv, nr, nullptr, xb, false, tile, &which, s));
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 32.0 * nr);
            k_fir_lcpr<<<grid_for(ctx, nr), 256, 0, s>>>(t, rv[which], lcpr, rrange);
        }
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_TMP, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "fir_reconstruct"));
        FirIndex fi;
        fi.isa = (const uint32_t *)isa.p;
        fi.Rslot = rk[which];
        fi.nstart = (const uint32_t *)sa.p;
        fi.R = rv[which];
        fi.lcpr = lcpr;
        fi.rrange = rrange;
        fi.minlen = std::max<int64_t>(1, (int64_t)ctx->pinned[0]);
        fi.kb = kb;
        fi.pairs = pk[0];
        fi.cap = (unsigned long long)cap;
        fi.count = cnt + CNT_CAND;
        {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 8.25 * N);   // isa and fragment id per position
            k_fir_query<<<grid_for(ctx, N), 256, 0, s>>>(t, fi);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_CAND, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "fir_reconstruct"));
        const int64_t np = (int64_t)ctx->pinned[0];
        if (np > cap) {
            if (attempt == 1) return fail(ctx, DNASA_CUDA_ERROR, "fir_reconstruct: pair count changed");
            cap = np + np / 8 + 1024;
            continue;
        }
        int which2 = 0;
        if (np > 0) {
            uint32_t *nov[2] = {nullptr, nullptr};
            DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs2, pk, nov, np, nullptr, kb + xb, false,
                                                           tile, &which2, s));
        }
        DevBuf xoffb;
        DNASA_TRY(dev_alloc(ctx, xoffb, (size_t)(N + 1) * 4, s));
        if (np == 0) {
            DNASA_CUDA(ctx, cudaMemsetAsync(xoffb.p, 0, (size_t)(N + 1) * 4, s));
        } else {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 4.0 * (N + 1) + 16.0 * np);
            k_fir_xoff<<<grid_for(ctx, np + 1), 256, 0, s>>>(pk[which2], np, kb, N, (uint32_t *)xoffb.p);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DevBuf movesb;
        DNASA_TRY(dev_alloc(ctx, movesb, (size_t)std::max<int64_t>(np, 1) * sizeof(FirMove), s));
        if (np > 0) {
            LaunchScope ls_(ctx, PK_OVERLAP, s, 24.0 * np);
            k_fir_moves<<<grid_for(ctx, np), 256, 0, s>>>(t, pk[which2], np, kb, (FirMove *)movesb.p);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        FirState S;
        S.moves = (const FirMove *)movesb.p;
        S.xoff = (const uint32_t *)xoffb.p;
        S.npairs = np;
        S.max_steps = max_steps;
        S.used = used;
        S.frames = frames;
        S.start = frag_start;
        S.status = status;
        S.steps = steps;
        S.rs_len = (int64_t *)rs_len.p;
        {
            LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
            k_fir_dfs<<<ceil_div(n_inst, 32), 32, 0, s>>>(t, S);
        }
        {
            LaunchScope ls_(ctx, PK_LAYOUT, s, 0);
            k_fir_scan<<<1, 32, 0, s>>>((const int64_t *)rs_len.p, n_inst, rs_off);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, rs_off + n_inst, 8, cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "fir_reconstruct"));
        *rs_total = (int64_t)ctx->pinned[0];
        if (*rs_total > rs_cap)
            return fail(ctx, DNASA_CAPACITY, "fir_reconstruct: result needs " + std::to_string(*rs_total) +
                                                 " bytes");
        {
            LaunchScope ls_(ctx, PK_LAYOUT, s, 2.0 * N);
            k_fir_spell<<<grid_for(ctx, 32 * nr), 256, 0, s>>>(t, text, frag_start, rs_off, status, rs,
                                                              rs_cap);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        return check_device_status(ctx, s, "fir_reconstruct");
    }
    return DNASA_OK;
}

}  // namespace dnasa

using namespace dnasa;

extern "C" {

int fir_reconstruct(dnasa_ctx *ctx, const uint8_t *text, int64_t N, int64_t max_steps,
                    int64_t *frag_start, int64_t frag_cap, uint8_t *rs, int64_t rs_cap,
                    int64_t *rs_len, int32_t *status, int64_t *steps, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (N <= 0 || N >= (int64_t(1) << 31) || max_steps < 1 || frag_cap < 1 || rs_cap < 0 || !rs_len ||
        !status || !steps)
        return fail(ctx, DNASA_INVALID_ARG, "fir_reconstruct: bad size, step bound or null output");
    if (!is_device_ptr(ctx, text) || !is_device_ptr(ctx, frag_start) || (rs_cap > 0 && !is_device_ptr(ctx, rs)))
        return fail(ctx, DNASA_INVALID_ARG, "fir_reconstruct: text, frag_start and rs must be device pointers");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf small;
    DNASA_TRY(dev_alloc(ctx, small, 64, s));
    int64_t *d_off = (int64_t *)small.p;            // rs_off[0..1]
    int32_t *d_status = (int32_t *)(d_off + 2);
    int64_t *d_steps = d_off + 3;
    int64_t total = 0, nf = 0;
    int rc = fir_impl(ctx, text, N, nullptr, 1, max_steps, frag_start, frag_cap, rs, rs_cap, d_off, d_status,
                      d_steps, &total, &nf, s);
    *rs_len = total;
    if (rc != DNASA_OK && rc != DNASA_CAPACITY) return rc;
    int64_t host[4] = {0, 0, 0, 0};
    DNASA_CUDA(ctx, cudaMemcpyAsync(host, d_off, 32, cudaMemcpyDeviceToHost, s));
    DNASA_CUDA(ctx, cudaStreamSynchronize(s));
    *status = (int32_t)(host[2] & 0xffffffff);
    *steps = host[3];
    return rc;
}

int fir_reconstruct_batched(dnasa_ctx *ctx, const uint8_t *texts, const int64_t *inst_off, int32_t n_inst,
                            int64_t max_steps, int64_t *frag_start, int64_t frag_cap, uint8_t *rs,
                            int64_t rs_cap, int64_t *rs_off, int32_t *status, int64_t *steps,
                            int64_t *rs_total, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (n_inst < 1 || !inst_off)
        return fail(ctx, DNASA_INVALID_ARG, "fir_reconstruct_batched: n_inst >= 1 and inst_off required");
    const int64_t N = inst_off[n_inst];
    if (N <= 0 || N >= (int64_t(1) << 31) || max_steps < 1 || frag_cap < 1 || rs_cap < 0 || !rs_total)
        return fail(ctx, DNASA_INVALID_ARG, "fir_reconstruct_batched: bad size, step bound or null output");
    if (!is_device_ptr(ctx, texts) || !is_device_ptr(ctx, frag_start) || !is_device_ptr(ctx, rs_off) ||
        !is_device_ptr(ctx, status) || !is_device_ptr(ctx, steps) || (rs_cap > 0 && !is_device_ptr(ctx, rs)))
        return fail(ctx, DNASA_INVALID_ARG, "fir_reconstruct_batched: buffers must be device pointers");
    cudaSetDevice(ctx->device);
    int64_t nf = 0;
    return fir_impl(ctx, texts, N, inst_off, n_inst, max_steps, frag_start, frag_cap, rs, rs_cap, rs_off,
                    status, steps, rs_total, &nf, (cudaStream_t)stream);
}

}  // extern "C"
