// sa.cu -- suffix array by prefix doubling over the 2-bit packed text.
//
// Sec. IV of the paper builds the suffix array "Pos" by radix sorting suffix
// keys on the GPU.  Here the keys are:
//   round 0   (kmer, lc): the first h0 bases of the suffix packed 2 bits each
//             (zero past the fragment end) and lc = min(bases left, h0).  With
//             '$' smaller than A this integer order is the suffix order on the
//             first h0 symbols; suffixes with lc < h0 contain their own '$'
//             and are final at once (distinct sentinels ordered by position).
//   round r   (rank[i], rank[i+h]) for the suffixes still in groups of equal
//             rank, h = h0 * 2^(r-1): the doubling step of Manber & Myers.
// Round 0 is a stable LSD radix sort (radix.cu) of every suffix, then a rerank
// in which each tile handles the groups whose head it holds (no look-back): SA
// entries, new ranks (rank = SA index of the group head, i.e. the number of
// smaller suffixes, Sec. IV's "rank") staged by position bucket and applied
// bucket by bucket, the singletons dropped and the rest compacted.  Each later
// round only orders the members of every group by rank[i+h] (in-group sorts on
// chip, global radix passes for the largest groups; a group that is one
// arithmetic progression of positions is ordered at once), then reranks in a
// single pass with decoupled look-back, writing the few changed ranks in place.
// The later rounds run as one captured CUDA graph with a device-side loop when
// every group fits the on-chip sorts.  For sa_lcp_build round 0 also writes the
// LCP of every SA pair its keys separate.  A finisher (optional) sorts each
// remaining group by comparing rank sequences directly.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "block.cuh"
#include "common.cuh"

namespace dnasa {

namespace {

// ------------------------------------------------------------------ initial keys
constexpr int kInitThreads = 256;
constexpr int kInitItems = 8;

// pb > 0: the position is packed under the key, (key << pb) | p, and no value
// array is written (a keys-only sort then moves 8 instead of 12 bytes per item).
// The digit histograms of every pass of the initial sort (8-bit digits of the
// sort word from bit lo_bit on) are counted here too, so that the sort does not
// read the keys once more for them.  Grid-stride over chunks of 32 * kInitItems
// positions per warp.
//
// hist4 (one sequence, h0 = 4 * passes): a digit of the sort word is then the
// 4-mer code at a fixed offset from the suffix start, so every pass's histogram
// is the text's 4-mer histogram except near the two ends; only that histogram
// is counted here (one atomic per key instead of one per pass), into pass 0's
// slot, and k_hist4_fix derives each pass's histogram from it.
__global__ void __launch_bounds__(kInitThreads) k_init_keys(TextDesc t, int h0, int inst_shift,
                                                            int pb, int single, int passes, int lo_bit,
                                                            int hist4, uint32_t *__restrict__ ghist,
                                                            unsigned long long *__restrict__ keys,
                                                            uint32_t *__restrict__ vals) {
    __shared__ uint32_t sh[8 * 256];
    for (int i = threadIdx.x; i < passes * 256; i += kInitThreads) sh[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * kInitThreads) >> 5;
    for (int64_t warp = ((int64_t)blockIdx.x * kInitThreads + threadIdx.x) >> 5;
         warp * 32 * kInitItems < t.N; warp += nwarps) {
        const int64_t p0 = warp * 32 * kInitItems + lane;
        int64_t r = read_of(t.toff, t.n_reads, min(p0, t.N - 1));
        int64_t inst = 0;
        if (t.n_inst > 1) inst = upper_index(t.inst_toff, 0, t.n_inst, min(p0, t.N - 1));
#pragma unroll
        for (int i = 0; i < kInitItems; ++i) {
            const int64_t p = p0 + (int64_t)i * 32;
            if (p >= t.N) break;
            while (__ldg(t.toff + r + 1) <= p) ++r;
            if (t.n_inst > 1)
                while (__ldg(t.inst_toff + inst + 1) <= p) ++inst;
            const int64_t left = __ldg(t.toff + r + 1) - 1 - p;   // bases before this fragment's '$'
            const uint64_t x = bases32(t.packed, (uint64_t)(p - r));
            uint64_t kmer = x >> (64 - 2 * h0);
            const int lc = (int)min(left, (int64_t)h0);
            if (lc < h0) kmer &= ~((1ull << (2 * (h0 - lc))) - 1ull);
            unsigned long long key = ((unsigned long long)kmer << 5) | (unsigned long long)lc;
            if (t.n_inst > 1) key |= (unsigned long long)inst << inst_shift;
            unsigned long long w;
            int64_t at = p;
            if (single) {
                // one sequence: bases only, and the word stored at index f (h0_single):
                // the sort orders key bits only and keeps equal keys in input order,
                // which is then f order -- ended suffixes first, shorter first
                const unsigned long long f = lc < h0 ? (unsigned long long)lc : (unsigned long long)(p + h0);
                w = ((unsigned long long)kmer << pb) | f;
                at = (int64_t)f;
            } else if (pb) {
                w = (key << pb) | (unsigned long long)p;
            } else {
                w = key;
                vals[p] = (uint32_t)p;
            }
            keys[at] = w;
            if (hist4) {
                if (left >= 4) atomicAdd(&sh[(uint32_t)(x >> 56)], 1u);
            } else {
                for (int q = 0; q < passes; ++q)
                    atomicAdd(&sh[q * 256 + (uint32_t)((w >> (lo_bit + 8 * q)) & 255ull)], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (hist4 ? 1 : passes) * 256; i += kInitThreads) {
        const uint32_t c = sh[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

// One block of 256 threads, thread d = digit value d.  The 4-mer histogram H
// counts the codes at x = 0 .. N-5 (four bases before the '$').  Pass q's digit
// of a suffix p with h0 bases left is the code at x = p + o, o = h0 - 4 - 4q, for
// p = 0 .. N-1-h0: H without x < o and without x > N-1-h0+o; the h0 suffixes
// with fewer bases left carry a zero-padded key, counted one by one.
__global__ void __launch_bounds__(256) k_hist4_fix(TextDesc t, int h0, int passes, uint32_t *ghist) {
    // the codes near both ends and the ended suffixes' keys, fetched once (h0 <= 32 here)
    __shared__ uint32_t s_head[32], s_tail[32];
    __shared__ unsigned long long s_kmer[32];
    const uint32_t d = threadIdx.x;
    const int64_t N = t.N;
    if (d < 32 && (int)d < h0) {
        s_head[d] = (uint32_t)(bases32(t.packed, (uint64_t)d) >> 56);                  // x = d
        s_tail[d] = (uint32_t)(bases32(t.packed, (uint64_t)(N - h0 - 4 + d)) >> 56);   // x = N-h0-4+d
        const int64_t p = N - h0 + d;                                                  // ended suffix
        const int lc = (int)(N - 1 - p);                                               // 0 .. h0 - 1
        uint64_t kmer = bases32(t.packed, (uint64_t)p) >> (64 - 2 * h0);
        s_kmer[d] = kmer & ~((1ull << (2 * (h0 - lc))) - 1ull);
    }
    const uint32_t H = ghist[d];
    __syncthreads();
    for (int q = 0; q < passes; ++q) {
        const int o = h0 - 4 - 4 * q;
        int64_t c = H;
        for (int x = 0; x < o; ++x) c -= s_head[x] == d;
        for (int i = o + 4; i < h0; ++i) c -= s_tail[i] == d;   // x = N-h0-4+i = N-h0+o .. N-5
        for (int i = 0; i < h0; ++i) c += (uint32_t)((s_kmer[i] >> (8 * q)) & 255ull) == d;
        ghist[q * 256 + d] = (uint32_t)c;
    }
}

// ------------------------------------------------------------------ rerank + compact
constexpr int kRrThreads = 256;
constexpr int kRrItems = 8;
constexpr int kRrTile = kRrThreads * kRrItems;

// look-back word: [63:62] flag, [61:31] max head index + 1 (0: none), [30:0] kept count
constexpr unsigned long long RR_AGG = 1ull << 62;
constexpr unsigned long long RR_INC = 2ull << 62;

__device__ __forceinline__ unsigned long long rr_pack(unsigned long long flag, int64_t head,
                                                      int64_t keep) {
    return flag | ((unsigned long long)(head + 1) << 31) | (unsigned long long)keep;
}

// rank[] writes are staged by position bucket (2^bshift positions each) and
// applied bucket by bucket afterwards (k_rank_apply): a random 4-byte write into
// an array larger than L2 costs a random read-modify-write of a whole DRAM
// sector, while writes applied one 8 MB bucket at a time merge in L2.
constexpr int kMaxBuckets = 1024;

struct RerankOut {
    int64_t N;          // text length: bound of every SA slot and text position
    int kb;             // rounds >= 1: keys hold (old head rank << kb) | rank[i+h]
    uint32_t *sa, *rank;
    uint32_t *nslots, *npos, *nhead;
    uint2 *groups;
    unsigned long long *kept, *ngroups, *maxgroup;
    uint2 *stage;       // round 0 only, [N]: bucket b's (pos, rank) pairs start at b << bshift
    uint32_t *bucket_fill;   // [kMaxBuckets]
    int bshift;
    int pb;             // round 0 only: keys hold (key << pb) | position, no value array
    int single;         // round 0 only: (bases << pb) | f, f as in h0_single
    int32_t *lcp;       // round 0 only, may be null: LCP of every pair the initial keys separate,
                        // -1 where both suffixes share their initial key (LCP >= h0)
};

// Shared memory of one rerank tile of a doubling round (dynamic, > 48 KB).
struct RerankSmem {
    union {
        unsigned long long k[kRrTile + 2];   // keys with one halo key on each side
        struct {                             // reused once the head flags are known;
            // item li at li + li / 32 (padded: the blocked writes, eight
            // consecutive items per thread, then hit 32 distinct banks)
            uint32_t head[kRrTile + kRrTile / 32];   // new rank (SA slot of the group head)
            int32_t kp[kRrTile + kRrTile / 32];      // output index of a kept item, -1 if dropped
        } o;
    } u;
    uint32_t v[kRrTile];                 // positions
    uint32_t sl[kRrTile];                // SA slots
    uint32_t oh[kRrTile];                // old head rank
    uint32_t hb[kRrTile / 32];           // bit l of word w: item 32w + l starts a group
    uint32_t nb[kRrTile / 32];           // ... the item after it starts one (or the data end)
    int64_t tmp[kRrThreads / 32 + 1];
    int64_t incmax[kRrThreads];
    int64_t prefix[2];
    int64_t win_h[kRrThreads / 32], win_k[kRrThreads / 32];
    uint32_t win_nr[kRrThreads / 32], win_inc[kRrThreads / 32];
    uint32_t tile;
    int abort;
    int stop;
};

// One tile of a doubling round's rerank: the next tile id from the counter (ids
// are taken in order, so every tile a look-back waits on is held by a running
// CTA).  Returns false when there is no tile left or the look-back gave up.
__device__ __forceinline__ bool rerank_tile(RerankSmem &S,
    const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ slots, int64_t n, const RerankOut &o,
    unsigned long long *status, uint32_t *tile_ctr, uint32_t *err) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        S.tile = atomicAdd(tile_ctr, 1u);
        S.abort = 0;
    }
    __syncthreads();
    const uint32_t tile = S.tile;
    const int64_t base = (int64_t)tile * kRrTile;
    if (base >= n) return false;
    const int tile_n = (int)min((int64_t)kRrTile, n - base);

    // ---- striped, coalesced loads
    for (int i = tid; i < tile_n + 2; i += kRrThreads) {
        int64_t j = base - 1 + i;
        unsigned long long w = (j >= 0 && j < n) ? keys[j] : 0ull;
        S.u.k[i] = w;
        if (i >= 1 && i <= tile_n) S.oh[i - 1] = (uint32_t)(w >> o.kb);
    }
    for (int i = tid; i < tile_n; i += kRrThreads) {
        S.v[i] = vals[base + i];
        S.sl[i] = slots[base + i];
    }
    __syncthreads();
    // ---- head flags, striped (conflict-free shared reads)
    auto is_head = [&](int64_t j) -> bool {   // j in [base, base + tile_n]
        if (j == 0) return true;
        return S.u.k[j - base + 1] != S.u.k[j - base];
    };
    {   // one ballot per 32 consecutive items; the next item's flag is the next lane's
        const int lane = tid & 31;
        for (int b0 = tid - lane; b0 < tile_n; b0 += kRrThreads) {   // warp-uniform
            const int li = b0 + lane;
            const int64_t j = base + li;
            const bool in = li < tile_n;
            const bool h = in && is_head(j);
            const uint32_t hm = __ballot_sync(0xffffffffu, h);
            const bool nh = in && (j == n - 1 || (lane < 31 ? ((hm >> (lane + 1)) & 1u) != 0u
                                                            : is_head(j + 1)));
            const uint32_t nm = __ballot_sync(0xffffffffu, nh);
            if (lane == 0) {
                S.hb[b0 >> 5] = hm;
                S.nb[b0 >> 5] = nm;
            }
        }
    }
    __syncthreads();
    // ---- blocked scan: max head index and kept count
    int64_t my_max = -1, my_keep = 0;
    uint32_t headbits = 0, keepbits = 0, lastbits = 0;
    {
        static_assert(kRrItems == 8, "a thread's items are one byte of a flag word");
        const int sh = (tid * kRrItems) & 31;
        const uint32_t vm = tid * kRrItems >= tile_n ? 0u
                            : (1u << min(kRrItems, tile_n - tid * kRrItems)) - 1u;
        headbits = (S.hb[(tid * kRrItems) >> 5] >> sh) & vm;
        lastbits = (S.nb[(tid * kRrItems) >> 5] >> sh) & vm;
        keepbits = ~(headbits & lastbits) & vm;
        my_keep = __popc(keepbits);
        if (headbits) my_max = base + tid * kRrItems + 31 - __clz(headbits);
    }
    int64_t tile_max, tile_keep;
    int64_t inc_max = block_inclusive_max<kRrThreads>(my_max, S.tmp, &tile_max, (int64_t)-1);
    S.incmax[tid] = inc_max;
    int64_t ex_keep = block_exclusive_sum<kRrThreads>(my_keep, S.tmp, &tile_keep);

    // ---- decoupled look-back with the whole CTA: thread i probes tile - 1 - i,
    // so one round trip covers 256 predecessors.  (The inclusive prefix can
    // advance at most one window per round trip; a 32-wide window capped the
    // kernel at 32 tiles per status round trip.)
    {
        const int lane = tid & 31, warp = tid >> 5;
        if (tid == 0)
            st_relaxed_u64(status + tile, rr_pack(tile == 0 ? RR_INC : RR_AGG, tile_max, tile_keep));
        int64_t pmax = -1, psum = 0;
        int64_t wend = tile;          // window = tiles [wend - 256, wend - 1]
        uint32_t spins = 0;
        bool gave_up = false;
        while (tile != 0) {
            int64_t tt = wend - 1 - tid;
            unsigned long long w = tt >= 0 ? ld_relaxed_u64(status + tt) : RR_INC;  // virtual INC
            unsigned long long flag = w & (3ull << 62);
            uint32_t nr = __ballot_sync(0xffffffffu, flag == 0);
            uint32_t inc = __ballot_sync(0xffffffffu, flag == RR_INC);
            if (lane == 0) {
                S.win_nr[warp] = nr;
                S.win_inc[warp] = inc;
            }
            if (tid == 0) S.stop = (spins & 1023) == 1023 && ld_relaxed_u32(err) != 0;
            __syncthreads();
            const bool stop = S.stop;   // read before the next barrier: tid 0 rewrites it later
            // nearest INC over the window (lowest thread index), and readiness before it
            int near = kRrThreads;
            bool blocked = false;
            for (int v = 0; v < kRrThreads / 32; ++v) {
                uint32_t iv = S.win_inc[v], nv = S.win_nr[v];
                uint32_t need = iv ? ((iv & (0u - iv)) << 1) - 1u : 0xffffffffu;
                if (nv & need) { blocked = true; break; }
                if (iv) { near = v * 32 + __ffs(iv) - 1; break; }
            }
            if (!blocked) {
                bool take = tid <= near && tt >= 0;
                int64_t hv = take ? (int64_t)((w >> 31) & 0x7FFFFFFFull) - 1 : -1;
                int64_t kv = take ? (int64_t)(w & 0x7FFFFFFFull) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    hv = max(hv, __shfl_xor_sync(0xffffffffu, hv, o));
                    kv += __shfl_xor_sync(0xffffffffu, kv, o);
                }
                if (lane == 0) {
                    S.win_h[warp] = hv;
                    S.win_k[warp] = kv;
                }
            }
            __syncthreads();
            if (blocked) {   // uniform: every thread read the same shared words
                if (++spins > kSpinLimit || stop) {
                    gave_up = true;
                    break;
                }
                __nanosleep(64);
                continue;
            }
            for (int v = 0; v < kRrThreads / 32; ++v) {
                pmax = max(pmax, S.win_h[v]);
                psum += S.win_k[v];
            }
            __syncthreads();   // window arrays are rewritten by the next probe
            if (near < kRrThreads) break;
            wend -= kRrThreads;
        }
        if (tid == 0) {
            if (gave_up) {
                atomicOr(err, DERR_TIMEOUT);
                S.abort = 1;
            }
            if (tile != 0)
                st_relaxed_u64(status + tile, rr_pack(RR_INC, max(pmax, tile_max), psum + tile_keep));
            S.prefix[0] = pmax;
            S.prefix[1] = psum;
            if (base + tile_n == n) *o.kept = (unsigned long long)(psum + tile_keep);
        }
    }
    __syncthreads();
    if (S.abort) return false;   // prefix unknown: write nothing
    // ---- blocked: new rank and output index of every item.  A kept item that
    // ends its group records (first kept index, size) in the group list; the
    // list slots and the largest size are claimed with one atomic per warp.
    {
        int64_t cur = max(S.prefix[0], tid > 0 ? S.incmax[tid - 1] : (int64_t)-1);
        int64_t kp = S.prefix[1] + ex_keep;
        const int lane = tid & 31;
        uint32_t gend = keepbits & lastbits;
        uint32_t ng = __popc(gend);
        uint32_t ng_inc = ng;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ng_inc, off);
            if (lane >= off) ng_inc += y;
        }
        unsigned long long gbase = 0;
        if (lane == 31 && ng_inc) gbase = atomicAdd(o.ngroups, (unsigned long long)ng_inc);
        gbase = __shfl_sync(0xffffffffu, gbase, 31) + (ng_inc - ng);
        uint32_t my_maxsize = 0;
#pragma unroll
        for (int i = 0; i < kRrItems; ++i) {
            int li = tid * kRrItems + i;
            if (li >= tile_n) break;
            int64_t j = base + li;
            if (headbits >> i & 1u) cur = j;
            uint32_t slot = S.sl[li];
            S.u.o.head[li + (li >> 5)] = slot - (uint32_t)(j - cur);
            if (keepbits >> i & 1u) {
                S.u.o.kp[li + (li >> 5)] = (int32_t)kp;
                if (lastbits >> i & 1u) {
                    uint32_t size = (uint32_t)(j - cur + 1);
                    o.groups[gbase++] = make_uint2((uint32_t)(kp - size + 1), size);
                    my_maxsize = max(my_maxsize, size);
                }
                ++kp;
            } else {
                S.u.o.kp[li + (li >> 5)] = -1;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            my_maxsize = max(my_maxsize, __shfl_xor_sync(0xffffffffu, my_maxsize, off));
        if (lane == 0 && my_maxsize) atomicMax(o.maxgroup, (unsigned long long)my_maxsize);
    }
    __syncthreads();
    // ---- striped, coalesced writes; rank[pos] changes only where the item's group
    // head moved, and is written in place: a doubling round changes few ranks
    // (round 0, which writes all of them, stages them by position bucket instead)
    auto moved = [&](int li) -> bool { return S.u.o.head[li + (li >> 5)] != S.oh[li]; };
#pragma unroll
    for (int i = 0; i < kRrItems; ++i) {
        int li = tid + i * kRrThreads;
        if (li >= tile_n) break;
        uint32_t slot = S.sl[li];
        uint32_t pos = S.v[li];
        uint32_t hs = S.u.o.head[li + (li >> 5)];
        int32_t kp = S.u.o.kp[li + (li >> 5)];
        if ((int64_t)slot >= o.N || (int64_t)pos >= o.N || kp >= n) {
            atomicOr(err, DERR_BOUNDS);
            continue;
        }
        o.sa[slot] = pos;
        if (moved(li)) o.rank[pos] = hs;
        if (kp >= 0) {
            o.nslots[kp] = slot;
            o.npos[kp] = pos;
            o.nhead[kp] = hs;
        }
    }
    return true;
}

// A doubling round's rerank.  Persistent: each CTA takes tiles until none is
// left, so any grid covers the items (n from d_n when given: the count the
// previous round left on the device).
__global__ void __launch_bounds__(kRrThreads) k_rerank(
    const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ slots, int64_t n_host, const unsigned long long *__restrict__ d_n,
    RerankOut o, unsigned long long *status, uint32_t *tile_ctr, uint32_t *err) {
    extern __shared__ __align__(16) unsigned char rr_raw[];
    RerankSmem &S = *reinterpret_cast<RerankSmem *>(rr_raw);
    const int64_t n = d_n ? (int64_t)*d_n : n_host;
    while (rerank_tile(S, keys, vals, slots, n, o, status, tile_ctr, err)) __syncthreads();
}

// ------------------------------------------------------------------ round 0 without a look-back
// Round 0 needs no cross-tile prefix: every group (items with equal initial
// keys) is handled whole by the tile that holds its head.  A tile writes SA for
// its own items; for the groups whose heads it holds it writes the ranks (rank =
// SA slot of the group head, staged by position bucket), and reserves room for
// their kept members in the active list with one atomic, so that each group
// stays contiguous there (the order of the groups in the list is free: every
// later step works group by group).  A last group that runs past the tile is
// followed into the next tiles in global memory; a tile with no head leaves its
// items to the tile of their head.  (Later rounds, where most groups are a few
// dozen members and many cross a tile boundary, keep k_rerank's look-back: the
// look-back-free form measured slower there.)
constexpr int kR0Threads = 256;
constexpr int kR0Items = 8;
constexpr int kR0Tile = kR0Threads * kR0Items;

// Round 0's sorted word -> the key heads are compared on, and the position.
__device__ __forceinline__ void r0_decode(unsigned long long w, uint32_t val, const RerankOut &o, int h0,
                                          unsigned long long *key, uint32_t *pos) {
    if (o.single) {   // bit 0: 0 for an ended suffix (f < h0), which is its own group
        const uint32_t f = (uint32_t)(w & ((1ull << o.pb) - 1ull));
        const bool ended = f < (uint32_t)h0;
        *key = ((w >> o.pb) << 1) | (ended ? 0ull : 1ull);
        *pos = ended ? (uint32_t)(o.N - 1 - f) : f - (uint32_t)h0;
    } else if (o.pb) {
        *key = w >> o.pb;
        *pos = (uint32_t)(w & ((1ull << o.pb) - 1ull));
    } else {
        *key = w;
        *pos = val;
    }
}

// Does the item with compared key k start a group (kp: the key before it)?
__device__ __forceinline__ bool own_head(unsigned long long k, unsigned long long kp, const RerankOut &o,
                                         int h0) {
    if (o.single) return (k & 1ull) == 0 || (kp & 1ull) == 0 || k != kp;
    if ((int)(k & 31ull) < h0) return true;   // its own '$' lies inside the key: final
    return k != kp;
}

// LCP (bases, a '$' never matching) of two suffixes with different initial keys,
// from the keys alone: the equal leading bases of their h0-mers, capped by the
// bases each has before its '$'; 0 across instances.  ka/kb as r0_decode gives them.
__device__ __forceinline__ int32_t r0_lcp(unsigned long long ka, uint32_t pa, unsigned long long kb,
                                          uint32_t pb_, const RerankOut &o, int h0) {
    const unsigned long long km = (1ull << (2 * h0)) - 1ull;
    unsigned long long xa, xb;
    int la, lb;
    if (o.single) {   // (h0-mer << 1) | not-ended; bases left from the position
        xa = ka >> 1;
        xb = kb >> 1;
        la = (int)min((int64_t)h0, o.N - 1 - (int64_t)pa);
        lb = (int)min((int64_t)h0, o.N - 1 - (int64_t)pb_);
    } else {          // (instance << (2 h0 + 5)) | (h0-mer << 5) | bases left
        if ((ka >> (2 * h0 + 5)) != (kb >> (2 * h0 + 5))) return 0;
        xa = (ka >> 5) & km;
        xb = (kb >> 5) & km;
        la = (int)(ka & 31ull);
        lb = (int)(kb & 31ull);
    }
    const unsigned long long d = (xa ^ xb) << (64 - 2 * h0);
    const int eq = d ? (__clzll((long long)d) >> 1) : h0;
    return (int32_t)min(eq, min(la, lb));
}

struct OwnSmem {
    unsigned long long k[kR0Tile + 2];   // compared keys, one halo key on each side
    uint32_t v[kR0Tile];                 // positions
    uint32_t hd[kR0Tile + kR0Tile / 32]; // rank of each owned item, item li at li + li / 32 (the
                                         // blocked writes, 8 items per thread, hit distinct banks)
    uint32_t hb[kR0Tile / 32];           // bit l of word w: item 32w + l starts a group
    uint32_t nb[kR0Tile / 32];           // ... the item after it starts one (or the data end)
    int64_t tmp[kR0Threads / 32 + 1];
    uint32_t bcnt[kMaxBuckets];          // per-bucket counts of a chunk, then global bases
    uint32_t vh;                         // position of the item before the tile (its halo)
    int64_t own_end;                     // end of the last group whose head is in the tile
    unsigned long long kp_base;          // list index of the tile's first kept item
    int first_head;                      // tile-local index of the first head (tile_n: none)
};

// Stages rank writes (pos -> rank) of a chunk of items: counts per position
// bucket in shared memory, one global atomic per bucket, then the writes.
// Every thread calls; item i of the chunk is (pos(i), rank(i)) for i < cnt when
// take(i) is true.
template <typename SM, typename Pos, typename Rank, typename Take>
__device__ __forceinline__ void own_stage(SM &S, const RerankOut &o, int cnt, Pos pos, Rank rank, Take take,
                                          uint32_t *err) {
    const int nb = (int)((o.N + (1ll << o.bshift) - 1) >> o.bshift);
    for (int b = threadIdx.x; b < nb; b += kR0Threads) S.bcnt[b] = 0;
    __syncthreads();
    uint32_t idx[kR0Items];
#pragma unroll
    for (int q = 0; q < kR0Items; ++q) {
        const int i = threadIdx.x + q * kR0Threads;
        idx[q] = (i < cnt && take(i)) ? atomicAdd(&S.bcnt[pos(i) >> o.bshift], 1u) : 0u;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += kR0Threads) {
        const uint32_t c = S.bcnt[b];
        if (c) S.bcnt[b] = atomicAdd(&o.bucket_fill[b], c);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kR0Items; ++q) {
        const int i = threadIdx.x + q * kR0Threads;
        if (i >= cnt || !take(i)) continue;
        const uint32_t p = pos(i);
        const uint32_t b = p >> o.bshift;
        const uint64_t st = ((uint64_t)b << o.bshift) + S.bcnt[b] + idx[q];
        if ((int64_t)p >= o.N || (int64_t)st >= o.N) {
            atomicOr(err, DERR_BOUNDS);
            continue;
        }
        o.stage[st] = make_uint2(p, rank(i));
    }
    __syncthreads();
}

__device__ __forceinline__ void own_load(const unsigned long long *__restrict__ keys,
                                         const uint32_t *__restrict__ vals, int64_t j, const RerankOut &o,
                                         int h0, unsigned long long *key, uint32_t *pos) {
    r0_decode(keys[j], o.pb ? 0u : vals[j], o, h0, key, pos);
}

__global__ void __launch_bounds__(kR0Threads, 5) k_rerank0(const unsigned long long *__restrict__ keys,
                                                        const uint32_t *__restrict__ vals, int64_t n, int h0,
                                                        RerankOut o, uint32_t *err) {
    __shared__ OwnSmem S;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t base = (int64_t)blockIdx.x * kR0Tile;
    if (base >= n) return;
    const int tile_n = (int)min((int64_t)kR0Tile, n - base);

    // ---- keys (one halo each side) and positions; SA of the tile's items.  All
    // of a thread's loads are issued before its first store (the SA store could
    // alias the keys as far as the compiler knows, which would serialise them).
    {
        unsigned long long w[kR0Items];
        uint32_t vv[kR0Items];
#pragma unroll
        for (int q = 0; q < kR0Items; ++q) {
            const int i = tid + q * kR0Threads;
            w[q] = i < tile_n ? keys[base + i] : 0ull;
            vv[q] = (i < tile_n && !o.pb) ? vals[base + i] : 0u;
        }
        int64_t hj = -1;   // threads 0 and 1: the halo items before and after the tile
        unsigned long long hw = 0;
        uint32_t hv = 0;
        if (tid < 2) {
            hj = tid == 0 ? base - 1 : base + tile_n;
            if (hj >= 0 && hj < n) {
                hw = keys[hj];
                hv = o.pb ? 0u : vals[hj];
            }
        }
#pragma unroll
        for (int q = 0; q < kR0Items; ++q) {
            const int i = tid + q * kR0Threads;
            if (i >= tile_n) break;
            unsigned long long key;
            uint32_t pos;
            r0_decode(w[q], vv[q], o, h0, &key, &pos);
            S.k[i + 1] = key;
            S.v[i] = pos;
            if ((int64_t)pos < o.N) o.sa[base + i] = pos;
            else atomicOr(err, DERR_BOUNDS);
        }
        if (tid < 2) {   // outside [0, n): the decode of a zero word, as a neighbour only
            unsigned long long key;
            uint32_t pos;
            if (hj >= 0 && hj < n) r0_decode(hw, hv, o, h0, &key, &pos);
            else r0_decode(0ull, 0u, o, h0, &key, &pos);
            S.k[tid == 0 ? 0 : tile_n + 1] = key;
            if (tid == 0) S.vh = pos;
        }
    }
    __syncthreads();
    // ---- head flags, one ballot per 32 consecutive items
    for (int b0 = tid - lane; b0 < tile_n; b0 += kR0Threads) {   // warp-uniform
        const int li = b0 + lane;
        const int64_t j = base + li;
        const bool in = li < tile_n;
        const bool h = in && (j == 0 || own_head(S.k[li + 1], S.k[li], o, h0));
        const uint32_t hm = __ballot_sync(0xffffffffu, h);
        bool nh = false;
        if (in) {
            if (j == n - 1) nh = true;
            else if (lane < 31 && li + 1 < tile_n) nh = ((hm >> (lane + 1)) & 1u) != 0u;
            else nh = own_head(S.k[li + 2], S.k[li + 1], o, h0);
        }
        const uint32_t nm = __ballot_sync(0xffffffffu, nh);
        if (lane == 0) {
            S.hb[b0 >> 5] = hm;
            S.nb[b0 >> 5] = nm;
        }
    }
    __syncthreads();
    // ---- LCP with the SA predecessor, where the initial keys decide it (coalesced)
    if (o.lcp) {
        for (int i = tid; i < tile_n; i += kR0Threads) {
            const int64_t j = base + i;
            int32_t v;
            if (j == 0) v = 0;
            else if (((S.hb[i >> 5] >> (i & 31)) & 1u) == 0u) v = -1;   // same initial key
            else v = r0_lcp(S.k[i], i > 0 ? S.v[i - 1] : S.vh, S.k[i + 1], S.v[i], o, h0);
            o.lcp[j] = v;
        }
    }
    // ---- first head of the tile; end of its last group (past the tile if needed)
    if (tid < 32) {
        int fh = tile_n;
        const int words = (tile_n + 31) / 32;
        for (int w0 = 0; w0 < words; w0 += 32) {
            const int w = w0 + lane;
            const uint32_t hm = w < words ? S.hb[w] : 0u;
            const uint32_t any = __ballot_sync(0xffffffffu, hm != 0u);
            if (any) {
                const int wl = __ffs(any) - 1;
                const uint32_t hw = __shfl_sync(0xffffffffu, hm, wl);
                fh = (w0 + wl) * 32 + __ffs(hw) - 1;
                break;
            }
        }
        int64_t end = base + tile_n;
        const int last = tile_n - 1;
        const bool closed = (S.nb[last >> 5] >> (last & 31)) & 1u;
        if (fh < tile_n && !closed) {
            // follow the last group into the next tiles.  The keys are sorted and a
            // group that runs past a tile has a key no ended suffix shares, so its
            // end is the first slot whose key differs: found by galloping (lane l
            // probes 2^l slots on), then by 32-way splits of the bracket
            const unsigned long long gk = S.k[tile_n];   // key of the tile's last item
            auto differs = [&](int64_t j) -> bool {
                if (j >= n) return true;
                unsigned long long key;
                uint32_t pos;
                own_load(keys, vals, j, o, h0, &key, &pos);
                return key != gk;
            };
            int64_t a = base + tile_n - 1;                  // last slot known in the group
            int64_t b;                                      // a slot known past it
            {
                const int64_t j = a + ((int64_t)1 << lane);
                const uint32_t dm = __ballot_sync(0xffffffffu, differs(j));
                const int l = __ffs(dm) - 1;                // lane 31 reaches past n: dm != 0
                b = a + ((int64_t)1 << l);
                if (l > 0) a += (int64_t)1 << (l - 1);
            }
            while (b - a > 1) {
                const int64_t step = (b - a + 32) / 33;     // 32 probes inside (a, b)
                const int64_t j = min(a + step * (lane + 1), b - 1);
                const uint32_t dm = __ballot_sync(0xffffffffu, differs(j));
                const int l = dm ? __ffs(dm) - 1 : 32;
                const int64_t nb = l < 32 ? min(a + step * (l + 1), b - 1) : b;
                const int64_t na = l > 0 ? min(a + step * l, b - 1) : a;
                a = na;
                b = nb;
            }
            end = b;
        }
        if (lane == 0) {
            S.first_head = fh;
            S.own_end = end;
        }
    }
    __syncthreads();
    const int fh = S.first_head;
    if (fh >= tile_n) return;   // every item belongs to a group whose head is in an earlier tile
    const int64_t spill = S.own_end - (base + tile_n);

    // ---- blocked: rank and kept index of every owned item
    static_assert(kR0Items == 8, "a thread's items are one byte of a flag word");
    const int sh = (tid * kR0Items) & 31;
    uint32_t vm = tid * kR0Items >= tile_n ? 0u : (1u << min(kR0Items, tile_n - tid * kR0Items)) - 1u;
    {   // items before the first head belong to an earlier tile
        const int lo = fh - tid * kR0Items;
        if (lo > 0) vm &= lo >= kR0Items ? 0u : ~((1u << lo) - 1u);
    }
    const uint32_t headbits = (S.hb[(tid * kR0Items) >> 5] >> sh) & vm;
    const uint32_t lastbits = (S.nb[(tid * kR0Items) >> 5] >> sh) & vm;
    const uint32_t keepbits = ~(headbits & lastbits) & vm;
    const int64_t my_max = headbits ? base + tid * kR0Items + 31 - __clz(headbits) : -1;
    int64_t tile_max, tile_keep;
    const int64_t inc_max = block_inclusive_max<kR0Threads>(my_max, S.tmp, &tile_max, (int64_t)-1);
    const int64_t ex_max = __shfl_up_sync(0xffffffffu, inc_max, 1);
    const int64_t ex_keep = block_exclusive_sum<kR0Threads>((int64_t)__popc(keepbits), S.tmp, &tile_keep);
    if (tid == 0) S.kp_base = atomicAdd(o.kept, (unsigned long long)(tile_keep + spill));
    int64_t cur;   // list index of the head before this thread's items
    {
        const int w = tid >> 5;
        __syncthreads();
        if (lane == 31) S.tmp[w] = inc_max;
        __syncthreads();
        int64_t before = -1;
        for (int x = 0; x < w; ++x) before = max(before, S.tmp[x]);
        cur = lane > 0 ? max(before, ex_max) : before;
    }
    __syncthreads();
    const unsigned long long kp0 = S.kp_base;
    {
        const uint32_t gend = keepbits & lastbits;
        const uint32_t ng = __popc(gend);
        uint32_t ng_inc = ng;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ng_inc, off);
            if (lane >= off) ng_inc += y;
        }
        unsigned long long gbase = 0;
        if (lane == 31 && ng_inc) gbase = atomicAdd(o.ngroups, (unsigned long long)ng_inc);
        gbase = __shfl_sync(0xffffffffu, gbase, 31) + (ng_inc - ng);
        uint32_t my_maxsize = 0;
        unsigned long long kp = kp0 + (unsigned long long)ex_keep;
#pragma unroll
        for (int i = 0; i < kR0Items; ++i) {
            const int li = tid * kR0Items + i;
            if (!((vm >> i) & 1u)) continue;
            const int64_t j = base + li;
            if ((headbits >> i) & 1u) cur = j;
            const uint32_t rk = (uint32_t)cur;
            S.hd[li + (li >> 5)] = rk;
            if ((keepbits >> i) & 1u) {
                if (kp >= (unsigned long long)n) {
                    atomicOr(err, DERR_BOUNDS);
                } else {
                    o.nslots[kp] = (uint32_t)j;
                    o.npos[kp] = S.v[li];
                    o.nhead[kp] = rk;
                }
                if ((lastbits >> i) & 1u) {
                    const uint32_t size = (uint32_t)(j - cur + 1);
                    o.groups[gbase++] = make_uint2((uint32_t)(kp - size + 1), size);
                    my_maxsize = max(my_maxsize, size);
                }
                ++kp;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            my_maxsize = max(my_maxsize, __shfl_xor_sync(0xffffffffu, my_maxsize, off));
        if (lane == 0 && my_maxsize) atomicMax(o.maxgroup, (unsigned long long)my_maxsize);
    }
    __syncthreads();
    // ---- ranks of the owned items in the tile
    own_stage(S, o, tile_n, [&](int i) { return S.v[i]; }, [&](int i) { return S.hd[i + (i >> 5)]; },
              [&](int i) { return i >= fh; }, err);
    if (spill <= 0) return;
    // ---- the last group continues past the tile: all of it kept, one rank
    const uint32_t rk = S.hd[(tile_n - 1) + ((tile_n - 1) >> 5)];
    const unsigned long long kps = kp0 + (unsigned long long)tile_keep;
    for (int64_t c0 = base + tile_n; c0 < S.own_end; c0 += kR0Tile) {
        const int cnt = (int)min((int64_t)kR0Tile, S.own_end - c0);
        for (int i = tid; i < cnt; i += kR0Threads) {
            unsigned long long key;
            uint32_t pos;
            own_load(keys, vals, c0 + i, o, h0, &key, &pos);
            S.v[i] = pos;
            const unsigned long long kp = kps + (unsigned long long)(c0 - base - tile_n + i);
            if (kp >= (unsigned long long)n || (int64_t)pos >= o.N) {
                atomicOr(err, DERR_BOUNDS);
                continue;
            }
            o.nslots[kp] = (uint32_t)(c0 + i);
            o.npos[kp] = pos;
            o.nhead[kp] = rk;
        }
        __syncthreads();
        own_stage(S, o, cnt, [&](int i) { return S.v[i]; }, [&](int) { return rk; }, [&](int) { return true; },
                  err);
    }
    if (tid == 0) {
        const uint32_t size = (uint32_t)(S.own_end - tile_max);
        o.groups[atomicAdd(o.ngroups, 1ull)] = make_uint2((uint32_t)(kp0 + tile_keep + spill - size), size);
        atomicMax(o.maxgroup, (unsigned long long)size);
    }
}

// Applies the staged rank writes, bucket-major: the buckets' filled parts are
// taken as one concatenated list, each CTA a kApplyItems slice of it, so the
// grid matches the items staged (CTAs are issued roughly in index order, so one
// bucket's 8 MB of rank[] is written at a time).
constexpr int kApplyItems = 4096;
__global__ void __launch_bounds__(256) k_rank_apply(const uint2 *__restrict__ stage,
                                                    const uint32_t *__restrict__ bucket_fill,
                                                    int nbuckets, int bshift, int64_t N,
                                                    uint32_t *__restrict__ rank, uint32_t *err) {
    __shared__ uint32_t s_off[kMaxBuckets + 1];   // exclusive prefix of the fills
    __shared__ uint32_t s_tmp[256 / 32 + 1];
    {
        static_assert(kMaxBuckets == 4 * 256, "four buckets per thread");
        uint32_t c[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int bb = 4 * threadIdx.x + q;
            c[q] = bb < nbuckets ? bucket_fill[bb] : 0u;
            sum += c[q];
        }
        uint32_t tot;
        uint32_t run = block_exclusive_sum<256>(sum, s_tmp, &tot);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int bb = 4 * threadIdx.x + q;
            if (bb < nbuckets) s_off[bb] = run;
            run += c[q];
        }
        if (threadIdx.x == 0) s_off[nbuckets] = tot;
    }
    __syncthreads();
    const uint32_t total = s_off[nbuckets];
    // slices of kApplyItems staged pairs, grid-stride (one CTA per slice when the
    // grid matches the items staged)
    for (uint64_t g0 = (uint64_t)blockIdx.x * kApplyItems; g0 < total;
         g0 += (uint64_t)gridDim.x * kApplyItems) {
        const uint32_t f0 = (uint32_t)g0;
        const uint32_t f1 = min(total, f0 + kApplyItems);
        // first bucket holding flat index f0
        int b = 0;
        {
            int lo = 0, hi = nbuckets - 1;
            while (lo < hi) {
                int m = (lo + hi + 1) >> 1;
                if (s_off[m] <= f0) lo = m; else hi = m - 1;
            }
            b = lo;
        }
        // all of a thread's staged pairs are loaded before any rank write, so that
        // the loads are in flight together
        constexpr int kPer = kApplyItems / 256;
        uint2 pr[kPer];
        int pb_[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t f = f0 + threadIdx.x + q * 256;
            pb_[q] = -1;
            if (f < f1) {
                while (f >= s_off[b + 1]) ++b;   // non-decreasing f per thread
                pb_[q] = b;
                pr[q] = stage[((uint64_t)b << bshift) + (f - s_off[b])];
            }
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            if (pb_[q] < 0) continue;
            if ((int64_t)pr[q].x < N && (pr[q].x >> bshift) == (uint32_t)pb_[q]) rank[pr[q].x] = pr[q].y;
            else atomicOr(err, DERR_BOUNDS);
        }
    }
}

// ------------------------------------------------------------------ doubling gather
// n and h from d_n / d_h when given (a device-driven round).
__global__ void __launch_bounds__(256) k_gather(const uint32_t *__restrict__ npos,
                                                const uint32_t *__restrict__ nhead, int64_t n_host,
                                                const unsigned long long *__restrict__ d_n,
                                                const uint32_t *__restrict__ rank, uint32_t h_host,
                                                const uint32_t *__restrict__ d_h,
                                                int b, unsigned long long *__restrict__ keys,
                                                uint32_t *__restrict__ vals, int64_t N,
                                                uint32_t *err) {
    const int64_t n = d_n ? (int64_t)*d_n : n_host;
    const uint32_t h = d_h ? *d_h : h_host;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t pos = npos[t];
        uint32_t r2 = 0;
        if ((int64_t)pos + h < N) r2 = __ldg(rank + pos + h);
        else atomicOr(err, DERR_BOUNDS);
        keys[t] = ((unsigned long long)nhead[t] << b) | r2;
        vals[t] = pos;
    }
}

// ------------------------------------------------------------------ direct finisher
// Each remaining group shares its first h symbols.  rank[] holds h-ranks (equal
// ranks <=> equal first h symbols; a rank that contains a '$' is unique), so two
// members p, q compare as the sequences rank[p+h], rank[p+2h], rank[p+3h], ...:
// every step compares the next h symbols at once, which keeps tandem repeats
// thousands of bases long to a handful of steps.  rank[p+h] is cached in shared
// memory; one CTA sorts one group with a bitonic network.
constexpr int kFinMax = 1024;
constexpr int kFinThreads = 512;

__device__ __forceinline__ bool fin_less(uint32_t pa, uint32_t ra, uint32_t pb, uint32_t rb,
                                         const uint32_t *__restrict__ rank, uint32_t h, int64_t N,
                                         uint32_t *err) {
    if (ra != rb) return ra < rb;
    for (int64_t k = 2;; ++k) {
        int64_t xa = (int64_t)pa + k * h, xb = (int64_t)pb + k * h;
        if (xa >= N || xb >= N) {   // cannot happen for valid ranks
            atomicOr(err, DERR_BOUNDS);
            return pa < pb;
        }
        uint32_t a = __ldg(rank + xa), b = __ldg(rank + xb);
        if (a != b) return a < b;
    }
}

__global__ void __launch_bounds__(kFinThreads) k_finish(const uint2 *__restrict__ groups,
                                                        const unsigned long long *__restrict__ ngroups,
                                                        const uint32_t *__restrict__ npos,
                                                        const uint32_t *__restrict__ nslots,
                                                        const uint32_t *__restrict__ rank,
                                                        uint32_t h, int64_t N,
                                                        uint32_t *__restrict__ sa, uint32_t *err) {
    __shared__ uint32_t s_pos[kFinMax];
    __shared__ uint32_t s_r1[kFinMax];
    __shared__ uint16_t s_idx[kFinMax];
    const int64_t ng = (int64_t)*ngroups;
    for (int64_t g = blockIdx.x; g < ng; g += gridDim.x) {
        uint2 gs = groups[g];
        const int size = (int)min(gs.y, (uint32_t)kFinMax);
        int n2 = 1;
        while (n2 < size) n2 <<= 1;
        for (int i = threadIdx.x; i < n2; i += kFinThreads) {
            s_idx[i] = (uint16_t)i;
            if (i < size) {
                uint32_t pos = npos[gs.x + i];
                s_pos[i] = pos;
                s_r1[i] = (int64_t)pos + h < N ? __ldg(rank + pos + h) : 0u;
            }
        }
        __syncthreads();
        for (int k = 2; k <= n2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < n2; i += kFinThreads) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        uint16_t a = s_idx[i], c = s_idx[ixj];
                        bool up = (i & k) == 0;
                        // padding members (index >= size) are larger than everything
                        bool swap;
                        if (a >= size || c >= size) {
                            swap = up ? (a >= size && c < size) : (c >= size && a < size);
                        } else if (up) {
                            swap = fin_less(s_pos[c], s_r1[c], s_pos[a], s_r1[a], rank, h, N, err);
                        } else {
                            swap = fin_less(s_pos[a], s_r1[a], s_pos[c], s_r1[c], rank, h, N, err);
                        }
                        if (swap) {
                            s_idx[i] = c;
                            s_idx[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        uint32_t slot0 = nslots[gs.x];
        for (int i = threadIdx.x; i < size; i += kFinThreads)
            if ((int64_t)slot0 + i < N) sa[slot0 + i] = s_pos[s_idx[i]];
        __syncthreads();
    }
}

// ------------------------------------------------------------------ in-group sorting
// From the first doubling round on, a round only has to order the members of each group by
// rank[i+h] (all members of a group share the high key part, the head rank),
// and members with equal keys stay together in one group that a later round
// sorts again, so no stable order is needed.  Groups of at most 8 members are
// sorted by one thread, up to 256 by one warp in registers (bitonic networks),
// up to kSegMax by one CTA (radix passes in shared memory); only the members of
// larger groups go through the global radix sort.  Each item is then read and
// written once instead of once per global radix pass, and a group whose members
// all carry the same rank[i+h] is left as it is.
constexpr int kSegMax = 12288;     // largest group sorted on chip (one CTA, shared memory)
constexpr int kSegWarpMax = 256;   // one warp, registers
constexpr int kSegThreads = 512;

// Inside one group every key has the same high part (the head rank), so a
// member is ordered by its low key part rank[i+h] and, to make every word
// distinct, its position: one 64-bit word (rank[i+h] << 32 | position) per
// member, compared as an integer.
__device__ __forceinline__ unsigned long long seg_word(unsigned long long k, uint32_t v,
                                                       unsigned long long rmask) {
    return ((k & rmask) << 32) | v;
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long x, int m) {
    uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)x, m);
    uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(x >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}

// A group whose members sit at the positions i, i+p, ..., i+(n-1)p of one arithmetic
// progression with p <= h (h: the number of symbols every member shares) lies in a
// periodic stretch of the text: T[x] = T[x+p] for every x from i up to past
// i+(n-1)p+h.  Any two members first differ at the same text position e, where that
// period breaks, and compare there as T[e] against T[e-p]; the whole group is
// therefore in position order or in the reverse order.  The last two members
// (max-p, max) tell which: they agree beyond their first h symbols, so they compare
// as the suffixes h further on, and those two differ within their first h symbols
// (max+p is not a member, so the period breaks before max+p+h), so their h-ranks
// rank[max-p+h] and rank[max+h], gathered as the members' low key parts, differ and
// order them.  Such a group is ordered at once instead of log2(run length / h) rounds
// later: the suffixes of one phase of a tandem array.  ap_period() returns p, or 0
// when the positions are not such a progression.
__device__ __forceinline__ uint32_t ap_period(uint32_t pmin, uint32_t pmax, int n, uint32_t h) {
    if (n < 3) return 0;   // two members: their low key parts already differ if it applies
    const uint32_t d = pmax - pmin;
    // a step above h is excluded first by a multiply, so most groups (members far
    // apart: copies of a repeat, reads of one locus) never reach the division
    if ((uint64_t)d > (uint64_t)h * (uint64_t)(n - 1)) return 0;
    if (d % (uint32_t)(n - 1) != 0) return 0;
    return d / (uint32_t)(n - 1);
}

// For sa_lcp_build: the LCP of every adjacent pair of an arithmetic-progression
// group, in closed form.  The members share the period up to the text position e
// where it breaks (the same e for every pair), so two members at positions a < b
// agree on exactly e - b bases; e = max + LCP(max - p, max), and that LCP is h
// plus the LCP of the suffixes h further on, which differ within h bases: one
// comparison of at most h bases per group.  lcp null: not wanted.
struct ApLcp {
    int32_t *lcp;
    const uint32_t *slots;   // SA slot of each active item (a group's are consecutive)
    TextDesc t;
};

// Common prefix (bases, a '$' never matching) of the suffixes at a and b, at most lim.
__device__ __forceinline__ int64_t text_lcp(const TextDesc &t, int64_t a, int64_t b, int64_t lim) {
    const int64_t ra = frag_of(t, a), rb = frag_of(t, b);
    const int64_t m = min(lim, min(__ldg(t.toff + ra + 1) - 1 - a, __ldg(t.toff + rb + 1) - 1 - b));
    for (int64_t k = 0; k < m; k += 32) {
        const uint64_t d = bases32(t.packed, (uint64_t)(a - ra + k)) ^ bases32(t.packed, (uint64_t)(b - rb + k));
        if (d) return min(m, k + (int64_t)(__clzll((long long)d) >> 1));
    }
    return m;
}

// The break position e of a progression group (members pmin .. pmax, step p,
// sharing h symbols).
__device__ __forceinline__ int64_t ap_break(const TextDesc &t, uint32_t pmax, uint32_t p, uint32_t h) {
    return (int64_t)pmax + h + text_lcp(t, (int64_t)pmax - p + h, (int64_t)pmax + h, h);
}

// LCP entry of the member at sorted index j >= 1 of a progression group.
__device__ __forceinline__ void ap_lcp_write(const ApLcp &al, uint32_t slot0, uint32_t j, uint32_t pmin,
                                             uint32_t pmax, uint32_t p, bool asc, int64_t e, uint32_t *err) {
    if (j == 0) return;   // the pair before the group was separated earlier
    const int64_t hi_pos = asc ? (int64_t)pmin + (int64_t)j * p : (int64_t)pmax - (int64_t)(j - 1) * p;
    const int64_t slot = (int64_t)slot0 + j;
    if (slot < al.t.N && e >= hi_pos) al.lcp[slot] = (int32_t)(e - hi_pos);
    else atomicOr(err, DERR_BOUNDS);
}

// Index of a member within an arithmetic-progression group in suffix order.
__device__ __forceinline__ uint32_t ap_index(uint32_t pos, uint32_t pmin, uint32_t pmax, uint32_t p,
                                             bool ascending) {
    return (ascending ? pos - pmin : pmax - pos) / p;
}

// Splits the group list into five lists by size (<= 8, <= 32, <= kSegWarpMax,
// <= seg_max, larger), one atomic per warp and list.
__global__ void __launch_bounds__(256) k_classify(const uint2 *__restrict__ groups, int64_t ng_host,
                                                  const unsigned long long *__restrict__ d_ng,
                                                  int seg_max, uint2 *__restrict__ tiny,
                                                  uint2 *__restrict__ small, uint2 *__restrict__ wmid,
                                                  uint2 *__restrict__ mid, uint2 *__restrict__ large,
                                                  unsigned long long *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t ng = d_ng ? (int64_t)*d_ng : ng_host;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; b < ng; b += stride) {
        const int64_t g = b + lane;
        uint2 gs = g < ng ? groups[g] : make_uint2(0, 0);
        const int sz = (int)gs.y;
        const int cls = g >= ng ? -1 : sz > seg_max ? 4 : sz <= 8 ? 0 : sz <= 32 ? 1
                                                 : sz <= kSegWarpMax ? 2 : 3;
        uint2 *lists[5] = {tiny, small, wmid, mid, large};
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            uint32_t m = __ballot_sync(0xffffffffu, cls == c);
            if (!m) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&counts[c], (unsigned long long)__popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (cls == c) lists[c][base + __popc(m & lanemask_lt())] = gs;
        }
    }
}

// Groups of at most 8 members: one thread each, insertion sort in registers.
__global__ void __launch_bounds__(256) k_seg_thread(const uint2 *__restrict__ groups,
                                                    const unsigned long long *__restrict__ d_ng,
                                                    int b, uint32_t h_host, const uint32_t *__restrict__ d_h,
                                                    unsigned long long *__restrict__ keys,
                                                    uint32_t *__restrict__ vals, ApLcp al, uint32_t *err) {
    const int64_t ng = (int64_t)*d_ng;
    const uint32_t h = d_h ? *d_h : h_host;
    const unsigned long long rmask = (1ull << b) - 1ull;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x) {
        const uint2 gs = groups[g];
        const int n = (int)gs.y;   // 2..8
        const unsigned long long hi = keys[gs.x] & ~rmask;
        unsigned long long w[8];
        uint32_t pmin = ~0u, pmax = 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            w[i] = i < n ? seg_word(keys[gs.x + i], vals[gs.x + i], rmask) : ~0ull;
            if (i < n) {
                pmin = min(pmin, (uint32_t)w[i]);
                pmax = max(pmax, (uint32_t)w[i]);
            }
        }
        if (const uint32_t p = ap_period(pmin, pmax, n, h)) {
            bool ok = true;
            uint32_t kmax = 0, kprev = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < n) {
                    const uint32_t v = (uint32_t)w[i];
                    ok = ok && (v - pmin) % p == 0;
                    if (v == pmax) kmax = (uint32_t)(w[i] >> 32);
                    if (v == pmax - p) kprev = (uint32_t)(w[i] >> 32);
                }
            if (ok && kmax != kprev) {
                const int64_t e = al.lcp ? ap_break(al.t, pmax, p, h) : 0;
                const uint32_t slot0 = al.lcp ? al.slots[gs.x] : 0u;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i < n) {
                        const uint32_t v = (uint32_t)w[i];
                        const uint32_t j = ap_index(v, pmin, pmax, p, kprev < kmax);
                        keys[gs.x + j] = hi | j;
                        vals[gs.x + j] = v;
                        if (al.lcp) ap_lcp_write(al, slot0, j, pmin, pmax, p, kprev < kmax, e, err);
                    }
                continue;
            }
        }
#pragma unroll
        for (int i = 1; i < 8; ++i) {
#pragma unroll
            for (int j = i; j > 0; --j) {
                unsigned long long a = w[j - 1], c = w[j];
                w[j - 1] = min(a, c);
                w[j] = max(a, c);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (i < n) {
                keys[gs.x + i] = hi | (w[i] >> 32);
                vals[gs.x + i] = (uint32_t)w[i];
            }
    }
}

// Bitonic network over 32 * E words held E per lane (word i = e * 32 + lane):
// strides below 32 exchange across lanes by shuffles, larger ones inside a lane.
// With E == 1 only the first n2 lanes take part (n2 a power of two, 2..32);
// with E > 1 all 32 * E words do.
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&w)[E], int lane, int n2) {
    const int lim = E == 1 ? n2 : 32 * E;
#pragma unroll
    for (int size = 2; size <= 32 * E; size <<= 1) {
        if (size > lim) continue;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int es = stride >> 5;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & es) == 0) {
                        const bool asc = ((e * 32) & size) == 0;   // size >= 64: lane bits are below it
                        unsigned long long a = w[e], c = w[e | es];
                        unsigned long long lo = min(a, c), hi = max(a, c);
                        w[e] = asc ? lo : hi;
                        w[e | es] = asc ? hi : lo;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    unsigned long long o = shfl_xor_u64(w[e], stride);
                    const bool keep_min = ((lane & stride) == 0) == (((e * 32 + lane) & size) == 0);
                    w[e] = keep_min ? min(w[e], o) : max(w[e], o);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void warp_sort_group(uint2 gs, int lane, int n2, unsigned long long rmask,
                                                uint32_t h, unsigned long long *__restrict__ keys,
                                                uint32_t *__restrict__ vals, const ApLcp &al, uint32_t *err) {
    const int n = (int)gs.y;
    const unsigned long long k0 = keys[gs.x];
    const unsigned long long hi = k0 & ~rmask;
    unsigned long long w[E];
    uint32_t x = 0;   // bits in which some rank differs from the first
    uint32_t pmin = ~0u, pmax = 0u;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = e * 32 + lane;
        w[e] = i < n ? seg_word(keys[gs.x + i], vals[gs.x + i], rmask) : ~0ull;
        if (i < n) {
            x |= (uint32_t)(w[e] >> 32) ^ (uint32_t)(k0 & rmask);
            pmin = min(pmin, (uint32_t)w[e]);
            pmax = max(pmax, (uint32_t)w[e]);
        }
    }
    if (!__any_sync(0xffffffffu, x != 0)) return;   // one rank for all: already in order
    pmin = __reduce_min_sync(0xffffffffu, pmin);
    pmax = __reduce_max_sync(0xffffffffu, pmax);
    if (const uint32_t p = ap_period(pmin, pmax, n, h)) {   // warp-uniform
        bool ok = true;
        uint32_t kmax = 0, kprev = 0;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (e * 32 + lane < n) {
                const uint32_t v = (uint32_t)w[e];
                ok = ok && (v - pmin) % p == 0;
                if (v == pmax) kmax = (uint32_t)(w[e] >> 32);
                if (v == pmax - p) kprev = (uint32_t)(w[e] >> 32);
            }
        kmax = __reduce_or_sync(0xffffffffu, kmax);     // one lane holds each
        kprev = __reduce_or_sync(0xffffffffu, kprev);
        if (__all_sync(0xffffffffu, ok) && kmax != kprev) {
            int64_t brk = 0;
            uint32_t slot0 = 0;
            if (al.lcp) {
                if (lane == 0) brk = ap_break(al.t, pmax, p, h);
                brk = __shfl_sync(0xffffffffu, brk, 0);
                slot0 = al.slots[gs.x];
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (e * 32 + lane < n) {
                    const uint32_t v = (uint32_t)w[e];
                    const uint32_t j = ap_index(v, pmin, pmax, p, kprev < kmax);
                    keys[gs.x + j] = hi | j;
                    vals[gs.x + j] = v;
                    if (al.lcp) ap_lcp_write(al, slot0, j, pmin, pmax, p, kprev < kmax, brk, err);
                }
            return;
        }
    }
    warp_bitonic<E>(w, lane, n2);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = e * 32 + lane;
        if (i < n) {
            keys[gs.x + i] = hi | (w[e] >> 32);
            vals[gs.x + i] = (uint32_t)w[e];
        }
    }
}

// Groups of 9..kSegWarpMax members: one warp per group, the words in registers
// (one per lane up to 32 members; 2, 4 or 8 per lane above).
__global__ void __launch_bounds__(256) k_seg_warp(const uint2 *__restrict__ groups,
                                                  const unsigned long long *__restrict__ d_ng, int b,
                                                  uint32_t h_host, const uint32_t *__restrict__ d_h,
                                                  unsigned long long *__restrict__ keys,
                                                  uint32_t *__restrict__ vals, ApLcp al, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    const int64_t ng = (int64_t)*d_ng;
    const uint32_t h = d_h ? *d_h : h_host;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned long long rmask = (1ull << b) - 1ull;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += nw) {
        const uint2 gs = groups[g];
        const int n = (int)gs.y;
        int n2 = 2;
        while (n2 < n) n2 <<= 1;   // network only as wide as the group
        if (n2 <= 32) warp_sort_group<1>(gs, lane, n2, rmask, h, keys, vals, al, err);
        else if (n2 <= 64) warp_sort_group<2>(gs, lane, n2, rmask, h, keys, vals, al, err);
        else if (n2 <= 128) warp_sort_group<4>(gs, lane, n2, rmask, h, keys, vals, al, err);
        else warp_sort_group<8>(gs, lane, n2, rmask, h, keys, vals, al, err);
    }
}

// Groups of kSegWarpMax+1 .. kSegMax members: one CTA per group, LSD radix sort
// on rank[i+h] in shared memory (ping-pong buffers of up to 512 * ROWS words).
// Only the bits in which the group's ranks differ are sorted, 8 per pass; each
// pass ranks the digits within each warp by ballots (stable: warp w holds the
// w-th contiguous slice, rows in order) and scatters through per-warp digit
// offsets.  Equal ranks keep their order, which is all a doubling round needs.
constexpr int kSegRadixWarps = kSegThreads / 32;

template <int ROWS>
constexpr size_t seg_radix_smem() {
    return (size_t)2 * kSegThreads * ROWS * 8 + (size_t)kSegRadixWarps * 256 * 4;
}

template <int ROWS>
__global__ void __launch_bounds__(kSegThreads) k_seg_radix(const uint2 *__restrict__ groups,
                                                           const unsigned long long *__restrict__ d_ng,
                                                           int b, uint32_t h_host,
                                                           const uint32_t *__restrict__ d_h, int min_n,
                                                           int max_n, unsigned long long *__restrict__ keys,
                                                           uint32_t *__restrict__ vals, uint32_t *err, ApLcp al) {
    constexpr int NW = kSegRadixWarps, CAP = kSegThreads * ROWS;
    extern __shared__ __align__(16) unsigned char seg_raw[];
    unsigned long long *buf0 = reinterpret_cast<unsigned long long *>(seg_raw);
    unsigned long long *buf1 = buf0 + CAP;
    uint32_t *wh = reinterpret_cast<uint32_t *>(buf1 + CAP);   // [NW][256] digit offsets
    __shared__ uint32_t s_tmp[NW + 1];
    __shared__ uint32_t s_min[NW], s_max[NW], s_k[2];
    __shared__ long long s_brk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ng = (int64_t)*d_ng;
    const uint32_t h = d_h ? *d_h : h_host;
    const unsigned long long rmask = (1ull << b) - 1ull;
    for (int64_t g = blockIdx.x; g < ng; g += gridDim.x) {
        const uint2 gs = groups[g];
        const int n = (int)gs.y;
        if (n <= min_n || n > max_n) continue;   // another variant's size class (device-driven rounds)
        if (n > CAP) {   // the host sizes ROWS for the list: never taken
            if (tid == 0) atomicOr(err, DERR_BOUNDS);
            continue;
        }
        const unsigned long long k0 = keys[gs.x];
        const unsigned long long hi = k0 & ~rmask;
        const uint32_t r0 = (uint32_t)(k0 & rmask);
        uint32_t x = 0;   // bits in which some rank differs from the first
        uint32_t pmin = ~0u, pmax = 0u;
        for (int i = tid; i < n; i += kSegThreads) {
            const unsigned long long k = keys[gs.x + i];
            const uint32_t v = vals[gs.x + i];
            buf0[i] = seg_word(k, v, rmask);
            x |= (uint32_t)(k & rmask) ^ r0;
            pmin = min(pmin, v);
            pmax = max(pmax, v);
        }
        x = __reduce_or_sync(0xffffffffu, x);
        pmin = __reduce_min_sync(0xffffffffu, pmin);
        pmax = __reduce_max_sync(0xffffffffu, pmax);
        if (lane == 0) {
            s_tmp[warp] = x;
            s_min[warp] = pmin;
            s_max[warp] = pmax;
        }
        __syncthreads();
        x = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            x |= s_tmp[w];
            pmin = min(pmin, s_min[w]);
            pmax = max(pmax, s_max[w]);
        }
        const int passes = x ? (32 - __clz(x) + 7) / 8 : 0;
        if (passes == 0) {   // one rank for all: the group is already in order
            __syncthreads();
            continue;
        }
        if (const uint32_t p = ap_period(pmin, pmax, n, h)) {   // block-uniform
            int ok = 1;
            for (int i = tid; i < n; i += kSegThreads) {
                const unsigned long long w = buf0[i];
                const uint32_t v = (uint32_t)w;
                ok &= (v - pmin) % p == 0;
                if (v == pmax) s_k[0] = (uint32_t)(w >> 32);
                if (v == pmax - p) s_k[1] = (uint32_t)(w >> 32);
            }
            ok = __syncthreads_and(ok);   // also publishes s_k
            const uint32_t kmax = s_k[0], kprev = s_k[1];
            if (ok && kmax != kprev) {
                if (al.lcp && tid == 0) s_brk = ap_break(al.t, pmax, p, h);
                __syncthreads();
                const uint32_t slot0 = al.lcp ? al.slots[gs.x] : 0u;
                for (int i = tid; i < n; i += kSegThreads) {
                    const uint32_t v = (uint32_t)buf0[i];
                    const uint32_t j = ap_index(v, pmin, pmax, p, kprev < kmax);
                    keys[gs.x + j] = hi | j;
                    vals[gs.x + j] = v;
                    if (al.lcp) ap_lcp_write(al, slot0, j, pmin, pmax, p, kprev < kmax, s_brk, err);
                }
                __syncthreads();
                continue;
            }
        }
        const int chunk = ((n + NW * 32 - 1) / (NW * 32)) * 32;   // warp slice, whole rows
        const int rows = chunk / 32;
        unsigned long long *src = buf0, *dst = buf1;
        uint32_t *mh = wh + warp * 256;
        for (int pass = 0; pass < passes; ++pass) {
            const int shift = 32 + 8 * pass;
            for (int i = tid; i < NW * 256; i += kSegThreads) wh[i] = 0;
            __syncthreads();
            uint16_t lr[ROWS];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                lr[r] = 0;
                if (r < rows) {   // warp-uniform
                    const int i = warp * chunk + r * 32 + lane;
                    const bool valid = i < n;
                    const uint32_t d = valid ? (uint32_t)(src[i] >> shift) & 255u : 0u;
                    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
                    uint32_t peers = vmask;
#pragma unroll
                    for (int bb = 0; bb < 8; ++bb) {
                        const uint32_t m = (uint32_t)((int32_t)(d << (31 - bb)) >> 31);
                        peers &= ~(__ballot_sync(0xffffffffu, m) ^ m);
                    }
                    const int leader = peers ? __ffs(peers) - 1 : 0;
                    uint32_t old = 0;
                    if (valid && lane == leader) {   // one lane per digit: plain update
                        old = mh[d];
                        mh[d] = old + (uint32_t)__popc(peers);
                    }
                    old = __shfl_sync(0xffffffffu, old, leader);
                    lr[r] = (uint16_t)(old + __popc(peers & lanemask_lt()));
                    __syncwarp();
                }
            }
            __syncthreads();
            // digit d starts after all smaller digits, and after digit d of lower warps
            uint32_t tot = 0;
            if (tid < 256)
                for (int w = 0; w < NW; ++w) tot += wh[w * 256 + tid];
            uint32_t total;
            const uint32_t start = block_exclusive_sum<kSegThreads>(tot, s_tmp, &total);
            if (tid < 256) {
                uint32_t run = start;
                for (int w = 0; w < NW; ++w) {
                    const uint32_t c = wh[w * 256 + tid];
                    wh[w * 256 + tid] = run;
                    run += c;
                }
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                if (r < rows) {
                    const int i = warp * chunk + r * 32 + lane;
                    if (i < n) {
                        const unsigned long long w = src[i];
                        dst[mh[(uint32_t)(w >> shift) & 255u] + lr[r]] = w;
                    }
                }
            }
            __syncthreads();
            unsigned long long *t = src;
            src = dst;
            dst = t;
        }
        for (int i = tid; i < n; i += kSegThreads) {
            keys[gs.x + i] = hi | (src[i] >> 32);
            vals[gs.x + i] = (uint32_t)src[i];
        }
        __syncthreads();
    }
}

// Marks the members of the groups larger than kSegMax (flags zeroed beforehand).
// Members of the groups sorted by global radix passes: flagged, and each one
// tagged with its group's start in the active list.
__global__ void k_flag_large(const uint2 *__restrict__ groups,
                             const unsigned long long *__restrict__ d_ng, uint8_t *__restrict__ flags,
                             uint32_t *__restrict__ gstart) {
    const int64_t ng = (int64_t)*d_ng;
    for (int64_t g = blockIdx.x; g < ng; g += gridDim.x) {
        const uint2 gs = groups[g];
        for (uint32_t i = threadIdx.x; i < gs.y; i += blockDim.x) {
            flags[(size_t)gs.x + i] = 1;
            gstart[(size_t)gs.x + i] = gs.x;
        }
    }
}

// Sort keys of the large-group members: (group start << kb) | rank[i+h].  The
// groups may lie in the active list in any order; keyed by their start, the
// sorted members come back group by group in list order.
__global__ void k_take(const uint32_t *__restrict__ idx, const unsigned long long *__restrict__ d_m,
                       const unsigned long long *__restrict__ keys, const uint32_t *__restrict__ vals,
                       const uint32_t *__restrict__ gstart, int kb, unsigned long long *__restrict__ ck,
                       uint32_t *__restrict__ cv) {
    const int64_t m = (int64_t)*d_m;
    const unsigned long long lo = (1ull << kb) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t t = idx[i];
        ck[i] = ((unsigned long long)gstart[t] << kb) | (keys[t] & lo);
        cv[i] = vals[t];
    }
}

// Sorted large-group members back to their ranges: the i-th of the sorted list
// belongs at the i-th large-group index, with its key restored to (old head
// rank << kb) | rank[i+h] (the head rank of a group is that of its first member).
__global__ void k_put(const uint32_t *__restrict__ idx, const unsigned long long *__restrict__ d_m,
                      const unsigned long long *__restrict__ ck, const uint32_t *__restrict__ cv,
                      const uint32_t *__restrict__ nhead, int kb,
                      unsigned long long *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int64_t m = (int64_t)*d_m;
    const unsigned long long lo = (1ull << kb) - 1ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t t = idx[i];
        const uint32_t start = (uint32_t)(ck[i] >> kb);
        keys[t] = ((unsigned long long)nhead[start] << kb) | (ck[i] & lo);
        vals[t] = cv[i];
    }
}

// Ranks of the members the finisher placed: rank[sa[slot]] = slot, so that the
// rank array ends as the inverse suffix array.  (A separate launch: the
// finisher's own comparisons read rank[] and must see it unchanged.)
__global__ void k_finish_ranks(const uint2 *__restrict__ groups,
                               const unsigned long long *__restrict__ ngroups,
                               const uint32_t *__restrict__ nslots, const uint32_t *__restrict__ sa,
                               int64_t N, uint32_t *__restrict__ rank) {
    const int64_t ng = (int64_t)*ngroups;
    for (int64_t g = blockIdx.x; g < ng; g += gridDim.x) {
        const uint2 gs = groups[g];
        const uint32_t slot0 = nslots[gs.x];
        for (uint32_t i = threadIdx.x; i < gs.y; i += blockDim.x) {
            int64_t slot = (int64_t)slot0 + i;
            if (slot < N) {
                uint32_t pos = sa[slot];
                if ((int64_t)pos < N) rank[pos] = (uint32_t)slot;
            }
        }
    }
}

// fid[p] = fragment of text position p: each warp walks 32 * 8 consecutive
// positions after one binary search per lane.
__global__ void __launch_bounds__(256) k_fid(TextDesc t, uint32_t *__restrict__ fid) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t p0 = warp * 32 * 8 + lane;
    if (warp * 32 * 8 >= t.N) return;
    int64_t r = read_of(t.toff, t.n_reads, min(p0, t.N - 1));
    for (int i = 0; i < 8; ++i) {
        int64_t p = p0 + (int64_t)i * 32;
        if (p >= t.N) break;
        while (__ldg(t.toff + r + 1) <= p) ++r;
        fid[p] = (uint32_t)r;
    }
}

__global__ void k_widen(const uint32_t *__restrict__ a, int64_t n, int64_t *__restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// ------------------------------------------------------------------ device-driven rounds
// The doubling rounds after round 0 can run as one captured CUDA graph: a WHILE
// node whose body holds two rounds (the list buffers alternate between them),
// with an IF node before the second.  Every launch of a round has a fixed grid
// (grid-stride or persistent kernels) and takes its counts and h from RoundDev,
// so the graph depends only on the buffers and sizes, and no count comes back to
// the host between rounds.  k_round_check ends the loop when no suffix is left
// active, when a group outgrows the on-chip sorts (the host then finishes the
// rounds), after kDevRoundsMax rounds, when h would reach N, or on an error flag.
constexpr int kDevRoundsMax = 59;

struct RoundDev {   // 64 words: read back whole into the pinned buffer
    unsigned long long kept, ngroups, maxgroup;   // the previous round's counts: this round's input
    uint32_t h;                                   // symbols every group member shares
    uint32_t round;                               // doubling rounds done
    unsigned long long max_rounds;
    unsigned long long active[59];                // trace: active suffixes after round r (index r - 1)
};
static_assert(sizeof(RoundDev) == 64 * 8, "one pinned read-back");

// Start of a round: the counts the last rerank left become the round's inputs
// (thread 0, before it clears them); the rerank's tile counter and look-back
// words are cleared.
__global__ void k_round_begin(RoundDev *rd, unsigned long long *cnt, uint32_t *tile_ctr,
                              unsigned long long *rr_status, int64_t rr_tiles) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (i0 == 0) {
        rd->kept = cnt[CNT_ACTIVE];
        rd->ngroups = cnt[CNT_GROUPS];
        rd->maxgroup = cnt[CNT_MAXGROUP];
        for (int k = 0; k < 4; ++k) cnt[k] = 0;
        for (int k = 0; k < 5; ++k) cnt[CNT_SEG + k] = 0;
        for (int k = 0; k < 4; ++k) tile_ctr[k] = 0;
    }
    for (int64_t i = i0; i < rr_tiles; i += stride) rr_status[i] = 0;
}

// Sets up the loop state before the graph runs (outside it: per call values).
__global__ void k_round_init(RoundDev *rd, uint32_t h0, int max_rounds) {
    rd->h = h0;
    rd->round = 0;
    rd->max_rounds = (unsigned long long)min(max_rounds, kDevRoundsMax);
}

// End of a round: count it, double h, record the trace, and decide whether the
// graph runs another round.  One thread sets the conditional handles.
__global__ void k_round_check(RoundDev *rd, const unsigned long long *cnt, const uint32_t *err, int64_t N,
                              int seg_max, cudaGraphConditionalHandle h_loop,
                              cudaGraphConditionalHandle h_second, int first) {
    const unsigned long long kept = cnt[CNT_ACTIVE], maxg = cnt[CNT_MAXGROUP];
    rd->kept = kept;   // the round's outputs (the next round_begin copies the same)
    rd->ngroups = cnt[CNT_GROUPS];
    rd->maxgroup = maxg;
    const uint32_t r = rd->round + 1;
    rd->round = r;
    if (r <= (uint32_t)kDevRoundsMax) rd->active[r - 1] = kept;
    const uint64_t h2 = 2ull * rd->h;
    rd->h = (uint32_t)min(h2, (uint64_t)0xffffffffu);
    const bool go = kept > 0 && maxg <= (unsigned long long)seg_max && r < rd->max_rounds &&
                    h2 < (uint64_t)N && *err == 0;
    cudaGraphSetConditional(h_loop, go ? 1u : 0u);
    if (first) cudaGraphSetConditional(h_second, go ? 1u : 0u);
}

}  // namespace

// The captured doubling loop of one sa_build configuration (held by the context).
struct SaGraph {
    std::vector<unsigned long long> key;   // buffers and sizes the kernels were given
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;             // capture stream
    int launches_per_round = 0;
};

static void sa_graph_free(SaGraph *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cs) cudaStreamDestroy(g->cs);
    delete g;
}

// The context's captured loops, most recently used last: a caller that alternates
// output buffers (double buffering) reuses one graph per buffer set.  A loop is
// captured only when its configuration comes back: the first call with new
// buffers or sizes runs its rounds from the host and is remembered in `seen`, so a
// stream of one-off sizes (a server's batches) never pays for a capture it would
// not reuse.
struct SaGraphCache {
    static constexpr size_t kMax = 4, kSeen = 8;
    std::vector<SaGraph *> g;
    std::vector<std::vector<unsigned long long>> seen;
};

static void sa_graph_cache_free(void *p) {
    SaGraphCache *c = static_cast<SaGraphCache *>(p);
    for (SaGraph *x : c->g) sa_graph_free(x);
    delete c;
}

// Symbols in the initial key.  Enough that i.i.d. text leaves few suffixes
// unsorted (4^h0 >= 32 * symbols per instance: expected colliding pairs at most
// N/64), then as many as fit in the same number of 8-bit passes: the key is
// [instance | 2*h0 bits of bases | 5 bits of lc], and its passes are the cost.
// A single sequence (one fragment, one instance) has only h0 suffixes that reach
// its '$' within h0 symbols, so the initial word can drop the bases-left field:
// word = (2*h0 bits of bases << pb) | f with f = bases left (0..h0-1) for those
// few "ended" suffixes and f = position + h0 for every other one, stored at
// index f of the sort input.  The radix passes order the bases and keep equal
// ones in input order, i.e. f order: the ended suffixes first, shorter first (as
// their '$' makes them smaller), then the rest by position.  f < N, so pb = bits
// of N - 1.  The key is 5 bits shorter: one 8-bit pass fewer for a 16-base key.
// Returns 0 when no packed word holds a key of at least the collision bound.
int h0_single(int64_t N, int *pack_bits) {
    int hmin = (int)std::ceil((std::log2(std::max((double)N, 2.0)) + 5.0) / 2.0);
    hmin = std::max(8, std::min(hmin, 29));
    const int passes = (2 * hmin + 7) / 8;
    const int pb = bits_for((uint64_t)(N - 1));
    const int h0 = std::min(std::min(4 * passes, 29), (64 - pb) / 2);
    if (h0 < hmin) return 0;
    *pack_bits = pb;
    return h0;
}

int h0_for(int64_t N, int n_inst, int *inst_bits, int *pack_bits) {
    int ib = n_inst > 1 ? bits_for((uint64_t)(n_inst - 1)) : 0;
    *inst_bits = ib;
    double per = (double)N / (double)(n_inst > 0 ? n_inst : 1);
    int hmin = (int)std::ceil((std::log2(std::max(per, 2.0)) + 5.0) / 2.0);
    hmin = std::max(8, std::min(hmin, 29));
    int passes = (ib + 2 * hmin + 5 + 7) / 8;
    int h0 = std::max(1, std::min((8 * passes - 5 - ib) / 2, 29));
    // the position fits under a key of at least hmin bases: sort one word per suffix
    const int pb = bits_for((uint64_t)(N - 1));
    const int hp = std::min((64 - pb - 5 - ib) / 2, h0);
    if (!pack_bits) return h0;
    *pack_bits = hp >= hmin ? pb : 0;
    return hp >= hmin ? hp : h0;
}

size_t sa_workspace_bytes(int64_t N, int tile_items) {
    const size_t n = (size_t)N;
    const int rr_tiles = ceil_div(N, kRrTile);
    size_t need = 0;
    auto add = [&](size_t bytes) { need += (bytes + 255) & ~size_t(255); };
    add(n * 8); add(n * 8);                 // keys x2
    add(n * 4); add(n * 4);                 // vals x2
    add(n * 4);                             // rank
    for (int i = 0; i < 6; ++i) add(n * 4); // lists A, B
    add((n / 2 + 1) * 8);                   // groups
    add((size_t)rr_tiles * 8);              // rerank status
    add((size_t)kMaxBuckets * 4);           // rank-write bucket fill counts
    add(n); add(n * 4); add(n * 8); add(n * 4);   // large-group flags, indices, sort buffers
    for (int i = 0; i < 5; ++i) add((n / 2 + 1) * 8);   // group lists by size class
    add(compact_scratch_bytes(N));
    add(radix_scratch_bytes(N, 64, tile_items));
    add(sizeof(RoundDev));                  // device-driven round state
    return need;
}

int sa_build_u32(dnasa_ctx *ctx, const TextDesc &t, uint32_t *sa32, const dnasa_opts *opts_in,
                 cudaStream_t s, uint32_t *isa_out, int32_t *lcp_out) {
    dnasa_opts opts{};
    if (opts_in) opts = *opts_in;
    if (opts.builder == 1) return sa_build_dc3(ctx, t, sa32, s, isa_out);
    const int tile_items = opts.tile_items ? opts.tile_items : radix_tile_default();
    const int64_t finish_threshold =
        opts.finish_threshold == 0 ? (int64_t)-1 : opts.finish_threshold;   // default: never
    const int max_rounds = opts.max_rounds > 0 ? std::min(opts.max_rounds, 63) : 63;
    const int lbw = opts.lookback == 1 ? 1 : 8;
    // largest group a doubling round sorts on chip (larger ones: radix passes)
    const int seg_max = opts.seg_max == 0 ? kSegMax : std::max(8, std::min(opts.seg_max, kSegMax));
    const int64_t N = t.N;
    int ib, pb;
    int h0 = h0_for(N, t.n_inst, &ib, &pb);
    if (opts.pack_position < 0 && pb) {
        pb = 0;
        h0 = h0_for(N, t.n_inst, &ib, nullptr);
    }
    // one sequence: the shorter key without the bases-left field (h0_single)
    bool single = false;
    if (t.n_reads == 1 && t.n_inst <= 1 && opts.pack_position >= 0) {
        int pbs = 0;
        const int hs = h0_single(N, &pbs);
        if (hs > 0) {
            single = true;
            h0 = hs;
            pb = pbs;
            ib = 0;
        }
    }
    const int inst_shift = 2 * h0 + 5;
    const int key_bits0 = single ? 2 * h0 : inst_shift + ib;
    const int b = bits_for((uint64_t)(N - 1));

    // ---- workspace
    const size_t n = (size_t)N;
    const int rr_tiles = ceil_div(N, kRrTile);
    const size_t need = sa_workspace_bytes(N, tile_items);
    DNASA_TRY(ws_reserve(ctx, need + 4096, s));
    Arena a = ws_arena(ctx);
    unsigned long long *keys[2] = {a.take<unsigned long long>(n), a.take<unsigned long long>(n)};
    uint32_t *vals[2] = {a.take<uint32_t>(n), a.take<uint32_t>(n)};
    uint32_t *rank = a.take<uint32_t>(n);
    uint32_t *L[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) L[i][j] = a.take<uint32_t>(n);
    uint2 *groups = a.take<uint2>(n / 2 + 1);
    unsigned long long *rr_status = a.take<unsigned long long>((size_t)rr_tiles);
    uint32_t *bucket_fill = a.take<uint32_t>((size_t)kMaxBuckets);
    uint8_t *lflags = a.take<uint8_t>(n);
    uint2 *gtiny = a.take<uint2>(n / 2 + 1);
    uint2 *gsmall = a.take<uint2>(n / 2 + 1), *gwmid = a.take<uint2>(n / 2 + 1);
    uint2 *gmid = a.take<uint2>(n / 2 + 1), *glarge = a.take<uint2>(n / 2 + 1);
    uint32_t *lidx = a.take<uint32_t>(n);
    unsigned long long *ck2 = a.take<unsigned long long>(n);
    uint32_t *cv2 = a.take<uint32_t>(n);
    RadixScratch rs = radix_scratch_take(a, N, 64, tile_items);
    RoundDev *rd = a.take<RoundDev>(1);
    if (!rs.hist || !rr_status || !rd) return fail(ctx, DNASA_OOM, "sa_build workspace");

    // dynamic shared-memory limits of this call's kernels, once per (kernel, device)
    DNASA_CUDA(ctx, smem_attr(k_rerank, sizeof(RerankSmem)));
    DNASA_CUDA(ctx, smem_attr(k_seg_radix<4>, seg_radix_smem<4>()));
    DNASA_CUDA(ctx, smem_attr(k_seg_radix<12>, seg_radix_smem<12>()));
    DNASA_CUDA(ctx, smem_attr(k_seg_radix<24>, seg_radix_smem<24>()));
    DevCtrl *c = ctx->ctrl;
    unsigned long long *cnt = c->count;
    dnasa_trace &tr = ctx->trace;
    memset(&tr, 0, sizeof(tr));
    tr.h0 = h0;
    tr.pack_bits = pb;

    auto reset_counters = [&]() -> int {
        DNASA_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 4, s));
        DNASA_CUDA(ctx, cudaMemsetAsync(c->tile_ctr + 32, 0, sizeof(uint32_t) * 4, s));
        DNASA_CUDA(ctx, cudaMemsetAsync(rr_status, 0, (size_t)rr_tiles * 8, s));
        DNASA_CUDA(ctx, cudaMemsetAsync(bucket_fill, 0, (size_t)kMaxBuckets * 4, s));
        return DNASA_OK;
    };
    // position buckets of 2^bshift (>= 2M) positions, at most kMaxBuckets of them
    int bshift = 21;
    while (((N - 1) >> bshift) + 1 > kMaxBuckets) ++bshift;
    const int nbuckets = (int)(((N - 1) >> bshift) + 1);
    auto apply_ranks = [&](int64_t n_items, int stage_buf) -> int {
        LaunchScope ls_(ctx, PK_APPLY, s, 12.0 * n_items);
        k_rank_apply<<<std::max(1, ceil_div(n_items, kApplyItems)), 256, 0, s>>>(
            reinterpret_cast<const uint2 *>(keys[stage_buf]), bucket_fill, nbuckets, bshift, N, rank,
            &c->err);
        return DNASA_OK;
    };
    auto read_counters = [&](int64_t *kept, int64_t *ngroups, int64_t *maxgroup) -> int {
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt, sizeof(unsigned long long) * 3,
                                        cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "sa_build"));
        volatile unsigned long long *pv = ctx->pinned;
        *kept = (int64_t)pv[CNT_ACTIVE];
        *ngroups = (int64_t)pv[CNT_GROUPS];
        *maxgroup = (int64_t)pv[CNT_MAXGROUP];
        return DNASA_OK;
    };
    RerankOut ro;
    ro.N = N;
    ro.sa = sa32;
    ro.rank = rank;
    ro.groups = groups;
    ro.kept = cnt + CNT_ACTIVE;
    ro.ngroups = cnt + CNT_GROUPS;
    ro.maxgroup = cnt + CNT_MAXGROUP;
    ro.bucket_fill = bucket_fill;
    ro.bshift = bshift;
    ro.kb = b;
    ro.pb = pb;
    ro.single = single ? 1 : 0;
    ro.lcp = lcp_out;

    // ---- one doubling round with fixed grids and device-side counts (captured)
    int rr_grid = 0;
    {
        int per_sm = 0;
        DNASA_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rerank, kRrThreads,
                                                                      sizeof(RerankSmem)));
        rr_grid = ctx->num_sms * std::max(per_sm, 1);
    }
    // the progression groups' LCP entries, for sa_lcp_build (lcp_out), in a round reading list cr
    auto ap_lcp = [&](int cr) -> ApLcp {
        ApLcp al;
        al.lcp = lcp_out;
        al.slots = L[cr][0];
        al.t = t;
        return al;
    };
    auto launch_round = [&](cudaStream_t cs, int cr) -> int {   // returns the launch count
        const int G = ctx->num_sms * 16;
        int nl = 0;
        k_round_begin<<<ctx->num_sms, 256, 0, cs>>>(rd, cnt, c->tile_ctr + 32, rr_status, rr_tiles);
        k_gather<<<G, 256, 0, cs>>>(L[cr][1], L[cr][2], 0, &rd->kept, rank, 0u, &rd->h, b, keys[0], vals[0],
                                    N, &c->err);
        k_classify<<<G, 256, 0, cs>>>(groups, 0, &rd->ngroups, seg_max, gtiny, gsmall, gwmid, gmid, glarge,
                                      cnt + CNT_SEG);
        const ApLcp al = ap_lcp(cr);
        k_seg_thread<<<G, 256, 0, cs>>>(gtiny, cnt + CNT_SEG, b, 0u, &rd->h, keys[0], vals[0], al, &c->err);
        k_seg_warp<<<G, 256, 0, cs>>>(gsmall, cnt + CNT_SEG + 1, b, 0u, &rd->h, keys[0], vals[0], al, &c->err);
        k_seg_warp<<<G, 256, 0, cs>>>(gwmid, cnt + CNT_SEG + 2, b, 0u, &rd->h, keys[0], vals[0], al, &c->err);
        nl += 6;
        // each CTA-radix variant takes its own size class of the one list
        auto radix = [&](auto kern, size_t smem, int lo, int hi) {
            if (seg_max <= lo) return;
            const int per_sm = std::max(1, (int)((200u << 10) / smem));
            kern<<<ctx->num_sms * per_sm, kSegThreads, smem, cs>>>(gmid, cnt + CNT_SEG + 3, b, 0u, &rd->h, lo,
                                                                    hi, keys[0], vals[0], &c->err, al);
            ++nl;
        };
        radix(k_seg_radix<4>, seg_radix_smem<4>(), kSegWarpMax, kSegThreads * 4);
        radix(k_seg_radix<12>, seg_radix_smem<12>(), kSegThreads * 4, kSegThreads * 12);
        radix(k_seg_radix<24>, seg_radix_smem<24>(), kSegThreads * 12, kSegThreads * 24);
        RerankOut r2 = ro;
        r2.nslots = L[cr ^ 1][0];
        r2.npos = L[cr ^ 1][1];
        r2.nhead = L[cr ^ 1][2];
        k_rerank<<<rr_grid, kRrThreads, sizeof(RerankSmem), cs>>>(keys[0], vals[0], L[cr][0], 0, &rd->kept, r2,
                                                                  rr_status, c->tile_ctr + 32, &c->err);
        return nl + 1;
    };
    // Runs the doubling rounds as the captured graph (captured on first use, or
    // again when a buffer or size differs from the cached one); returns the
    // rounds done and the counts the last one left.
    auto device_rounds = [&](int *rounds, int64_t *kept, int64_t *ngroups, int64_t *maxgroup) -> int {
        const std::vector<unsigned long long> key = {
            (unsigned long long)N, (unsigned long long)b, (unsigned long long)seg_max,
            (unsigned long long)bshift, (unsigned long long)nbuckets, (unsigned long long)rr_grid,
            (unsigned long long)(uintptr_t)keys[0], (unsigned long long)(uintptr_t)keys[1],
            (unsigned long long)(uintptr_t)vals[0], (unsigned long long)(uintptr_t)rank,
            (unsigned long long)(uintptr_t)sa32, (unsigned long long)(uintptr_t)groups,
            (unsigned long long)(uintptr_t)gtiny, (unsigned long long)(uintptr_t)gsmall,
            (unsigned long long)(uintptr_t)gwmid, (unsigned long long)(uintptr_t)gmid,
            (unsigned long long)(uintptr_t)glarge, (unsigned long long)(uintptr_t)L[0][0],
            (unsigned long long)(uintptr_t)L[1][0], (unsigned long long)(uintptr_t)rr_status,
            (unsigned long long)(uintptr_t)bucket_fill, (unsigned long long)(uintptr_t)rd,
            (unsigned long long)(uintptr_t)c,
            // the progression groups' LCP writes read the text
            (unsigned long long)(uintptr_t)lcp_out, (unsigned long long)(uintptr_t)t.packed,
            (unsigned long long)(uintptr_t)t.toff, (unsigned long long)t.n_reads,
            (unsigned long long)(uintptr_t)t.inst_toff, (unsigned long long)(uintptr_t)t.inst_roff,
            (unsigned long long)t.n_inst, (unsigned long long)(uintptr_t)t.fid};
        SaGraphCache *cache = static_cast<SaGraphCache *>(ctx->sa_graph);
        if (!cache) {
            cache = new SaGraphCache();
            ctx->sa_graph = cache;
            ctx->sa_graph_free = sa_graph_cache_free;
        }
        SaGraph *gph = nullptr;
        for (size_t i = 0; i < cache->g.size(); ++i)
            if (cache->g[i]->key == key) {   // reuse, and mark most recently used
                gph = cache->g[i];
                cache->g.erase(cache->g.begin() + (std::ptrdiff_t)i);
                cache->g.push_back(gph);
                break;
            }
        if (!gph) {   // capture only a configuration seen before
            auto it = std::find(cache->seen.begin(), cache->seen.end(), key);
            if (it == cache->seen.end()) {
                if (cache->seen.size() >= SaGraphCache::kSeen) cache->seen.erase(cache->seen.begin());
                cache->seen.push_back(key);
                *rounds = -1;   // declined: the host runs the rounds this time
                return DNASA_OK;
            }
            cache->seen.erase(it);
        }
        if (!gph) {
            if (cache->g.size() >= SaGraphCache::kMax) {   // evict the least recently used
                sa_graph_free(cache->g.front());
                cache->g.erase(cache->g.begin());
            }
            gph = new SaGraph();
            auto drop = [&](cudaError_t e, const char *where) -> int {   // no half-built graph is kept
                sa_graph_free(gph);
                return cuda_fail(ctx, e, where);
            };
            cudaError_t e = cudaStreamCreateWithFlags(&gph->cs, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaGraphCreate(&gph->graph, 0);
            cudaGraphConditionalHandle h_loop = 0, h_second = 0;
            if (e == cudaSuccess)
                e = cudaGraphConditionalHandleCreate(&h_loop, gph->graph, 1, cudaGraphCondAssignDefault);
            if (e == cudaSuccess)
                e = cudaGraphConditionalHandleCreate(&h_second, gph->graph, 0, cudaGraphCondAssignDefault);
            if (e != cudaSuccess) return drop(e, "sa_build: graph setup");
            cudaGraphNodeParams wp = {};
            wp.type = cudaGraphNodeTypeConditional;
            wp.conditional.handle = h_loop;
            wp.conditional.type = cudaGraphCondTypeWhile;
            wp.conditional.size = 1;
            cudaGraphNode_t wnode;
            e = cudaGraphAddNode(&wnode, gph->graph, nullptr, nullptr, 0, &wp);
            if (e != cudaSuccess) return drop(e, "sa_build: loop node");
            cudaGraph_t body = wp.conditional.phGraph_out[0];
            // pass body: round (lists 0 -> 1), check, IF node holding round (1 -> 0) and check
            e = cudaStreamBeginCaptureToGraph(gph->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return drop(e, "sa_build: capture");
            gph->launches_per_round = launch_round(gph->cs, 0) + 1;
            k_round_check<<<1, 1, 0, gph->cs>>>(rd, cnt, &c->err, N, seg_max, h_loop, h_second, 1);
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t *deps = nullptr;
            size_t ndeps = 0;
            e = cudaStreamGetCaptureInfo(gph->cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
            cudaGraphNodeParams ip = {};
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = h_second;
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            cudaGraphNode_t inode;
            if (e == cudaSuccess) e = cudaGraphAddNode(&inode, body, deps, nullptr, ndeps, &ip);
            cudaGraph_t captured = nullptr;
            const cudaError_t e_end = cudaStreamEndCapture(gph->cs, &captured);
            if (e == cudaSuccess) e = e_end;
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) return drop(e, "sa_build: first round capture");
            e = cudaStreamBeginCaptureToGraph(gph->cs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return drop(e, "sa_build: capture");
            launch_round(gph->cs, 1);
            k_round_check<<<1, 1, 0, gph->cs>>>(rd, cnt, &c->err, N, seg_max, h_loop, h_second, 0);
            e = cudaStreamEndCapture(gph->cs, &captured);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaGraphInstantiate(&gph->exec, gph->graph, 0);
            if (e != cudaSuccess) return drop(e, "sa_build: second round capture");
            gph->key = key;
            cache->g.push_back(gph);
        }
        k_round_init<<<1, 1, 0, s>>>(rd, (uint32_t)h0, max_rounds);
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_CUDA(ctx, cudaGraphLaunch(gph->exec, s));
        DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, rd, sizeof(RoundDev), cudaMemcpyDeviceToHost, s));
        DNASA_TRY(check_device_status(ctx, s, "sa_build"));
        RoundDev hr;
        memcpy(&hr, (const void *)ctx->pinned, sizeof(hr));
        *rounds = (int)hr.round;
        *kept = (int64_t)hr.kept;
        *ngroups = (int64_t)hr.ngroups;
        *maxgroup = (int64_t)hr.maxgroup;
        for (int r = 1; r <= *rounds && r <= kDevRoundsMax && r < 64; ++r) tr.active[r] = (int64_t)hr.active[r - 1];
        ctx->launches += 1 + (unsigned long long)hr.round * (unsigned long long)gph->launches_per_round;
        return DNASA_OK;
    };

    // ---- round 0: initial keys, sort, rerank
    {
        PhaseRange nvtx_("dnasa.sa_round0");
        const int passes0 = ceil_div(key_bits0, 8);
        // one sequence whose key is whole 4-mers: count one 4-mer histogram (k_hist4_fix)
        const bool hist4 = single && h0 == 4 * passes0 && h0 <= 32 && N >= 2 * h0 + 8;
        DNASA_CUDA(ctx, cudaMemsetAsync(rs.hist, 0, (size_t)passes0 * 256 * 4, s));
        {
            LaunchScope ls_(ctx, PK_INIT, s, (pb ? 8.25 : 12.25) * N);
            const int warps = ceil_div(N, 32 * kInitItems);
            const int grid = (int)std::min<int64_t>(ceil_div(warps, kInitThreads / 32),
                                                    (int64_t)ctx->num_sms * 8);
            k_init_keys<<<std::max(grid, 1), kInitThreads, 0, s>>>(t, h0, inst_shift, pb, single ? 1 : 0,
                                                                   passes0, pb, hist4 ? 1 : 0,
                                                                   rs.hist, keys[0], vals[0]);
        }
        if (hist4) {
            LaunchScope ls_(ctx, PK_HIST, s, 0.0);
            k_hist4_fix<<<1, 256, 0, s>>>(t, h0, passes0, rs.hist);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        int which;
        uint32_t *novals[2] = {nullptr, nullptr};
        DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs, keys, pb ? novals : vals, N, nullptr,
                                                       key_bits0, true, tile_items, &which, s, lbw, pb));
        DNASA_TRY(reset_counters());
        ro.nslots = L[0][0]; ro.npos = L[0][1]; ro.nhead = L[0][2];
        ro.stage = reinterpret_cast<uint2 *>(keys[which ^ 1]);   // the free key buffer
        {
            LaunchScope ls_(ctx, PK_RERANK, s, (lcp_out ? 24.0 : 20.0) * N);   // + 4 B of LCP per slot
            k_rerank0<<<ceil_div(N, kR0Tile), kR0Threads, 0, s>>>(keys[which], vals[which], N, h0, ro, &c->err);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_TRY(apply_ranks(N, which ^ 1));
        DNASA_CUDA(ctx, cudaGetLastError());
    }
    int64_t kept, ngroups, maxgroup;
    DNASA_TRY(read_counters(&kept, &ngroups, &maxgroup));
    tr.active[0] = kept;
    int cur = 0;
    uint64_t h = (uint64_t)h0;
    int round = 0;
    if (kept > 0 && opts.rounds_on_host == 0 && finish_threshold < 0 && !ctx->prof_on &&
        maxgroup <= seg_max && h < (uint64_t)N) {
        int rounds = 0;
        PhaseRange nvtx_("dnasa.sa_rounds_graph");
        DNASA_TRY(device_rounds(&rounds, &kept, &ngroups, &maxgroup));
        if (rounds >= 0) {   // else: a first call with these buffers and sizes, rounds from the host
            round = rounds;
            cur = rounds & 1;
            h = (uint64_t)h0 << rounds;
            tr.rounds = rounds;
            tr.graph_rounds = rounds;
        }
    }
    while (kept > 0) {
        if (finish_threshold >= 0 && kept <= finish_threshold && maxgroup <= kFinMax) {
            int grid = (int)std::min<int64_t>(ngroups, (int64_t)ctx->num_sms * 4);
            {
                LaunchScope ls_(ctx, PK_FINISH, s, 0);
                k_finish<<<std::max(grid, 1), kFinThreads, 0, s>>>(groups, cnt + CNT_GROUPS, L[cur][1],
                                                                   L[cur][0], rank, (uint32_t)h, N,
                                                                   sa32, &c->err);
            }
            {
                LaunchScope ls_(ctx, PK_FINISH, s, 0);
                k_finish_ranks<<<std::max(grid, 1), 256, 0, s>>>(groups, cnt + CNT_GROUPS, L[cur][0],
                                                                 sa32, N, rank);
            }
            DNASA_CUDA(ctx, cudaGetLastError());
            tr.finished_direct = 1;
            break;
        }
        if (++round > max_rounds) return fail(ctx, DNASA_INVALID_ARG, "sa_build: max_rounds exceeded");
        PhaseRange nvtx_("dnasa.sa_round");
        if (h >= (uint64_t)N) return fail(ctx, DNASA_CUDA_ERROR, "sa_build: doubling did not converge");
        // keys for this round
        int grid = (int)std::min<int64_t>(ceil_div(kept, 256), (int64_t)ctx->num_sms * 16);
        {
            LaunchScope ls_(ctx, PK_GATHER, s, 24.0 * kept);
            k_gather<<<std::max(grid, 1), 256, 0, s>>>(L[cur][1], L[cur][2], kept, nullptr, rank,
                                                       (uint32_t)h, nullptr, b, keys[0], vals[0], N, &c->err);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        // order every group by rank[i+h]: small groups on chip, large ones by radix
        const uint32_t hs = (uint32_t)h;   // h < N < 2^32 here: the members share h symbols
        DNASA_CUDA(ctx, cudaMemsetAsync(cnt + CNT_SEG, 0, 5 * sizeof(unsigned long long), s));
        {
            LaunchScope ls_(ctx, PK_SEGSORT, s, 8.0 * ngroups);
            int gc = (int)std::min<int64_t>(ceil_div(ngroups, 256), (int64_t)ctx->num_sms * 16);
            k_classify<<<std::max(gc, 1), 256, 0, s>>>(groups, ngroups, nullptr, seg_max, gtiny, gsmall, gwmid,
                                                       gmid, glarge, cnt + CNT_SEG);
        }
        {
            LaunchScope ls_(ctx, PK_SEGSORT, s, 24.0 * kept);
            int gt = (int)std::min<int64_t>(ceil_div(ngroups, 256), (int64_t)ctx->num_sms * 16);
            k_seg_thread<<<std::max(gt, 1), 256, 0, s>>>(gtiny, cnt + CNT_SEG, b, hs, nullptr, keys[0], vals[0],
                                                         ap_lcp(cur), &c->err);
        }
        for (int cls = 1; cls <= 2; ++cls) {   // 9..32 and 33..kSegWarpMax members: a warp each
            if (maxgroup <= (cls == 1 ? 8 : 32) || seg_max <= (cls == 1 ? 8 : 32)) break;
            LaunchScope ls_(ctx, PK_SEGSORT, s, 0.0);
            int gw = (int)std::min<int64_t>(ceil_div(ngroups, 8), (int64_t)ctx->num_sms * 16);
            k_seg_warp<<<std::max(gw, 1), 256, 0, s>>>(cls == 1 ? gsmall : gwmid, cnt + CNT_SEG + cls, b,
                                                       hs, nullptr, keys[0], vals[0], ap_lcp(cur), &c->err);
        }
        if (maxgroup > kSegWarpMax && seg_max > kSegWarpMax) {
            const int64_t biggest = std::min<int64_t>(maxgroup, seg_max);
            LaunchScope ls_(ctx, PK_SEGSORT, s, 0.0);
            auto launch = [&](auto kern, size_t smem) {
                const int per_sm = std::max(1, (int)((200u << 10) / smem));
                const int gb = (int)std::min<int64_t>(ngroups, (int64_t)ctx->num_sms * per_sm);
                kern<<<std::max(gb, 1), kSegThreads, smem, s>>>(gmid, cnt + CNT_SEG + 3, b, hs, nullptr, 0,
                                                                0x7fffffff, keys[0], vals[0], &c->err,
                                                                ap_lcp(cur));
            };
            if (biggest <= kSegThreads * 4) launch(k_seg_radix<4>, seg_radix_smem<4>());
            else if (biggest <= kSegThreads * 12) launch(k_seg_radix<12>, seg_radix_smem<12>());
            else launch(k_seg_radix<24>, seg_radix_smem<24>());
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        if (maxgroup > seg_max) {
            DNASA_CUDA(ctx, cudaMemsetAsync(lflags, 0, (size_t)kept, s));
            {
                LaunchScope ls_(ctx, PK_SEGSORT, s, 0.0);
                k_flag_large<<<ctx->num_sms * 2, 256, 0, s>>>(glarge, cnt + CNT_SEG + 4, lflags,
                                                              reinterpret_cast<uint32_t *>(ck2));
            }
            Arena rest = a;
            DNASA_TRY(compact_flags(ctx, rest, lflags, kept, lidx, cnt + CNT_TMP, s));
            DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, cnt + CNT_TMP, 8, cudaMemcpyDeviceToHost, s));
            DNASA_TRY(check_device_status(ctx, s, "sa_build"));
            const int64_t m = (int64_t)ctx->pinned[0];
            unsigned long long *ck[2] = {keys[1], ck2};
            uint32_t *cv[2] = {vals[1], cv2};
            int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 256), (int64_t)ctx->num_sms * 16));
            {
                LaunchScope ls_(ctx, PK_SEGSORT, s, 24.0 * m);
                // ck2 (the radix sort's spare buffer, free until the sort) holds the group starts
                k_take<<<g2, 256, 0, s>>>(lidx, cnt + CNT_TMP, keys[0], vals[0],
                                          reinterpret_cast<const uint32_t *>(ck2), b, ck[0], cv[0]);
            }
            int which;
            DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs, ck, cv, m, nullptr, 2 * b,
                                                           false, tile_items, &which, s, lbw));
            {
                LaunchScope ls_(ctx, PK_SEGSORT, s, 24.0 * m);
                k_put<<<g2, 256, 0, s>>>(lidx, cnt + CNT_TMP, ck[which], cv[which], L[cur][2], b, keys[0],
                                         vals[0]);
            }
            DNASA_CUDA(ctx, cudaGetLastError());
        }
        DNASA_TRY(reset_counters());
        ro.nslots = L[cur ^ 1][0]; ro.npos = L[cur ^ 1][1]; ro.nhead = L[cur ^ 1][2];
        int tiles = ceil_div(kept, kRrTile);
        {
            // later rounds keep the decoupled look-back: measured faster here than the
            // look-back-free form, whose tiles wait on following the many groups that
            // cross a tile boundary once most groups are a few dozen members
            LaunchScope ls_(ctx, PK_RERANK, s, 24.0 * kept);
            k_rerank<<<tiles, kRrThreads, sizeof(RerankSmem), s>>>(keys[0], vals[0], L[cur][0], kept,
                                                         nullptr, ro, rr_status, c->tile_ctr + 32, &c->err);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        DNASA_TRY(read_counters(&kept, &ngroups, &maxgroup));
        cur ^= 1;
        h *= 2;
        tr.rounds = round;
        if (round < 64) tr.active[round] = kept;
    }
    if (isa_out)   // every rank is now final: the rank array is the inverse SA
        DNASA_CUDA(ctx, cudaMemcpyAsync(isa_out, rank, (size_t)N * 4, cudaMemcpyDeviceToDevice, s));
    if (lcp_out)   // the pairs round 0 left (-1), walked in text order through the inverse SA;
                   // the free key buffer holds the walk's bitmap
        DNASA_TRY(lcp_finish_with_isa(ctx, t, sa32, rank, lcp_out, h0, reinterpret_cast<uint32_t *>(keys[1]), s));
    return check_device_status(ctx, s, "sa_build");
}

int fragment_ids(dnasa_ctx *ctx, const TextDesc &t, uint32_t *fid, cudaStream_t s) {
    int warps = ceil_div(t.N, 32 * 8);
    LaunchScope ls_(ctx, PK_OTHER, s, 4.0 * t.N);
    k_fid<<<std::max(1, ceil_div(warps, 8)), 256, 0, s>>>(t, fid);
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}

int widen_u32_to_i64(dnasa_ctx *ctx, const uint32_t *a, int64_t n, int64_t *b, cudaStream_t s) {
    int grid = (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 16);
    {
        LaunchScope ls_(ctx, PK_OTHER, s, 12.0 * n);
        k_widen<<<std::max(grid, 1), 256, 0, s>>>(a, n, b);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}

}  // namespace dnasa
