// lcp.cu -- LCP array over the suffix array.
//
// lcp[0] = 0 and lcp[j] = the number of equal bases at the start of suffixes
// SA[j-1] and SA[j], never counting a '$' (so no LCP crosses a fragment end),
// and 0 where an instance of a batch starts.  Each thread compares one adjacent
// pair 32 bases at a time: XOR of two packed words and a count of leading zero
// bits, capped by the bases left in both fragments.  The paper's prefix tests
// between fragments (Sec. IV) rest on these common-prefix lengths; here they
// drive the containment test and the overlap interval scan.
#include <algorithm>

#include "common.cuh"

namespace dnasa {

namespace {

constexpr int kShortBases = 64;   // resolved by one thread; longer LCPs go to a warp

struct PairInfo {
    uint64_t bp, bq;
    int64_t m;      // bases left in the shorter of the two suffixes
};

__device__ __forceinline__ bool instance_start(const TextDesc &t, int64_t j) {
    if (t.n_inst <= 1) return false;
    int64_t i = upper_index(t.inst_toff, 0, t.n_inst, j);
    return __ldg(t.inst_toff + i) == j;
}

__device__ __forceinline__ PairInfo pair_info(const TextDesc &t, const uint32_t *__restrict__ sa,
                                              int64_t j) {
    int64_t p = sa[j - 1], q = sa[j];
    int64_t rp = frag_of(t, p);
    int64_t rq = frag_of(t, q);
    PairInfo r;
    r.m = min(__ldg(t.toff + rp + 1) - 1 - p, __ldg(t.toff + rq + 1) - 1 - q);
    r.bp = (uint64_t)(p - rp);
    r.bq = (uint64_t)(q - rq);
    return r;
}

// One thread per adjacent pair: the first 64 bases.  Each lane fetches the
// first 32 bases of its own suffix SA[j] and takes those of SA[j-1] from the
// lane before it (lane 0 fetches both), so a pair costs one random text fetch
// instead of two.  Pairs still equal after 64 bases (repeats) are queued for
// k_lcp_chain.
__global__ void __launch_bounds__(256) k_lcp(TextDesc t, const uint32_t *__restrict__ sa,
                                             int32_t *__restrict__ lcp, uint32_t *__restrict__ qpos,
                                             uint32_t *__restrict__ qj,
                                             unsigned long long *__restrict__ nlong) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; b < t.N; b += stride) {
        const int64_t j = b + lane;
        const bool in = j < t.N;
        // own suffix q = SA[j]: base coordinate, bases left in its fragment, first 32 bases
        int64_t q = in ? (int64_t)sa[j] : 0;
        int64_t rq = in ? frag_of(t, q) : 0;
        int64_t left_q = in ? __ldg(t.toff + rq + 1) - 1 - q : 0;
        uint64_t bq = (uint64_t)(q - rq);
        uint64_t wq = in ? bases32(t.packed, bq) : 0ull;
        // the previous suffix p = SA[j-1]: from the lane before, or fetched by lane 0
        int64_t left_p = __shfl_up_sync(0xffffffffu, left_q, 1);
        uint64_t bp = __shfl_up_sync(0xffffffffu, bq, 1);
        uint64_t wp = __shfl_up_sync(0xffffffffu, wq, 1);
        bool queue = false;
        if (in) {
            if (j == 0 || instance_start(t, j)) {
                lcp[j] = 0;
            } else {
                if (lane == 0) {
                    const int64_t p = sa[j - 1];
                    const int64_t rp = frag_of(t, p);
                    left_p = __ldg(t.toff + rp + 1) - 1 - p;
                    bp = (uint64_t)(p - rp);
                    wp = bases32(t.packed, bp);
                }
                const int64_t m = min(left_p, left_q);
                int64_t h;
                uint64_t d = wp ^ wq;
                if (d || m <= 32) {
                    h = d ? (int64_t)(__clzll((long long)d) >> 1) : 32;
                } else {
                    d = bases32(t.packed, bp + 32) ^ bases32(t.packed, bq + 32);
                    h = d ? 32 + (int64_t)(__clzll((long long)d) >> 1) : kShortBases;
                }
                if (h < kShortBases || h >= m) lcp[j] = (int32_t)min(h, m);
                else queue = true;
            }
        }
        uint32_t qm = __ballot_sync(0xffffffffu, queue);
        if (qm) {
            unsigned long long qb = 0;
            if (lane == 0) qb = atomicAdd(nlong, (unsigned long long)__popc(qm));
            qb = __shfl_sync(0xffffffffu, qb, 0);
            if (queue) {
                unsigned long long at = qb + __popc(qm & lanemask_lt());
                qpos[at] = sa[j];
                qj[at] = (uint32_t)j;
            }
        }
    }
}

// The queued pairs (LCP over 64 bases: repeats), sorted by the text position p
// of their lower suffix.  Kasai's bound: the LCP of suffix p+1 with its SA
// predecessor is at least that of p minus one, so along a run of consecutive
// positions each comparison starts where the previous one ended instead of at
// base 64.  One thread walks kChain consecutive entries, four words (128 bases)
// per round trip (one word first: past the bound most pairs differ within it).
// The walk is a chain of dependent loads, so short chains (many
// threads in flight) beat the comparisons the bound saves inside a long one: a
// 16 Mbp genome queued ~1.3 M pairs, which at 128 entries per thread left the GPU
// 6 % occupied.
constexpr int kChain = 16;

__global__ void __launch_bounds__(256) k_lcp_chain(TextDesc t, const uint32_t *__restrict__ sa,
                                                   int32_t *__restrict__ lcp,
                                                   const uint32_t *__restrict__ qpos,
                                                   const uint32_t *__restrict__ qj, int64_t nq) {
    const int64_t chunks = (nq + kChain - 1) / kChain;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t prev_p = -2, prev_h = 0;
        const int64_t e1 = min((c + 1) * kChain, nq);
        for (int64_t e = c * kChain; e < e1; ++e) {
            const int64_t p = qpos[e], j = qj[e];
            PairInfo pi = pair_info(t, sa, j);
            int64_t h = (p == prev_p + 1 && prev_h - 1 > kShortBases) ? prev_h - 1 : kShortBases;
            int64_t res = pi.m;
            bool found = false;
            if (h < pi.m) {   // one word first: past Kasai's bound most pairs differ within it
                const uint64_t d0 = bases32(t.packed, pi.bp + h) ^ bases32(t.packed, pi.bq + h);
                if (d0) {
                    res = min(h + (int64_t)(__clzll((long long)d0) >> 1), pi.m);
                    found = true;
                }
                h += 32;
            }
            for (; !found && h < pi.m; h += 4 * 32) {
                uint64_t d[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int64_t o = h + 32 * u;   // past the shorter suffix's end: a "mismatch" at o
                    d[u] = o < pi.m ? bases32(t.packed, pi.bp + o) ^ bases32(t.packed, pi.bq + o) : ~0ull;
                }
                int64_t at = -1;
#pragma unroll
                for (int u = 3; u >= 0; --u)
                    if (d[u]) at = h + 32 * u + (__clzll((long long)d[u]) >> 1);
                if (at >= 0) { res = min(at, pi.m); break; }
            }
            lcp[j] = (int32_t)res;
            prev_p = p;
            prev_h = res;
        }
    }
}

// With the inverse SA at hand: PLCP in text order (Kaerkkaeinen, Manzini &
// Puglisi's Phi algorithm).  PLCP[p] = LCP of suffix p with its SA predecessor
// sa[isa[p] - 1]; PLCP[p] >= PLCP[p-1] - 1, so each thread walks kPhiChunk
// consecutive positions and starts each comparison where the previous one
// ended.  '$' positions have PLCP 0 (among them every instance's first slot).
constexpr int kPhiChunk = 64;

__global__ void __launch_bounds__(128) k_plcp(TextDesc t, const uint32_t *__restrict__ sa,
                                              const uint32_t *__restrict__ isa,
                                              uint32_t *__restrict__ plcp) {
    const int64_t chunks = (t.N + kPhiChunk - 1) / kPhiChunk;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p0 = c * kPhiChunk, p1 = min(p0 + kPhiChunk, t.N);
        int64_t prev = 0;
        int64_t rp = frag_of(t, p0);
        for (int64_t p = p0; p < p1; ++p) {
            while (__ldg(t.toff + rp + 1) <= p) ++rp;
            const int64_t remp = __ldg(t.toff + rp + 1) - 1 - p;
            const uint32_t j = isa[p];
            int64_t h = 0;
            if (remp > 0 && j > 0) {
                const int64_t q = sa[j - 1];
                const int64_t rq = frag_of(t, q);
                const int64_t m = min(remp, __ldg(t.toff + rq + 1) - 1 - q);
                const uint64_t bp = (uint64_t)(p - rp), bq = (uint64_t)(q - rq);
                h = min(max(prev - 1, (int64_t)0), m);
                for (; h < m; h += 4 * 32) {
                    uint64_t d[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        int64_t o = h + 32 * u;
                        d[u] = o < m ? bases32(t.packed, bp + o) ^ bases32(t.packed, bq + o) : ~0ull;
                    }
                    int64_t at = -1;
#pragma unroll
                    for (int u = 3; u >= 0; --u)
                        if (d[u]) at = h + 32 * u + (__clzll((long long)d[u]) >> 1);
                    if (at >= 0) { h = at; break; }
                }
                h = min(h, m);
            }
            plcp[p] = (uint32_t)h;
            prev = h;
        }
    }
}

__global__ void k_lcp_gather(const uint32_t *__restrict__ sa, const uint32_t *__restrict__ plcp,
                             int64_t N, int32_t *__restrict__ lcp) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x)
        lcp[j] = (int32_t)__ldg(plcp + sa[j]);
}

// ---- finishing the LCP inside a suffix-array build (sa_lcp_build), with the
// inverse SA at hand: the pairs round 0 left (-1: they share their first `skip`
// bases) are marked by the text position of their lower suffix in a bitmap, then
// walked in text order, 16 positions per thread (more threads in flight beat
// longer chains: 32 or 64 positions measured slower).  Kasai's bound chains the walk:
// the LCP of position p with its SA predecessor is at least that of p - 1 minus
// one, so a comparison starts where the previous one ended.  No sort by position
// is needed: the bitmap is the order.
__global__ void __launch_bounds__(256) k_lcp_mark(const uint32_t *__restrict__ sa,
                                                  const int32_t *__restrict__ lcp, int64_t N,
                                                  uint32_t *__restrict__ bits) {
    // four entries per 16-byte load when lcp is 16-byte aligned (else all scalar);
    // the SA is read only where an entry is left (-1)
    const int64_t quads = ((uintptr_t)lcp & 15u) == 0 ? (N >> 2) : 0;
    const int4 *lcp4 = reinterpret_cast<const int4 *>(lcp);
    for (int64_t qd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; qd < quads;
         qd += (int64_t)gridDim.x * blockDim.x) {
        const int4 v = lcp4[qd];
        const int64_t j = qd << 2;
        const int32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e[u] < 0) {
                const uint32_t p = sa[j + u];
                atomicOr(bits + (p >> 5), 1u << (p & 31u));
            }
    }
    for (int64_t j = (quads << 2) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N;
         j += (int64_t)gridDim.x * blockDim.x) {   // the last N mod 4 entries
        if (lcp[j] < 0) {
            const uint32_t p = sa[j];
            atomicOr(bits + (p >> 5), 1u << (p & 31u));
        }
    }
}

__global__ void __launch_bounds__(128) k_lcp_walk(TextDesc t, const uint32_t *__restrict__ sa,
                                                  const uint32_t *__restrict__ isa,
                                                  const uint32_t *__restrict__ bits, int skip,
                                                  int32_t *__restrict__ lcp) {
    const int64_t halves = ((t.N + 31) >> 5) * 2;   // 16 positions per thread
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < halves;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = c >> 1;
        const int sh = (int)(c & 1) * 16;
        uint32_t m = (bits[w] >> sh) & 0xffffu;
        int64_t prev_p = -2, prev_h = 0;
        while (m) {
            const int b = __ffs(m) - 1 + sh;
            m &= m - 1u;
            const int64_t p = (w << 5) + b;
            const int64_t j = isa[p];
            if (j <= 0 || j >= t.N) continue;   // never marked: slot 0 has LCP 0
            const int64_t q = sa[j - 1];
            const int64_t rp = frag_of(t, p), rq = frag_of(t, q);
            const int64_t mlen = min(__ldg(t.toff + rp + 1) - 1 - p, __ldg(t.toff + rq + 1) - 1 - q);
            const uint64_t bp = (uint64_t)(p - rp), bq = (uint64_t)(q - rq);
            int64_t h = (p == prev_p + 1 && prev_h - 1 > skip) ? prev_h - 1 : skip;
            int64_t res = mlen;
            bool found = false;
            if (h < mlen) {   // one word first: past Kasai's bound most pairs differ within it
                const uint64_t d0 = bases32(t.packed, bp + h) ^ bases32(t.packed, bq + h);
                if (d0) {
                    res = min(h + (int64_t)(__clzll((long long)d0) >> 1), mlen);
                    found = true;
                }
                h += 32;
            }
            for (; !found && h < mlen; h += 4 * 32) {
                uint64_t d[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t o = h + 32 * u;   // past the shorter suffix's end: a "mismatch"
                    d[u] = o < mlen ? bases32(t.packed, bp + o) ^ bases32(t.packed, bq + o) : ~0ull;
                }
                int64_t at = -1;
#pragma unroll
                for (int u = 3; u >= 0; --u)
                    if (d[u]) at = h + 32 * u + (__clzll((long long)d[u]) >> 1);
                if (at >= 0) {
                    res = min(at, mlen);
                    break;
                }
            }
            lcp[j] = (int32_t)res;
            prev_p = p;
            prev_h = res;
        }
    }
}

}  // namespace

int lcp_build_impl(dnasa_ctx *ctx, const TextDesc &t, const uint32_t *sa32, int32_t *lcp,
                   cudaStream_t s, const uint32_t *isa) {
    PhaseRange nvtx_("dnasa.lcp");
    if (isa) {   // Phi / PLCP in text order, then one gather
        DNASA_TRY(ws_reserve(ctx, ((size_t)t.N * 4 + 255) / 256 * 256 + 4096, s));
        Arena a = ws_arena(ctx);
        uint32_t *plcp = a.take<uint32_t>((size_t)t.N);
        int chunks = ceil_div(t.N, kPhiChunk);
        {
            LaunchScope ls_(ctx, PK_LCP, s, 12.0 * t.N);
            int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(chunks, 128), (int64_t)ctx->num_sms * 64));
            k_plcp<<<g, 128, 0, s>>>(t, sa32, isa, plcp);
        }
        {
            LaunchScope ls_(ctx, PK_LCP, s, 12.0 * t.N);
            int g = (int)std::min<int64_t>(ceil_div(t.N, 256), (int64_t)ctx->num_sms * 16);
            k_lcp_gather<<<std::max(g, 1), 256, 0, s>>>(sa32, plcp, t.N, lcp);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
        return DNASA_OK;
    }
    const int tile = radix_tile_default();
    const int key_bits = bits_for((uint64_t)(t.N - 1));
    const size_t q = ((size_t)t.N * 4 + 255) / 256 * 256;
    DNASA_TRY(ws_reserve(ctx, 4 * q + radix_scratch_bytes(t.N, key_bits, tile) + 8192, s));
    Arena a = ws_arena(ctx);
    uint32_t *qk[2] = {a.take<uint32_t>((size_t)t.N), a.take<uint32_t>((size_t)t.N)};
    uint32_t *qv[2] = {a.take<uint32_t>((size_t)t.N), a.take<uint32_t>((size_t)t.N)};
    RadixScratch rs = radix_scratch_take(a, t.N, key_bits, tile);
    if (!rs.hist) return fail(ctx, DNASA_OOM, "lcp_build workspace");
    unsigned long long *nlong = ctx->ctrl->count + CNT_TMP;
    DNASA_CUDA(ctx, cudaMemsetAsync(nlong, 0, 8, s));
    int grid = (int)std::min<int64_t>(ceil_div(t.N, 256), (int64_t)ctx->num_sms * 16);
    {
        LaunchScope ls_(ctx, PK_LCP, s, 8.5 * t.N);
        k_lcp<<<std::max(grid, 1), 256, 0, s>>>(t, sa32, lcp, qk[0], qv[0], nlong);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->pinned, nlong, 8, cudaMemcpyDeviceToHost, s));
    DNASA_TRY(check_device_status(ctx, s, "lcp_build"));
    const int64_t nq = (int64_t)ctx->pinned[0];
    if (nq == 0) return DNASA_OK;
    int which = 0;
    DNASA_TRY(radix_sort_pairs<uint32_t>(ctx, rs, qk, qv, nq, nullptr, key_bits, false, tile, &which, s));
    {
        LaunchScope ls_(ctx, PK_LCP, s, 16.0 * nq);
        int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ceil_div(nq, kChain), 128),
                                                           (int64_t)ctx->num_sms * 64));
        k_lcp_chain<<<g2, 128, 0, s>>>(t, sa32, lcp, qk[which], qv[which], nq);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}


int lcp_finish_with_isa(dnasa_ctx *ctx, const TextDesc &t, const uint32_t *sa32, const uint32_t *isa,
                        int32_t *lcp, int skip, uint32_t *bits, cudaStream_t s) {
    PhaseRange nvtx_("dnasa.lcp_walk");
    const int64_t words = (t.N + 31) >> 5;
    DNASA_CUDA(ctx, cudaMemsetAsync(bits, 0, (size_t)words * 4, s));
    {
        LaunchScope ls_(ctx, PK_LCP, s, 4.0 * t.N);
        const int g = (int)std::min<int64_t>(ceil_div(t.N, 256), (int64_t)ctx->num_sms * 16);
        k_lcp_mark<<<std::max(g, 1), 256, 0, s>>>(sa32, lcp, t.N, bits);
    }
    {
        LaunchScope ls_(ctx, PK_LCP, s, (double)words * 4.0);
        const int g = (int)std::min<int64_t>(ceil_div(words * 2, 128), (int64_t)ctx->num_sms * 64);
        k_lcp_walk<<<std::max(g, 1), 128, 0, s>>>(t, sa32, isa, bits, skip, lcp);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}

}  // namespace dnasa
