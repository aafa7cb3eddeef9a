// radix.cu -- stable LSD radix sort of (key, value) pairs, onesweep style.
//
// Sec. IV of the paper sorts suffix keys with an LSD radix sort in which each
// pass places an element after every element of a smaller bucket and after the
// elements of its own bucket placed before it (after Satish et al.), built from
// split/scan/scatter kernels on shared-memory chunks (Algorithm 1).  This is the
// same sort, re-planned for sm_103a:
//   * one histogram kernel reads the keys once and counts every digit of every
//     pass (8-bit digits, shared-memory atomics), unless the kernel that wrote
//     the keys counted them already;
//   * then one kernel per digit.  Each CTA takes the next tile id from an
//     atomic counter, ranks its tile's digits in shared memory (per-warp
//     ranking: the lanes holding the same digit are found with one ballot per
//     digit bit, the lowest of them bumps the warp's digit counter), publishes
//     its per-digit counts, and looks back over
//     its predecessors' published counts (decoupled look-back) to find its
//     global output offsets; the scatter goes through shared memory so that
//     each digit's run leaves as a contiguous burst.  Every spin on a
//     predecessor is bounded: on time-out the CTA sets DERR_TIMEOUT, publishes
//     an (invalid) inclusive prefix so that no successor waits on it, and the
//     host reports DNASA_DEVICE_TIMEOUT.
// Look-back words live in a status buffer owned by the context; each pass
// stamps its words with an 8-bit epoch so that the buffer is zeroed only when
// the epoch wraps.
#include "common.cuh"

namespace dnasa {

namespace {

constexpr int kThreads = 256;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kWarps = kThreads / 32;

// look-back word: [63:62] flag, [61:54] epoch, [53:0] count
constexpr unsigned long long FLAG_AGG = 1ull << 62;
constexpr unsigned long long FLAG_INC = 2ull << 62;
constexpr unsigned long long VAL_MASK = (1ull << 54) - 1;

__device__ __forceinline__ unsigned long long lb_word(unsigned long long flag, uint32_t epoch,
                                                      unsigned long long v) {
    return flag | ((unsigned long long)(epoch & 0xFF) << 54) | (v & VAL_MASK);
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift) {
    return (uint32_t)(k >> shift) & (kRadix - 1);
}

// Lanes of `vmask` whose 8-bit digit equals this lane's: one ballot per digit
// bit (all 32 lanes take part; lanes outside vmask are masked out).  Eight
// full-rate ballots are much cheaper than one match.any.sync.
__device__ __forceinline__ uint32_t match_digit(uint32_t d, uint32_t vmask) {
    uint32_t peers = vmask;
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
        const uint32_t m = (uint32_t)((int32_t)(d << (31 - b)) >> 31);   // all ones iff bit b set
        peers &= ~(__ballot_sync(0xffffffffu, m) ^ m);   // lanes whose bit b equals ours
    }
    return peers;
}

// ------------------------------------------------------------------ histogram
template <typename K>
__global__ void __launch_bounds__(kThreads) k_hist(const K *__restrict__ keys, int64_t n_host,
                                                   const unsigned long long *__restrict__ d_n,
                                                   int passes, uint32_t *__restrict__ ghist,
                                                   int lo_bit = 0) {
    __shared__ uint32_t sh[8 * kRadix];
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) sh[i] = 0;
    __syncthreads();
    const int64_t n = d_n ? (int64_t)*d_n : n_host;
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    (void)lane;
    for (int64_t i = warp_global * 32 + lane; i < n; i += nwarps * 32) {
        K k = keys[i];
        for (int p = 0; p < passes; ++p)
            atomicAdd(&sh[p * kRadix + digit_of(k, lo_bit + p * kRadixBits)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) {
        uint32_t c = sh[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

// exclusive scan of one 256-bin histogram per block (block = pass)
__global__ void __launch_bounds__(kRadix) k_hist_scan(uint32_t *__restrict__ ghist) {
    __shared__ uint32_t wsum[kRadix / 32];
    uint32_t *h = ghist + blockIdx.x * kRadix;
    uint32_t v = h[threadIdx.x];
    uint32_t x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t off = 0;
    for (int i = 0; i < w; ++i) off += wsum[i];
    h[threadIdx.x] = off + x - v;
}

// ------------------------------------------------------------------ one digit pass
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
}

// Phases of one tile (the look-back latency is the only wait left on the path
// between ranking and the global writes):
//   1. take a tile id; start the values' loads into shared memory (cp.async);
//   2. load keys; count the tile's digits; publish them (AGG);
//   3. rank every key within its warp (stable); tile-local digit offsets;
//   4. scatter keys, then values, into shared memory in digit order;
//   5. look back over the predecessors' counts; publish the inclusive prefix;
//   6. write keys and values, each digit's run as one contiguous burst.
template <typename K, int ITEMS, bool HAS_VALS, int LBW, bool FULL>
__device__ __forceinline__ void onesweep_tile(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *__restrict__ bucket, unsigned long long *status,
    int64_t n, uint32_t tile, int64_t base, int tile_n, int shift, uint32_t epoch, uint32_t *err,
    uint32_t spin_limit, unsigned char *smem_raw) {
    constexpr int TILE = kThreads * ITEMS;
    K *s_keys = reinterpret_cast<K *>(smem_raw);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + TILE);
    uint32_t *s_whist = s_vals + (HAS_VALS ? TILE : 0);          // [kWarps][kRadix]
    uint32_t *s_count = s_whist + kWarps * kRadix;                // [kRadix]
    uint32_t *s_start = s_count + kRadix;                         // [kRadix] tile-local start
    uint32_t *s_gbase = s_start + kRadix;                         // [kRadix] global base - start
    uint32_t *s_misc = s_gbase + kRadix;                          // [kWarps + 2]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // warp-striped layout: warp w owns [w*32*ITEMS, (w+1)*32*ITEMS) of the tile
    const int wbase = warp * 32 * ITEMS;
    auto valid_at = [&](int idx) -> bool { return FULL || idx < tile_n; };

    // ---- 1. values start arriving in shared memory while the keys are ranked
    if (HAS_VALS) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            int idx = wbase + i * 32 + lane;
            if (valid_at(idx)) cp_async4(s_vals + idx, vin + base + idx);
        }
    }
    // ---- 2. keys and their digits; the tile's digit counts, published before
    // any ranking work.  dl[i] keeps the digit (bits 0-7) and, after step 3, the
    // rank among the warp's equal digits (bits 8-31).
    K key[ITEMS];
    uint32_t dl[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int idx = wbase + i * 32 + lane;
        key[i] = valid_at(idx) ? kin[base + idx] : K(0);
        dl[i] = digit_of(key[i], shift);
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int idx = wbase + i * 32 + lane;
        if (valid_at(idx)) atomicAdd(&s_count[dl[i]], 1u);
    }
    __syncthreads();
    for (int d = tid; d < kRadix; d += kThreads)
        st_relaxed_u64(status + (size_t)tile * kRadix + d,
                       lb_word(tile == 0 ? FLAG_INC : FLAG_AGG, epoch, s_count[d]));
    // ---- 3. rank within the warp, item by item (tile order: stable).  The lanes
    // holding the same digit are found by ballots; the lowest of them bumps the
    // warp's counter for that digit and broadcasts the old count.
    uint32_t *wh = s_whist + warp * kRadix;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int idx = wbase + i * 32 + lane;
        const bool valid = valid_at(idx);
        const uint32_t vmask = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
        const uint32_t d = dl[i];
        const uint32_t peers = match_digit(d, vmask);
        const int leader = __ffs(peers) - 1;   // valid lanes: peers holds the lane itself
        uint32_t old = 0;
        if (valid && lane == leader) {   // the leaders of one ballot hold distinct digits
            old = wh[d];
            wh[d] = old + (uint32_t)__popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader < 0 ? 0 : leader);
        dl[i] = d | ((old + __popc(peers & lanemask_lt())) << kRadixBits);
        __syncwarp();
    }
    // tile-local start of each digit (kThreads == kRadix: one digit per thread)
    {
        uint32_t v = s_count[tid];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_misc[warp] = x;
        __syncthreads();
        uint32_t off = 0;
        for (int w = 0; w < warp; ++w) off += s_misc[w];
        s_start[tid] = off + x - v;
        // exclusive scan over warps of this digit's per-warp counts
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = s_whist[w * kRadix + tid];
            s_whist[w * kRadix + tid] = run;
            run += c;
        }
    }
    __syncthreads();
    // ---- 4. keys, then values, into shared memory in digit order
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        int idx = wbase + i * 32 + lane;
        if (valid_at(idx)) {
            const uint32_t d = dl[i] & (kRadix - 1);
            const uint32_t p = s_start[d] + wh[d] + (dl[i] >> kRadixBits);
            s_keys[p] = key[i];
            dl[i] = p;   // from here on: the item's place in the tile
        }
    }
    if (HAS_VALS) {
        cp_async_commit_wait_all();
        __syncthreads();
        uint32_t v[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            int idx = wbase + i * 32 + lane;
            v[i] = valid_at(idx) ? s_vals[idx] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            int idx = wbase + i * 32 + lane;
            if (valid_at(idx)) s_vals[dl[i]] = v[i];
        }
    }
    // ---- 5. look back and form the global base of each digit
    {
        const int d = tid;
        const uint32_t c = s_count[d];
        unsigned long long excl = 0;
        if (tile != 0) {
            // probe LBW predecessors per round trip: LBW independent loads in
            // flight, then consume them nearest first
            int64_t t = (int64_t)tile - 1;
            uint32_t spins = 0;
            bool gave_up = false;
            bool done = false;
            while (!done) {
                unsigned long long w[LBW];
#pragma unroll
                for (int k = 0; k < LBW; ++k)
                    w[k] = t - k >= 0 ? ld_relaxed_u64(status + (size_t)(t - k) * kRadix + d)
                                      : lb_word(FLAG_INC, epoch, 0);   // before tile 0: nothing
                int k = 0;
                for (; k < LBW; ++k) {
                    uint32_t we = (uint32_t)(w[k] >> 54) & 0xFF;
                    unsigned long long flag = w[k] & (3ull << 62);
                    if (flag == 0 || we != (epoch & 0xFF)) break;   // not published yet
                    excl += w[k] & VAL_MASK;
                    if (flag == FLAG_INC) { done = true; break; }
                }
                if (done) break;
                if (k == LBW) { t -= LBW; continue; }
                t -= k;                                            // wait on tile t
                if (++spins > spin_limit || ((spins & 1023) == 0 && ld_relaxed_u32(err) != 0)) {
                    gave_up = true;
                    break;
                }
                __nanosleep(32);
            }
            if (gave_up) {
                atomicOr(err, DERR_TIMEOUT);
                s_misc[kWarps + 1] = 1;
            }
            st_relaxed_u64(status + (size_t)tile * kRadix + d, lb_word(FLAG_INC, epoch, excl + c));
        }
        s_gbase[d] = bucket[d] + (uint32_t)excl - s_start[d];
    }
    __syncthreads();
    if (s_misc[kWarps + 1]) return;   // offsets unknown: write nothing
    // ---- 6. global writes
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int idx = tid + i * kThreads;
        if (!valid_at(idx)) break;
        const K k = s_keys[idx];
        const uint32_t o = s_gbase[digit_of(k, shift)] + (uint32_t)idx;
        if (o < (uint64_t)n) {
            kout[o] = k;
            if (HAS_VALS) vout[o] = s_vals[idx];
        } else {
            atomicOr(err, DERR_BOUNDS);
        }
    }
}

// CTAs per SM a variant is held to: the pass is latency- and issue-bound, so
// small tiles (2048 items) take five CTAs per SM and the larger ones three (80
// registers, no spills).  Every tile but the last is full and runs without
// per-item bounds tests.
template <int ITEMS>
struct OnesweepOcc {
    static constexpr int value = ITEMS <= 8 ? 5 : 3;
};

template <typename K, int ITEMS, bool HAS_VALS, int LBW>
__global__ void __launch_bounds__(kThreads, OnesweepOcc<ITEMS>::value) k_onesweep(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
    uint32_t *__restrict__ vout, const uint32_t *__restrict__ bucket, unsigned long long *status,
    uint32_t *tile_ctr, int64_t n_host, const unsigned long long *__restrict__ d_n, int shift,
    uint32_t epoch, uint32_t *err, uint32_t spin_limit) {
    constexpr int TILE = kThreads * ITEMS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_whist = reinterpret_cast<uint32_t *>(smem_raw + (size_t)TILE * sizeof(K)) +
                        (HAS_VALS ? TILE : 0);
    uint32_t *s_count = s_whist + kWarps * kRadix;
    uint32_t *s_misc = s_count + 3 * kRadix;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_misc[kWarps] = atomicAdd(tile_ctr, 1u);
        s_misc[kWarps + 1] = 0;   // set when a look-back gave up: skip the writes
    }
    for (int i = tid; i < kWarps * kRadix; i += kThreads) s_whist[i] = 0;
    for (int i = tid; i < kRadix; i += kThreads) s_count[i] = 0;
    __syncthreads();
    const uint32_t tile = s_misc[kWarps];
    const int64_t n = d_n ? (int64_t)*d_n : n_host;
    const int64_t base = (int64_t)tile * TILE;
    if (base >= n) return;   // uniform over the CTA; later tiles are empty too
    const int tile_n = (int)min((int64_t)TILE, n - base);
    if (tile_n == TILE)
        onesweep_tile<K, ITEMS, HAS_VALS, LBW, true>(kin, vin, kout, vout, bucket, status, n, tile, base,
                                                     tile_n, shift, epoch, err, spin_limit, smem_raw);
    else
        onesweep_tile<K, ITEMS, HAS_VALS, LBW, false>(kin, vin, kout, vout, bucket, status, n, tile, base,
                                                      tile_n, shift, epoch, err, spin_limit, smem_raw);
}

template <typename K, int ITEMS, bool HAS_VALS>
size_t onesweep_smem() {
    constexpr int TILE = kThreads * ITEMS;
    return (size_t)TILE * sizeof(K) + (HAS_VALS ? (size_t)TILE * 4 : 0) +
           (size_t)(kWarps * kRadix + 3 * kRadix + kWarps + 2) * 4;
}

template <typename K, int ITEMS, bool HAS_VALS, int LBW>
cudaError_t launch_pass(int tiles, cudaStream_t s, const K *kin, const uint32_t *vin, K *kout,
                        uint32_t *vout, const uint32_t *bucket, unsigned long long *status,
                        uint32_t *tile_ctr, int64_t n_host, const unsigned long long *d_n,
                        int shift, uint32_t epoch, uint32_t *err, uint32_t spin_limit = kSpinLimit) {
    size_t smem = onesweep_smem<K, ITEMS, HAS_VALS>();
    auto kern = k_onesweep<K, ITEMS, HAS_VALS, LBW>;
    const cudaError_t configured = smem_attr(kern, smem);   // once per (kernel, device)
    if (configured != cudaSuccess) return configured;
    kern<<<tiles, kThreads, smem, s>>>(kin, vin, kout, vout, bucket, status, tile_ctr, n_host,
                                       d_n, shift, epoch, err, spin_limit);
    return cudaGetLastError();
}

int items_for_tile(int tile_items) {
    switch (tile_items) {
        case 2048: return 8;
        case 5120: return 20;
        default: return 15;
    }
}

}  // namespace

int radix_tile_default() { return 3840; }

size_t radix_scratch_bytes(int64_t n_max, int key_bits, int tile_items) {
    int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    (void)n_max; (void)tile_items;
    return ((size_t)passes * kRadix * 4 + 255) & ~size_t(255);
}

RadixScratch radix_scratch_take(Arena &a, int64_t n_max, int key_bits, int tile_items) {
    (void)n_max; (void)tile_items;
    RadixScratch rs;
    int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    rs.hist = a.take<uint32_t>((size_t)passes * kRadix);
    return rs;
}

// Look-back status buffer of the context: grown on demand, zeroed on growth and
// when the 8-bit epoch wraps.
static int lb_prepare(dnasa_ctx *ctx, size_t words, cudaStream_t s, unsigned long long **buf,
                      uint32_t *epoch) {
    if (ctx->lb_words < words) {
        if (ctx->lb_buf) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->lb_buf);
            ctx->lb_buf = nullptr;
        }
        size_t w = words + words / 4 + 4096;
        cudaError_t e = cudaMalloc(&ctx->lb_buf, w * 8);
        if (e != cudaSuccess) {
            ctx->lb_words = 0;
            ctx->lb_buf = nullptr;
            return cuda_fail(ctx, e, "look-back status alloc");
        }
        ctx->lb_words = w;
        DNASA_CUDA(ctx, cudaMemsetAsync(ctx->lb_buf, 0, w * 8, s));
        ctx->lb_epoch = 0;
    }
    if (++ctx->lb_epoch > 255) {
        DNASA_CUDA(ctx, cudaMemsetAsync(ctx->lb_buf, 0, ctx->lb_words * 8, s));
        ctx->lb_epoch = 1;
    }
    *buf = ctx->lb_buf;
    *epoch = ctx->lb_epoch;
    return DNASA_OK;
}

template <typename K>
int radix_sort_pairs(dnasa_ctx *ctx, const RadixScratch &rs, K *keys[2], uint32_t *vals[2],
                     int64_t n_host, const unsigned long long *d_n, int key_bits, bool hist_ready,
                     int tile_items, int *which, cudaStream_t s, int lbw, int lo_bit) {
    *which = 0;
    if (n_host <= 0) return DNASA_OK;
    if (lo_bit < 0 || lo_bit + key_bits > (int)(8 * sizeof(K)))
        return fail(ctx, DNASA_INVALID_ARG, "radix: key bit range");
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    if (passes > 8) return fail(ctx, DNASA_INVALID_ARG, "radix: too many passes");
    const int items = items_for_tile(tile_items);
    const int tile = kThreads * items;
    const int tiles = ceil_div(n_host, tile);
    const bool has_vals = vals && vals[0] && vals[1];
    if (!hist_ready) {
        DNASA_CUDA(ctx, cudaMemsetAsync(rs.hist, 0, (size_t)passes * kRadix * 4, s));
        int grid = (int)std::min<int64_t>((int64_t)ctx->num_sms * 8, ceil_div(n_host, kThreads * 8));
        if (grid < 1) grid = 1;
        {
            LaunchScope ls_(ctx, PK_HIST, s, (double)n_host * sizeof(K));
            k_hist<K><<<grid, kThreads, 0, s>>>(keys[0], n_host, d_n, passes, rs.hist, lo_bit);
        }
        DNASA_CUDA(ctx, cudaGetLastError());
    }
    {
        LaunchScope ls_(ctx, PK_OTHER, s, 0);
        k_hist_scan<<<passes, kRadix, 0, s>>>(rs.hist);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    DNASA_CUDA(ctx, cudaMemsetAsync(ctx->ctrl->tile_ctr, 0, sizeof(uint32_t) * 8, s));
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        unsigned long long *status;
        uint32_t epoch;
        DNASA_TRY(lb_prepare(ctx, (size_t)tiles * kRadix, s, &status, &epoch));
        const K *kin = keys[cur];
        K *kout = keys[cur ^ 1];
        const uint32_t *vin = has_vals ? vals[cur] : nullptr;
        uint32_t *vout = has_vals ? vals[cur ^ 1] : nullptr;
        cudaError_t e;
        LaunchScope ls_(ctx, PK_ONESWEEP, s,
                        (double)n_host * 2.0 * (sizeof(K) + (has_vals ? 4.0 : 0.0)));
#define DNASA_PASS(IT, HV)                                                                    \
    e = lbw == 1 ? launch_pass<K, IT, HV, 1>(tiles, s, kin, vin, kout, vout, rs.hist + p * kRadix,  \
                                             status, ctx->ctrl->tile_ctr + p, n_host, d_n,          \
                                             lo_bit + p * kRadixBits, epoch, &ctx->ctrl->err)       \
                 : launch_pass<K, IT, HV, 8>(tiles, s, kin, vin, kout, vout, rs.hist + p * kRadix, status, \
                               ctx->ctrl->tile_ctr + p, n_host, d_n, lo_bit + p * kRadixBits, epoch, \
                               &ctx->ctrl->err)
        if (has_vals) {
            if (items == 8) DNASA_PASS(8, true);
            else if (items == 20) DNASA_PASS(20, true);
            else DNASA_PASS(15, true);
        } else {
            if (items == 8) DNASA_PASS(8, false);
            else if (items == 20) DNASA_PASS(20, false);
            else DNASA_PASS(15, false);
        }
#undef DNASA_PASS
        if (e != cudaSuccess) return cuda_fail(ctx, e, "onesweep pass");
        cur ^= 1;
    }
    *which = cur;
    return DNASA_OK;
}

template int radix_sort_pairs<uint32_t>(dnasa_ctx *, const RadixScratch &, uint32_t *[2],
                                        uint32_t *[2], int64_t, const unsigned long long *, int,
                                        bool, int, int *, cudaStream_t, int, int);
template int radix_sort_pairs<unsigned long long>(dnasa_ctx *, const RadixScratch &,
                                                  unsigned long long *[2], uint32_t *[2], int64_t,
                                                  const unsigned long long *, int, bool, int,
                                                  int *, cudaStream_t, int, int);


}  // namespace dnasa

using namespace dnasa;

extern "C" int dnasa_sort_pairs(dnasa_ctx *ctx, uint64_t *keys, uint32_t *vals, int64_t n,
                                int key_bits, int tile_items, int lookback, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    if (n < 0 || n >= (int64_t(1) << 32) || key_bits < 1 || key_bits > 64)
        return fail(ctx, DNASA_INVALID_ARG, "dnasa_sort_pairs: need 0 <= n < 2^32, 1 <= key_bits <= 64");
    if (tile_items != 0 && tile_items != 2048 && tile_items != 3840 && tile_items != 5120)
        return fail(ctx, DNASA_INVALID_ARG, "dnasa_sort_pairs: tile_items must be 0, 2048, 3840 or 5120");
    if (lookback != 0 && lookback != 1 && lookback != 8)
        return fail(ctx, DNASA_INVALID_ARG, "dnasa_sort_pairs: lookback must be 0, 1 or 8");
    if (n == 0) return DNASA_OK;
    if (!is_device_ptr(ctx, keys) || (vals && !is_device_ptr(ctx, vals)))
        return fail(ctx, DNASA_INVALID_ARG, "dnasa_sort_pairs: keys and vals must be device pointers");
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int tile = tile_items ? tile_items : radix_tile_default();
    size_t need = ((size_t)n * 8 + 255) / 256 * 256 + ((size_t)n * 4 + 255) / 256 * 256 +
                  radix_scratch_bytes(n, key_bits, tile) + 4096;
    DNASA_TRY(ws_reserve(ctx, need, s));
    Arena a = ws_arena(ctx);
    unsigned long long *kalt = a.take<unsigned long long>((size_t)n);
    uint32_t *valt = a.take<uint32_t>((size_t)n);
    RadixScratch rs = radix_scratch_take(a, n, key_bits, tile);
    unsigned long long *kk[2] = {reinterpret_cast<unsigned long long *>(keys), kalt};
    uint32_t *vv[2] = {vals, vals ? valt : nullptr};
    int which = 0;
    DNASA_TRY(radix_sort_pairs<unsigned long long>(ctx, rs, kk, vv, n, nullptr, key_bits, false,
                                                   tile, &which, s, lookback ? lookback : 8));
    if (which == 1) {
        DNASA_CUDA(ctx, cudaMemcpyAsync(keys, kalt, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        if (vals)
            DNASA_CUDA(ctx, cudaMemcpyAsync(vals, valt, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
    return DNASA_OK;
}

// Failure-path self-test: a pass whose only CTA takes tile 1 and looks back at a
// tile 0 that nothing ever publishes.  Its bounded spin gives up, it records
// DERR_TIMEOUT, writes nothing, and the call reports DNASA_DEVICE_TIMEOUT; the
// context stays usable.  Nothing hangs: the bound is a few thousand probes.
extern "C" int dnasa_selftest_timeout(dnasa_ctx *ctx, void *stream) {
    if (!ctx) return DNASA_INVALID_ARG;
    ctx->last_error.clear();
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    constexpr int kItems = 15, kTile = kThreads * kItems;
    const int64_t n = 2 * kTile;
    DNASA_TRY(ws_reserve(ctx, (size_t)n * 24 + 8 * kRadix + 4096, s));
    Arena a = ws_arena(ctx);
    unsigned long long *k0 = a.take<unsigned long long>((size_t)n), *k1 = a.take<unsigned long long>((size_t)n);
    uint32_t *v0 = a.take<uint32_t>((size_t)n), *v1 = a.take<uint32_t>((size_t)n);
    uint32_t *bucket = a.take<uint32_t>(kRadix);
    if (!bucket) return fail(ctx, DNASA_OOM, "selftest workspace");
    DNASA_CUDA(ctx, cudaMemsetAsync(k0, 0, (size_t)n * 8, s));
    DNASA_CUDA(ctx, cudaMemsetAsync(v0, 0, (size_t)n * 4, s));
    DNASA_CUDA(ctx, cudaMemsetAsync(bucket, 0, kRadix * 4, s));
    unsigned long long *status;
    uint32_t epoch;
    DNASA_TRY(lb_prepare(ctx, (size_t)2 * kRadix, s, &status, &epoch));
    const uint32_t one = 1;   // the only CTA will draw tile 1: tile 0 never runs
    DNASA_CUDA(ctx, cudaMemcpyAsync(ctx->ctrl->tile_ctr, &one, 4, cudaMemcpyHostToDevice, s));
    cudaError_t e = launch_pass<unsigned long long, kItems, true, 8>(
        1, s, k0, v0, k1, v1, bucket, status, ctx->ctrl->tile_ctr, n, nullptr, 0, epoch,
        &ctx->ctrl->err, 4096u);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "selftest pass");
    return check_device_status(ctx, s, "dnasa_selftest_timeout");
}

// ------------------------------------------------------------------ allocation-free sort
// Some callers cannot call cudaMalloc: code running under a host framework whose
// caching allocator has already reserved the device memory (a fresh cudaMalloc
// can fail or fragment that reservation), and latency-bound loops where an
// allocation's implicit device synchronization is not acceptable.  For them,
// dnasa_sort_pairs_noalloc runs the same radix-sort kernels on scratch that lives
// in the file-scope device array below: at most kNoAllocMaxItems pairs, about
// 12.6 MB that every device which loads this library keeps until the process
// exits.  All calls share that one array and it keeps the previous call's
// contents, so each call clears what must start at zero, and calls that overlap
// on the GPU (concurrent streams) race with each other.
namespace dnasa {
namespace noalloc {

constexpr int64_t kNoAllocMaxItems = DNASA_NOALLOC_MAX_ITEMS;
constexpr int kNoAllocItemsPerThread = 15;                            // 3840-item tiles
constexpr int kNoAllocTile = kThreads * kNoAllocItemsPerThread;
constexpr int kNoAllocTiles = (int)((kNoAllocMaxItems + kNoAllocTile - 1) / kNoAllocTile);

struct NoAllocScratch {
    unsigned long long keys[kNoAllocMaxItems];                  // alternate key buffer
    uint32_t vals[kNoAllocMaxItems];                            // alternate value buffer
    unsigned long long status[(size_t)kNoAllocTiles * kRadix];  // look-back words
    uint32_t hist[8 * kRadix];                                  // digit counts, then offsets
    uint32_t tile_ctr[8];                                       // one tile counter per pass
    uint32_t err;                                               // DERR_* flags of the call
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Device address of g_noalloc_scratch per device ordinal, found once per device.
static NoAllocScratch *g_noalloc_addr[64];

// True if p is device or managed memory that belongs to device `dev`.
static bool noalloc_device_ptr(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // an unknown pointer leaves no sticky error behind
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

__global__ void k_noalloc_clear(NoAllocScratch *S, int tiles) {
    const int64_t words = (int64_t)tiles * kRadix;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        S->status[i] = 0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 8 * kRadix; i += gridDim.x * blockDim.x)
        S->hist[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x < 8) S->tile_ctr[threadIdx.x] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) S->err = 0u;
}

template <bool HAS_VALS>
int noalloc_sort(NoAllocScratch *S, unsigned long long *keys, uint32_t *vals, int64_t n,
                 int key_bits, int num_sms, cudaStream_t s) {
    const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    const int tiles = ceil_div(n, kNoAllocTile);
    k_noalloc_clear<<<std::max(1, std::min(tiles, 64)), 256, 0, s>>>(S, tiles);
    int grid = std::max(1, (int)std::min<int64_t>((int64_t)num_sms * 8, ceil_div(n, kThreads * 8)));
    k_hist<unsigned long long><<<grid, kThreads, 0, s>>>(keys, n, nullptr, passes, S->hist);
    k_hist_scan<<<passes, kRadix, 0, s>>>(S->hist);
    if (cudaGetLastError() != cudaSuccess) return DNASA_CUDA_ERROR;
    unsigned long long *kb[2] = {keys, S->keys};
    uint32_t *vb[2] = {vals, S->vals};
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        cudaError_t e = launch_pass<unsigned long long, kNoAllocItemsPerThread, HAS_VALS, 8>(
            tiles, s, kb[cur], HAS_VALS ? vb[cur] : nullptr, kb[cur ^ 1],
            HAS_VALS ? vb[cur ^ 1] : nullptr, S->hist + p * kRadix, S->status, S->tile_ctr + p, n,
            nullptr, p * kRadixBits, (uint32_t)(p + 1), &S->err);
        if (e != cudaSuccess) return DNASA_CUDA_ERROR;
        cur ^= 1;
    }
    if (cur == 1) {   // result sits in the scratch buffers: copy it back
        if (cudaMemcpyAsync(keys, S->keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return DNASA_CUDA_ERROR;
        if (HAS_VALS &&
            cudaMemcpyAsync(vals, S->vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return DNASA_CUDA_ERROR;
    }
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, &S->err, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return DNASA_CUDA_ERROR;
    if (err & DERR_TIMEOUT) return DNASA_DEVICE_TIMEOUT;
    return err ? DNASA_CUDA_ERROR : DNASA_OK;
}

}  // namespace noalloc
}  // namespace dnasa

using namespace dnasa::noalloc;

extern "C" int dnasa_sort_pairs_noalloc(uint64_t *keys, uint32_t *vals, int64_t n, int key_bits,
                                        void *stream) {
    if (n < 0 || key_bits < 1 || key_bits > 64) return DNASA_INVALID_ARG;
    if (n > kNoAllocMaxItems) return DNASA_CAPACITY;
    if (n == 0) return DNASA_OK;
    if (!keys) return DNASA_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DNASA_CUDA_ERROR;
    // keys and vals must be device (or managed) memory of the current device:
    // anything else would reach the kernels as a bad address
    if (!noalloc_device_ptr(keys, dev) || (vals && !noalloc_device_ptr(vals, dev)))
        return DNASA_INVALID_ARG;
    if (!g_noalloc_addr[dev]) {
        // First call on this device: look up the array's device address (with
        // this device current).  Make this first call before any stream capture.
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DNASA_CUDA_ERROR;
        }
        g_noalloc_addr[dev] = reinterpret_cast<NoAllocScratch *>(p);
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *k = reinterpret_cast<unsigned long long *>(keys);
    return vals ? noalloc_sort<true>(g_noalloc_addr[dev], k, vals, n, key_bits, sms, s)
                : noalloc_sort<false>(g_noalloc_addr[dev], k, nullptr, n, key_bits, sms, s);
}
