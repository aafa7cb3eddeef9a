// common.cuh -- internal declarations shared by the CUDA translation units of
// libdnasa.so: the context, its workspace arena, status handling, and the
// device helpers for the 2-bit packed text.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "dnasa.h"

namespace dnasa {

// ---------------------------------------------------------------- errors

// Device-side error flags (bit set in DevCtrl::err).
enum : uint32_t {
    DERR_TIMEOUT = 1u,      // a bounded spin-wait gave up
    DERR_BOUNDS = 2u,       // a guarded index fell outside its buffer
    DERR_ALPHABET = 4u,     // pack found a byte outside A/C/G/T/'$'
    DERR_EMPTY_READ = 8u,   // pack found an empty fragment
};

// Small control block in device memory, one per context.
struct DevCtrl {
    uint32_t err;              // OR of DERR_* flags
    uint32_t err_info;
    uint32_t tile_ctr[64];     // dynamic tile counters (onesweep passes, look-back scans)
    unsigned long long count[16];  // general device counters (see CNT_*)
};
enum { CNT_ACTIVE = 0, CNT_GROUPS = 1, CNT_MAXGROUP = 2, CNT_CAND = 3, CNT_EDGES = 4,
       CNT_DOLLARS = 5, CNT_TMP = 6, CNT_SEG = 8 /* 8..12: group counts by size class */ };

// ---------------------------------------------------------------- context

struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0;
    template <typename T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (used + bytes > size) return nullptr;
        T *p = reinterpret_cast<T *>(base + used);
        used += bytes;
        return p;
    }
};

}  // namespace dnasa

namespace dnasa {
// Kernel classes the profiler aggregates (same numbering as DNASA_PROF_* in dnasa.h).
enum ProfKind { PK_ONESWEEP = 0, PK_HIST = 1, PK_RERANK = 2, PK_GATHER = 3, PK_INIT = 4,
                PK_FINISH = 5, PK_LCP = 6, PK_OVERLAP = 7, PK_LAYOUT = 8, PK_PACK = 9,
                PK_OTHER = 10, PK_SEGSORT = 11, PK_APPLY = 12, PK_COUNT = 13 };
struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double bytes;
};
}  // namespace dnasa

struct dnasa_ctx {
    int device = 0;
    size_t ws_cap = 0;        // 0 = unbounded
    void *ws = nullptr;       // device workspace
    size_t ws_size = 0;
    dnasa::DevCtrl *ctrl = nullptr;   // device
    unsigned long long *pinned = nullptr;  // host pinned readback buffer (64 words)
    std::string last_error;
    dnasa_trace trace{};
    int num_sms = 0;
    unsigned long long *lb_buf = nullptr;  // onesweep look-back status words (device)
    size_t lb_words = 0;
    uint32_t lb_epoch = 0;
    // profiling: launch counter (always on) and, when enabled, an event pair per launch
    unsigned long long launches = 0;
    bool prof_on = false;
    std::vector<dnasa::ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    // sa_build's doubling loop as a captured graph (owned by sa.cu; freed with the context)
    void *sa_graph = nullptr;
    void (*sa_graph_free)(void *) = nullptr;
};

namespace dnasa {

// Records msg as the context's last error and returns code.
int fail(dnasa_ctx *ctx, int code, const std::string &msg);
// Converts a CUDA error into DNASA_CUDA_ERROR (or DNASA_OOM) with context.
int cuda_fail(dnasa_ctx *ctx, cudaError_t e, const char *where);
// Grows the workspace to at least `bytes` (synchronizes `s` first if it must
// reallocate).  Returns DNASA_OK or DNASA_OOM.
int ws_reserve(dnasa_ctx *ctx, size_t bytes, cudaStream_t s);
// Arena over the whole workspace.
inline Arena ws_arena(dnasa_ctx *ctx) { Arena a; a.base = (char *)ctx->ws; a.size = ctx->ws_size; return a; }
// True if p is a device (or managed) pointer on the context's device.
bool is_device_ptr(dnasa_ctx *ctx, const void *p);
// Reads the device error flags (synchronizes s) and maps them to a status;
// clears them.
int check_device_status(dnasa_ctx *ctx, cudaStream_t s, const char *where);
// Raises kernel `fn`'s dynamic shared-memory limit to `bytes` on the CURRENT
// device.  The attribute belongs to a (kernel, device) pair, so it is set the
// first time each pair is seen (a process may use several devices) and
// remembered under a lock; later calls only look it up.
cudaError_t smem_attr_fn(const void *fn, size_t bytes);
template <typename F>
inline cudaError_t smem_attr(F *fn, size_t bytes) { return smem_attr_fn((const void *)fn, bytes); }

// Counts one kernel launch of class `kind` and, when profiling is on, brackets
// it with CUDA events on its stream; `bytes` is the launch's algorithmic
// traffic.  Construct immediately before the launch, destroy right after it.
// A named range for profilers (NVTX v3, header-only: a no-op unless a tool such as
// Nsight Systems is attached).  One per phase: pack, initial sort, doubling
// rounds, LCP, overlap search, layout.
struct PhaseRange {
    explicit PhaseRange(const char *name) { nvtxRangePushA(name); }
    ~PhaseRange() { nvtxRangePop(); }
    PhaseRange(const PhaseRange &) = delete;
    PhaseRange &operator=(const PhaseRange &) = delete;
};

struct LaunchScope {
    dnasa_ctx *ctx;
    int idx = -1;
    cudaStream_t s;
    LaunchScope(dnasa_ctx *c, int kind, cudaStream_t st, double bytes);
    ~LaunchScope();
};

#define DNASA_CUDA(ctx, call)                                         \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::dnasa::cuda_fail(ctx, e_, #call); \
    } while (0)

#define DNASA_TRY(call)                 \
    do {                                \
        int rc_ = (call);               \
        if (rc_ != DNASA_OK) return rc_; \
    } while (0)

// ---------------------------------------------------------------- radix sort

// Stable LSD radix sort of n (key, value) pairs on key bits [0, key_bits),
// 8-bit digits, onesweep passes with decoupled look-back.  keys[0]/vals[0]
// hold the input; keys[1]/vals[1] are the alternate buffers.  vals may be
// {nullptr, nullptr} for a keys-only sort.  The item count is n_host, or, if
// d_n is non-null, *d_n read on the device (n_host is then an upper bound).
// If `hist_ready` the digit histograms were already accumulated into the
// sorter's histogram buffer by the producer kernel.  On return *which is the
// index of the buffer pair holding the sorted data.
struct RadixScratch {
    uint32_t *hist = nullptr;        // [passes][256] digit counts, then exclusive offsets
    unsigned long long *status = nullptr;  // [tiles][256] look-back words
    size_t status_words = 0;
};
size_t radix_scratch_bytes(int64_t n_max, int key_bits, int tile_items);
RadixScratch radix_scratch_take(Arena &a, int64_t n_max, int key_bits, int tile_items);
// lbw = look-back loads in flight per digit (1 or 8).  The sort is on key bits
// [lo_bit, lo_bit + key_bits).
template <typename K>
int radix_sort_pairs(dnasa_ctx *ctx, const RadixScratch &rs, K *keys[2], uint32_t *vals[2],
                     int64_t n_host, const unsigned long long *d_n, int key_bits, bool hist_ready,
                     int tile_items, int *which, cudaStream_t s, int lbw = 8, int lo_bit = 0);
// Launch of the histogram kernel alone (used when a producer cannot fuse it).
int radix_tile_default();

// ---------------------------------------------------------------- compaction

// out[k] = index of the k-th set flag (flags[i] != 0), i in [0, n); *d_count =
// number of set flags.  Order preserving.  Scratch: compact_scratch_bytes(n).
size_t compact_scratch_bytes(int64_t n);
int compact_flags(dnasa_ctx *ctx, Arena &a, const uint8_t *flags, int64_t n, uint32_t *out,
                  unsigned long long *d_count, cudaStream_t s);

// ---------------------------------------------------------------- SA build internals

struct TextDesc {
    const uint64_t *packed;
    const int64_t *toff;       // device, n_reads + 1
    int64_t n_reads;
    int64_t N;
    const int64_t *inst_toff;  // device, n_inst + 1 text offsets of instances (nullptr: one)
    const int64_t *inst_roff;  // device, n_inst + 1 fragment offsets of instances
    int32_t n_inst;
    const uint32_t *fid;       // device, N: fragment of each text position (nullptr: search toff)
};

// Stream-ordered device buffer, freed on the stream when it goes out of scope.
struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, s);
    }
};
int dev_alloc(dnasa_ctx *ctx, DevBuf &b, size_t bytes, cudaStream_t s);
// Device copies of the instance offsets of a batch: text offsets (from the host
// array inst_toff_host, n_inst + 1 entries) and the first fragment of each
// instance; *max_reads = most fragments in one instance.  Synchronizes s.
int make_instances(dnasa_ctx *ctx, const int64_t *toff, int64_t n_reads, int64_t N,
                   const int64_t *inst_toff_host, int32_t n_inst, DevBuf &inst_toff, DevBuf &inst_roff,
                   int64_t *max_reads, cudaStream_t s);
// Device workspace sa_build_u32 takes for an N-symbol text (bytes, before the
// context's growth margin).
size_t sa_workspace_bytes(int64_t N, int tile_items);
// Builds the SA into sa32 (uint32, N entries, text coordinates).  If isa_out is
// non-null it also receives the inverse SA (the final rank array), N uint32.
// lcp_out (may be null): also the LCP array (as lcp_build_impl) -- round 0 writes
// the LCP of every SA pair the initial keys separate, lcp_finish_with_isa the rest.
int sa_build_u32(dnasa_ctx *ctx, const TextDesc &t, uint32_t *sa32, const dnasa_opts *opts,
                 cudaStream_t s, uint32_t *isa_out = nullptr, int32_t *lcp_out = nullptr);
// x[i] = x[0] + ... + x[i] in place (dc3.cu; sums below 2^32).
int scan_inclusive_u32(dnasa_ctx *ctx, uint32_t *x, int64_t n, cudaStream_t s);
// The same suffix array by DC3 (dc3.cu), one instance; isa_out may be null.
int sa_build_dc3(dnasa_ctx *ctx, const TextDesc &t, uint32_t *sa32, cudaStream_t s, uint32_t *isa_out);
// fid[p] = fragment holding text position p, for p in [0, N).
int fragment_ids(dnasa_ctx *ctx, const TextDesc &t, uint32_t *fid, cudaStream_t s);
// isa (may be null) = inverse of sa32: the LCP is then computed in text order.
// Finishes sa_build_u32's lcp_out with the inverse SA (the build's final ranks):
// the -1 slots (pairs equal on their first `skip` bases) are computed by a walk in
// text order.  bits: (N + 31) / 32 words of device scratch.
int lcp_finish_with_isa(dnasa_ctx *ctx, const TextDesc &t, const uint32_t *sa32, const uint32_t *isa,
                        int32_t *lcp, int skip, uint32_t *bits, cudaStream_t s);
int lcp_build_impl(dnasa_ctx *ctx, const TextDesc &t, const uint32_t *sa32, int32_t *lcp,
                   cudaStream_t s, const uint32_t *isa = nullptr);
// isa (may be null: rebuilt from sa32) is the inverse of sa32.
int overlap_impl(dnasa_ctx *ctx, const TextDesc &t, const uint32_t *sa32, const int32_t *lcp,
                 int32_t min_overlap, dnasa_edge *edges, int64_t cap, int64_t *n_edges,
                 uint8_t *contained, cudaStream_t s, const uint32_t *isa = nullptr);
int widen_u32_to_i64(dnasa_ctx *ctx, const uint32_t *a, int64_t n, int64_t *b, cudaStream_t s);
// Symbols in the initial packed key for an N-symbol text of n_inst instances,
// the instance bits, and the position bits packed under the key (0: none;
// pack_bits == nullptr asks for the unpacked key).
int h0_for(int64_t N, int n_inst, int *inst_bits, int *pack_bits);
int pack_impl(dnasa_ctx *ctx, const uint8_t *text, int64_t N, uint64_t *packed, int64_t *toff,
              int64_t toff_cap, int64_t *n_reads, cudaStream_t s);

// ---------------------------------------------------------------- device helpers

// 32 bases starting at base coordinate b (MSB-first), zero beyond the data
// only as far as the padding words reach (callers mask by remaining length).
__device__ __forceinline__ uint64_t bases32(const uint64_t *__restrict__ packed, uint64_t b) {
    uint64_t w = b >> 5;
    uint32_t sh = (uint32_t)(b & 31u) * 2u;
    uint64_t hi = __ldg(packed + w);
    if (sh == 0) return hi;
    uint64_t lo = __ldg(packed + w + 1);
    return (hi << sh) | (lo >> (64u - sh));
}

// Largest r in [lo, hi) with off[r] <= p  (off ascending; off[lo] <= p).
__device__ __forceinline__ int64_t upper_index(const int64_t *__restrict__ off, int64_t lo,
                                               int64_t hi, int64_t p) {
    while (hi - lo > 1) {
        int64_t m = lo + ((hi - lo) >> 1);
        if (__ldg(off + m) <= p) lo = m; else hi = m;
    }
    return lo;
}

// Fragment holding text position p.
__device__ __forceinline__ int64_t read_of(const int64_t *__restrict__ toff, int64_t n_reads,
                                           int64_t p) {
    return upper_index(toff, 0, n_reads, p);
}

// Fragment holding text position p: one load from the per-position table when
// the caller built one, otherwise a binary search of the fragment offsets.
__device__ __forceinline__ int64_t frag_of(const TextDesc &t, int64_t p) {
    return t.fid ? (int64_t)__ldg(t.fid + p) : read_of(t.toff, t.n_reads, p);
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Iterations a look-back spin may take before it gives up (each iteration
// sleeps ~100 ns at most, so the bound is well under a second).
constexpr uint32_t kSpinLimit = 1u << 22;

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int bits_for(uint64_t x) {  // bits to represent values in [0, x]
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b == 0 ? 1 : b;
}

}  // namespace dnasa
