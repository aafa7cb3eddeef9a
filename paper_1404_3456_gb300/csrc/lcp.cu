// lcp.cu -- LCP array over the suffix array (S7).
//
// lcp[0] = 0 and lcp[j] = the number of equal bases at the start of suffixes
// SA[j-1] and SA[j], never counting a '$' (so no LCP crosses a fragment end),
// and 0 where an instance of a batch starts.  Each thread compares one adjacent
// pair 32 bases at a time: XOR of two packed words and a count of leading zero
// bits, capped by the bases left in both fragments.  The paper needs these
// prefix lengths for its "is one fragment a prefix of X" tests (Sec. IV); they
// drive the containment test and the overlap interval scan here.
#include <algorithm>

#include "common.cuh"

namespace dnasa {

namespace {

__global__ void __launch_bounds__(256) k_lcp(TextDesc t, const uint32_t *__restrict__ sa,
                                             int32_t *__restrict__ lcp) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < t.N;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (j == 0) { lcp[0] = 0; continue; }
        if (t.n_inst > 1) {
            int64_t i = upper_index(t.inst_toff, 0, t.n_inst, j);
            if (__ldg(t.inst_toff + i) == j) { lcp[j] = 0; continue; }
        }
        int64_t p = sa[j - 1], q = sa[j];
        int64_t rp = read_of(t.toff, t.n_reads, p);
        int64_t rq = read_of(t.toff, t.n_reads, q);
        int64_t m = min(__ldg(t.toff + rp + 1) - 1 - p, __ldg(t.toff + rq + 1) - 1 - q);
        uint64_t bp = (uint64_t)(p - rp), bq = (uint64_t)(q - rq);
        int64_t h = 0;
        while (h < m) {
            uint64_t d = bases32(t.packed, bp + h) ^ bases32(t.packed, bq + h);
            if (d) { h += __clzll((long long)d) >> 1; break; }
            h += 32;
        }
        lcp[j] = (int32_t)min(h, m);
    }
}

}  // namespace

int lcp_build_impl(dnasa_ctx *ctx, const TextDesc &t, const uint32_t *sa32, int32_t *lcp,
                   cudaStream_t s) {
    int grid = (int)std::min<int64_t>(ceil_div(t.N, 256), (int64_t)ctx->num_sms * 16);
    {
        LaunchScope ls_(ctx, PK_LCP, s, 8.5 * t.N);
        k_lcp<<<std::max(grid, 1), 256, 0, s>>>(t, sa32, lcp);
    }
    DNASA_CUDA(ctx, cudaGetLastError());
    return DNASA_OK;
}

}  // namespace dnasa
