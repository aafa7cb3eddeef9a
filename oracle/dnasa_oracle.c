/*
 * dnasa_oracle.c -- the ORACLE of this repository.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C that states what
 * the GPU path computes, so that tests can compare the two element by element.
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
 * load it.  It shares no code, header, table or helper with the CUDA library
 * (paper_1404_3456_gb300/csrc); neither includes nor links the other.
 *
 * Text model (Sec. III, "given D = (d1, d2, ...)"): the fragments are joined into
 * one byte text T[0..N); every fragment is followed by one separator byte '$'.
 * Fragment r occupies T[toff[r] .. toff[r+1]-1) and T[toff[r+1]-1] == '$';
 * toff[n_reads] == N.  A single genome is one fragment.
 *
 * Separator reading (the paper never says how fragments are separated): every
 * '$' is its own sentinel, smaller than every other symbol, and sentinels are
 * ordered by their position.  So two suffixes compare symbol by symbol until
 * a mismatch or a '$'; if both reach a '$' at the same offset the suffix that
 * starts earlier is smaller.  No comparison ever runs past a '$'.
 *
 * Functions and the passage each follows:
 *   oracle_suffix_array     Sec. IV: the suffix array "Pos", all suffixes sorted
 *                           (direct comparison; merge sort, stable)
 *   oracle_lcp_kasai        LCP of adjacent SA entries, Kasai et al. 2001
 *   oracle_lcp_direct       the same, measured pair by pair (a pin for Kasai)
 *   oracle_sa_check         Burkhardt & Kaerkkaeinen (CPM 2003) linear SA checker
 *   oracle_inverse_sa, oracle_sa_check_range, oracle_lcp_kasai_range
 *                           the checker and Kasai split into independent ranges
 *                           (for billion-entry arrays, one range per thread)
 *   oracle_check_pairs      sampled SA neighbours (order and LCP) checked one by one
 *   oracle_split_sort_u64   Sec. IV / Algorithm 1: LSD radix sort made of 1-bit
 *                           stable "split" passes (flag, exclusive scan, scatter)
 *   oracle_overlaps_brute   Sec. III "fir" relation generalised to suffix-prefix
 *                           overlaps: all pairs, all lengths
 *   oracle_overlaps_sorted  Sec. IV: the same set by binary search over the
 *                           fragments sorted by their strings
 *   oracle_contained        Sec. III: fragments that occur inside another one
 *   oracle_layout           Sec. III (Fig. 3 path -> superstring, RS concatenation):
 *                           greedy unique-overlap layout, then spelling
 *   oracle_overlaps_approx  Sec. III DEFINITION: overlaps between fragments read on
 *                           either strand, with at most a rate mu of substitutions
 *   oracle_fir_reconstruct  Sec. III (Figs. 2, 5-8): a sequence cut by two shotguns
 *                           rebuilt from fir relations by depth-first search with
 *                           back-tracking
 *
 * Return codes: >= 0 success (or a count), -1 bad argument, -2 capacity,
 * -3 allocation failure.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SEP ((uint8_t)'$')

/* ------------------------------------------------------------------------ */
/* Suffix order under the distinct-sentinel reading.                          */
/* ------------------------------------------------------------------------ */

/* <0, 0, >0 as suffix p is smaller than, equal to, larger than suffix q.
 * T must end with '$', so every walk meets a '$' before the end of T. */
static int suffix_cmp(const uint8_t *T, int64_t p, int64_t q)
{
    if (p == q) return 0;
    for (int64_t k = 0;; ++k) {
        uint8_t a = T[p + k], b = T[q + k];
        int ea = (a == SEP), eb = (b == SEP);
        if (ea && eb) return p < q ? -1 : 1;   /* both end here: earlier start first */
        if (ea) return -1;                      /* '$' is smaller than any symbol */
        if (eb) return 1;
        if (a != b) return a < b ? -1 : 1;
    }
}

static int text_ok(const uint8_t *T, int64_t N)
{
    return T != NULL && N > 0 && T[N - 1] == SEP;
}

/* Suffix array by direct comparison: bottom-up merge sort of 0..N-1. */
int oracle_suffix_array(const uint8_t *T, int64_t N, int64_t *sa)
{
    if (!text_ok(T, N) || sa == NULL) return -1;
    int64_t *tmp = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    if (!tmp) return -3;
    for (int64_t i = 0; i < N; ++i) sa[i] = i;
    int64_t *src = sa, *dst = tmp;
    for (int64_t width = 1; width < N; width *= 2) {
        for (int64_t lo = 0; lo < N; lo += 2 * width) {
            int64_t mid = lo + width < N ? lo + width : N;
            int64_t hi = lo + 2 * width < N ? lo + 2 * width : N;
            int64_t a = lo, b = mid, o = lo;
            while (a < mid && b < hi)
                dst[o++] = suffix_cmp(T, src[b], src[a]) < 0 ? src[b++] : src[a++];
            while (a < mid) dst[o++] = src[a++];
            while (b < hi) dst[o++] = src[b++];
        }
        int64_t *t = src; src = dst; dst = t;
    }
    if (src != sa) memcpy(sa, src, (size_t)N * sizeof(int64_t));
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* LCP array.  lcp[0] = 0; lcp[j] = common prefix of suffixes sa[j-1] and     */
/* sa[j], where '$' never matches (so an LCP never crosses a fragment end).   */
/* ------------------------------------------------------------------------ */

static int64_t common_prefix(const uint8_t *T, int64_t p, int64_t q)
{
    int64_t h = 0;
    while (T[p + h] == T[q + h] && T[p + h] != SEP) ++h;
    return h;
}

int oracle_lcp_direct(const uint8_t *T, int64_t N, const int64_t *sa, int32_t *lcp)
{
    if (!text_ok(T, N) || !sa || !lcp) return -1;
    lcp[0] = 0;
    for (int64_t j = 1; j < N; ++j) lcp[j] = (int32_t)common_prefix(T, sa[j - 1], sa[j]);
    return 0;
}

/* Kasai, Lee, Arimura, Arikawa, Park (CPM 2001): walk the text in position
 * order; the LCP of suffix i+1 with its SA predecessor is at least the LCP of
 * suffix i with its predecessor, minus one. */
int oracle_lcp_kasai(const uint8_t *T, int64_t N, const int64_t *sa, int32_t *lcp)
{
    if (!text_ok(T, N) || !sa || !lcp) return -1;
    int64_t *isa = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    if (!isa) return -3;
    for (int64_t j = 0; j < N; ++j) isa[sa[j]] = j;
    int64_t h = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t r = isa[i];
        if (r == 0) { lcp[0] = 0; h = 0; continue; }
        int64_t j = sa[r - 1];
        while (T[i + h] == T[j + h] && T[i + h] != SEP) ++h;
        lcp[r] = (int32_t)h;
        if (h > 0) --h;
    }
    free(isa);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Burkhardt & Kaerkkaeinen linear-time suffix array checker.                 */
/* Returns 0 if sa is THE suffix array of T, otherwise a positive code:       */
/*   1 not a permutation; 2 + j for the first adjacent pair (j-1, j) whose    */
/*   first symbols are out of order or whose tails are out of order.          */
/* ------------------------------------------------------------------------ */
int64_t oracle_sa_check(const uint8_t *T, int64_t N, const int64_t *sa)
{
    if (!text_ok(T, N) || !sa) return -1;
    int64_t *isa = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    if (!isa) return -3;
    for (int64_t i = 0; i < N; ++i) isa[i] = -1;
    for (int64_t j = 0; j < N; ++j) {
        int64_t p = sa[j];
        if (p < 0 || p >= N || isa[p] != -1) { free(isa); return 1; }
        isa[p] = j;
    }
    int64_t bad = 0;
    for (int64_t j = 1; j < N && !bad; ++j) {
        int64_t p = sa[j - 1], q = sa[j];
        uint8_t a = T[p], b = T[q];
        if (a == SEP && b == SEP) { if (!(p < q)) bad = 2 + j; }
        else if (a == SEP) { /* '$' before a symbol: in order */ }
        else if (b == SEP) bad = 2 + j;
        else if (a < b) { /* in order */ }
        else if (a > b) bad = 2 + j;
        else if (!(isa[p + 1] < isa[q + 1])) bad = 2 + j;
    }
    free(isa);
    return bad;
}

/* The same checker and Kasai's LCP split into independent pieces, for arrays
 * of a billion entries and more (the large single-genome case): the caller
 * builds the inverse once, then checks pair ranges and computes LCP position
 * ranges in as many threads as it likes.  Each piece is the algorithm above
 * restricted to its range; nothing is shared but read-only inputs.
 *
 * oracle_inverse_sa: isa[sa[j]] = j.  Returns 0, or 1 if sa is not a
 * permutation of 0..N-1 (the first test of the checker). */
int64_t oracle_inverse_sa(const int64_t *sa, int64_t N, int64_t *isa)
{
    if (!sa || !isa || N <= 0) return -1;
    for (int64_t i = 0; i < N; ++i) isa[i] = -1;
    for (int64_t j = 0; j < N; ++j) {
        int64_t p = sa[j];
        if (p < 0 || p >= N || isa[p] != -1) return 1;
        isa[p] = j;
    }
    return 0;
}

/* The order tests of oracle_sa_check for the adjacent pairs (j-1, j), j in
 * [j0, j1), given the inverse.  Returns 0 or 2 + the first j that fails. */
int64_t oracle_sa_check_range(const uint8_t *T, int64_t N, const int64_t *sa, const int64_t *isa,
                              int64_t j0, int64_t j1)
{
    if (!text_ok(T, N) || !sa || !isa || j0 < 1 || j1 > N || j0 > j1) return -1;
    for (int64_t j = j0; j < j1; ++j) {
        int64_t p = sa[j - 1], q = sa[j];
        uint8_t a = T[p], b = T[q];
        if (a == SEP && b == SEP) { if (!(p < q)) return 2 + j; }
        else if (a == SEP) { /* '$' before a symbol: in order */ }
        else if (b == SEP) return 2 + j;
        else if (a < b) { /* in order */ }
        else if (a > b) return 2 + j;
        else if (!(isa[p + 1] < isa[q + 1])) return 2 + j;
    }
    return 0;
}

/* Kasai's walk over text positions [p0, p1) only: lcp[isa[i]] for those i.
 * It starts with h = 0 at p0 instead of the bound carried from p0 - 1, which
 * costs extra comparisons at the start of the range but never changes a value
 * (the bound only skips symbols already known to match). */
int oracle_lcp_kasai_range(const uint8_t *T, int64_t N, const int64_t *sa, const int64_t *isa,
                           int64_t p0, int64_t p1, int32_t *lcp)
{
    if (!text_ok(T, N) || !sa || !isa || !lcp || p0 < 0 || p1 > N || p0 > p1) return -1;
    int64_t h = 0;
    for (int64_t i = p0; i < p1; ++i) {
        int64_t r = isa[i];
        if (r == 0) { lcp[0] = 0; h = 0; continue; }
        int64_t j = sa[r - 1];
        while (T[i + h] == T[j + h] && T[i + h] != SEP) ++h;
        lcp[r] = (int32_t)h;
        if (h > 0) --h;
    }
    return 0;
}

/* Checks sampled neighbours of a (possibly huge) suffix array one by one: for
 * each j in idx[0..m), suffix sa[j-1] must be smaller than suffix sa[j] and, if
 * lcp is non-NULL, lcp[j] must be their common prefix.  Returns the number of
 * violations (0 = all sampled pairs correct). */
int64_t oracle_check_pairs(const uint8_t *T, int64_t N, const int64_t *sa, const int32_t *lcp,
                           const int64_t *idx, int64_t m)
{
    if (!text_ok(T, N) || !sa || !idx || m < 0) return -1;
    int64_t bad = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t j = idx[i];
        if (j < 1 || j >= N) { ++bad; continue; }
        int64_t p = sa[j - 1], q = sa[j];
        if (p < 0 || p >= N || q < 0 || q >= N || suffix_cmp(T, p, q) >= 0) { ++bad; continue; }
        if (lcp && lcp[j] != (int32_t)common_prefix(T, p, q)) ++bad;
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: LSD radix sort as repeated 1-bit split.  For each bit i in    */
/* [lo_bit, hi_bit): b = bit i of the key, e = not b, f = exclusive scan of e, */
/* total_false = e[n-1] + f[n-1], t = id - f + total_false, d = b ? t : f,    */
/* out[d] = in.  keys and vals are permuted together, in place.               */
/* ------------------------------------------------------------------------ */
int oracle_split_sort_u64(uint64_t *keys, uint64_t *vals, int64_t n, int lo_bit, int hi_bit)
{
    if (n < 0 || lo_bit < 0 || hi_bit > 64 || lo_bit > hi_bit) return -1;
    if (n == 0) return 0;
    if (!keys || !vals) return -1;
    uint64_t *ok = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint64_t *ov = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    int64_t *f = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!ok || !ov || !f) { free(ok); free(ov); free(f); return -3; }
    for (int i = lo_bit; i < hi_bit; ++i) {
        int64_t run = 0;
        for (int64_t id = 0; id < n; ++id) {       /* f = exclusive scan of e */
            int e = !((keys[id] >> i) & 1u);
            f[id] = run;
            run += e;
        }
        int64_t e_last = !((keys[n - 1] >> i) & 1u);
        int64_t total_false = e_last + f[n - 1];
        for (int64_t id = 0; id < n; ++id) {
            int b = (int)((keys[id] >> i) & 1u);
            int64_t t = id - f[id] + total_false;
            int64_t d = b ? t : f[id];
            ok[d] = keys[id];
            ov[d] = vals[id];
        }
        memcpy(keys, ok, (size_t)n * sizeof(uint64_t));
        memcpy(vals, ov, (size_t)n * sizeof(uint64_t));
    }
    free(ok); free(ov); free(f);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Fragments.  Read r = T[toff[r] .. toff[r+1]-1), its '$' excluded.          */
/* ------------------------------------------------------------------------ */

static int reads_ok(const uint8_t *T, const int64_t *toff, int64_t nr)
{
    if (!T || !toff || nr < 0) return 0;
    if (toff[0] != 0) return 0;
    for (int64_t r = 0; r < nr; ++r) {
        if (toff[r + 1] <= toff[r]) return 0;
        if (T[toff[r + 1] - 1] != SEP) return 0;
        for (int64_t p = toff[r]; p < toff[r + 1] - 1; ++p)
            if (T[p] == SEP) return 0;
    }
    return 1;
}

static int64_t read_len(const int64_t *toff, int64_t r) { return toff[r + 1] - toff[r] - 1; }

/* Overlap set: every ordered pair (j, k), j != k, with the largest L such that
 * lmin <= L <= min(|r_j|, |r_k|) - 1 and the last L symbols of r_j equal the
 * first L symbols of r_k.  Written in (j, k) order.  Returns the number of
 * edges (even when it exceeds cap; only the first cap are written). */
int64_t oracle_overlaps_brute(const uint8_t *T, const int64_t *toff, int64_t nr, int32_t lmin,
                              int32_t *ej, int32_t *ek, int32_t *eL, int64_t cap)
{
    if (!reads_ok(T, toff, nr) || lmin < 1) return -1;
    int64_t ne = 0;
    for (int64_t j = 0; j < nr; ++j) {
        int64_t lj = read_len(toff, j);
        for (int64_t k = 0; k < nr; ++k) {
            if (k == j) continue;
            int64_t lk = read_len(toff, k);
            int64_t Lmax = (lj < lk ? lj : lk) - 1;
            for (int64_t L = Lmax; L >= lmin; --L) {
                if (memcmp(T + toff[j] + lj - L, T + toff[k], (size_t)L) == 0) {
                    if (ne < cap && ej && ek && eL) {
                        ej[ne] = (int32_t)j; ek[ne] = (int32_t)k; eL[ne] = (int32_t)L;
                    }
                    ++ne;
                    break;
                }
            }
        }
    }
    return ne;
}

/* Order of fragments by their strings ('$' smallest), ties by index. */
static _Thread_local const uint8_t *g_T;   /* per thread: callers may run in parallel */
static _Thread_local const int64_t *g_toff;
static int read_cmp(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    int c = suffix_cmp(g_T, g_toff[a], g_toff[b]);
    if (c != 0) return c;
    return a < b ? -1 : (a > b);
}

/* Compare the first min(|r|, L) symbols of fragment r with Q[0..L); a fragment
 * shorter than L that is a prefix of Q is smaller. */
static int prefix_cmp(const uint8_t *T, const int64_t *toff, int64_t r, const uint8_t *Q, int64_t L)
{
    int64_t lr = read_len(toff, r);
    int64_t m = lr < L ? lr : L;
    int c = memcmp(T + toff[r], Q, (size_t)m);
    if (c != 0) return c;
    return lr < L ? -1 : 0;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y);
}

/* The same overlap set as oracle_overlaps_brute, found the way Sec. IV
 * describes: sort the fragments, then for each candidate suffix X of r_j
 * binary-search the fragments that have X as a prefix. */
int64_t oracle_overlaps_sorted(const uint8_t *T, const int64_t *toff, int64_t nr, int32_t lmin,
                               int32_t *ej, int32_t *ek, int32_t *eL, int64_t cap)
{
    if (!reads_ok(T, toff, nr) || lmin < 1) return -1;
    int64_t *ord = (int64_t *)malloc((size_t)(nr ? nr : 1) * sizeof(int64_t));
    int64_t *best = (int64_t *)malloc((size_t)(nr ? nr : 1) * sizeof(int64_t));
    int64_t *touched = (int64_t *)malloc((size_t)(nr ? nr : 1) * sizeof(int64_t));
    if (!ord || !best || !touched) { free(ord); free(best); free(touched); return -3; }
    for (int64_t r = 0; r < nr; ++r) { ord[r] = r; best[r] = -1; }
    g_T = T; g_toff = toff;
    qsort(ord, (size_t)nr, sizeof(int64_t), read_cmp);
    int64_t ne = 0;
    for (int64_t j = 0; j < nr; ++j) {
        int64_t lj = read_len(toff, j), nt = 0;
        for (int64_t L = lmin; L <= lj - 1; ++L) {
            const uint8_t *Q = T + toff[j] + lj - L;
            int64_t lo = 0, hi = nr;           /* first with prefix_cmp >= 0 */
            while (lo < hi) {
                int64_t m = lo + (hi - lo) / 2;
                if (prefix_cmp(T, toff, ord[m], Q, L) < 0) lo = m + 1; else hi = m;
            }
            int64_t a = lo;
            lo = a; hi = nr;                   /* first with prefix_cmp > 0 */
            while (lo < hi) {
                int64_t m = lo + (hi - lo) / 2;
                if (prefix_cmp(T, toff, ord[m], Q, L) <= 0) lo = m + 1; else hi = m;
            }
            for (int64_t x = a; x < lo; ++x) {
                int64_t k = ord[x];
                if (k == j || L > read_len(toff, k) - 1) continue;
                if (best[k] < 0) touched[nt++] = k;
                best[k] = L;                   /* L grows, so the last write is the max */
            }
        }
        qsort(touched, (size_t)nt, sizeof(int64_t), cmp_i64);
        for (int64_t t = 0; t < nt; ++t) {
            int64_t k = touched[t];
            if (ne < cap && ej && ek && eL) {
                ej[ne] = (int32_t)j; ek[ne] = (int32_t)k; eL[ne] = (int32_t)best[k];
            }
            ++ne;
            best[k] = -1;
        }
    }
    free(ord); free(best); free(touched);
    return ne;
}

/* Containment: fragment k is contained when it occurs inside another fragment
 * j != k.  Two identical fragments contain each other; the one with the larger
 * index is the one marked. */
int oracle_contained(const uint8_t *T, const int64_t *toff, int64_t nr, uint8_t *contained)
{
    if (!reads_ok(T, toff, nr) || !contained) return -1;
    for (int64_t k = 0; k < nr; ++k) {
        int64_t lk = read_len(toff, k);
        const uint8_t *rk = T + toff[k];
        contained[k] = 0;
        for (int64_t j = 0; j < nr && !contained[k]; ++j) {
            if (j == k) continue;
            int64_t lj = read_len(toff, j);
            const uint8_t *rj = T + toff[j];
            if (lj < lk) continue;
            if (lj == lk) {
                if (j < k && memcmp(rj, rk, (size_t)lk) == 0) contained[k] = 1;
                continue;
            }
            for (int64_t p = 0; p + lk <= lj; ++p)
                if (memcmp(rj + p, rk, (size_t)lk) == 0) { contained[k] = 1; break; }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Greedy layout.  Edges between non-contained fragments are taken in order    */
/* of (L descending, j ascending, k ascending); (j, k) is accepted when j has  */
/* no successor yet, k no predecessor yet, and j, k lie on different chains    */
/* (union-find).  Each chain head -- a non-contained fragment without a        */
/* predecessor, in ascending index -- starts a contig spelled as the head      */
/* followed by each successor minus its first L symbols.                       */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t j, k, L; } edge_t;

static int edge_cmp(const void *pa, const void *pb)
{
    const edge_t *a = (const edge_t *)pa, *b = (const edge_t *)pb;
    if (a->L != b->L) return a->L > b->L ? -1 : 1;
    if (a->j != b->j) return a->j < b->j ? -1 : 1;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    return 0;
}

static int64_t uf_find(int64_t *parent, int64_t x)
{
    while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
    return x;
}

/* Writes the contigs one after another into out[0..cap) and their offsets into
 * contig_off[0..n_contigs] (contig c is out[contig_off[c] .. contig_off[c+1])).
 * Returns 0, or -2 when out or contig_off is too small, with the sizes needed
 * in *needed_bytes and *n_contigs. */
int oracle_layout(const uint8_t *T, const int64_t *toff, int64_t nr,
                  const int32_t *ej, const int32_t *ek, const int32_t *eL, int64_t ne,
                  const uint8_t *contained, uint8_t *out, int64_t cap,
                  int64_t *contig_off, int64_t off_cap, int64_t *n_contigs, int64_t *needed_bytes)
{
    if (!reads_ok(T, toff, nr) || !contained || !n_contigs || !needed_bytes || ne < 0) return -1;
    if (ne > 0 && (!ej || !ek || !eL)) return -1;
    size_t nalloc = (size_t)(nr ? nr : 1);
    edge_t *E = (edge_t *)malloc((size_t)(ne ? ne : 1) * sizeof(edge_t));
    int64_t *succ = (int64_t *)malloc(nalloc * sizeof(int64_t));
    int64_t *succL = (int64_t *)malloc(nalloc * sizeof(int64_t));
    int64_t *pred = (int64_t *)malloc(nalloc * sizeof(int64_t));
    int64_t *parent = (int64_t *)malloc(nalloc * sizeof(int64_t));
    if (!E || !succ || !succL || !pred || !parent) {
        free(E); free(succ); free(succL); free(pred); free(parent); return -3;
    }
    int64_t m = 0;
    for (int64_t e = 0; e < ne; ++e) {
        if (ej[e] < 0 || ej[e] >= nr || ek[e] < 0 || ek[e] >= nr) {
            free(E); free(succ); free(succL); free(pred); free(parent); return -1;
        }
        if (contained[ej[e]] || contained[ek[e]]) continue;
        E[m].j = ej[e]; E[m].k = ek[e]; E[m].L = eL[e]; ++m;
    }
    qsort(E, (size_t)m, sizeof(edge_t), edge_cmp);
    for (int64_t r = 0; r < nr; ++r) { succ[r] = -1; pred[r] = -1; succL[r] = 0; parent[r] = r; }
    for (int64_t e = 0; e < m; ++e) {
        int64_t j = E[e].j, k = E[e].k;
        if (succ[j] != -1 || pred[k] != -1) continue;
        int64_t a = uf_find(parent, j), b = uf_find(parent, k);
        if (a == b) continue;
        succ[j] = k; succL[j] = E[e].L; pred[k] = j; parent[a] = b;
    }
    int64_t nc = 0, nb = 0;
    for (int64_t r = 0; r < nr; ++r) {
        if (contained[r] || pred[r] != -1) continue;
        if (nc < off_cap && contig_off) contig_off[nc] = nb;
        int64_t cur = r, skip = 0;
        for (;;) {
            int64_t len = read_len(toff, cur) - skip;
            for (int64_t i = 0; i < len; ++i) {
                if (nb + i < cap && out) out[nb + i] = T[toff[cur] + skip + i];
            }
            nb += len;
            if (succ[cur] == -1) break;
            skip = succL[cur];
            cur = succ[cur];
        }
        ++nc;
    }
    if (nc < off_cap && contig_off) contig_off[nc] = nb;
    *n_contigs = nc;
    *needed_bytes = nb;
    free(E); free(succ); free(succL); free(pred); free(parent);
    if (nb > cap || nc + 1 > off_cap) return -2;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. III, Figs. 2 and 5-8: reconstruction of a sequence cut by two          */
/* shotguns from "fir" relations, with back-tracking.                          */
/*                                                                            */
/* The fragments are the pieces of two cuttings of one sequence S, shuffled   */
/* (Fig. 2: m + n fragments), every break position different (Fig. 4).  Both */
/* cuttings start at the beginning of S, so the first piece of one is a      */
/* prefix of the first piece of the other: a "fir" pair.  Cutting the shorter */
/* from the longer leaves a remainder X (Fig. 6), and the next piece of the   */
/* shorter one's cutting starts where X starts: either it is a prefix of X    */
/* (cut it off X and continue with the rest of X) or X is a prefix of it      */
/* (continue with the part of it past X).  When a choice leads to a state     */
/* with no fir fragment, or to a result that leaves fragments unselected,    */
/* the search backs up and takes the next choice (Figs. 7-8).                */
/*                                                                            */
/* Readings (the paper gives no listing):                                     */
/*  - start pairs (i, k): d_i a proper prefix of d_k, tried for k ascending,   */
/*    then i ascending; the remainder is d_k past |d_i|;                      */
/*  - with remainder X (length l), the unused fragments c are tried in        */
/*    ascending index: |c| < l and c a prefix of X -> remainder X past |c|;   */
/*    |c| > l and X a prefix of c -> remainder c past l; |c| == l and c == X  */
/*    only as the very last fragment (both cuttings end together: done);     */
/*  - every placed fragment starts where its remainder starts in the result  */
/*    RS (the start pair at 0), and RS ends where the last fragment ends;    */
/*  - a step is one placed fragment (the start pair counts as one); after    */
/*    max_steps steps the search gives up.                                    */
/* Writes frag_start[r] (offset of fragment r in RS, -1 when not solved),     */
/* *status (0 solved, 1 no reconstruction exists, 2 gave up) and *rs_len.    */
/* Returns the number of steps taken, or < 0 on a bad argument.              */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t k, o, c; } fir_frame_t;   /* remainder (k, o); c: fragment placed from it */

/* 1 if the first la symbols of a equal those of b (la <= available length of b). */
static int same_prefix(const uint8_t *a, const uint8_t *b, int64_t la)
{
    return memcmp(a, b, (size_t)la) == 0;
}

int64_t oracle_fir_reconstruct(const uint8_t *T, const int64_t *toff, int64_t nr, int64_t max_steps,
                               int64_t *frag_start, int32_t *status, int64_t *rs_len)
{
    if (!reads_ok(T, toff, nr) || !frag_start || !status || !rs_len || max_steps < 1) return -1;
    uint8_t *used = (uint8_t *)calloc((size_t)(nr ? nr : 1), 1);
    fir_frame_t *F = (fir_frame_t *)malloc((size_t)(nr ? nr : 1) * sizeof(fir_frame_t));
    if (!used || !F) { free(used); free(F); return -3; }
    for (int64_t r = 0; r < nr; ++r) frag_start[r] = -1;
    *status = 1;
    *rs_len = 0;
    int64_t steps = 0;
    int done = 0;
    for (int64_t k = 0; k < nr && !done && *status != 2; ++k) {
        const int64_t lk = read_len(toff, k);
        for (int64_t i = 0; i < nr && !done; ++i) {
            const int64_t li = read_len(toff, i);
            if (i == k || li >= lk || !same_prefix(T + toff[i], T + toff[k], li)) continue;
            if (++steps > max_steps) { *status = 2; break; }
            used[i] = used[k] = 1;
            frag_start[i] = frag_start[k] = 0;
            int64_t top = 0;
            F[0].k = k; F[0].o = li; F[0].c = -1;
            while (top >= 0 && !done) {
                fir_frame_t *f = &F[top];
                int64_t from = 0;
                if (f->c >= 0) {               /* back from the child: undo its fragment */
                    used[f->c] = 0;
                    frag_start[f->c] = -1;
                    from = f->c + 1;
                    f->c = -1;
                }
                const int64_t l = read_len(toff, f->k) - f->o;     /* remainder length */
                const uint8_t *X = T + toff[f->k] + f->o;
                const int64_t pos = frag_start[f->k] + f->o;
                const int64_t nused = 2 + top;
                int64_t c = from;
                int64_t nk = -1, no = 0;
                for (; c < nr; ++c) {
                    if (used[c]) continue;
                    const int64_t lc = read_len(toff, c);
                    const uint8_t *C = T + toff[c];
                    if (lc < l && same_prefix(C, X, lc)) { nk = f->k; no = f->o + lc; break; }
                    if (lc > l && same_prefix(X, C, l)) { nk = c; no = l; break; }
                    if (lc == l && nused + 1 == nr && same_prefix(C, X, l)) { nk = -2; break; }
                }
                if (c >= nr) { --top; continue; }   /* no fir fragment: back-track */
                if (++steps > max_steps) { *status = 2; break; }
                used[c] = 1;
                frag_start[c] = pos;
                f->c = c;
                if (nk == -2) {                    /* both cuttings end here */
                    done = 1;
                    *status = 0;
                    *rs_len = pos + l;
                    break;
                }
                ++top;
                F[top].k = nk; F[top].o = no; F[top].c = -1;
            }
            if (!done) {
                for (int64_t r = 0; r < nr; ++r) { used[r] = 0; frag_start[r] = -1; }
            }
            if (*status == 2) break;
        }
    }
    if (*status != 0)
        for (int64_t r = 0; r < nr; ++r) frag_start[r] = -1;
    free(used);
    free(F);
    return steps;
}

/* ------------------------------------------------------------------------ */
/* Sec. III DEFINITION: fragments may come from either strand and carry      */
/* errors -- every fragment A must lie within an error rate mu of a piece of */
/* the result, read directly or as its reverse complement.  The overlap      */
/* relation under that definition, as this repository reads it:             */
/*  - errors are substitutions: the distance is the Hamming distance;        */
/*  - mu is the rational mu_num / mu_den; an overlap of length L may have at */
/*    most floor(L * mu_num / mu_den) mismatches;                            */
/*  - with rc != 0 the fragments are oriented: oriented fragment 2r is        */
/*    fragment r as given and 2r + 1 its reverse complement (A<->T, C<->G,   */
/*    read backwards); otherwise oriented fragment r is fragment r.          */
/* Edge set: every ordered pair (a, b) of oriented fragments of different    */
/* fragments with the largest L, lmin <= L <= min(|a|, |b|) - 1, whose last  */
/* L symbols of a and first L symbols of b differ in at most the allowed     */
/* number of places; written in (a, b) order with the mismatch count.        */
/* Returns the number of edges (only the first cap written), < 0 on error.   */
/* ------------------------------------------------------------------------ */
static uint8_t complement(uint8_t c)
{
    switch (c) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    default: return 'A';
    }
}

int64_t oracle_overlaps_approx(const uint8_t *T, const int64_t *toff, int64_t nr, int32_t lmin,
                               int32_t mu_num, int32_t mu_den, int rc, int32_t *ea, int32_t *eb,
                               int32_t *eL, int32_t *emm, int64_t cap)
{
    if (!reads_ok(T, toff, nr) || lmin < 1 || mu_num < 0 || mu_den < 1 || cap < 0) return -1;
    const int64_t m = rc ? 2 * nr : nr;
    /* oriented fragment strings, one after another */
    int64_t *off = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    uint8_t *S = (uint8_t *)malloc((size_t)(2 * toff[nr] + 1));
    if (!off || !S) { free(off); free(S); return -3; }
    int64_t w = 0;
    for (int64_t a = 0; a < m; ++a) {
        const int64_t r = rc ? a / 2 : a;
        const int64_t len = read_len(toff, r);
        off[a] = w;
        if (!rc || a % 2 == 0) {
            memcpy(S + w, T + toff[r], (size_t)len);
        } else {
            for (int64_t i = 0; i < len; ++i) S[w + i] = complement(T[toff[r] + len - 1 - i]);
        }
        w += len;
    }
    off[m] = w;
    int64_t ne = 0;
    for (int64_t a = 0; a < m; ++a) {
        const int64_t la = off[a + 1] - off[a];
        for (int64_t b = 0; b < m; ++b) {
            if ((rc ? a / 2 : a) == (rc ? b / 2 : b)) continue;   /* same fragment */
            const int64_t lb = off[b + 1] - off[b];
            const int64_t top = (la < lb ? la : lb) - 1;
            for (int64_t L = top; L >= lmin; --L) {
                const int64_t allow = (L * (int64_t)mu_num) / mu_den;
                const uint8_t *x = S + off[a] + la - L, *y = S + off[b];
                int64_t mm = 0;
                for (int64_t i = 0; i < L && mm <= allow; ++i) mm += x[i] != y[i];
                if (mm <= allow) {
                    if (ne < cap) { ea[ne] = (int32_t)a; eb[ne] = (int32_t)b; eL[ne] = (int32_t)L; emm[ne] = (int32_t)mm; }
                    ++ne;
                    break;
                }
            }
        }
    }
    free(off);
    free(S);
    return ne;
}
