// serve.cu -- a continuous-batching assembly server on one GPU.
//
// Jobs (one fragment text each, host memory) are queued in arrival order.  The
// server runs `slots` workers, each with its own context (workspace) and CUDA
// stream.  A free worker admits, from the head of the queue, the longest run of
// jobs with the same min_overlap whose estimated device memory fits in what the
// HBM budget has left after the batches already in flight, and runs them as one
// batched assembly (assemble_batched).  So jobs that arrive while other batches
// are on the GPU are admitted as soon as a slot and memory free up, and the
// batches of different slots overlap on the device.  Results (contigs, offsets,
// timestamps) wait in a completion list until polled.  Each result is the same
// as assembling that job alone: no overlap or chain crosses two jobs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace dnasa {
int assemble_impl(dnasa_ctx *ctx, const uint8_t *text, int64_t N, const int64_t *inst_toff_host,
                  int32_t n_inst, int32_t min_overlap, uint8_t *contigs, int64_t cap,
                  int64_t *contig_off, int64_t off_cap, int64_t *inst_contig_off, int64_t *n_contigs,
                  int64_t *needed, const dnasa_opts *opts, cudaStream_t s);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
    uint64_t id;
    std::vector<uint8_t> text;
    int32_t min_overlap;
    double t_submit;
    size_t est;
};

struct Done {
    uint64_t id;
    int32_t status;
    std::vector<uint8_t> contigs;
    std::vector<int64_t> offs;
    double t_submit, t_start, t_done;
};

// Device bytes one job of N symbols and n_reads fragments may hold at its peak
// while it is assembled: the context workspace of the suffix-array build (the
// largest step; the context grows it with a 1/8 margin and never shrinks it),
// plus the buffers assemble keeps alongside (packed text, fragment offsets,
// SA, LCP, inverse SA, fragment ids, containment flags, the edge list), plus
// the slot's own text, contig and offset buffers, plus a fixed allowance for
// the context's small buffers.
size_t job_bytes(int64_t N, int64_t n_reads) {
    const size_t n = (size_t)N, r = (size_t)std::max<int64_t>(n_reads, 1);
    const size_t ws = dnasa::sa_workspace_bytes(N, 0 /* default tile */) + 4096;
    const size_t ws_held = ws + ws / 8 + (1u << 20);
    const size_t assemble_bufs = (n / 32 + 3) * 8          // packed text
                                 + (n / 2 + 2) * 8         // fragment offsets (capacity)
                                 + 4 * n * 4               // SA, LCP, inverse SA, fragment ids
                                 + r                       // containment flags
                                 + std::max<size_t>(8 * r, 1024) * sizeof(dnasa_edge);
    const size_t slot_bufs = 2 * n + (n / 2 + 2) * 8;      // text, contigs, contig offsets
    return ws_held + assemble_bufs + slot_bufs + (32u << 20);
}

struct Slot {
    size_t held() const {   // device bytes this slot keeps between batches
        return (ctx ? ctx->ws_size + ctx->lb_words * 8 : 0) + text_cap + contig_cap +
               off_cap * 8 + ioff_cap * 8;
    }
    dnasa_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    // device and pinned host buffers, grown on demand
    uint8_t *d_text = nullptr, *d_contigs = nullptr;
    int64_t *d_off = nullptr, *d_ioff = nullptr;
    size_t text_cap = 0, off_cap = 0, ioff_cap = 0, contig_cap = 0;
    uint8_t *h_text = nullptr, *h_contigs = nullptr;
    int64_t *h_off = nullptr, *h_ioff = nullptr;
    size_t h_text_cap = 0, h_off_cap = 0, h_ioff_cap = 0, h_contig_cap = 0;
};

}  // namespace

struct dnasa_server {
    int device = 0;
    size_t budget = 0;
    int max_batch = 64;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::deque<Done> done;
    std::vector<Done> polled;       // results handed out by the last poll (kept alive)
    size_t reserved = 0;
    int in_flight = 0;
    bool stop = false;
    std::vector<Slot> slots;
    std::vector<std::thread> workers;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
};

namespace {

template <typename T>
bool grow_dev(T **p, size_t *cap, size_t n) {
    if (*cap >= n) return true;
    if (*p) cudaFree(*p);
    *p = nullptr;
    size_t want = std::max(n, *cap * 2);
    if (cudaMalloc(p, want * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *cap = 0;
        *p = nullptr;
        return false;
    }
    *cap = want;
    return true;
}

template <typename T>
bool grow_host(T **p, size_t *cap, size_t n) {
    if (*cap >= n) return true;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    size_t want = std::max(n, *cap * 2);
    if (cudaMallocHost(p, want * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *cap = 0;
        *p = nullptr;
        return false;
    }
    *cap = want;
    return true;
}

// Runs one batch on a slot; fills one Done per job.
void run_batch(dnasa_server *srv, Slot &sl, std::vector<Pending> &batch, std::vector<Done> &out) {
    const double t_start = srv->now_ms();
    const int n = (int)batch.size();
    std::vector<int64_t> inst_off(n + 1, 0);
    for (int i = 0; i < n; ++i) inst_off[i + 1] = inst_off[i] + (int64_t)batch[i].text.size();
    const int64_t N = inst_off[n];
    int rc = DNASA_OK;
    int64_t nc = 0, nb = 0;
    const size_t offs = (size_t)N / 2 + 2;
    if (!grow_host(&sl.h_text, &sl.h_text_cap, (size_t)N) ||
        !grow_dev(&sl.d_text, &sl.text_cap, (size_t)N) ||
        !grow_dev(&sl.d_off, &sl.off_cap, offs) || !grow_dev(&sl.d_ioff, &sl.ioff_cap, (size_t)n + 1) ||
        !grow_host(&sl.h_off, &sl.h_off_cap, offs) || !grow_host(&sl.h_ioff, &sl.h_ioff_cap, (size_t)n + 1)) {
        rc = DNASA_OOM;
    }
    // contigs never exceed the text size
    if (rc == DNASA_OK && (!grow_dev(&sl.d_contigs, &sl.contig_cap, (size_t)N) ||
                           !grow_host(&sl.h_contigs, &sl.h_contig_cap, (size_t)N)))
        rc = DNASA_OOM;
    if (rc == DNASA_OK) {
        for (int i = 0; i < n; ++i)
            memcpy(sl.h_text + inst_off[i], batch[i].text.data(), batch[i].text.size());
        if (cudaMemcpyAsync(sl.d_text, sl.h_text, (size_t)N, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            rc = DNASA_CUDA_ERROR;
    }
    if (rc == DNASA_OK)
        rc = dnasa::assemble_impl(sl.ctx, sl.d_text, N, inst_off.data(), n, batch[0].min_overlap,
                                  sl.d_contigs, (int64_t)sl.contig_cap, sl.d_off, (int64_t)offs,
                                  n > 1 ? sl.d_ioff : nullptr, &nc, &nb, nullptr, sl.stream);
    if (rc == DNASA_OK) {
        cudaMemcpyAsync(sl.h_contigs, sl.d_contigs, (size_t)nb, cudaMemcpyDeviceToHost, sl.stream);
        cudaMemcpyAsync(sl.h_off, sl.d_off, (size_t)(nc + 1) * 8, cudaMemcpyDeviceToHost, sl.stream);
        if (n > 1)
            cudaMemcpyAsync(sl.h_ioff, sl.d_ioff, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost, sl.stream);
        if (cudaStreamSynchronize(sl.stream) != cudaSuccess) rc = DNASA_CUDA_ERROR;
        if (n == 1) {
            sl.h_ioff[0] = 0;
            sl.h_ioff[1] = nc;
        }
    }
    if (rc != DNASA_OK && n > 1) {
        // the batch failed as a whole (e.g. out of memory): every job again on its
        // own, so that one job's failure is reported for that job alone
        std::vector<Done> all, one;
        for (int i = 0; i < n; ++i) {
            std::vector<Pending> single(1, batch[i]);
            run_batch(srv, sl, single, one);
            all.push_back(std::move(one[0]));
        }
        out = std::move(all);
        return;
    }
    const double t_done = srv->now_ms();
    out.clear();
    for (int i = 0; i < n; ++i) {
        Done d;
        d.id = batch[i].id;
        d.status = rc;
        d.t_submit = batch[i].t_submit;
        d.t_start = t_start;
        d.t_done = t_done;
        if (rc == DNASA_OK) {
            int64_t c0 = sl.h_ioff[i], c1 = sl.h_ioff[i + 1];
            int64_t b0 = sl.h_off[c0], b1 = sl.h_off[c1];
            d.contigs.assign(sl.h_contigs + b0, sl.h_contigs + b1);
            d.offs.resize((size_t)(c1 - c0 + 1));
            for (int64_t c = c0; c <= c1; ++c) d.offs[(size_t)(c - c0)] = sl.h_off[c] - b0;
        }
        out.push_back(std::move(d));
    }
}

// What admission may fill: the server's budget, but never more than the device
// memory that is free right now plus what the batches in flight have reserved
// (their memory is counted in `reserved`, allocated or not) plus what this slot
// already holds (its buffers are reused).  Called with srv->mu held.
size_t effective_budget(dnasa_server *srv, const Slot &sl) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return srv->budget;
    }
    const size_t live = (size_t)((double)(free_b + sl.held()) * 0.95) + srv->reserved;
    return std::min(srv->budget, live);
}

void worker(dnasa_server *srv, int k) {
    cudaSetDevice(srv->device);
    Slot &sl = srv->slots[k];
    std::vector<Pending> batch;
    std::vector<Done> out;
    for (;;) {
        size_t est = 0, budget = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->stop && srv->queue.empty()) return;
                if (!srv->queue.empty()) {
                    // admit the FIFO head (alone if it exceeds the budget and nothing else runs)
                    budget = effective_budget(srv, sl);
                    const Pending &h = srv->queue.front();
                    bool fits = srv->reserved + h.est <= budget;
                    if (fits || srv->in_flight == 0) break;
                }
                srv->cv_work.wait_for(lk, std::chrono::milliseconds(50));   // free HBM may change
            }
            batch.clear();
            const int32_t lmin = srv->queue.front().min_overlap;
            while (!srv->queue.empty() && (int)batch.size() < srv->max_batch) {
                Pending &h = srv->queue.front();
                if (h.min_overlap != lmin) break;
                if (!batch.empty() && srv->reserved + est + h.est > budget) break;
                est += h.est;
                batch.push_back(std::move(h));
                srv->queue.pop_front();
            }
            srv->reserved += est;
            srv->in_flight += 1;
        }
        run_batch(srv, sl, batch, out);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->reserved -= est;
            srv->in_flight -= 1;
            for (auto &d : out) srv->done.push_back(std::move(d));
        }
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
}

void free_slot(Slot &sl) {
    if (sl.d_text) cudaFree(sl.d_text);
    if (sl.d_contigs) cudaFree(sl.d_contigs);
    if (sl.d_off) cudaFree(sl.d_off);
    if (sl.d_ioff) cudaFree(sl.d_ioff);
    if (sl.h_text) cudaFreeHost(sl.h_text);
    if (sl.h_contigs) cudaFreeHost(sl.h_contigs);
    if (sl.h_off) cudaFreeHost(sl.h_off);
    if (sl.h_ioff) cudaFreeHost(sl.h_ioff);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctx) dnasa_destroy(sl.ctx);
    sl = Slot();
}

}  // namespace

extern "C" {

int dnasa_server_create(int device, size_t hbm_budget, int32_t slots, int32_t max_batch,
                        dnasa_server **out) {
    if (!out || slots < 1 || slots > 16 || max_batch < 1) return DNASA_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return DNASA_INVALID_ARG;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return DNASA_CUDA_ERROR;
    dnasa_server *srv = new dnasa_server();
    srv->device = device;
    srv->budget = std::min(hbm_budget ? hbm_budget : free_b, (size_t)(free_b * 0.9));
    srv->max_batch = max_batch;
    srv->t0 = Clock::now();
    srv->slots.resize((size_t)slots);
    for (auto &sl : srv->slots) {
        if (dnasa_create(device, 0, &sl.ctx) != DNASA_OK ||
            cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (auto &x : srv->slots) free_slot(x);
            delete srv;
            return DNASA_OOM;
        }
    }
    for (int k = 0; k < slots; ++k) srv->workers.emplace_back(worker, srv, k);
    *out = srv;
    return DNASA_OK;
}

int dnasa_server_submit(dnasa_server *srv, const dnasa_job *job, uint64_t id) {
    if (!srv || !job || !job->text || job->N <= 0 || job->min_overlap < 1) return DNASA_INVALID_ARG;
    // a malformed text is refused here, so that it can never fail a batch it shares
    if (job->text[job->N - 1] != '$' || job->text[0] == '$') return DNASA_BAD_ALPHABET;
    for (int64_t i = 0; i < job->N; ++i) {
        const uint8_t c = job->text[i];
        if (c == '$') {
            if (i > 0 && job->text[i - 1] == '$') return DNASA_BAD_ALPHABET;   // empty fragment
        } else if (c != 'A' && c != 'C' && c != 'G' && c != 'T') {
            return DNASA_BAD_ALPHABET;
        }
    }
    Pending p;
    p.id = id;
    p.text.assign(job->text, job->text + job->N);
    p.min_overlap = job->min_overlap;
    int64_t n_reads = 0;
    for (int64_t i = 0; i < job->N; ++i) n_reads += job->text[i] == '$';
    p.est = job_bytes(job->N, n_reads);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) return DNASA_INVALID_ARG;
        p.t_submit = srv->now_ms();
        srv->queue.push_back(std::move(p));
    }
    srv->cv_work.notify_one();
    return DNASA_OK;
}

int dnasa_server_poll(dnasa_server *srv, dnasa_result *out, int32_t max_results, int32_t wait_ms,
                      int32_t *n_out) {
    if (!srv || !n_out || max_results < 0 || (max_results > 0 && !out)) return DNASA_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->done.empty() && wait_ms > 0)
        srv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !srv->done.empty(); });
    srv->polled.clear();
    int n = 0;
    while (n < max_results && !srv->done.empty()) {
        srv->polled.push_back(std::move(srv->done.front()));
        srv->done.pop_front();
        ++n;
    }
    for (int i = 0; i < n; ++i) {
        Done &d = srv->polled[(size_t)i];
        dnasa_result r;
        r.id = d.id;
        r.status = d.status;
        r.reserved = 0;
        r.n_contigs = d.offs.empty() ? 0 : (int64_t)d.offs.size() - 1;
        r.bytes = (int64_t)d.contigs.size();
        r.contigs = d.contigs.data();
        r.contig_off = d.offs.data();
        r.t_submit_ms = d.t_submit;
        r.t_start_ms = d.t_start;
        r.t_done_ms = d.t_done;
        out[i] = r;
    }
    *n_out = n;
    return DNASA_OK;
}

int64_t dnasa_server_job_bytes(int64_t N, int64_t n_reads) {
    if (N <= 0 || n_reads < 1 || n_reads > N) return -1;
    return (int64_t)job_bytes(N, n_reads);
}

int dnasa_server_pending(dnasa_server *srv) {
    if (!srv) return DNASA_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    return (int)srv->queue.size() + srv->in_flight;
}

void dnasa_server_destroy(dnasa_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->workers) t.join();
    cudaSetDevice(srv->device);
    for (auto &sl : srv->slots) free_slot(sl);
    delete srv;
}

}  // extern "C"
