// rklt_serve.cpp -- native request loop for compress + decompress + PSNR requests
// (Sec. 4.1 per image: forward, zonal retention, inverse, PSNR), replaying a trace
// of timed arrivals in real time on the calling thread.
//
// Continuous batching: a waiting request is admitted as soon as its device buffers
// (input, 8-bit reconstruction, compact coefficients) fit in a first-fit arena over
// one preallocated device buffer of `budget` bytes; every request admitted in one
// pass of the loop goes out in one rklt_fused_items launch on the next of several
// streams, so batches admitted while earlier ones are on the GPU overlap with them.
// Inputs arrive in the caller's pageable memory: each is copied into a pinned
// mirror of its arena slot and moved to the device as whole padded rows (one
// contiguous transfer); reconstruction, coefficients, SSE and PSNR come back into
// pinned memory, and a request completes when its batch's event has fired.
//
// Plain: one rklt_fused call per request, strictly one at a time (copy in, launch,
// copy out, synchronise), on buffers sized for the largest request of the trace.
//
// Both record, per request, the completion time on the same clock as the arrivals.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "rklt_internal.h"

namespace rklt {
namespace {

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// First-fit allocator over [0, size) (offsets in bytes, 256-byte granules).
class Arena {
  public:
    explicit Arena(size_t size) : free_{{0, size}} {}
    bool alloc(size_t n, size_t &off) {
        for (size_t k = 0; k < free_.size(); k++) {
            if (free_[k].second >= n) {
                off = free_[k].first;
                if (free_[k].second == n) free_.erase(free_.begin() + long(k));
                else free_[k] = {free_[k].first + n, free_[k].second - n};
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, size_t(0)));
        it = free_.insert(it, {off, n});
        size_t k = size_t(it - free_.begin());
        if (k + 1 < free_.size() && free_[k].first + free_[k].second == free_[k + 1].first) {
            free_[k].second += free_[k + 1].second;
            free_.erase(free_.begin() + long(k) + 1);
        }
        if (k > 0 && free_[k - 1].first + free_[k - 1].second == free_[k].first) {
            free_[k - 1].second += free_[k].second;
            free_.erase(free_.begin() + long(k));
        }
    }

  private:
    std::vector<std::pair<size_t, size_t>> free_;  // sorted (offset, length)
};

struct Layout {  // a request's buffers inside its arena slot
    size_t in, rec, coef, total;
    int64_t ld;
};

Layout layout_of(const rklt_request &q, int N) {
    Layout L{};
    L.ld = int64_t(align_up(size_t(q.W), 16));
    const size_t bi = size_t(q.H) * size_t(L.ld);
    const size_t bc = size_t(q.H / N) * size_t(q.W / N) * size_t(q.r) * sizeof(float);
    L.in = 0;
    L.rec = align_up(bi);
    L.coef = L.rec + align_up(bi);
    L.total = L.coef + align_up(bc);
    return L;
}

// Host staging copies of one admitted batch, spread over worker threads: the loop
// thread publishes the batch's row chunks and copies alongside the workers, then
// waits until every worker has finished with them.  Under load one core's memcpy
// bandwidth would otherwise bound how fast admitted images reach pinned memory.
class CopyPool {
  public:
    struct Chunk {
        uint8_t *dst;          // pinned, pitch ld
        const uint8_t *src;    // caller's image rows, pitch W
        int64_t ld;
        int W, rows;
    };
    explicit CopyPool(int workers) : n_(workers) {
        for (int k = 0; k < workers; k++) th_.emplace_back([this] { loop(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
            ++gen_;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    void run(const Chunk *c, size_t n) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            jobs_ = c;
            njobs_ = n;
            next_.store(0, std::memory_order_relaxed);
            acked_ = 0;
            ++gen_;
        }
        cv_.notify_all();
        drain(c, n);
        std::unique_lock<std::mutex> lk(mu_);
        done_cv_.wait(lk, [&] { return acked_ == n_; });
    }

  private:
    static void copy(const Chunk &k) {
        if (k.ld == k.W) {
            std::memcpy(k.dst, k.src, size_t(k.rows) * size_t(k.W));
            return;
        }
        for (int y = 0; y < k.rows; y++)
            std::memcpy(k.dst + size_t(y) * size_t(k.ld), k.src + size_t(y) * size_t(k.W), size_t(k.W));
    }
    void drain(const Chunk *c, size_t n) {
        for (size_t i = next_.fetch_add(1, std::memory_order_relaxed); i < n;
             i = next_.fetch_add(1, std::memory_order_relaxed))
            copy(c[i]);
    }
    void loop() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_.wait(lk, [&] { return gen_ != seen; });
            seen = gen_;
            if (stop_) return;
            const Chunk *c = jobs_;
            const size_t n = njobs_;
            lk.unlock();
            drain(c, n);
            lk.lock();
            if (++acked_ == n_) done_cv_.notify_all();
        }
    }
    const int n_;
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    const Chunk *jobs_ = nullptr;
    size_t njobs_ = 0;
    std::atomic<size_t> next_{0};
    int acked_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

// Batches whose images total at least this many bytes are staged by the pool; smaller
// ones by the loop thread alone (waking the workers costs more than it saves there).
constexpr size_t kPoolBytes = size_t(2) << 20;
constexpr int kChunkBytes = 1 << 20;   // rows per chunk: about 1 MB of pixels
constexpr int kCopyWorkers = 3;

}  // namespace
}  // namespace rklt

struct rklt_server {
    std::vector<const rklt_plan *> plans;
    int N = 0;
    size_t budget = 0;
    int max_batch = 0;
    uint8_t *d_arena = nullptr;
    uint8_t *h_arena = nullptr;         // pinned mirror of the device arena
    std::vector<cudaStream_t> streams;
    int slots = 0;                      // batches in flight at most (two per stream)
    double *d_sse = nullptr;            // [slots][max_batch]
    float *d_psnr = nullptr;
    double *h_sse = nullptr;            // pinned
    float *h_psnr = nullptr;
    std::vector<cudaEvent_t> events;    // one per slot
    std::unique_ptr<rklt::CopyPool> pool;   // staging copies of large batches
};

using namespace rklt;

namespace {

void server_free(rklt_server *s) {
    if (!s) return;
    for (auto st : s->streams) cudaStreamSynchronize(st);
    for (auto e : s->events) cudaEventDestroy(e);
    for (auto st : s->streams) cudaStreamDestroy(st);
    cudaFree(s->d_arena);
    cudaFree(s->d_sse);
    cudaFree(s->d_psnr);
    cudaFreeHost(s->h_arena);
    cudaFreeHost(s->h_sse);
    cudaFreeHost(s->h_psnr);
    delete s;
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Sleep until about `until` seconds after t0 (wakes ~0.2 ms early, then spins).
void wait_until(std::chrono::steady_clock::time_point t0, double until) {
    double gap = until - seconds_since(t0);
    if (gap > 3e-4) std::this_thread::sleep_for(std::chrono::duration<double>(gap - 2e-4));
    while (seconds_since(t0) < until) {
    }
}

rklt_status check_requests(const rklt_server *s, const rklt_request *q, int n) {
    if (n < 0 || (n > 0 && !q)) return fail(RKLT_ERR_ARG, "bad request array");
    for (int i = 0; i < n; i++) {
        if (q[i].plan < 0 || q[i].plan >= int(s->plans.size())) return fail(RKLT_ERR_ARG, "request plan out of range");
        if (q[i].r < 0 || q[i].r > s->N * s->N) return fail(RKLT_ERR_ARG, "request r must lie in [0, N*N]");
        if (q[i].H <= 0 || q[i].W <= 0 || q[i].H % s->N || q[i].W % s->N)
            return fail(RKLT_ERR_SHAPE, "request H and W must be positive multiples of N");
        if (!q[i].h_img) return fail(RKLT_ERR_ARG, "request image is NULL");
        if (i > 0 && q[i].arrival_s < q[i - 1].arrival_s) return fail(RKLT_ERR_ARG, "arrivals must be sorted");
    }
    return RKLT_OK;
}

// Copies an H x W image (pitch W) into a pinned buffer of pitch ld.
void copy_rows(uint8_t *dst, int64_t ld, const uint8_t *src, int H, int W) {
    if (ld == W) {
        std::memcpy(dst, src, size_t(H) * size_t(W));
        return;
    }
    for (int y = 0; y < H; y++) std::memcpy(dst + size_t(y) * size_t(ld), src + size_t(y) * size_t(W), size_t(W));
}

void unpack_rows(uint8_t *dst, const uint8_t *src, int64_t ld, int H, int W) {
    for (int y = 0; y < H; y++) std::memcpy(dst + size_t(y) * size_t(W), src + size_t(y) * size_t(ld), size_t(W));
}

struct Inflight {
    int slot;
    std::vector<int> reqs;
    std::vector<size_t> offs;
    size_t block_off, block_len;   // the batch's arena block
};

rklt_status run_continuous(rklt_server *s, const rklt_request *q, int n, uint8_t *const *h_recon,
                           float *const *h_coef, rklt_result *res, double *wall) {
    Arena arena(s->budget);
    std::vector<int> free_slots;
    for (int k = s->slots - 1; k >= 0; k--) free_slots.push_back(k);
    std::deque<int> waiting;
    std::vector<Inflight> inflight;
    std::vector<rklt_item> items;
    std::vector<CopyPool::Chunk> chunks;
    std::vector<std::pair<size_t, size_t>> runs;   // (first, last) batch positions of a contiguous run
    std::vector<size_t> order;
    std::vector<size_t> prefix;
    std::vector<Layout> lay(static_cast<size_t>(n));
    for (int i = 0; i < n; i++) lay[size_t(i)] = layout_of(q[i], s->N);
    int next_stream = 0, k = 0, completed = 0;
    const auto t0 = std::chrono::steady_clock::now();
    while (completed < n) {
        const double now = seconds_since(t0);
        while (k < n && q[k].arrival_s <= now) waiting.push_back(k++);
        // admission by budget, first come first served; a request larger than the
        // whole budget is rejected.  A batch takes one contiguous arena block (its
        // requests' slots back to back), the longest prefix of the waiting requests
        // that fits, so that its copies are one call per direction whatever the
        // arena's fragmentation.
        std::vector<int> batch;
        std::vector<size_t> offs;
        size_t block_off = 0, block_len = 0;
        while (!waiting.empty() && lay[size_t(waiting.front())].total > s->budget) {
            const int i = waiting.front();
            waiting.pop_front();
            res[i].status = RKLT_ERR_BUDGET;
            res[i].done_s = now;
            completed++;
        }
        if (!waiting.empty() && !free_slots.empty()) {
            size_t cand = 0, total = 0;
            prefix.clear();
            while (cand < waiting.size() && int(cand) < s->max_batch) {
                const size_t t = lay[size_t(waiting[cand])].total;
                if (t > s->budget) break;   // rejected when it reaches the front
                total += t;
                prefix.push_back(total);
                cand++;
            }
            while (cand > 0 && !arena.alloc(prefix[cand - 1], block_off)) cand--;
            if (cand > 0) {
                block_len = prefix[cand - 1];
                size_t off = block_off;
                for (size_t c = 0; c < cand; c++) {
                    const int i = waiting.front();
                    waiting.pop_front();
                    batch.push_back(i);
                    offs.push_back(off);
                    off += lay[size_t(i)].total;
                }
            }
        }
        if (!batch.empty()) {
            const cudaStream_t st = s->streams[size_t(next_stream)];
            next_stream = (next_stream + 1) % int(s->streams.size());
            const int slot = free_slots.back();
            free_slots.pop_back();
            items.clear();
            cudaError_t e = cudaSuccess;
            // the admitted images into their pinned slots (by the pool when large)
            size_t bytes = 0;
            for (size_t b = 0; b < batch.size(); b++) bytes += size_t(q[batch[b]].H) * size_t(q[batch[b]].W);
            if (s->pool && bytes >= kPoolBytes) {
                chunks.clear();
                for (size_t b = 0; b < batch.size(); b++) {
                    const rklt_request &r = q[batch[b]];
                    const Layout &L = lay[size_t(batch[b])];
                    const int step = std::max(1, kChunkBytes / r.W);
                    for (int y = 0; y < r.H; y += step)
                        chunks.push_back({s->h_arena + offs[b] + L.in + size_t(y) * size_t(L.ld),
                                          r.h_img + size_t(y) * size_t(r.W), L.ld, r.W, std::min(step, r.H - y)});
                }
                s->pool->run(chunks.data(), chunks.size());
            } else {
                for (size_t b = 0; b < batch.size(); b++) {
                    const rklt_request &r = q[batch[b]];
                    copy_rows(s->h_arena + offs[b] + lay[size_t(batch[b])].in, lay[size_t(batch[b])].ld, r.h_img, r.H,
                              r.W);
                }
            }
            // copies as few contiguous spans as possible: slots that touch in the arena
            // form one run, copied in one call per direction (a run holds only this
            // batch's slots).  One call per request and direction filled the stream's
            // command queue at high rates, and the host then blocked for hundreds of ms.
            runs.clear();
            order.resize(batch.size());
            for (size_t b = 0; b < batch.size(); b++) order[b] = b;
            std::sort(order.begin(), order.end(), [&](size_t a, size_t b2) { return offs[a] < offs[b2]; });
            for (size_t t = 0; t < order.size(); t++) {
                const size_t b = order[t];
                if (!runs.empty()) {
                    const size_t p = runs.back().second;
                    if (offs[p] + lay[size_t(batch[p])].total == offs[b]) {
                        runs.back().second = b;
                        continue;
                    }
                }
                runs.push_back({b, b});
            }
            for (const auto &run : runs) {
                const Layout &Lf = lay[size_t(batch[run.first])], &Ll = lay[size_t(batch[run.second])];
                const size_t from = offs[run.first] + Lf.in;
                const size_t to = offs[run.second] + Ll.in + size_t(q[batch[run.second]].H) * size_t(Ll.ld);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(s->d_arena + from, s->h_arena + from, to - from, cudaMemcpyHostToDevice, st);
            }
            for (size_t b = 0; b < batch.size(); b++) {
                const rklt_request &r = q[batch[b]];
                const Layout &L = lay[size_t(batch[b])];
                uint8_t *d = s->d_arena + offs[b];
                rklt_item it{};
                it.d_img = d + L.in;
                it.H = r.H;
                it.W = r.W;
                it.ld = L.ld;
                it.plan = r.plan;
                it.r = r.r;
                it.d_zcoef = r.r > 0 ? reinterpret_cast<float *>(d + L.coef) : nullptr;
                it.d_recon = d + L.rec;
                it.ld_recon = L.ld;
                items.push_back(it);
            }
            if (e != cudaSuccess) return cuda_fail(e, "request copy-in");
            double *dsse = s->d_sse + size_t(slot) * size_t(s->max_batch);
            float *dps = s->d_psnr + size_t(slot) * size_t(s->max_batch);
            const rklt_status ls = rklt_fused_items(items.data(), int(items.size()), s->plans.data(),
                                                    int(s->plans.size()), dsse, dps, st);
            if (ls != RKLT_OK) return ls;
            for (const auto &run : runs) {
                if (e != cudaSuccess) break;
                const Layout &Lf = lay[size_t(batch[run.first])], &Ll = lay[size_t(batch[run.second])];
                const size_t from = offs[run.first] + Lf.rec, to = offs[run.second] + Ll.total;
                e = cudaMemcpyAsync(s->h_arena + from, s->d_arena + from, to - from, cudaMemcpyDeviceToHost, st);
            }
            const size_t nb = batch.size();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->h_sse + size_t(slot) * size_t(s->max_batch), dsse, nb * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->h_psnr + size_t(slot) * size_t(s->max_batch), dps, nb * sizeof(float),
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(s->events[size_t(slot)], st);
            if (e != cudaSuccess) return cuda_fail(e, "request launch");
            const double tl = seconds_since(t0);
            for (int i : batch) res[i].admit_s = tl;
            inflight.push_back({slot, std::move(batch), std::move(offs), block_off, block_len});
        }
        // completions
        for (size_t f = 0; f < inflight.size();) {
            Inflight &it = inflight[f];
            const cudaError_t qe = cudaEventQuery(s->events[size_t(it.slot)]);
            if (qe == cudaErrorNotReady) {
                f++;
                continue;
            }
            if (qe != cudaSuccess) return cuda_fail(qe, "request completion");
            const double tdone = seconds_since(t0);
            for (size_t b = 0; b < it.reqs.size(); b++) {
                const int i = it.reqs[b];
                const Layout &L = lay[size_t(i)];
                rklt_result &o = res[i];
                o.done_s = tdone;
                o.sse = s->h_sse[size_t(it.slot) * size_t(s->max_batch) + b];
                o.psnr = s->h_psnr[size_t(it.slot) * size_t(s->max_batch) + b];
                o.status = RKLT_OK;
                if (h_recon && h_recon[i]) unpack_rows(h_recon[i], s->h_arena + it.offs[b] + L.rec, L.ld, q[i].H, q[i].W);
                if (h_coef && h_coef[i] && q[i].r > 0)
                    std::memcpy(h_coef[i], s->h_arena + it.offs[b] + L.coef,
                                size_t(q[i].H / s->N) * size_t(q[i].W / s->N) * size_t(q[i].r) * sizeof(float));
                completed++;
            }
            arena.release(it.block_off, it.block_len);
            free_slots.push_back(it.slot);
            inflight.erase(inflight.begin() + long(f));
        }
        if (waiting.empty() && inflight.empty() && k < n) wait_until(t0, q[k].arrival_s);
    }
    *wall = seconds_since(t0);
    return RKLT_OK;
}

rklt_status run_plain(rklt_server *s, const rklt_request *q, int n, uint8_t *const *h_recon, float *const *h_coef,
                      rklt_result *res, double *wall) {
    // one request's buffers at the front of the arenas, sized for the largest request
    size_t most = 0;
    for (int i = 0; i < n; i++) most = std::max(most, layout_of(q[i], s->N).total);
    if (most > s->budget) return fail(RKLT_ERR_BUDGET, "a request exceeds the device-memory budget");
    const cudaStream_t st = s->streams[0];
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < n; i++) {
        wait_until(t0, q[i].arrival_s);
        res[i].admit_s = seconds_since(t0);
        const rklt_request &r = q[i];
        const Layout L = layout_of(r, s->N);
        copy_rows(s->h_arena + L.in, L.ld, r.h_img, r.H, r.W);
        cudaError_t e = cudaMemcpyAsync(s->d_arena + L.in, s->h_arena + L.in, size_t(r.H) * size_t(L.ld),
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "request copy-in");
        float *zc = r.r > 0 ? reinterpret_cast<float *>(s->d_arena + L.coef) : nullptr;
        const rklt_status ls = rklt_fused(s->plans[size_t(r.plan)], s->d_arena + L.in, r.H, r.W, L.ld, r.r, zc,
                                          s->d_arena + L.rec, L.ld, s->d_sse, s->d_psnr, st);
        if (ls != RKLT_OK) return ls;
        e = cudaMemcpyAsync(s->h_arena + L.rec, s->d_arena + L.rec, size_t(r.H) * size_t(L.ld), cudaMemcpyDeviceToHost,
                            st);
        if (e == cudaSuccess && r.r > 0)
            e = cudaMemcpyAsync(s->h_arena + L.coef, s->d_arena + L.coef, L.total - L.coef, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_sse, s->d_sse, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_psnr, s->d_psnr, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "request");
        rklt_result &o = res[i];
        o.done_s = seconds_since(t0);
        o.sse = s->h_sse[0];
        o.psnr = s->h_psnr[0];
        o.status = RKLT_OK;
        if (h_recon && h_recon[i]) unpack_rows(h_recon[i], s->h_arena + L.rec, L.ld, r.H, r.W);
        if (h_coef && h_coef[i] && r.r > 0)
            std::memcpy(h_coef[i], s->h_arena + L.coef,
                        size_t(r.H / s->N) * size_t(r.W / s->N) * size_t(r.r) * sizeof(float));
    }
    *wall = seconds_since(t0);
    return RKLT_OK;
}

rklt_status server_warm(rklt_server *s) {
    const int N = s->N, H = 4 * N, W = 256;
    const cudaStream_t st = s->streams[0];
    if (cudaMemsetAsync(s->d_arena, 0, size_t(H) * W * 2, st) != cudaSuccess) return fail(RKLT_ERR_CUDA, "warm-up");
    uint8_t *img = s->d_arena, *rec = s->d_arena + size_t(H) * W;
    float *zc = reinterpret_cast<float *>(s->d_arena + align_up(size_t(H) * W * 2));
    for (int r = 0; r <= N * N; r++) {
        for (int p = 0; p < int(s->plans.size()); p++) {
            rklt_item it{img, H, W, W, p, r, r > 0 ? zc : nullptr, rec, W};
            rklt_status ls = rklt_fused_items(&it, 1, s->plans.data(), int(s->plans.size()), s->d_sse, s->d_psnr, st);
            if (ls == RKLT_OK)
                ls = rklt_fused(s->plans[size_t(p)], img, H, W, W, r, r > 0 ? zc : nullptr, rec, W, s->d_sse, s->d_psnr,
                                st);
            if (ls != RKLT_OK) return ls;
        }
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? RKLT_OK : cuda_fail(e, "warm-up");
}

}  // namespace

extern "C" {

rklt_status rklt_server_create(const rklt_plan *const *plans, int nplans, size_t budget_bytes, int nstreams,
                               int max_batch, rklt_server **out) {
    if (!out) return fail(RKLT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nplans < 1 || !plans) return fail(RKLT_ERR_ARG, "need at least one plan");
    if (budget_bytes < 4096 || nstreams < 1 || nstreams > 64 || max_batch < 1 || max_batch > 4096)
        return fail(RKLT_ERR_ARG, "budget, stream count or batch size out of range");
    rklt_server *s = new (std::nothrow) rklt_server;
    if (!s) return fail(RKLT_ERR_OOM, "host allocation failed");
    for (int p = 0; p < nplans; p++) {
        if (!plans[p]) {
            delete s;
            return fail(RKLT_ERR_ARG, "NULL plan");
        }
        if (p == 0) s->N = plans[p]->p.N;
        if (plans[p]->p.N != s->N || plans[p]->p.kind != 0) {
            delete s;
            return fail(RKLT_ERR_ARG, "plans must be rounded (integer) plans of one block size");
        }
        s->plans.push_back(plans[p]);
    }
    if (s->N != 4 && s->N != 8) {
        delete s;
        return fail(RKLT_ERR_UNSUPPORTED, "the request loop batches N = 4 and N = 8");
    }
    s->budget = budget_bytes / 256 * 256;
    s->max_batch = max_batch;
    // two batches in flight per stream: a batch waits for a slot rather than piling
    // launches onto the streams, so under load the requests that arrive meanwhile
    // join the next batch
    s->slots = std::min(64, 2 * nstreams);
    try {
        s->pool.reset(new CopyPool(kCopyWorkers));
    } catch (...) {
        s->pool.reset();   // no worker threads: the loop stages every batch itself
    }
    cudaError_t e = cudaMalloc(&s->d_arena, s->budget);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_arena), s->budget, cudaHostAllocDefault);
    const size_t nres = size_t(s->slots) * size_t(max_batch);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_sse, nres * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_psnr, nres * sizeof(float));
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_sse), nres * sizeof(double), 0);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s->h_psnr), nres * sizeof(float), 0);
    for (int k = 0; k < nstreams && e == cudaSuccess; k++) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    for (int k = 0; k < s->slots && e == cudaSuccess; k++) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) s->events.push_back(ev);
    }
    if (e != cudaSuccess) {
        server_free(s);
        return e == cudaErrorMemoryAllocation ? fail(RKLT_ERR_OOM, "server allocation failed")
                                              : cuda_fail(e, "server set-up");
    }
    // load every kernel both loops can reach (every r, batched and single) before any
    // trace starts, so that no request pays for module loading
    const rklt_status ws = server_warm(s);
    if (ws != RKLT_OK) {
        server_free(s);
        return ws;
    }
    *out = s;
    return RKLT_OK;
}

rklt_status rklt_server_run(rklt_server *s, const rklt_request *reqs, int n, int mode, uint8_t *const *h_recon,
                            float *const *h_coef, rklt_result *results, double *wall_s) {
    if (!s || !results || !wall_s) return fail(RKLT_ERR_ARG, "server, results and wall_s are required");
    if (mode != 0 && mode != 1) return fail(RKLT_ERR_ARG, "mode must be 0 (continuous) or 1 (plain)");
    rklt_status st = check_requests(s, reqs, n);
    if (st != RKLT_OK) return st;
    for (int i = 0; i < n; i++) results[i] = rklt_result{-1.0, -1.0, 0.0, 0.0f, RKLT_ERR_ARG};
    *wall_s = 0.0;
    if (n == 0) return RKLT_OK;
    return mode == 0 ? run_continuous(s, reqs, n, h_recon, h_coef, results, wall_s)
                     : run_plain(s, reqs, n, h_recon, h_coef, results, wall_s);
}

void rklt_server_destroy(rklt_server *s) { server_free(s); }

rklt_status rklt_copypool_selftest(unsigned seed, int rounds) {
    // rounds of staging copies through a pool of worker threads: random images with
    // random pitches cut into row chunks of random height; every destination row must
    // hold its source row and the pitch padding must keep its sentinel byte
    unsigned x = seed ? seed : 1u;
    auto rnd = [&x]() {
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        return x;
    };
    std::unique_ptr<rklt::CopyPool> pool;
    try {
        pool.reset(new rklt::CopyPool(3));
    } catch (...) {
        return fail(RKLT_ERR_ARG, "could not start the copy workers");
    }
    std::vector<uint8_t> src, dst;
    std::vector<rklt::CopyPool::Chunk> chunks;
    struct Img {
        size_t s_off, d_off;
        int H, W;
        int64_t ld;
    };
    std::vector<Img> imgs;
    for (int t = 0; t < rounds; t++) {
        imgs.clear();
        chunks.clear();
        size_t s_len = 0, d_len = 0;
        const int nimg = 1 + int(rnd() % 6);
        for (int i = 0; i < nimg; i++) {
            Img m{};
            m.H = 1 + int(rnd() % 97);
            m.W = 1 + int(rnd() % 301);
            m.ld = m.W + int64_t(rnd() % 17);
            m.s_off = s_len;
            m.d_off = d_len;
            s_len += size_t(m.H) * size_t(m.W);
            d_len += size_t(m.H) * size_t(m.ld);
            imgs.push_back(m);
        }
        src.resize(s_len);
        for (auto &b : src) b = uint8_t(rnd());
        dst.assign(d_len, 0xA5);
        for (const Img &m : imgs) {
            const int step = 1 + int(rnd() % 13);
            for (int y = 0; y < m.H; y += step)
                chunks.push_back({dst.data() + m.d_off + size_t(y) * size_t(m.ld), src.data() + m.s_off + size_t(y) * m.W,
                                  m.ld, m.W, std::min(step, m.H - y)});
        }
        pool->run(chunks.data(), chunks.size());
        for (const Img &m : imgs)
            for (int y = 0; y < m.H; y++) {
                const uint8_t *d = dst.data() + m.d_off + size_t(y) * size_t(m.ld);
                if (std::memcmp(d, src.data() + m.s_off + size_t(y) * m.W, size_t(m.W)) != 0)
                    return fail(RKLT_ERR_ARG, "a staged row differs from its source");
                for (int64_t c = m.W; c < m.ld; c++)
                    if (d[c] != 0xA5) return fail(RKLT_ERR_ARG, "a copy wrote into the pitch padding");
            }
    }
    pool.reset();   // joins the workers
    return RKLT_OK;
}

rklt_status rklt_arena_selftest(unsigned seed, int steps) {
    // random allocations and releases against a byte map of the arena: no two live
    // ranges overlap, offsets are 256-byte aligned, and releasing everything
    // coalesces the free list back into the whole arena
    const size_t size = size_t(1) << 16;
    rklt::Arena a(size);
    std::vector<std::pair<size_t, size_t>> live;
    std::vector<unsigned char> owner(size, 0);
    unsigned x = seed ? seed : 1u;
    auto rnd = [&x]() {
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        return x;
    };
    for (int t = 0; t < steps; t++) {
        if (!live.empty() && (rnd() & 1)) {
            const size_t k = rnd() % live.size();
            for (size_t b = live[k].first; b < live[k].first + live[k].second; b++) owner[b] = 0;
            a.release(live[k].first, live[k].second);
            live.erase(live.begin() + long(k));
        } else {
            const size_t n = rklt::align_up(1 + rnd() % 4000);
            size_t off = 0;
            if (!a.alloc(n, off)) continue;
            if (off % 256 || off + n > size) return fail(RKLT_ERR_ARG, "arena returned a bad range");
            for (size_t b = off; b < off + n; b++) {
                if (owner[b]) return fail(RKLT_ERR_ARG, "arena ranges overlap");
                owner[b] = 1;
            }
            live.push_back({off, n});
        }
    }
    for (auto &l : live) a.release(l.first, l.second);
    size_t off = 0;
    if (!a.alloc(size, off) || off != 0) return fail(RKLT_ERR_ARG, "free list did not coalesce");
    return RKLT_OK;
}

}  // extern "C"
