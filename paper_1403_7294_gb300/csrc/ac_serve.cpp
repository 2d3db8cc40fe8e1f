// ac_serve.cpp - continuous batching of scan requests over resident dfas.
//
// Requests arrive with ac_serve_submit (host texts, copied at submit) and
// wait in one queue. n_streams worker threads each own a CUDA stream. A free
// worker takes the oldest waiting request, adds younger requests for the same
// dfa (oldest first) up to max_batch, as long as the device bytes of the
// work in flight on all workers stay within the budget (memory admission),
// and runs them as one batched scan on its stream. While it runs, other
// workers form and launch further batches from requests that arrived in the
// meantime, so scans of different sizes overlap on the device.
//
// A request's device bytes: its packed text (n/4), its ASCII text if it came
// as ASCII (n), its output reservation (16 B per reserved occurrence, twice:
// the batch's output and the per-request split of it) and its per-keyword
// counts (8 B per keyword of its dfa). The reservation per base is learned
// per dfa from the batches it has served (twice the densest seen, decaying
// slowly), so batches rarely outgrow it.
// Per-request results are exactly the stand-alone scan's: the batch writes
// every occurrence with its text index; for a batch of several requests two
// device passes split them into one range per request and count each
// request's occurrences per keyword (no host loop over occurrences), and one
// copy brings all of it into a pinned block the batch's requests share. A
// batch of one request takes the batch's own counts. If a batch overflows
// its reservation (its occurrence count is still exact), the batch runs once
// more with exactly that much room.
//
// Host copies are what a large request's latency is made of, so texts of
// 1 MiB or more are copied at submit into pinned blocks from a pool and go to
// the device from there (small ones are gathered in a per-worker pinned
// staging buffer), and a batch of one request with 1 MiB or more of
// occurrences leaves them in a pinned block the request keeps until it is
// waited for.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ac_internal.h"
#include "ac_trace.h"

namespace {

using Clock = std::chrono::steady_clock;

// Pinned host blocks reused across requests: a block stays with the request
// whose text or results it holds until the request is forgotten, then goes
// back to the free list (beyond kKeepFree free bytes it is released).
class PinnedPool : public std::enable_shared_from_this<PinnedPool> {
  public:
    struct Block {  // keeps its pool alive: a taken result may outlive the server
        void* p = nullptr;
        size_t cap = 0;
        std::shared_ptr<PinnedPool> pool;
        ~Block() { pool->put(p, cap); }
    };
    ~PinnedPool() {
        for (auto& f : free_) cudaFreeHost(f.second);
    }
    // a block of at least `bytes` (sizes are powers of two from 1 MiB), or null
    std::shared_ptr<Block> get(size_t bytes) {
        size_t cap = (size_t)1 << 20;
        while (cap < bytes) cap <<= 1;
        void* p = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto it = free_.find(cap);
            if (it != free_.end()) {
                p = it->second;
                free_.erase(it);
                free_bytes_ -= cap;
            }
        }
        if (!p && cudaHostAlloc(&p, cap, cudaHostAllocPortable) != cudaSuccess) return nullptr;  // any thread's context
        auto b = std::make_shared<Block>();
        b->p = p;
        b->cap = cap;
        b->pool = shared_from_this();
        return b;
    }

  private:
    static constexpr size_t kKeepFree = (size_t)1 << 30;
    void put(void* p, size_t cap) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (free_bytes_ + cap <= kKeepFree) {
                free_.emplace(cap, p);
                free_bytes_ += cap;
                return;
            }
        }
        cudaFreeHost(p);
    }
    std::mutex mu_;
    std::multimap<size_t, void*> free_;
    size_t free_bytes_ = 0;
};

struct Request {
    uint64_t ticket = 0;
    uint32_t slot = 0;
    int32_t encoding = AC_TEXT_ASCII;
    uint64_t n = 0;
    std::vector<uint8_t> bytes;  // ASCII bytes or packed words
    // a text of kHandoffBytes or more is copied at submit into a pinned block
    // instead (ASCII padded with 'A' to a multiple of 64), which the worker
    // copies to the device directly
    std::shared_ptr<PinnedPool::Block> text_block;
    uint64_t reserve = 0;        // occurrences reserved
    uint64_t dev_bytes = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
    int status = AC_OK;
    std::vector<ac_match> matches;
    std::vector<uint64_t> counts;
    uint64_t n_matches = 0;
    // or in a pinned block the request holds (shared by the requests of one
    // batch): n_matches occurrences at match_off, the counts at count_off
    std::shared_ptr<PinnedPool::Block> block;
    size_t match_off = 0, count_off = 0;  // bytes into block
    const ac_match* match_data() const {
        return block ? (const ac_match*)((const uint8_t*)block->p + match_off) : matches.data();
    }
    const uint64_t* count_data() const {
        return block ? (const uint64_t*)((const uint8_t*)block->p + count_off) : counts.data();
    }
    size_t n_counts = 0;
};

uint64_t round_up(uint64_t x, uint64_t m) { return (x + m - 1) / m * m; }

// Texts at least this large are held in pinned blocks from submit on, and the
// results of a one-request batch at least this large stay in a pinned block
// handed to the request; smaller ones go through the worker's buffers.
constexpr size_t kHandoffBytes = (size_t)1 << 20;

// Copies n bytes from src to dst; with `check`, also tells whether every byte
// is one of A, C, G, T. One pass over the caller's bytes: 64 per step through
// the compiler's generic 16-byte vectors (no target-specific code; the host
// compiler maps them to the machine's SIMD registers), the tail byte by byte.
typedef uint8_t v16u8 __attribute__((vector_size(16)));
typedef int8_t v16i8 __attribute__((vector_size(16)));

bool copy_text(uint8_t* dst, const uint8_t* src, uint64_t n, bool check) {
    if (!check) {
        if (n) std::memcpy(dst, src, n);
        return true;
    }
    uint64_t i = 0;
    v16i8 bad = {};
    for (; i + 64 <= n; i += 64) {
        for (int k = 0; k < 4; ++k) {
            v16u8 x;
            std::memcpy(&x, src + i + 16 * k, 16);
            bad |= (x != 'A') & (x != 'C') & (x != 'G') & (x != 'T');  // lanes: -1 where not a base
            std::memcpy(dst + i + 16 * k, &x, 16);
        }
    }
    uint64_t w[2];
    std::memcpy(w, &bad, 16);
    bool ok = (w[0] | w[1]) == 0;
    for (; i < n; ++i) {
        const uint8_t c = src[i];
        dst[i] = c;
        ok &= c == 'A' || c == 'C' || c == 'G' || c == 'T';
    }
    return ok;
}

// Large submitted texts are copied (and checked) by the submitting thread
// together with a few helper threads of the server, each taking one
// contiguous part: one core's memory copy would otherwise be most of the
// time a large request spends in ac_serve_submit.
constexpr uint64_t kSplitCopyBytes = 2ull << 20;  // smaller texts: the caller's thread alone
constexpr int kCopyHelpers = 3;

class CopyHelpers {
   public:
    CopyHelpers() {
        try {
            for (int i = 0; i < kCopyHelpers; ++i) threads_.emplace_back([this] { run(); });
        } catch (...) {  // fewer helpers (none at worst): copy() splits over the ones running
        }
    }
    ~CopyHelpers() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : threads_) t.join();
    }
    // copy_text over (helpers + 1) parts; true when every part passed the check
    bool copy(uint8_t* dst, const uint8_t* src, uint64_t n, bool check) {
        const uint64_t parts = threads_.size() + 1;
        if (parts == 1 || n < kSplitCopyBytes) return copy_text(dst, src, n, check);
        const uint64_t part = round_up((n + parts - 1) / parts, 64);
        Job job;
        job.pending = (int)(parts - 1);  // set before any helper can see a task of this job
        {
            std::lock_guard<std::mutex> lk(mu_);
            for (uint64_t i = 0; i + 1 < parts; ++i) {
                const uint64_t a = std::min(n, i * part), b = std::min(n, a + part);
                tasks_.push_back(Task{&job, dst + a, src + a, b - a, check});
            }
        }
        cv_.notify_all();
        const uint64_t a = std::min(n, (parts - 1) * part);
        const bool ok = copy_text(dst + a, src + a, n - a, check);
        std::unique_lock<std::mutex> lk(job.mu);
        job.cv.wait(lk, [&] { return job.pending == 0; });
        return ok && job.ok;
    }

   private:
    struct Job {
        std::mutex mu;
        std::condition_variable cv;
        int pending = 0;
        bool ok = true;
    };
    struct Task {
        Job* job;
        uint8_t* dst;
        const uint8_t* src;
        uint64_t n;
        bool check;
    };
    void run() {
        for (;;) {
            Task t;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || !tasks_.empty(); });
                if (tasks_.empty()) return;  // stopping, nothing left to copy
                t = tasks_.front();
                tasks_.pop_front();
            }
            const bool ok = copy_text(t.dst, t.src, t.n, t.check);
            std::lock_guard<std::mutex> lk(t.job->mu);  // the waiter wakes only after this is released
            t.job->ok = t.job->ok && ok;
            if (--t.job->pending == 0) t.job->cv.notify_one();
        }
    }
    std::vector<std::thread> threads_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<Task> tasks_;
    bool stop_ = false;
};

struct PinnedBuf {
    void* p = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes) {
        if (bytes <= cap) return true;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max(bytes, (size_t)1 << 24);
        if (cudaMallocHost(&p, want) != cudaSuccess) return false;
        cap = want;
        return true;
    }
    ~PinnedBuf() {
        if (p) cudaFreeHost(p);
    }
};

}  // namespace

struct ac_server {
    std::shared_ptr<PinnedPool> pool = std::make_shared<PinnedPool>();  // pinned text and result blocks
    ac_serve_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // workers: new requests / freed budget / stop
    std::condition_variable cv_done;  // waiters: completions
    std::vector<const ac_dfa*> dfas;
    // learned occurrences per base of each dfa's requests: twice the densest
    // batch seen, decaying slowly, so reservations rarely fall short
    std::vector<double> density;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> by_ticket;
    uint64_t next_ticket = 1;
    uint64_t in_flight_bytes = 0;
    uint32_t in_flight_reqs = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    CopyHelpers copiers;  // threads that share the copy of large submitted texts
    // stats
    uint64_t submitted = 0, completed = 0, rejected = 0, failed = 0, bases_completed = 0, batches = 0;
    uint64_t overflow_batches = 0;  // batches run twice for want of output room
    uint64_t cancelled = 0;         // requests withdrawn before they ran
    std::vector<double> lat_ms;
    double busy_s = 0.0;
    Clock::time_point busy_since;
    uint32_t active_batches = 0;

    void worker_main(int idx);
    void run_batch(cudaStream_t st, std::vector<std::shared_ptr<Request>>& batch, PinnedBuf& stage,
                   PinnedBuf& results);
};

void ac_server::run_batch(cudaStream_t st, std::vector<std::shared_ptr<Request>>& batch, PinnedBuf& stage,
                          PinnedBuf& results) {
    AcRange trace_("ac_serve batch");
    const ac_dfa* dfa = dfas[batch[0]->slot];
    const uint32_t P = dfa->host.n_patterns;
    // ASCII requests first (one pack over their contiguous slots), packed after
    std::stable_sort(batch.begin(), batch.end(), [](const std::shared_ptr<Request>& a,
                                                     const std::shared_ptr<Request>& b) {
        return a->encoding == AC_TEXT_ASCII && b->encoding != AC_TEXT_ASCII;
    });
    const size_t B = batch.size();
    std::vector<uint64_t> slot(B + 1, 0);  // bases, 64-aligned
    uint64_t ascii_bases = 0, reserve = 0;
    for (size_t i = 0; i < B; ++i) {
        slot[i + 1] = slot[i] + round_up(batch[i]->n, 64);
        if (batch[i]->encoding == AC_TEXT_ASCII) ascii_bases = slot[i + 1];
        reserve += batch[i]->reserve;
    }
    const uint64_t all = slot[B];
    const size_t packed_bytes = all / 4;
    int status = AC_OK;
    bool overflowed = false;
    uint8_t* d_ascii = nullptr;
    uint32_t* d_packed = nullptr;
    ac_match* d_m = nullptr;
    unsigned long long* d_cnt = nullptr;
    ac_match* d_split = nullptr;              // several requests: the occurrences split per request
    unsigned long long* d_aux_keep = nullptr;  // their offsets, cursors and per-request counts
    auto fail_all = [&](int s) { status = s; };

    // ---- stage: ASCII bytes padded with 'A', then packed words (texts held in
    // pinned blocks are not staged: they are copied to the device from there)
    if (!stage.ensure(std::max<size_t>(ascii_bases + packed_bytes, 16))) fail_all(AC_ERR_OOM);
    uint8_t* h_ascii = (uint8_t*)stage.p;
    uint8_t* h_packed = h_ascii + ascii_bases;
    if (status == AC_OK) {
        for (size_t i = 0; i < B; ++i) {
            Request& r = *batch[i];
            if (r.text_block) continue;
            if (r.encoding == AC_TEXT_ASCII) {
                std::memcpy(h_ascii + slot[i], r.bytes.data(), r.n);
                std::memset(h_ascii + slot[i] + r.n, 'A', slot[i + 1] - slot[i] - r.n);
            } else {
                const size_t wb = (r.n + 15) / 16 * 4;
                std::memcpy(h_packed + slot[i] / 4 - ascii_bases / 4, r.bytes.data(), wb);
            }
        }
        if (ac_dev_alloc_async((void**)&d_packed, std::max<size_t>(packed_bytes, 16), st) != cudaSuccess ||
            (ascii_bases && ac_dev_alloc_async((void**)&d_ascii, ascii_bases, st) != cudaSuccess) ||
            ac_dev_alloc_async((void**)&d_m, std::max<uint64_t>(reserve, 1) * sizeof(ac_match), st) != cudaSuccess)
            fail_all(AC_ERR_OOM);
    }
    if (status == AC_OK) {
        auto h2d = [&](void* d, const void* h, size_t bytes) {
            if (bytes) cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st);
        };
        // ASCII slots: runs of staged ones, and each pinned text (with its padding) on its own
        uint64_t run = 0;  // first base of the current run of staged slots
        for (size_t i = 0; i < B && batch[i]->encoding == AC_TEXT_ASCII; ++i) {
            if (!batch[i]->text_block) continue;
            h2d(d_ascii + run, h_ascii + run, slot[i] - run);
            h2d(d_ascii + slot[i], batch[i]->text_block->p, slot[i + 1] - slot[i]);
            run = slot[i + 1];
        }
        h2d(d_ascii + run, h_ascii + run, ascii_bases - run);
        // packed slots (after the ASCII ones), the same way
        run = ascii_bases;
        for (size_t i = 0; i < B; ++i) {
            const Request& r = *batch[i];
            if (r.encoding == AC_TEXT_ASCII || !r.text_block) continue;
            h2d((uint8_t*)d_packed + run / 4, h_packed + (run - ascii_bases) / 4, (slot[i] - run) / 4);
            h2d((uint8_t*)d_packed + slot[i] / 4, r.text_block->p, (r.n + 15) / 16 * 4);
            run = slot[i + 1];
        }
        h2d((uint8_t*)d_packed + run / 4, h_packed + (run - ascii_bases) / 4, (all - run) / 4);
        if (ascii_bases) {
            uint64_t bad = ~0ull;
            int s = ac_pack(d_ascii, ascii_bases, d_packed, 0, &bad, st);
            if (s == AC_ERR_ALPHABET) {
                // find the request that holds the bad byte; fail only that one
                for (size_t i = 0; i < B; ++i)
                    if (bad >= slot[i] && bad < slot[i + 1]) batch[i]->status = AC_ERR_ALPHABET;
            } else if (s != AC_OK) {
                fail_all(s);
            }
        }
    }
    // ---- the batched scan
    uint64_t nm = 0;
    if (status == AC_OK) {
        std::vector<ac_text> texts(B);
        for (size_t i = 0; i < B; ++i) texts[i] = ac_text{d_packed + slot[i] / 16, batch[i]->n, AC_TEXT_PACKED2, 1};
        ac_result res;
        std::memset(&res, 0, sizeof res);
        res.matches = d_m;
        res.capacity = reserve;
        res.on_device = 1;
        // a batch of one: the batch's counts are the request's counts
        int s = AC_OK;
        if (B == 1 && ac_dev_alloc_async((void**)&d_cnt, (size_t)P * 8, st) != cudaSuccess) s = AC_ERR_OOM;
        res.counts = (uint64_t*)d_cnt;
        if (s == AC_OK) s = ac_scan_batch(dfa, texts.data(), (uint32_t)B, &res, nullptr, st, nullptr);
        nm = res.n_matches;
        if (s == AC_ERR_OVERFLOW) {
            // more occurrences than reserved: the count is exact, so the batch runs once more with room for all
            overflowed = true;
            cudaFreeAsync(d_m, st);
            d_m = nullptr;
            if (ac_dev_alloc_async((void**)&d_m, std::max<uint64_t>(nm, 1) * sizeof(ac_match), st) != cudaSuccess) {
                s = AC_ERR_OOM;
            } else {
                res.matches = d_m;
                res.capacity = nm;
                res.n_matches = 0;
                s = ac_scan_batch(dfa, texts.data(), (uint32_t)B, &res, nullptr, st, nullptr);
                nm = res.n_matches;
            }
        }
        if (s != AC_OK) {
            fail_all(s);
        } else {
            const size_t mb = nm * sizeof(ac_match);
            if (B == 1) {
                // one request: the batch's occurrences (text index 0 already) and
                // counts are the request's. With many occurrences they land in a
                // pinned block the request keeps until it is waited for.
                std::shared_ptr<PinnedPool::Block> blk;
                if (d_cnt && mb >= kHandoffBytes) blk = pool->get(mb + (size_t)P * 8);  // none: the worker's buffer
                const bool handoff = blk != nullptr;
                void* dst = nullptr;
                if (handoff) {
                    dst = blk->p;
                } else if (results.ensure(std::max<size_t>(mb + (d_cnt ? (size_t)P * 8 : 0), 16))) {
                    dst = results.p;
                }
                if (!dst) {
                    fail_all(AC_ERR_OOM);
                } else {
                    if (nm) cudaMemcpyAsync(dst, d_m, mb, cudaMemcpyDeviceToHost, st);
                    if (d_cnt) cudaMemcpyAsync((uint8_t*)dst + mb, d_cnt, (size_t)P * 8, cudaMemcpyDeviceToHost, st);
                    if (cudaStreamSynchronize(st) != cudaSuccess) fail_all(AC_ERR_CUDA);
                }
                Request& r = *batch[0];
                if (status == AC_OK && r.status == AC_OK) {
                    if (handoff) {
                        r.block = std::move(blk);
                        r.match_off = 0;
                        r.count_off = mb;
                    } else {
                        const ac_match* m = (const ac_match*)dst;
                        const uint64_t* c = (const uint64_t*)((const uint8_t*)dst + mb);
                        r.matches.assign(m, m + nm);
                        r.counts.assign(c, c + P);
                    }
                    r.n_matches = nm;
                    r.n_counts = P;
                }
            } else {
                // several requests: split on the device (each request's occurrences
                // in one range, its per-keyword counts in a row of B x P), then one
                // copy into a pinned block the batch's requests share
                const size_t cb = (size_t)B * P * 8, ob = (B + 1) * sizeof(unsigned long long);
                unsigned long long* d_aux = nullptr;  // [n_per B][cursor B][offs B+1][counts B*P]
                const size_t aux = (3 * (size_t)B + 1) * 8 + cb;
                if (ac_dev_alloc_async((void**)&d_split, std::max<size_t>(mb, 16), st) != cudaSuccess ||
                    ac_dev_alloc_async((void**)&d_aux, aux, st) != cudaSuccess) {
                    fail_all(AC_ERR_OOM);
                } else {
                    d_aux_keep = d_aux;
                    unsigned long long* n_per = d_aux;
                    unsigned long long* cursor = d_aux + B;
                    unsigned long long* offs = d_aux + 2 * B;
                    unsigned long long* rc = d_aux + 3 * B + 1;
                    if (cudaMemsetAsync(d_aux, 0, aux, st) != cudaSuccess) fail_all(AC_ERR_CUDA);
                    if (status == AC_OK &&
                        ac_launch_serve_split(d_m, nm, (uint32_t)B, P, d_split, rc, n_per, offs, cursor, st) != 0)
                        fail_all(AC_ERR_CUDA);
                    std::shared_ptr<PinnedPool::Block> blk;
                    void* dst = nullptr;
                    if (status == AC_OK) {
                        blk = pool->get(mb + cb + ob);
                        if (blk) dst = blk->p;
                        else if (results.ensure(mb + cb + ob)) dst = results.p;  // no pooled block: the worker's
                        if (!dst) fail_all(AC_ERR_OOM);
                    }
                    if (status == AC_OK) {
                        if (nm) cudaMemcpyAsync(dst, d_split, mb, cudaMemcpyDeviceToHost, st);
                        cudaMemcpyAsync((uint8_t*)dst + mb, rc, cb, cudaMemcpyDeviceToHost, st);
                        cudaMemcpyAsync((uint8_t*)dst + mb + cb, offs, ob, cudaMemcpyDeviceToHost, st);
                        if (cudaStreamSynchronize(st) != cudaSuccess) fail_all(AC_ERR_CUDA);
                    }
                    if (status == AC_OK) {
                        const uint64_t* off = (const uint64_t*)((const uint8_t*)dst + mb + cb);
                        for (size_t i = 0; i < B; ++i) {
                            Request& r = *batch[i];
                            if (r.status != AC_OK) continue;
                            r.n_matches = off[i + 1] - off[i];
                            r.n_counts = P;
                            const size_t mo = off[i] * sizeof(ac_match), co = mb + i * (size_t)P * 8;
                            if (blk) {
                                r.block = blk;
                                r.match_off = mo;
                                r.count_off = co;
                            } else {
                                const ac_match* m = (const ac_match*)((const uint8_t*)dst + mo);
                                const uint64_t* c = (const uint64_t*)((const uint8_t*)dst + co);
                                r.matches.assign(m, m + r.n_matches);
                                r.counts.assign(c, c + P);
                            }
                        }
                    }
                }
            }
        }
    }
    if (d_ascii) cudaFreeAsync(d_ascii, st);
    if (d_packed) cudaFreeAsync(d_packed, st);
    if (d_m) cudaFreeAsync(d_m, st);
    if (d_cnt) cudaFreeAsync(d_cnt, st);
    if (d_split) cudaFreeAsync(d_split, st);
    if (d_aux_keep) cudaFreeAsync(d_aux_keep, st);
    cudaStreamSynchronize(st);
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    if (overflowed) overflow_batches++;
    if (status == AC_OK && all) {
        double& dn = density[batch[0]->slot];
        dn = std::max(dn * 0.999, 2.0 * (double)nm / (double)all);
    }
    for (auto& r : batch) {
        if (status != AC_OK && r->status == AC_OK) r->status = status;
        r->text_block.reset();  // the text is on the device no longer: its host copy goes now
        std::vector<uint8_t>().swap(r->bytes);
        r->done = true;
        r->t_done = now;
        in_flight_bytes -= r->dev_bytes;
        in_flight_reqs -= 1;
        if (r->status == AC_OK) {
            completed++;
            bases_completed += r->n;
            lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        } else {
            failed++;
        }
    }
    cv_done.notify_all();
    cv_work.notify_all();
}

void ac_server::worker_main(int idx) {
    (void)idx;
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    PinnedBuf stage, results;
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stop && pending.empty()) {
                    lk.unlock();
                    cudaStreamDestroy(st);
                    return;
                }
                if (!pending.empty()) {
                    const uint32_t slot = pending.front()->slot;
                    uint64_t bytes = in_flight_bytes;
                    for (auto it = pending.begin(); it != pending.end() && batch.size() < opts.max_batch;) {
                        if ((*it)->slot == slot && bytes + (*it)->dev_bytes <= opts.device_budget_bytes) {
                            bytes += (*it)->dev_bytes;
                            batch.push_back(*it);
                            it = pending.erase(it);
                        } else if (batch.empty()) {
                            break;  // the oldest waits until the budget frees up
                        } else {
                            ++it;
                        }
                    }
                    if (!batch.empty()) {
                        in_flight_bytes = bytes;
                        in_flight_reqs += (uint32_t)batch.size();
                        if (active_batches++ == 0) busy_since = Clock::now();
                        batches++;
                        break;
                    }
                }
                cv_work.wait(lk);
            }
        }
        run_batch(st, batch, stage, results);
        {
            std::lock_guard<std::mutex> lk(mu);
            if (--active_batches == 0)
                busy_s += std::chrono::duration<double>(Clock::now() - busy_since).count();
        }
    }
}

extern "C" int ac_serve_create(const ac_serve_opts* opts, ac_server** out) {
    if (!out) return AC_ERR_INVALID_ARG;
    ac_server* s = new (std::nothrow) ac_server();
    if (!s) return AC_ERR_OOM;
    if (opts) s->opts = *opts;
    if (!s->opts.device_budget_bytes) s->opts.device_budget_bytes = 40ull << 30;
    if (!s->opts.n_streams) s->opts.n_streams = 4;
    if (!s->opts.max_batch) s->opts.max_batch = 256;
    if (!s->opts.max_queue) s->opts.max_queue = 1u << 16;
    if (!s->opts.match_capacity_per_base_x1000) s->opts.match_capacity_per_base_x1000 = 64;
    cudaGetDevice(&s->device);
    try {
        for (uint32_t i = 0; i < s->opts.n_streams; ++i) s->workers.emplace_back(&ac_server::worker_main, s, (int)i);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto& t : s->workers) t.join();
        delete s;
        return AC_ERR_OOM;
    }
    *out = s;
    return AC_OK;
}

extern "C" int ac_serve_add_dfa(ac_server* s, const ac_dfa* dfa, uint32_t* slot) {
    if (!s || !dfa || !slot) return AC_ERR_INVALID_ARG;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lk(s->mu);
    s->dfas.push_back(dfa);
    s->density.push_back(0.0);
    *slot = (uint32_t)(s->dfas.size() - 1);
    return AC_OK;
}

extern "C" int ac_serve_submit(ac_server* s, uint32_t slot, const ac_text* t, uint64_t* ticket) {
    AcRange trace_("ac_serve_submit");
    if (!s || !t || !ticket) return AC_ERR_INVALID_ARG;
    if (t->on_device) return AC_ERR_INVALID_ARG;
    if (t->encoding != AC_TEXT_ASCII && t->encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
    if (t->n_bases && !t->data) return AC_ERR_INVALID_ARG;
    if (t->n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
    auto r = std::make_shared<Request>();
    r->slot = slot;
    r->encoding = t->encoding;
    r->n = t->n_bases;
    const uint64_t nb = t->encoding == AC_TEXT_ASCII ? t->n_bases : (t->n_bases + 15) / 16 * 4;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (slot >= s->dfas.size()) return AC_ERR_NOT_FOUND;
        const double per_base = std::max(s->opts.match_capacity_per_base_x1000 / 1000.0, s->density[slot]);
        r->reserve = (uint64_t)((double)t->n_bases * per_base) + 1024;
        r->dev_bytes = round_up(t->n_bases, 64) / 4 + (t->encoding == AC_TEXT_ASCII ? round_up(t->n_bases, 64) : 0) +
                       2 * r->reserve * sizeof(ac_match) + (uint64_t)s->dfas[slot]->host.n_patterns * 8;
        if (s->stop || s->pending.size() >= s->opts.max_queue || r->dev_bytes > s->opts.device_budget_bytes) {
            s->rejected++;
            return AC_ERR_BUSY;
        }
    }
    // the text is copied now, and an ASCII text checked in the same pass: bad
    // input is refused here, before it is queued
    const bool ascii = t->encoding == AC_TEXT_ASCII;
    bool ok = true;
    try {
        const uint64_t held = ascii ? round_up(t->n_bases, 64) : nb;
        if (nb >= kHandoffBytes) r->text_block = s->pool->get(held);  // no pinned memory: staged instead
        if (r->text_block) {
            ok = s->copiers.copy((uint8_t*)r->text_block->p, (const uint8_t*)t->data, nb, ascii);
            std::memset((uint8_t*)r->text_block->p + nb, 'A', held - nb);
        } else {
            r->bytes.resize(nb);
            ok = copy_text(r->bytes.data(), (const uint8_t*)t->data, nb, ascii);
        }
    } catch (const std::bad_alloc&) {
        return AC_ERR_OOM;
    }
    if (!ok) return AC_ERR_ALPHABET;  // the request and its block go with r
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->by_ticket[r->ticket] = r;
        s->pending.push_back(r);
        s->submitted++;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return AC_OK;
}

extern "C" int ac_serve_wait(ac_server* s, uint64_t ticket, ac_result* res, int64_t timeout_us) {
    AcRange trace_("ac_serve_wait");
    if (!s || !res) return AC_ERR_INVALID_ARG;
    if (res->on_device || (res->capacity && !res->matches)) return AC_ERR_INVALID_ARG;
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->by_ticket.find(ticket);
        if (it == s->by_ticket.end()) return AC_ERR_NOT_FOUND;
        r = it->second;
        auto ready = [&] { return r->done; };
        if (timeout_us < 0) {
            s->cv_done.wait(lk, ready);
        } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
            return AC_ERR_TIMEOUT;
        }
        res->bad_offset = ~0ull;
        res->n_matches = r->n_matches;
        if (r->status == AC_OK && r->n_matches > res->capacity) return AC_ERR_OVERFLOW;  // ticket stays valid
        s->by_ticket.erase(ticket);
    }
    if (r->status != AC_OK) return r->status;
    if (r->n_matches) std::memcpy(res->matches, r->match_data(), r->n_matches * sizeof(ac_match));
    if (res->counts && r->n_counts) std::memcpy(res->counts, r->count_data(), r->n_counts * 8);
    return AC_OK;
}

namespace {
struct Taken {  // what an ac_serve_take handle owns
    std::shared_ptr<Request> r;
};
}  // namespace

extern "C" int ac_serve_take(ac_server* s, uint64_t ticket, ac_served* out, int64_t timeout_us) {
    AcRange trace_("ac_serve_take");
    if (!s || !out) return AC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->by_ticket.find(ticket);
        if (it == s->by_ticket.end()) return AC_ERR_NOT_FOUND;
        r = it->second;
        auto ready = [&] { return r->done; };
        if (timeout_us < 0) {
            s->cv_done.wait(lk, ready);
        } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
            return AC_ERR_TIMEOUT;
        }
        s->by_ticket.erase(ticket);
    }
    if (r->status != AC_OK) return r->status;
    Taken* t = new (std::nothrow) Taken{r};
    if (!t) return AC_ERR_OOM;
    out->matches = r->match_data();
    out->n_matches = r->n_matches;
    out->counts = r->count_data();
    out->n_counts = r->n_counts;
    out->handle = t;
    return AC_OK;
}

extern "C" void ac_serve_release(void* handle) { delete static_cast<Taken*>(handle); }

extern "C" int ac_serve_cancel(ac_server* s, uint64_t ticket) {
    if (!s) return AC_ERR_INVALID_ARG;
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->by_ticket.find(ticket);
        if (it == s->by_ticket.end()) return AC_ERR_NOT_FOUND;
        r = it->second;
        if (r->done) {  // finished, not yet waited for: drop its results
            s->by_ticket.erase(it);
            return AC_OK;
        }
        auto q = std::find(s->pending.begin(), s->pending.end(), r);
        if (q == s->pending.end()) return AC_ERR_BUSY;  // its batch is on the device
        s->pending.erase(q);
        s->by_ticket.erase(it);
        s->cancelled++;
    }
    s->cv_work.notify_all();  // the queue changed: a worker may now admit the next request
    return AC_OK;  // r (and its text) goes when the last reference does
}

extern "C" int ac_serve_stats(ac_server* s, ac_serve_stats_t* o) {
    if (!s || !o) return AC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(o, 0, sizeof *o);
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->rejected = s->rejected;
    o->failed = s->failed;
    o->bases_completed = s->bases_completed;
    o->batches_launched = s->batches;
    o->overflow_batches = s->overflow_batches;
    o->cancelled = s->cancelled;
    double busy = s->busy_s;
    if (s->active_batches) busy += std::chrono::duration<double>(Clock::now() - s->busy_since).count();
    o->busy_s = busy;
    o->gbases_per_s = busy > 0 ? (double)s->bases_completed / busy / 1e9 : 0.0;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        auto pct = [&](double q) {
            size_t k = (size_t)std::min<double>((double)v.size() - 1, std::max(0.0, q * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + k, v.end());
            return v[k];
        };
        o->p50_ms = pct(0.50);
        o->p99_ms = pct(0.99);
        double sum = 0, mx = 0;
        for (double x : s->lat_ms) {
            sum += x;
            mx = std::max(mx, x);
        }
        o->mean_ms = sum / (double)s->lat_ms.size();
        o->max_ms = mx;
    }
    return AC_OK;
}

extern "C" void ac_serve_destroy(ac_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}
