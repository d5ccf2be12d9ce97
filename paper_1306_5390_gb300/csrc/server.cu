// Request server: continuous batching of denoising requests on one GPU.
//
// Requests (one image each, any size, their own alpha / beta / max_k) are
// queued by hgrms_server_submit and served by `slots` worker threads.  Each
// slot owns a denoising handle with its own CUDA stream and its own share of
// the device-memory budget.  A slot that becomes free takes, in arrival
// order, every queued request with the same (alpha, beta, max_k) as the
// oldest one while their device memory (the resident images and the batched
// schedule's buffers) fits its share, and runs them as one batched call
// (hgrms_denoise_batch): requests that arrive while others are on the GPU
// join the next batch of the next free slot, and the batches of different
// slots overlap on the device (their list-pass launches, whose CTAs wait
// for one another, take turns on one shared stream).  A request's result does not depend on the
// batch it joins (each image's passes and k are its own; see
// hgrms_denoise_batch), so a request gives the same bytes and k alone and in
// any mix.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hgrms.h"
#include "kernels.h"

#define HG_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
    unsigned long long id = 0;
    const uint8_t* src = nullptr;
    uint8_t* dst = nullptr;
    int rows = 0, cols = 0, alpha = 0, beta = 0, max_k = 0;
    bool device = false;  // src is device memory, denoised in place
    long long need = 0;   // device bytes while it is being served
    Clock::time_point t_submit, t_start, t_done;
    int k = 0;
    int status = 0;       // 0 queued, 1 running, 2 done
    int batch_size = 0;
    int slot = -1;
};

// Device bytes one request needs while served: its resident copy (host
// requests) plus what the batched schedule allocates per pixel (three
// canvases with padding, four change lists and bitmaps; an upper estimate).
long long request_bytes(int rows, int cols, bool device) {
    const long long px = (long long)rows * cols;
    const long long padded = (long long)(rows + 96) * (long long)(cols + 288);
    return (device ? 0 : px) + 3 * padded + 4 * px + px / 2 + 4096;
}

}  // namespace

struct hgrms_server {
    int device = 0;
    long long budget = 0;
    long long share = 0;  // per slot
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<unsigned long long, Request*> reqs;
    unsigned long long next_id = 1;
    bool stopping = false;
    std::vector<std::thread> workers;
    std::vector<hgrms_t> handles;
    std::vector<cudaStream_t> streams;
    cudaStream_t coop = nullptr;  // the slots' list-pass launches, one at a time
    long long served = 0, batches = 0, in_flight = 0, max_in_flight = 0;
    int error = 0;
    int fail_allocs = 0;  // allocations still to fail (hgrms_server_fail_allocations; under mu)

    void work(int slot);
};

void hgrms_server::work(int slot) {
    cudaSetDevice(device);
    hgrms_t h = handles[slot];
    cudaStream_t st = streams[slot];
    uint8_t* dbuf = nullptr;  // resident copies of this slot's host requests
    size_t dbuf_bytes = 0;
    std::vector<Request*> batch;
    std::vector<uint8_t*> ptrs;
    std::vector<int> rows, cols, ks;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_work.wait(lock, [&] { return stopping || !queue.empty(); });
            if (queue.empty()) break;  // stopping and drained
            const Request* head = queue.front();
            const int alpha = head->alpha, beta = head->beta, max_k = head->max_k;
            long long used = 0;
            for (auto it = queue.begin(); it != queue.end();) {
                Request* r = *it;
                if (r->alpha != alpha || r->beta != beta || r->max_k != max_k) {
                    ++it;
                    continue;
                }
                // The oldest request is always taken (alone if it exceeds the share).
                if (!batch.empty() && used + r->need > share) break;
                used += r->need;
                r->status = 1;
                r->slot = slot;
                r->t_start = Clock::now();
                batch.push_back(r);
                it = queue.erase(it);
                if ((int)batch.size() >= 4096) break;
            }
            in_flight += (long long)batch.size();
            if (in_flight > max_in_flight) max_in_flight = in_flight;
        }
        // Device copies of the host requests, one after another in this
        // slot's buffer.
        size_t host_bytes = 0;
        for (Request* r : batch)
            if (!r->device) host_bytes += ((size_t)r->rows * r->cols + 255) / 256 * 256;
        int rc = HGRMS_OK;
        if (host_bytes > dbuf_bytes) {
            if (dbuf) cudaFree(dbuf);
            dbuf = nullptr;
            dbuf_bytes = 0;
            bool fake = false;  // a failure requested by hgrms_server_fail_allocations
            {
                std::lock_guard<std::mutex> lock(mu);
                if (fail_allocs > 0) {
                    --fail_allocs;
                    fake = true;
                }
            }
            if (fake) {
                rc = HGRMS_ENOMEM;
            } else if (cudaMalloc(&dbuf, host_bytes) != cudaSuccess) {
                cudaGetLastError();
                dbuf = nullptr;
                rc = HGRMS_ENOMEM;
            } else {
                dbuf_bytes = host_bytes;
            }
        }
        ptrs.clear();
        rows.clear();
        cols.clear();
        size_t off = 0;
        for (Request* r : batch) {
            uint8_t* p = const_cast<uint8_t*>(r->src);
            if (!r->device && rc == HGRMS_OK) {
                p = dbuf + off;
                off += ((size_t)r->rows * r->cols + 255) / 256 * 256;
                if (cudaMemcpyAsync(p, r->src, (size_t)r->rows * r->cols, cudaMemcpyHostToDevice, st) != cudaSuccess)
                    rc = HGRMS_ECUDA;
            }
            ptrs.push_back(p);
            rows.push_back(r->rows);
            cols.push_back(r->cols);
        }
        ks.assign(batch.size(), 0);
        if (rc == HGRMS_OK)
            rc = hgrms_denoise_batch(h, ptrs.data(), rows.data(), cols.data(), (int)batch.size(), batch[0]->alpha,
                                     batch[0]->beta, batch[0]->max_k, ks.data());
        if (rc == HGRMS_OK) {
            for (size_t i = 0; i < batch.size(); ++i) {
                Request* r = batch[i];
                if (r->device) continue;
                if (cudaMemcpyAsync(r->dst, ptrs[i], (size_t)r->rows * r->cols, cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess)
                    rc = HGRMS_ECUDA;
            }
            if (cudaStreamSynchronize(st) != cudaSuccess) rc = HGRMS_ECUDA;
        }
        {
            std::lock_guard<std::mutex> lock(mu);
            const Clock::time_point now = Clock::now();
            for (size_t i = 0; i < batch.size(); ++i) {
                Request* r = batch[i];
                r->k = rc == HGRMS_OK ? ks[i] : rc;
                r->status = 2;
                r->t_done = now;
                r->batch_size = (int)batch.size();
            }
            if (rc != HGRMS_OK && !error) error = rc;
            served += (long long)batch.size();
            batches += 1;
            in_flight -= (long long)batch.size();
        }
        cv_done.notify_all();
    }
    if (dbuf) cudaFree(dbuf);
}

HG_EXPORT int hgrms_server_create(hgrms_server_t* out, int device, long long hbm_budget_bytes, int slots) {
    if (!out) return HGRMS_EINVAL;
    *out = nullptr;
    if (slots < 1 || slots > 64 || hbm_budget_bytes < (64ll << 20)) return HGRMS_EINVAL;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return HGRMS_ENODEV;
    }
    if (device < 0 || device >= n) return HGRMS_ENODEV;
    hgrms_server* s = new (std::nothrow) hgrms_server();
    if (!s) return HGRMS_ENOMEM;
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->share = hbm_budget_bytes / slots;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int rc = HGRMS_OK;
    if (cudaStreamCreateWithFlags(&s->coop, cudaStreamNonBlocking) != cudaSuccess) rc = HGRMS_ECUDA;
    for (int i = 0; i < slots && rc == HGRMS_OK; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            rc = HGRMS_ECUDA;
            break;
        }
        s->streams.push_back(st);
        hgrms_t h = nullptr;
        rc = hgrms_create(&h, device, st);
        if (rc != HGRMS_OK) break;
        s->handles.push_back(h);
        rc = hg::set_coop_stream(h, s->coop);
        if (rc != HGRMS_OK) break;
        // Batched launches stay within the slot's share of the budget.
        hgrms_set_option(h, HGRMS_OPT_BATCH_MB, (int)(s->share >> 20) > 64 ? (int)(s->share >> 20) : 64);
    }
    cudaSetDevice(prev);
    if (rc != HGRMS_OK) {
        for (hgrms_t h : s->handles) hgrms_destroy(h);
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        if (s->coop) cudaStreamDestroy(s->coop);
        delete s;
        return rc;
    }
    for (int i = 0; i < slots; ++i) s->workers.emplace_back(&hgrms_server::work, s, i);
    *out = s;
    return HGRMS_OK;
}

HG_EXPORT int hgrms_server_submit(hgrms_server_t s, const uint8_t* img, uint8_t* out, int rows, int cols, int alpha,
                                  int beta, int max_k, unsigned long long* id) {
    if (!s || !img || !id || rows < 1 || cols < 1 || rows > 65536 || cols > 65536) return HGRMS_EINVAL;
    if (alpha < 0 || alpha > 255 || beta < 1 || beta > 7 || max_k < 0 || max_k > 1000000) return HGRMS_EINVAL;
    cudaPointerAttributes at;
    bool dev = false;
    if (cudaPointerGetAttributes(&at, img) == cudaSuccess) {
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
            if (at.device != s->device) return HGRMS_EINVAL;
            dev = true;
        }
    } else {
        cudaGetLastError();
    }
    if (dev && out && out != img) return HGRMS_EINVAL;  // device images are denoised in place
    if (!dev && !out) return HGRMS_EINVAL;
    Request* r = new (std::nothrow) Request();
    if (!r) return HGRMS_ENOMEM;
    r->src = img;
    r->dst = dev ? const_cast<uint8_t*>(img) : out;
    r->rows = rows;
    r->cols = cols;
    r->alpha = alpha;
    r->beta = beta;
    r->max_k = max_k;
    r->device = dev;
    r->need = request_bytes(rows, cols, dev);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) {
            delete r;
            return HGRMS_EINVAL;
        }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->queue.push_back(r);
        *id = r->id;
    }
    s->cv_work.notify_one();
    return HGRMS_OK;
}

HG_EXPORT int hgrms_server_wait(hgrms_server_t s, unsigned long long id, double timeout_s, hgrms_request_info_t* info) {
    if (!s) return HGRMS_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return HGRMS_EINVAL;
    Request* r = it->second;
    const auto pred = [&] { return r->status == 2; };
    if (timeout_s < 0) {
        s->cv_done.wait(lock, pred);
    } else if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), pred)) {
        return HGRMS_EAGAIN;
    }
    const int k = r->k;
    if (info) {
        info->k = k;
        info->latency_ms = ms_between(r->t_submit, r->t_done);
        info->queue_ms = ms_between(r->t_submit, r->t_start);
        info->batch_size = r->batch_size;
        info->slot = r->slot;
    }
    s->reqs.erase(it);
    delete r;
    return k;
}

HG_EXPORT int hgrms_server_stats(hgrms_server_t s, long long* served, long long* batches, long long* queued,
                                 long long* max_in_flight) {
    if (!s) return HGRMS_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (served) *served = s->served;
    if (batches) *batches = s->batches;
    if (queued) *queued = (long long)s->queue.size();
    if (max_in_flight) *max_in_flight = s->max_in_flight;
    return s->error;
}

HG_EXPORT int hgrms_server_fail_allocations(hgrms_server_t s, int n) {
    if (!s || n < 0) return HGRMS_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    s->fail_allocs = n;
    return HGRMS_OK;
}

HG_EXPORT void hgrms_server_destroy(hgrms_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (std::thread& t : s->workers) t.join();
    for (hgrms_t h : s->handles) hgrms_destroy(h);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (s->coop) cudaStreamDestroy(s->coop);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}
