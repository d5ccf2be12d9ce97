// Host runtime behind the C ABI declared in include/hgrms.h.
//
// One call of hgrms_denoise:
//   1. copy the image into canvas A (padded, 16-byte aligned rows),
//   2. reset the device control block (k = 0, current canvas = A),
//   3. enqueue the passes (Section 2's iteration): by default one fused
//      launch of T passes on shared-memory tiles (the passes where many
//      pixels change), then one list-pass launch per remaining pass, which
//      evaluates only the windows around the pixels the previous pass
//      changed.  The last CTA of each launch updates k, the converged flag
//      and the current canvas on the device, so no launch waits for the
//      host; launches after the end return at once,
//   4. copy the current canvas back and read k with one device-to-host copy.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <new>
#include <vector>

#include "../../include/hgrms.h"
#include "fused.cuh"
#include "kernels.h"

#define HG_EXPORT extern "C" __attribute__((visibility("default")))

struct hgrms_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    uint8_t* canvas[3] = {nullptr, nullptr, nullptr};
    size_t canvas_bytes = 0;
    uint32_t* chg_maps = nullptr;  // three pixel change bitmaps (repeated fused launches)
    size_t chg_map_bytes = 0;
    uint32_t* lists = nullptr;     // four change lists (list passes)
    size_t list_cap = 0;
    uint32_t* bitmaps = nullptr;   // four per-pixel change bitmaps (list passes)
    size_t bitmap_words = 0;
    hg::GridBar* bar = nullptr;    // list-pass loop barrier
    hg::Ctrl* ctrl = nullptr;
    hg::Ctrl* host_ctrl = nullptr;
    int last_cuda_error = 0;
    int converged = 0;
    int opt_kernel = 0;
    int opt_passes = 0;
    int opt_timing = 0;
    int opt_list_cap = 0;
    hgrms_stats_t stats{};
    std::vector<cudaEvent_t> events;
    std::vector<float> launch_ms;  // per-launch durations of the last call (HGRMS_OPT_TIMING)
    std::vector<int> launch_kind;  // 0 = fused, 1 = list pass, 2 = unfused
};

namespace hg {

const FusedEntry* find_fused(int beta, int T) {
    const hg::FusedEntry* tabs[3] = {hg::kFusedB1, hg::kFusedB2, hg::kFusedB3};
    const int counts[3] = {hg::kFusedB1Count, hg::kFusedB2Count, hg::kFusedB3Count};
    for (int t = 0; t < 3; ++t)
        for (int i = 0; i < counts[t]; ++i)
            if (tabs[t][i].beta == beta && tabs[t][i].T == T) return &tabs[t][i];
    return nullptr;
}

int default_passes(int beta) {
    switch (beta) {
        case 1: return 8;
        case 2: return 4;
        case 3: return 2;
        case 4: return 2;
        default: return 1;
    }
}

}  // namespace hg

namespace {

using hg::default_passes;
using hg::find_fused;

int cuda_fail(hgrms_ctx* h, cudaError_t e) {
    h->last_cuda_error = (int)e;
    if (e == cudaErrorMemoryAllocation) return HGRMS_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInvalidDevice) return HGRMS_ENODEV;
    return HGRMS_ECUDA;
}

#define HG_TRY(h, call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail((h), e_); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int check_args(int rows, int cols, int alpha, int beta, int max_k) {
    if (rows < 1 || cols < 1 || rows > 65536 || cols > 65536) return HGRMS_EINVAL;
    if (alpha < 0 || alpha > 255) return HGRMS_EINVAL;
    if (beta < 1 || beta > hg::kMaxBeta) return HGRMS_EINVAL;
    if (max_k < 0 || max_k > 1000000) return HGRMS_EINVAL;
    return HGRMS_OK;
}

// Where a pointer lives: 1 = device memory of `device`, 0 = host, -1 = device
// memory of another device (rejected).
int pointer_kind(const void* p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return at.device == device ? 1 : -1;
    return 0;
}

enum Schedule { kHybrid = 0, kPlain = 1, kFusedOnly = 2 };

struct Plan {
    int schedule;
    bool fused;
    const hg::FusedEntry* fe;
    int T;
    int tiles_x, tiles_y;
    long long pitch;
    long long crows;
    int launches;       // all launches
    int fused_launches; // of which fused
    int map_words;
    size_t list_cap;
    int bm_words;
};

int make_plan(hgrms_ctx* h, int rows, int cols, int beta, int max_k, Plan* p) {
    p->schedule = h->opt_kernel;
    p->fused = p->schedule != kPlain;
    p->fe = nullptr;
    p->list_cap = 0;
    p->bm_words = 0;
    if (p->fused) {
        p->T = h->opt_passes > 0 ? h->opt_passes : default_passes(beta);
        p->fe = find_fused(beta, p->T);
        if (!p->fe) return HGRMS_EINVAL;
        p->tiles_x = (cols + p->fe->TW - 1) / p->fe->TW;
        p->tiles_y = (rows + p->fe->TH - 1) / p->fe->TH;
        const long long need_w = hg::kPadX + (long long)p->tiles_x * p->fe->TW + 16;
        p->pitch = (need_w + 127) / 128 * 128;
        p->crows = hg::kPadY + (long long)p->tiles_y * p->fe->TH + 16;
        if (p->schedule == kHybrid) {
            p->fused_launches = max_k > 0 ? 1 : 0;
            p->launches = max_k > p->T ? 2 : p->fused_launches;  // + one launch running every list pass
            p->map_words = 0;
            p->list_cap = h->opt_list_cap > 0 ? (size_t)h->opt_list_cap
                                              : (size_t)rows * (size_t)cols / 4 + 65536;
            p->bm_words = (cols + 31) / 32 + 1;
        } else {
            p->fused_launches = p->launches = (max_k + p->T - 1) / p->T;
            p->map_words = (p->tiles_x * p->fe->TW + 31) / 32 + 2;
        }
    } else {
        p->T = 1;
        p->tiles_x = p->tiles_y = 0;
        const long long need_w = hg::kPadX + (long long)cols + 16;
        p->pitch = (need_w + 127) / 128 * 128;
        p->crows = hg::kPadY + (long long)rows + 16;
        p->launches = max_k;
        p->fused_launches = 0;
        p->map_words = 0;
    }
    return HGRMS_OK;
}

int ensure_canvas(hgrms_ctx* h, size_t bytes) {
    if (bytes <= h->canvas_bytes) return HGRMS_OK;
    for (int i = 0; i < 3; ++i) {
        if (h->canvas[i]) cudaFree(h->canvas[i]);
        h->canvas[i] = nullptr;
    }
    h->canvas_bytes = 0;
    for (int i = 0; i < 3; ++i) {
        HG_TRY(h, cudaMalloc(&h->canvas[i], bytes));
        HG_TRY(h, cudaMemsetAsync(h->canvas[i], 0, bytes, h->stream));
    }
    h->canvas_bytes = bytes;
    return HGRMS_OK;
}

int ensure_maps(hgrms_ctx* h, size_t bytes) {
    if (bytes <= h->chg_map_bytes) return HGRMS_OK;
    if (h->chg_maps) cudaFree(h->chg_maps);
    h->chg_maps = nullptr;
    h->chg_map_bytes = 0;
    HG_TRY(h, cudaMalloc(&h->chg_maps, bytes));
    h->chg_map_bytes = bytes;
    return HGRMS_OK;
}

int ensure_lists(hgrms_ctx* h, size_t cap, size_t bm_words) {
    if (cap > h->list_cap) {
        if (h->lists) cudaFree(h->lists);
        h->lists = nullptr;
        h->list_cap = 0;
        HG_TRY(h, cudaMalloc(&h->lists, 4 * cap * sizeof(uint32_t)));
        h->list_cap = cap;
    }
    if (bm_words > h->bitmap_words) {
        if (h->bitmaps) cudaFree(h->bitmaps);
        h->bitmaps = nullptr;
        h->bitmap_words = 0;
        HG_TRY(h, cudaMalloc(&h->bitmaps, 4 * bm_words * sizeof(uint32_t)));
        h->bitmap_words = bm_words;
    }
    return HGRMS_OK;
}

int ensure_events(hgrms_ctx* h, size_t n) {
    while (h->events.size() < n) {
        cudaEvent_t e;
        HG_TRY(h, cudaEventCreate(&e));
        h->events.push_back(e);
    }
    return HGRMS_OK;
}

// Everything of one denoise except argument checks.  `dev` tells whether img
// is device memory.
int denoise_one(hgrms_ctx* h, uint8_t* img, int rows, int cols, int alpha, int beta, int max_k,
                bool dev, bool sync_and_finish) {
    Plan p;
    int rc = make_plan(h, rows, cols, beta, max_k, &p);
    if (rc < 0) return rc;
    rc = ensure_canvas(h, (size_t)(p.pitch * p.crows));
    if (rc < 0) return rc;
    const size_t map_bytes = (size_t)rows * (size_t)p.map_words * sizeof(uint32_t);
    if (p.map_words > 0) {
        rc = ensure_maps(h, 3 * map_bytes);
        if (rc < 0) return rc;
    }
    const size_t bm_size = (size_t)rows * (size_t)p.bm_words;
    if (p.list_cap > 0) {
        rc = ensure_lists(h, p.list_cap, bm_size);
        if (rc < 0) return rc;
    }
    cudaStream_t s = h->stream;
    uint8_t* ca = h->canvas[0];
    if (dev) {
        HG_TRY(h, hg::launch_copy_in(img, rows, cols, ca, p.pitch, h->sms, s));
    } else {
        HG_TRY(h, cudaMemcpy2DAsync(ca + hg::kPadY * p.pitch + hg::kPadX, (size_t)p.pitch, img,
                                    (size_t)cols, (size_t)cols, (size_t)rows, cudaMemcpyHostToDevice, s));
    }
    HG_TRY(h, hg::launch_ctrl_init(h->ctrl, (unsigned)max_k, s));
    // Map 0 is written by the first launch; the launches clear the others.
    if (p.map_words > 0) HG_TRY(h, cudaMemsetAsync(h->chg_maps, 0, map_bytes, s));
    // The change bitmaps start empty; each list pass clears one for a later pass.
    if (p.list_cap > 0) {
        HG_TRY(h, cudaMemsetAsync(h->bitmaps, 0, 4 * bm_size * sizeof(uint32_t), s));
        HG_TRY(h, cudaMemsetAsync(h->bar, 0, sizeof(hg::GridBar), s));
    }
    hg::PassArgs a;
    for (int i = 0; i < 3; ++i) a.canvas[i] = h->canvas[i];
    a.pitch = p.pitch;
    a.rows = rows;
    a.cols = cols;
    a.alpha = alpha;
    a.tiles_x = p.tiles_x;
    a.ctrl = h->ctrl;
    a.chg_maps = p.map_words > 0 ? h->chg_maps : nullptr;
    a.map_words = p.map_words;
    for (int i = 0; i < 4; ++i) {
        a.lists[i] = p.list_cap > 0 ? h->lists + i * p.list_cap : nullptr;
        a.bitmaps[i] = p.list_cap > 0 ? h->bitmaps + i * bm_size : nullptr;
    }
    a.list_cap = (unsigned)p.list_cap;
    a.bm_words = p.bm_words;
    a.bar = h->bar;
    a.write_prev = p.schedule == kHybrid ? 1 : 0;
    // Per-launch timing is limited to calls of at most kMaxTimedLaunches launches.
    constexpr int kMaxTimedLaunches = 4096;
    const bool timed = h->opt_timing && p.launches <= kMaxTimedLaunches;
    if (timed) {
        rc = ensure_events(h, 2 * (size_t)p.launches);
        if (rc < 0) return rc;
    }
    for (int i = 0; i < p.launches; ++i) {
        if (timed) HG_TRY(h, cudaEventRecord(h->events[2 * i], s));
        if (i < p.fused_launches)
            HG_TRY(h, p.fe->launch(a, p.tiles_y, s));
        else if (p.fused)
            HG_TRY(h, hg::launch_list(beta, a, h->sms, s));
        else
            HG_TRY(h, hg::launch_plain(beta, a, s));
        if (timed) HG_TRY(h, cudaEventRecord(h->events[2 * i + 1], s));
    }
    if (dev) HG_TRY(h, hg::launch_copy_out(h->ctrl, h->canvas, p.pitch, img, rows, cols, h->sms, s));
    h->stats.launches += p.launches;
    h->stats.passes_per_launch = p.T;
    h->stats.tile_rows = p.fused ? p.fe->TH : 0;
    h->stats.tile_cols = p.fused ? p.fe->TW : 0;
    h->stats.ctas_per_launch = p.fused ? (long long)p.tiles_x * p.tiles_y
                                       : (long long)((cols + 31) / 32) * ((rows + 7) / 8);
    if (!sync_and_finish) return HGRMS_OK;
    HG_TRY(h, cudaMemcpyAsync(h->host_ctrl, h->ctrl, sizeof(hg::Ctrl), cudaMemcpyDeviceToHost, s));
    HG_TRY(h, cudaStreamSynchronize(s));
    const hg::Ctrl c = *h->host_ctrl;
    if (!dev) {
        const uint8_t* fin = h->canvas[c.cur];
        HG_TRY(h, cudaMemcpy2DAsync(img, (size_t)cols, fin + hg::kPadY * p.pitch + hg::kPadX, (size_t)p.pitch,
                                    (size_t)cols, (size_t)rows, cudaMemcpyDeviceToHost, s));
        HG_TRY(h, cudaStreamSynchronize(s));
    }
    if (timed) {
        // Launches after the call finished return at once; once one does, all
        // later ones do, so the first work_launches launches are the working ones.
        for (int i = 0; i < p.launches; ++i) {
            float ms = 0.f;
            HG_TRY(h, cudaEventElapsedTime(&ms, h->events[2 * i], h->events[2 * i + 1]));
            h->launch_ms.push_back(ms);
            h->launch_kind.push_back(i < p.fused_launches ? 0 : (p.fused ? 1 : 2));
            if (i < (int)c.work_launches)
                h->stats.kernel_ms += ms;
            else
                h->stats.idle_kernel_ms += ms;
        }
    }
    if (c.error) {
        h->last_cuda_error = 0;
        return HGRMS_ETIMEOUT;
    }
    h->stats.passes_executed += (int)c.executed;
    h->stats.evals_fused += (long long)c.evals_fused;
    h->stats.evals_list += (long long)c.evals_list;
    h->stats.work_launches += (int)c.work_launches;
    h->stats.passes += (int)(c.k + c.converged);
    h->converged = (int)c.converged;
    return (int)c.k;
}

}  // namespace

HG_EXPORT int hgrms_create(hgrms_t* out, int device, void* cuda_stream) {
    if (!out) return HGRMS_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return HGRMS_ENODEV;
    }
    if (device < 0 || device >= n) return HGRMS_ENODEV;
    hgrms_ctx* h = new (std::nothrow) hgrms_ctx();
    if (!h) return HGRMS_ENOMEM;
    DeviceGuard g(device);
    h->device = device;
    h->stream = (cudaStream_t)cuda_stream;
    int rc = HGRMS_OK;
    cudaError_t e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&h->ctrl, sizeof(hg::Ctrl));
    if (e == cudaSuccess) e = cudaMalloc(&h->bar, sizeof(hg::GridBar));
    if (e == cudaSuccess) e = cudaMemset(h->ctrl, 0, sizeof(hg::Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost(&h->host_ctrl, sizeof(hg::Ctrl));
    if (e != cudaSuccess) {
        rc = cuda_fail(h, e);
        hgrms_destroy(h);
        return rc;
    }
    *out = h;
    return HGRMS_OK;
}

HG_EXPORT void hgrms_destroy(hgrms_t h) {
    if (!h) return;
    {
        DeviceGuard g(h->device);
        if (h->stream) cudaStreamSynchronize(h->stream);
        for (int i = 0; i < 3; ++i)
            if (h->canvas[i]) cudaFree(h->canvas[i]);
        if (h->ctrl) cudaFree(h->ctrl);
        if (h->bar) cudaFree(h->bar);
        if (h->chg_maps) cudaFree(h->chg_maps);
        if (h->lists) cudaFree(h->lists);
        if (h->bitmaps) cudaFree(h->bitmaps);
        if (h->host_ctrl) cudaFreeHost(h->host_ctrl);
        for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    }
    delete h;
}

HG_EXPORT int hgrms_denoise(hgrms_t h, uint8_t* img, int rows, int cols, int alpha, int beta, int max_k) {
    if (!h || !img) return HGRMS_EINVAL;
    int rc = check_args(rows, cols, alpha, beta, max_k);
    if (rc < 0) return rc;
    DeviceGuard g(h->device);
    const int kind = pointer_kind(img, h->device);
    if (kind < 0) return HGRMS_EINVAL;
    h->stats = hgrms_stats_t{};
    h->launch_ms.clear();
    h->launch_kind.clear();
    return denoise_one(h, img, rows, cols, alpha, beta, max_k, kind == 1, true);
}

HG_EXPORT int hgrms_denoise_batch(hgrms_t h, uint8_t* const* imgs, const int* rows, const int* cols, int n,
                                  int alpha, int beta, int max_k, int* k_out) {
    if (!h || n < 0 || (n > 0 && (!imgs || !rows || !cols || !k_out))) return HGRMS_EINVAL;
    DeviceGuard g(h->device);
    int kind0 = -2;
    for (int i = 0; i < n; ++i) {
        if (!imgs[i]) return HGRMS_EINVAL;
        int rc = check_args(rows[i], cols[i], alpha, beta, max_k);
        if (rc < 0) return rc;
        const int kind = pointer_kind(imgs[i], h->device);
        if (kind < 0) return HGRMS_EINVAL;
        if (kind0 == -2) kind0 = kind;
        if (kind != kind0) return HGRMS_EINVAL;
    }
    hgrms_stats_t acc{};
    int all_conv = 1;
    h->launch_ms.clear();
    h->launch_kind.clear();
    for (int i = 0; i < n; ++i) {
        h->stats = hgrms_stats_t{};
        const int k = denoise_one(h, imgs[i], rows[i], cols[i], alpha, beta, max_k, kind0 == 1, true);
        if (k < 0) return k;
        k_out[i] = k;
        all_conv &= h->converged;
        acc.launches += h->stats.launches;
        acc.work_launches += h->stats.work_launches;
        acc.passes += h->stats.passes;
        acc.kernel_ms += h->stats.kernel_ms;
        acc.idle_kernel_ms += h->stats.idle_kernel_ms;
        acc.passes_executed += h->stats.passes_executed;
        acc.evals_fused += h->stats.evals_fused;
        acc.evals_list += h->stats.evals_list;
        acc.passes_per_launch = h->stats.passes_per_launch;
        acc.tile_rows = h->stats.tile_rows;
        acc.tile_cols = h->stats.tile_cols;
        acc.ctas_per_launch += h->stats.ctas_per_launch;
    }
    h->stats = acc;
    h->converged = all_conv;
    return HGRMS_OK;
}

HG_EXPORT int hgrms_converged(hgrms_t h) {
    if (!h) return HGRMS_EINVAL;
    return h->converged;
}

HG_EXPORT const char* hgrms_strerror(int code) {
    switch (code) {
        case HGRMS_OK: return "success";
        case HGRMS_EINVAL: return "invalid argument";
        case HGRMS_ENOMEM: return "out of memory";
        case HGRMS_ECUDA: return "CUDA error";
        case HGRMS_ETIMEOUT: return "device wait timed out";
        case HGRMS_ENODEV: return "no CUDA device";
        case HGRMS_ETOOBIG: return "image too large for the fixed scratch of hgrms_denoise_noalloc";
        default: return code >= 0 ? "success" : "unknown error";
    }
}

HG_EXPORT int hgrms_last_cuda_error(hgrms_t h) {
    if (!h) return HGRMS_EINVAL;
    return h->last_cuda_error;
}

HG_EXPORT int hgrms_set_option(hgrms_t h, int option, int value) {
    if (!h) return HGRMS_EINVAL;
    switch (option) {
        case HGRMS_OPT_KERNEL:
            if (value < 0 || value > 2) return HGRMS_EINVAL;
            h->opt_kernel = value;
            return HGRMS_OK;
        case HGRMS_OPT_PASSES:
            if (value < 0 || value > 32) return HGRMS_EINVAL;
            h->opt_passes = value;
            return HGRMS_OK;
        case HGRMS_OPT_TIMING:
            if (value != 0 && value != 1) return HGRMS_EINVAL;
            h->opt_timing = value;
            return HGRMS_OK;
        case HGRMS_OPT_LIST_CAP:
            if (value < 0) return HGRMS_EINVAL;
            h->opt_list_cap = value;
            return HGRMS_OK;
        default: return HGRMS_EINVAL;
    }
}

HG_EXPORT int hgrms_stats(hgrms_t h, hgrms_stats_t* out) {
    if (!h || !out) return HGRMS_EINVAL;
    *out = h->stats;
    return HGRMS_OK;
}

HG_EXPORT int hgrms_launch_times(hgrms_t h, float* ms, int* kind, int n) {
    if (!h || n < 0 || (n > 0 && !ms)) return HGRMS_EINVAL;
    const int m = (int)h->launch_ms.size();
    for (int i = 0; i < n && i < m; ++i) {
        ms[i] = h->launch_ms[i];
        if (kind) kind[i] = h->launch_kind[i];
    }
    return m;
}

HG_EXPORT int hgrms_default_passes(int beta) {
    if (beta < 1 || beta > hg::kMaxBeta) return HGRMS_EINVAL;
    return default_passes(beta);
}

HG_EXPORT int hgrms_has_kernel(int beta, int passes) {
    return find_fused(beta, passes) != nullptr ? 1 : 0;
}
