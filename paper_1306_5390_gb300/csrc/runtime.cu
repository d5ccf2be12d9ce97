// Host runtime behind the C ABI declared in include/hgrms.h.
//
// One call of hgrms_denoise (or one chunk of hgrms_denoise_batch, whose
// images are laid out side by side in the same buffers):
//   1. host images the device cannot read are copied into canvas A (padded,
//      16-byte aligned rows); the first fused launch reads the others
//      (device memory, mapped page-locked host memory) directly,
//   2. reset the device control block (k = 0, current canvas = A),
//   3. enqueue the passes (Section 2's iteration): by default one fused
//      launch of T passes on shared-memory tiles of every image (the passes
//      where many pixels change), then one persistent launch that runs each
//      remaining pass as a list pass, evaluating only the windows around the
//      pixels the previous pass changed.  k, the converged flag and the
//      current canvas are kept on the device, so no launch waits for the
//      host,
//   4. copy the current canvas back and read k with one device-to-host copy.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/hgrms.h"
#include "fused.cuh"
#include "kernels.h"

#define HG_EXPORT extern "C" __attribute__((visibility("default")))

// Fused passes per launch and in-tile list/dense switch point of one call
// (0: the built-in one for the call's tiles).
struct Tuning {
    int T;
    int eval_max;
};

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
    // Image table of the hybrid schedule (device copy, pinned staging copy),
    // the fused tile -> image map and the per-image k of a batch.
    hg::ImgDesc* d_desc = nullptr;
    size_t desc_cap = 0;
    hg::ImgDesc* host_desc = nullptr;
    size_t host_desc_cap = 0;
    int* tile_img = nullptr;
    size_t tile_cap = 0;
    unsigned* img_k = nullptr;
    unsigned* host_img_k = nullptr;
    size_t img_k_cap = 0;
    std::vector<hg::ImgDesc> table_cache;  // what d_desc and tile_img hold now
    int table_tiles = -1;
    int opt_batch_mb = 0;
    int opt_relaunch_ppm = 0;
    int opt_tile_eval_max = 0;
    int opt_autotune = 0;
    int opt_list_ctas = 0;
    int opt_wait_test = 0;
    int opt_tma = 1;
    // Tensor maps of the fused kernel's TMA tile loads (kTmaMapsPerImage per
    // image), on the device, and the layout they were made for.
    CUtensorMap* tmaps = nullptr;
    CUtensorMap* tmaps_host = nullptr;  // page-locked staging of the maps' upload
    cudaEvent_t tmaps_ev = nullptr;     // recorded after the upload from tmaps_host
    size_t tmaps_cap = 0;
    std::vector<uint8_t> tmaps_key;
    int tmaps_user = 0;
    std::map<long long, Tuning> tuned;  // autotuner choices by (beta, batch, size class)
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    // Stream shared with other handles whose work overlaps this one's (the
    // request server's slots): the list-pass launch, a cooperative launch
    // whose CTAs wait for one another, runs there, so two such launches never
    // share the device.  Null: the handle's own stream.
    cudaStream_t coop_stream = nullptr;
    cudaEvent_t coop_ev[2] = {nullptr, nullptr};
    // Recorded after this handle's latest list-pass launch (see chain_coop).
    cudaEvent_t chain_ev = nullptr;
    // Learned k-predictor (weights loaded by hgrms_predictor_load) and its
    // image table.
    hg::Predictor* pred[hg::kMaxBeta + 1] = {};  // by beta
    hg::ImgDesc* pred_desc = nullptr;
    int pred_desc_cap = 0;
    int opt_predict_k = 0;
    // HGRMS_OPT_GRAPH: captured CUDA graphs of whole hybrid calls, by the
    // bytes of everything the call's device work depends on (oldest first),
    // and the stream they are captured on (the legacy default stream cannot
    // be captured).
    int opt_graph = 0;
    std::vector<std::pair<std::vector<uint8_t>, cudaGraphExec_t>> graphs;
    cudaStream_t cap_stream = nullptr;
    // The call that hgrms_denoise_async queued and hgrms_wait has not yet
    // finished (see PendingCall).
    struct PendingCall {
        bool active = false;  // a call is outstanding
        bool done = false;    // it already ran synchronously; `result` holds its return value
        int result = 0;
        int n = 0, max_k = 0, launches = 0, fused_launches = 0, T = 0, eval_max = 0, TH = 0, TW = 0;
        long long tiles_total = 0;
        bool per_image_k = false, write_back = false, timed = false;
    } pending;
};

namespace hg {

const FusedEntry* find_fused(int beta, int T, int rn) {
    const hg::FusedEntry* tabs[3] = {hg::kFusedB1, hg::kFusedB2, hg::kFusedB3};
    const int counts[3] = {hg::kFusedB1Count, hg::kFusedB2Count, hg::kFusedB3Count};
    for (int t = 0; t < 3; ++t)
        for (int i = 0; i < counts[t]; ++i)
            if (tabs[t][i].beta == beta && tabs[t][i].T == T && tabs[t][i].RN == rn) return &tabs[t][i];
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

// Hybrid schedule: fused launches after the first (each runs only when the
// previous one left many changed pixels; a launch that does not run still
// costs a few microseconds).  Default: for beta 1 (T = 8, the cheapest fused
// pass) up to 3 of them, when a list pass would evaluate more than 2.5 % of
// the pixels (measured on GB300: list passes stay faster below that); none
// for wider windows, whose fused passes cost more than list passes even on
// dense change sets.  With HGRMS_OPT_RELAUNCH_PPM set, up to 8 for any beta.
constexpr int kDefaultRelaunches = 3;
// Calls of at least this many pixels use the 128-row tiles (where compiled
// and they compute fewer rows): measured faster on 8192 x 8192 and on the
// 629 M-pixel uneven batch; smaller calls keep the 64-row tiles, whose larger
// tile count spreads better over the SMs.
constexpr long long kTallMinPixels = 32ll << 20;
constexpr long long kRelaunchMinPixels = 4ll << 20;
constexpr size_t kMaxGraphs = 8;  // captured graphs kept per handle (HGRMS_OPT_GRAPH)
constexpr int kMaxRelaunches = 8;
long long default_relaunch_ppm(int beta) {
    return beta == 1 ? 25000 : 1000000;
}

using hg::default_passes;
using hg::find_fused;

// Cooperative list-pass launches of every handle of the process on one device
// run one after another, in the order they are issued.  The CTAs of such a
// launch wait for one another at every pass, so two of them overlapping on
// the device could each hold SM slots that the other's CTAs need, and both
// would wait until their bounded barrier gives up.  Each launch (or replayed
// graph that holds one) first makes its stream wait for the event recorded
// after the previous one, whichever stream and handle that was.
constexpr int kMaxChainDevices = 64;
std::mutex g_chain_mu;
cudaEvent_t g_chain_last[kMaxChainDevices] = {};
cudaStream_t g_chain_stream[kMaxChainDevices] = {};

// Run `launch` (which queues work holding a cooperative launch on stream s)
// behind the device's previous cooperative launch, then record h->chain_ev
// after it.  Not for use while a stream is being captured.
template <class F>
cudaError_t chain_coop(hgrms_ctx* h, cudaStream_t s, F&& launch) {
    const int dev = h->device;
    if (dev < 0 || dev >= kMaxChainDevices) return launch();
    std::lock_guard<std::mutex> lock(g_chain_mu);
    cudaError_t e = cudaSuccess;
    if (!h->chain_ev) e = cudaEventCreateWithFlags(&h->chain_ev, cudaEventDisableTiming);
    if (e == cudaSuccess && g_chain_last[dev] && g_chain_stream[dev] != s)
        e = cudaStreamWaitEvent(s, g_chain_last[dev], 0);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(h->chain_ev, s);
    if (e == cudaSuccess) {
        g_chain_last[dev] = h->chain_ev;
        g_chain_stream[dev] = s;
    }
    return e;
}

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

// A named NVTX range over the scope: profilers (ncu --nvtx, Nsight Systems)
// show the library's calls and the enqueue of its launches by name; without
// a profiler attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

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

// Where a pointer lives: 1 = memory the device reads and writes directly
// (device memory of `device`, or page-locked host memory mapped into the
// device's address space, whose device address goes to *devp), 0 = other
// host memory (staged by copies), -1 = device memory of another device
// (rejected).
int pointer_kind(const void* p, int device, uint8_t** devp) {
    *devp = const_cast<uint8_t*>(static_cast<const uint8_t*>(p));
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return at.device == device ? 1 : -1;
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        *devp = static_cast<uint8_t*>(at.devicePointer);
        return 1;
    }
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

// Launch plan of the unfused and fused-only schedules (the hybrid schedule
// is run_hybrid's).
int make_plan(hgrms_ctx* h, int rows, int cols, int beta, int max_k, Plan* p) {
    p->schedule = h->opt_kernel;
    if (p->schedule == kHybrid) return HGRMS_EINVAL;
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
        p->fused_launches = p->launches = (max_k + p->T - 1) / p->T;
        p->map_words = (p->tiles_x * p->fe->TW + 31) / 32 + 2;
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

// The handle's buffers grow geometrically (to at least 1.5 times their old
// size), so that a stream of calls of slowly growing size - the request
// server's batches - reallocates rarely: cudaFree waits for the whole device.
// A growth that does not fit falls back to the exact size.
size_t grown(size_t need, size_t have) {
    return have > 0 && need < have + have / 2 ? have + have / 2 : need;
}
// cudaMalloc of `want` bytes (a grown size), else of `need` bytes; *got
// receives the size allocated.
cudaError_t malloc_grown(void** p, size_t want, size_t need, size_t* got) {
    cudaError_t e = cudaMalloc(p, want);
    if (e == cudaErrorMemoryAllocation && want > need) {
        cudaGetLastError();
        want = need;
        e = cudaMalloc(p, want);
    }
    *got = e == cudaSuccess ? want : 0;
    return e;
}

int ensure_canvas(hgrms_ctx* h, size_t bytes) {
    if (bytes <= h->canvas_bytes) return HGRMS_OK;
    size_t got = grown(bytes, h->canvas_bytes);
    for (int i = 0; i < 3; ++i) {
        if (h->canvas[i]) cudaFree(h->canvas[i]);
        h->canvas[i] = nullptr;
    }
    h->canvas_bytes = 0;
    for (int i = 0; i < 3; ++i) {
        size_t g = 0;
        HG_TRY(h, malloc_grown(reinterpret_cast<void**>(&h->canvas[i]), got, bytes, &g));
        got = g;  // a later canvas never asks for more than an earlier one got
    }
    for (int i = 0; i < 3; ++i) HG_TRY(h, cudaMemsetAsync(h->canvas[i], 0, got, h->stream));
    h->canvas_bytes = got;
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
        const size_t want = grown(cap, h->list_cap);
        if (h->lists) cudaFree(h->lists);
        h->lists = nullptr;
        h->list_cap = 0;
        size_t got = 0;
        HG_TRY(h, malloc_grown(reinterpret_cast<void**>(&h->lists), 4 * want * sizeof(uint32_t),
                               4 * cap * sizeof(uint32_t), &got));
        h->list_cap = got / (4 * sizeof(uint32_t));
    }
    if (bm_words > h->bitmap_words) {
        const size_t want = grown(bm_words, h->bitmap_words);
        if (h->bitmaps) cudaFree(h->bitmaps);
        h->bitmaps = nullptr;
        h->bitmap_words = 0;
        size_t got = 0;
        HG_TRY(h, malloc_grown(reinterpret_cast<void**>(&h->bitmaps), 4 * want * sizeof(uint32_t),
                               4 * bm_words * sizeof(uint32_t), &got));
        h->bitmap_words = got / (4 * sizeof(uint32_t));
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

// Device and pinned host buffers of the image table for n images and
// `tiles` fused tiles; a reallocation invalidates the cached table.
int ensure_table(hgrms_ctx* h, size_t n, size_t tiles, bool per_image_k) {
    if (n > h->desc_cap) {
        n = grown(n, h->desc_cap);
        if (h->d_desc) cudaFree(h->d_desc);
        if (h->host_desc) cudaFreeHost(h->host_desc);
        h->d_desc = nullptr;
        h->host_desc = nullptr;
        h->desc_cap = 0;
        h->table_tiles = -1;
        HG_TRY(h, cudaMalloc(&h->d_desc, n * sizeof(hg::ImgDesc)));
        HG_TRY(h, cudaMallocHost(&h->host_desc, n * sizeof(hg::ImgDesc)));
        h->desc_cap = n;
    }
    if (tiles > h->tile_cap) {
        tiles = grown(tiles, h->tile_cap);
        if (h->tile_img) cudaFree(h->tile_img);
        h->tile_img = nullptr;
        h->tile_cap = 0;
        h->table_tiles = -1;
        HG_TRY(h, cudaMalloc(&h->tile_img, tiles * sizeof(int)));
        h->tile_cap = tiles;
    }
    if (per_image_k && n > h->img_k_cap) {
        if (h->img_k) cudaFree(h->img_k);
        if (h->host_img_k) cudaFreeHost(h->host_img_k);
        h->img_k = nullptr;
        h->host_img_k = nullptr;
        h->img_k_cap = 0;
        HG_TRY(h, cudaMalloc(&h->img_k, n * sizeof(unsigned)));
        HG_TRY(h, cudaMallocHost(&h->host_img_k, n * sizeof(unsigned)));
        h->img_k_cap = n;
    }
    return HGRMS_OK;
}

// cuTensorMapEncodeTiled from the driver (looked up once; null if absent).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// A 3-D byte view for tile loads: (16 bytes, 16-byte chunks of a row, rows)
// of a row-major array with `pitch` bytes per row (a multiple of 16), whose
// box is one tile with its halo: 17 chunks (272 bytes) by `box_rows` rows.
bool encode_tile_map(CUtensorMap* m, const void* base, long long pitch, long long rows, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || ((uintptr_t)base & 15u) != 0 || pitch % 16 != 0 || pitch < 16 || rows < 1) return false;
    const cuuint64_t dims[3] = {16, (cuuint64_t)(pitch / 16), (cuuint64_t)rows};
    const cuuint64_t strides[2] = {16, (cuuint64_t)pitch};
    const cuuint32_t box[3] = {16, 17, (cuuint32_t)box_rows};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Bits needed for values 0 .. v (at least 1).
int bits_for(long long v) {
    int b = 1;
    while (b < 62 && (1ll << b) <= v) ++b;
    return b;
}

struct BatchImg {
    uint8_t* ptr;
    int rows, cols;
    bool dev;  // device memory of the handle's device (else host memory)
};

// Built-in in-tile list/dense switch point per beta (measured on GB300).
int default_eval_max(int beta) {
    return beta == 2 ? 2048 : 4096;
}

// Canvas, bitmap and list bytes the hybrid schedule needs for one image (a
// chunk needs the sum, plus a small constant).
long long hybrid_bytes(const hg::FusedEntry* fe, int rows, int cols) {
    const long long tiles_x = (cols + fe->TW - 1) / fe->TW, tiles_y = (rows + fe->TH - 1) / fe->TH;
    const long long pitch = (hg::kPadX + tiles_x * fe->TW + 16 + 127) / 128 * 128;
    const long long crows = hg::kPadY + tiles_y * fe->TH + 16;
    const long long px = (long long)rows * cols;
    return 3 * pitch * crows + 4 * 4 * (long long)rows * ((cols + 31) / 32 + 1) + 4 * 4 * (px / 4) + 4 * tiles_x * tiles_y;
}

// Tensor maps for the fused kernel's TMA tile loads of one call (kernel `fe`,
// images `im` laid out as h->host_desc): per image, its canvas in each of the
// three arenas and, for an image in device memory that is 16-byte aligned
// with a width that is a multiple of 16, the image itself (the first fused
// launch reads it directly; the box's rows and columns outside the image read
// zeros).  They are rebuilt only when the layout changes and uploaded in
// stream order from page-locked memory (an upload from pageable memory would
// wait for the stream), outside any captured graph.  Returns false when TMA cannot be
// used for this call (ordinary loads then); *user_ok is 1 when every image
// the first launch reads in place has a map.
bool ensure_tile_maps(hgrms_ctx* h, const hg::FusedEntry* fe, const BatchImg* im, int n, cudaStream_t s,
                      int* user_ok) {
    *user_ok = 0;
    if (!h->opt_tma || !fe->tma || !tensor_map_encoder()) return false;
    std::vector<uint8_t> key;
    auto put = [&key](const void* p, size_t b) {
        const uint8_t* c = static_cast<const uint8_t*>(p);
        key.insert(key.end(), c, c + b);
    };
    put(h->canvas, sizeof(h->canvas));
    put(&fe->SH, sizeof(fe->SH));
    put(&fe->TH, sizeof(fe->TH));
    put(&n, sizeof(n));
    put(h->host_desc, (size_t)n * sizeof(hg::ImgDesc));
    for (int i = 0; i < n; ++i) {
        put(&im[i].ptr, sizeof(im[i].ptr));
        put(&im[i].dev, sizeof(im[i].dev));
    }
    if (key == h->tmaps_key) {
        *user_ok = h->tmaps_user;
        return true;
    }
    h->tmaps_key.clear();
    const size_t nm = (size_t)n * hg::kTmaMapsPerImage;
    // The staging buffer may still be the source of the previous upload.
    if (h->tmaps_ev && cudaEventSynchronize(h->tmaps_ev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (!h->tmaps_ev && cudaEventCreateWithFlags(&h->tmaps_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (nm > h->tmaps_cap) {
        if (h->tmaps) cudaFree(h->tmaps);
        if (h->tmaps_host) cudaFreeHost(h->tmaps_host);
        h->tmaps = nullptr;
        h->tmaps_host = nullptr;
        h->tmaps_cap = 0;
        if (cudaMalloc(&h->tmaps, nm * sizeof(CUtensorMap)) != cudaSuccess ||
            cudaMallocHost(&h->tmaps_host, nm * sizeof(CUtensorMap)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        h->tmaps_cap = nm;
    }
    CUtensorMap* maps = h->tmaps_host;
    memset(maps, 0, nm * sizeof(CUtensorMap));
    int uok = 1;
    for (int i = 0; i < n; ++i) {
        const hg::ImgDesc& d = h->host_desc[i];
        const long long tiles_y = (d.rows + fe->TH - 1) / fe->TH;
        const long long crows = hg::kPadY + tiles_y * fe->TH + 16;
        for (int c = 0; c < 3; ++c)
            if (!encode_tile_map(&maps[(size_t)i * hg::kTmaMapsPerImage + c], h->canvas[c] + d.off, d.pitch, crows,
                                 fe->SH))
                return false;
        if (!im[i].dev) continue;  // copied into canvas 0 first
        cudaPointerAttributes at;
        bool ok = cudaPointerGetAttributes(&at, im[i].ptr) == cudaSuccess && at.type == cudaMemoryTypeDevice;
        if (!ok) cudaGetLastError();
        ok = ok && d.cols % 16 == 0 &&
             encode_tile_map(&maps[(size_t)i * hg::kTmaMapsPerImage + 3], im[i].ptr, d.cols, d.rows, fe->SH);
        if (!ok) uok = 0;
    }
    if (cudaMemcpyAsync(h->tmaps, maps, nm * sizeof(CUtensorMap), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(h->tmaps_ev, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    h->tmaps_key = std::move(key);
    h->tmaps_user = uok;
    *user_ok = uok;
    return true;
}

// The hybrid schedule (one fused launch of T passes over the tiles of every
// image, then one persistent launch running the remaining passes as list
// passes) for n images at once.  k_out[i] gets image i's k; the return value
// is HGRMS_OK or a negative code.  Every image runs the same sequence of
// passes; the sequence ends when a pass changes no pixel of any image or
// after max_k passes, and image i's k is the number of the last pass that
// changed one of its pixels (an image that a pass leaves unchanged is at a
// fixed point, so later passes leave it unchanged too).
//
// `tu` gives the fused passes per launch and the in-tile list/dense switch
// point.  With write_back false the images are not written (an autotuning
// trial); *ms, when given, receives the device time of the call's work.
int finish_hybrid(hgrms_ctx* h, const hgrms_ctx::PendingCall& pd, const BatchImg* im, int* k_out, float* ms);

// Queue one hybrid call (or one chunk of a batch) on the handle's stream.
// Synchronous calls then wait for it and finish (finish_hybrid); with
// `async_call` the call returns after queueing and hgrms_wait finishes it
// (only for images the device reads directly: nothing is copied back on the
// host).
int run_hybrid(hgrms_ctx* h, const BatchImg* im, int n, int alpha, int beta, int max_k, int* k_out,
               const Tuning& tu, bool write_back, float* ms, int forced_fused = 0, bool async_call = false) {
    const int T = tu.T;
    // Large calls (one image or a batch) take the tall tiles when they are
    // compiled for (beta, T) and compute fewer rows with them: at this size
    // every SM still gets many tiles.
    const hg::FusedEntry* fe = find_fused(beta, T);
    if (!fe) return HGRMS_EINVAL;
    {
        const hg::FusedEntry* tall = find_fused(beta, T, 128);
        long long px_call = 0, rows64 = 0, rows128 = 0;
        for (int i = 0; i < n && tall; ++i) {
            const long long tx = (im[i].cols + fe->TW - 1) / fe->TW;
            px_call += (long long)im[i].rows * im[i].cols;
            rows64 += tx * ((im[i].rows + fe->TH - 1) / fe->TH) * 64;
            rows128 += tx * ((im[i].rows + tall->TH - 1) / tall->TH) * 128;
        }
        if (tall && px_call >= kTallMinPixels && rows128 < rows64) fe = tall;
    }
    // The built-in in-tile switch point counts evaluations per 64-row tile.
    const int eval_max = tu.eval_max > 0 ? tu.eval_max : default_eval_max(beta) * (fe->RN / 64);
    const bool per_image_k = n > 1;
    // Layout: image i's canvas at offset off_i of each arena, its bitmap at
    // word bm_off_i of each bitmap arena, its tiles from tile0_i.
    long long canvas_total = 0, bm_total = 0, tiles_total = 0, px_total = 0, max_words = 0;
    int max_rows = 1, max_cols = 1;
    int rc = ensure_table(h, (size_t)n, 0, false);
    if (rc < 0) return rc;
    for (int i = 0; i < n; ++i) {
        const int rows = im[i].rows, cols = im[i].cols;
        const int tiles_x = (cols + fe->TW - 1) / fe->TW, tiles_y = (rows + fe->TH - 1) / fe->TH;
        const long long pitch = (hg::kPadX + (long long)tiles_x * fe->TW + 16 + 127) / 128 * 128;
        const long long crows = hg::kPadY + (long long)tiles_y * fe->TH + 16;
        hg::ImgDesc d;
        memset(&d, 0, sizeof(d));
        d.off = canvas_total;
        d.bm_off = bm_total;
        d.pitch = (int)pitch;
        d.rows = rows;
        d.cols = cols;
        d.tiles_x = tiles_x;
        d.tile0 = (int)tiles_total;
        d.bm_words = (cols + 31) / 32 + 1;
        d.user = (n > 1 && im[i].dev) ? im[i].ptr : nullptr;
        h->host_desc[i] = d;
        canvas_total += pitch * crows;
        bm_total += (long long)rows * d.bm_words;
        tiles_total += (long long)tiles_x * tiles_y;
        px_total += (long long)rows * cols;
        const long long words = ((long long)rows * cols + 3) / 4 + 1;
        if (words > max_words) max_words = words;
        if (rows > max_rows) max_rows = rows;
        if (cols > max_cols) max_cols = cols;
    }
    if (tiles_total > 0x7fffffffll) return HGRMS_EINVAL;
    // Entry packing: a single image uses 16 + 16 bits (the list loop's
    // single-image form assumes it), a batch the fewest bits its sizes need.
    const int xb = n > 1 ? bits_for(max_cols - 1) : 16, yb = n > 1 ? bits_for(max_rows - 1) : 16;
    if (xb + yb + (n > 1 ? bits_for(n - 1) : 0) > 32) return HGRMS_EINVAL;  // chunking keeps this from happening
    const size_t list_cap = h->opt_list_cap > 0 ? (size_t)h->opt_list_cap : (size_t)(px_total / 4 + 65536);
    rc = ensure_canvas(h, (size_t)canvas_total);
    if (rc < 0) return rc;
    rc = ensure_lists(h, list_cap, (size_t)bm_total);
    if (rc < 0) return rc;
    rc = ensure_table(h, (size_t)n, (size_t)tiles_total, per_image_k);
    if (rc < 0) return rc;
    cudaStream_t s = h->stream;
    // The table and tile map on the device (skipped when unchanged).
    const bool same = h->table_tiles == (int)tiles_total && h->table_cache.size() == (size_t)n &&
                      memcmp(h->table_cache.data(), h->host_desc, (size_t)n * sizeof(hg::ImgDesc)) == 0;
    if (!same) {
        HG_TRY(h, cudaMemcpyAsync(h->d_desc, h->host_desc, (size_t)n * sizeof(hg::ImgDesc), cudaMemcpyHostToDevice, s));
        HG_TRY(h, hg::launch_tile_map(h->d_desc, n, (int)tiles_total, h->tile_img, s));
        h->table_cache.assign(h->host_desc, h->host_desc + n);
        h->table_tiles = (int)tiles_total;
    }
    hg::PassArgs a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < 3; ++i) a.canvas[i] = h->canvas[i];
    a.pitch = h->host_desc[0].pitch;
    a.rows = h->host_desc[0].rows;
    a.cols = h->host_desc[0].cols;
    a.alpha = alpha;
    a.tiles_x = h->host_desc[0].tiles_x;
    a.ctrl = h->ctrl;
    a.chg_maps = nullptr;
    a.map_words = 0;
    for (int i = 0; i < 4; ++i) {
        a.lists[i] = h->lists + i * list_cap;
        a.bitmaps[i] = h->bitmaps + i * (size_t)bm_total;
    }
    a.list_cap = (unsigned)list_cap;
    a.bm_words = h->host_desc[0].bm_words;
    a.write_prev = 1;
    a.bar = h->bar;
    a.imgs = h->d_desc;
    a.nimg = n;
    a.xb = xb;
    a.yb = yb;
    a.tile_img = h->tile_img;
    a.bm_total = bm_total;
    a.img_k = per_image_k ? h->img_k : nullptr;
    a.ntiles = (int)tiles_total;
    a.hybrid = 1;
    a.tile_eval_max = eval_max;
    a.user0 = (n == 1 && im[0].dev) ? im[0].ptr : nullptr;
    {
        int user_ok = 0;
        if (ensure_tile_maps(h, fe, im, n, s, &user_ok)) {
            a.tmaps = h->tmaps;
            a.tma_user = user_ok;
        }
    }
    // List-pass CTAs: one per SM below 16 M pixels (fewer CTAs at the
    // barrier; measured faster on GB300 up to 2048 x 2048), two per SM above.
    a.list_ctas = h->opt_list_ctas > 0 ? h->opt_list_ctas : (px_total < (16ll << 20) ? h->sms : 0);
    a.bar_extra = h->opt_wait_test > 0 ? 1u : 0u;
    a.bar_spins = (unsigned)h->opt_wait_test;
    const bool user_ppm = h->opt_relaunch_ppm > 0;
    const long long ppm = user_ppm ? h->opt_relaunch_ppm : default_relaunch_ppm(beta);
    a.relaunch_evals = ppm >= 1000000 ? (1ll << 62) : px_total / 1000000 * ppm + px_total % 1000000 * ppm / 1000000;
    // Built-in: relaunch slots only for calls of at least kRelaunchMinPixels
    // (below that the list passes are cheap, and each slot a launch that
    // usually finds nothing to do: ~5 us of a ~100 us call on 256 x 256).
    int relaunches = ppm >= 1000000 ? 0
                                    : (user_ppm ? kMaxRelaunches
                                                : (px_total >= kRelaunchMinPixels ? kDefaultRelaunches : 0));
    if (forced_fused > 0) {
        // A predicted k: that many passes run as fused launches (each still
        // stops once a pass changed nothing), the list passes do the rest.
        a.relaunch_evals = 0;
        relaunches = std::min(forced_fused - 1, kMaxRelaunches);
    }
    // Fused launches: the first always runs; each later one runs only while
    // the previous one left many changed pixels (decided on the device).
    // Then one launch runs every remaining pass as a list pass.
    const int fused_launches = max_k > 0 ? std::min((max_k + T - 1) / T, 1 + relaunches) : 0;
    const bool list_loop = max_k > T;
    const int launches = fused_launches + (list_loop ? 1 : 0);
    const bool timed = h->opt_timing != 0;
    if (timed) {
        rc = ensure_events(h, 2 * (size_t)launches);
        if (rc < 0) return rc;
    }
    // The call's device work, on stream `st` (the handle's stream, or the
    // capture stream while a graph is recorded).
    auto enqueue = [&](cudaStream_t st, bool capturing) -> int {
        cudaStream_t s = st;
        // Timing events inside a recorded graph must be record nodes (an
        // ordinary record during capture only orders the capture).
        auto record = [&](cudaEvent_t e) {
            return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
        };
        // Images in: the first fused launch reads the images the device can read
        // (device memory, mapped page-locked host memory) directly; other host
        // images are copied into canvas 0, which it reads for them.
        for (int i = 0; i < n; ++i) {
            if (im[i].dev) continue;
            const hg::ImgDesc& d = h->host_desc[i];
            HG_TRY(h, cudaMemcpy2DAsync(h->canvas[0] + d.off + (long long)hg::kPadY * d.pitch + hg::kPadX, (size_t)d.pitch,
                                        im[i].ptr, (size_t)d.cols, (size_t)d.cols, (size_t)d.rows,
                                        cudaMemcpyHostToDevice, s));
        }
        HG_TRY(h, hg::launch_ctrl_init(h->ctrl, (unsigned)max_k, s));
        HG_TRY(h, cudaMemsetAsync(h->bitmaps, 0, 4 * (size_t)bm_total * sizeof(uint32_t), s));
        HG_TRY(h, cudaMemsetAsync(h->bar, 0, sizeof(hg::GridBar), s));
        if (per_image_k) HG_TRY(h, cudaMemsetAsync(h->img_k, 0, (size_t)n * sizeof(unsigned), s));
        for (int i = 0; i < launches; ++i) {
            if (timed) HG_TRY(h, record(h->events[2 * i]));
            if (i < fused_launches) {
                NvtxRange nr("hgrms fused launch");
                HG_TRY(h, fe->launch(a, (int)tiles_total, s));
            } else if (h->coop_stream) {
                NvtxRange nr("hgrms list-pass launch");
                HG_TRY(h, cudaEventRecord(h->coop_ev[0], s));
                HG_TRY(h, cudaStreamWaitEvent(h->coop_stream, h->coop_ev[0], 0));
                HG_TRY(h, chain_coop(h, h->coop_stream,
                                     [&] { return hg::launch_list(beta, a, h->sms, h->coop_stream); }));
                HG_TRY(h, cudaEventRecord(h->coop_ev[1], h->coop_stream));
                HG_TRY(h, cudaStreamWaitEvent(s, h->coop_ev[1], 0));
            } else if (capturing) {
                // The replay of the recorded graph is chained as a whole.
                NvtxRange nr("hgrms list-pass launch");
                HG_TRY(h, hg::launch_list(beta, a, h->sms, s));
            } else {
                NvtxRange nr("hgrms list-pass launch");
                HG_TRY(h, chain_coop(h, s, [&] { return hg::launch_list(beta, a, h->sms, s); }));
            }
            if (timed) HG_TRY(h, record(h->events[2 * i + 1]));
        }
        if (!write_back || max_k == 0) {
            // a trial, or no pass ran (the images are unchanged): no copy-out
        } else if (n == 1 && im[0].dev) {
            HG_TRY(h, hg::launch_copy_out(h->ctrl, h->canvas, h->host_desc[0].pitch, im[0].ptr, im[0].rows, im[0].cols,
                                          h->sms, s));
        } else {
            HG_TRY(h, hg::launch_copy_out_batch(h->ctrl, h->canvas, h->d_desc, n, max_words, h->sms, s));
        }
        HG_TRY(h, cudaMemcpyAsync(h->host_ctrl, h->ctrl, sizeof(hg::Ctrl), cudaMemcpyDeviceToHost, s));
        if (per_image_k)
            HG_TRY(h, cudaMemcpyAsync(h->host_img_k, h->img_k, (size_t)n * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        return HGRMS_OK;
    };
    if (ms) HG_TRY(h, cudaEventRecord(h->tune_ev[0], s));
    bool all_dev = true;
    for (int i = 0; i < n; ++i) all_dev = all_dev && im[i].dev;
    if (h->opt_graph && !ms && !h->coop_stream && all_dev) {
        // Replay the graph of an identical earlier call, or record one.
        std::vector<uint8_t> key(sizeof(a) + 16 * sizeof(long long));
        memcpy(key.data(), &a, sizeof(a));
        const long long extra[16] = {beta, T, fused_launches, list_loop, launches, write_back, max_k, n,
                                     (long long)(uintptr_t)im[0].ptr, im[0].rows, im[0].cols, max_words,
                                     timed, bm_total, (long long)(uintptr_t)h->host_ctrl,
                                     (long long)(uintptr_t)h->host_img_k};
        memcpy(key.data() + sizeof(a), extra, sizeof(extra));
        cudaGraphExec_t ex = nullptr;
        for (auto& g : h->graphs)
            if (g.first == key) ex = g.second;
        if (ex) {
            h->stats.graph = 1;
        } else {
            if (!h->cap_stream) HG_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
            HG_TRY(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
            const int erc = enqueue(h->cap_stream, true);
            cudaGraph_t g = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &g);
            if (erc == HGRMS_OK && ee == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                if (h->graphs.size() >= kMaxGraphs) {
                    cudaGraphExecDestroy(h->graphs.front().second);
                    h->graphs.erase(h->graphs.begin());
                }
                h->graphs.emplace_back(std::move(key), ex);
                h->stats.graph = 2;
            } else {
                ex = nullptr;
                (void)cudaGetLastError();  // a failed capture falls back to plain launches
            }
            if (g) cudaGraphDestroy(g);
        }
        if (ex) {
            if (list_loop)
                HG_TRY(h, chain_coop(h, s, [&] { return cudaGraphLaunch(ex, s); }));
            else
                HG_TRY(h, cudaGraphLaunch(ex, s));
        } else {
            rc = enqueue(s, false);
            if (rc < 0) return rc;
        }
    } else {
        rc = enqueue(s, false);
        if (rc < 0) return rc;
    }
    if (ms) HG_TRY(h, cudaEventRecord(h->tune_ev[1], s));
    hgrms_ctx::PendingCall pd;
    pd.n = n;
    pd.max_k = max_k;
    pd.launches = launches;
    pd.fused_launches = fused_launches;
    pd.T = T;
    pd.eval_max = eval_max;
    pd.TH = fe->TH;
    pd.TW = fe->TW;
    pd.tiles_total = tiles_total;
    pd.per_image_k = per_image_k;
    pd.write_back = write_back;
    pd.timed = timed;
    if (async_call) {
        pd.active = true;
        h->pending = pd;
        return HGRMS_OK;
    }
    HG_TRY(h, cudaStreamSynchronize(s));
    return finish_hybrid(h, pd, im, k_out, ms);
}

// The host side of a hybrid call after its queued work finished: copy host
// images back (synchronous calls only), read k, the launch times and the
// statistics.  `im` may be null when every image was device-readable.
int finish_hybrid(hgrms_ctx* h, const hgrms_ctx::PendingCall& pd, const BatchImg* im, int* k_out, float* ms) {
    cudaStream_t s = h->stream;
    const int n = pd.n, max_k = pd.max_k, launches = pd.launches, fused_launches = pd.fused_launches;
    const bool per_image_k = pd.per_image_k, write_back = pd.write_back, timed = pd.timed;
    const hg::Ctrl c = *h->host_ctrl;
    bool host_out = false;
    for (int i = 0; im && i < n && write_back && max_k > 0; ++i) {
        if (im[i].dev) continue;
        const hg::ImgDesc& d = h->host_desc[i];
        HG_TRY(h, cudaMemcpy2DAsync(im[i].ptr, (size_t)d.cols,
                                    h->canvas[c.cur] + d.off + (long long)hg::kPadY * d.pitch + hg::kPadX,
                                    (size_t)d.pitch, (size_t)d.cols, (size_t)d.rows, cudaMemcpyDeviceToHost, s));
        host_out = true;
    }
    if (host_out) HG_TRY(h, cudaStreamSynchronize(s));
    if (ms) HG_TRY(h, cudaEventElapsedTime(ms, h->tune_ev[0], h->tune_ev[1]));
    if (timed) {
        // Fused launches that ran passes come first; the list-pass launch
        // ran passes when work_launches counts it.
        const bool list_worked = c.work_launches > c.fused_work;
        for (int i = 0; i < launches; ++i) {
            float ms = 0.f;
            HG_TRY(h, cudaEventElapsedTime(&ms, h->events[2 * i], h->events[2 * i + 1]));
            const bool worked = i < fused_launches ? i < (int)c.fused_work : list_worked;
            h->launch_ms.push_back(ms);
            h->launch_kind.push_back(worked ? (i < fused_launches ? 0 : 1) : 3);
            if (worked)
                h->stats.kernel_ms += ms;
            else
                h->stats.idle_kernel_ms += ms;
        }
    }
    if (c.error) {
        h->last_cuda_error = 0;
        return HGRMS_ETIMEOUT;
    }
    for (int i = 0; i < n; ++i) k_out[i] = per_image_k ? (int)h->host_img_k[i] : (int)c.k;
    h->stats.launches += launches;
    h->stats.passes_per_launch = pd.T;
    h->stats.tile_eval_max = pd.eval_max;
    h->stats.tile_rows = pd.TH;
    h->stats.tile_cols = pd.TW;
    h->stats.ctas_per_launch += pd.tiles_total;
    h->stats.passes_executed += (int)c.executed;
    h->stats.evals_fused += (long long)c.evals_fused;
    h->stats.evals_list += (long long)c.evals_list;
    h->stats.work_launches += (int)c.work_launches;
    h->stats.passes += (int)(c.k + c.converged);
    h->converged = (int)c.converged;
    return HGRMS_OK;
}

// The tuning of a hybrid call: the options when set, else the autotuner's
// choice for (beta, single image or batch, size class) when autotuning is on
// (the first call of a class times every compiled T with four switch points
// on the call's own images, which are not written by the trials, and keeps
// the fastest; every candidate gives the same result), else the built-in
// values.
int choose_tuning(hgrms_ctx* h, const BatchImg* im, int n, int alpha, int beta, int max_k, int* k_scratch,
                  Tuning* out) {
    Tuning tu{h->opt_passes > 0 ? h->opt_passes : default_passes(beta), h->opt_tile_eval_max};
    if (!h->opt_autotune || (h->opt_passes > 0 && h->opt_tile_eval_max > 0)) {
        *out = tu;
        return HGRMS_OK;
    }
    long long px = 0;
    for (int i = 0; i < n; ++i) px += (long long)im[i].rows * im[i].cols;
    const long long key = ((long long)beta << 8) | ((n > 1 ? 1ll : 0ll) << 7) | (long long)bits_for(px);
    auto it = h->tuned.find(key);
    if (it != h->tuned.end()) {
        *out = it->second;
        h->stats.autotuned = 1;
        return HGRMS_OK;
    }
    std::vector<int> Ts;
    if (h->opt_passes > 0) {
        Ts.push_back(h->opt_passes);
    } else {
        for (int T = 1; T <= 32; ++T)
            if (find_fused(beta, T)) Ts.push_back(T);
    }
    std::vector<int> ems;
    if (h->opt_tile_eval_max > 0)
        ems.push_back(h->opt_tile_eval_max);
    else
        ems = {1024, 2048, 4096, 8192};
    const int reps = px < (4ll << 20) ? 3 : 1;
    Tuning best = tu;
    float best_ms = 3.0e38f;
    float tune_total = 0.f;
    for (int T : Ts)
        for (int em : ems) {
            const Tuning c{T, em};
            float t_min = 3.0e38f;
            for (int r = 0; r < reps; ++r) {
                float ms = 0.f;
                const int rc = run_hybrid(h, im, n, alpha, beta, max_k, k_scratch, c, false, &ms);
                if (rc < 0) return rc;
                tune_total += ms;
                if (ms < t_min) t_min = ms;
            }
            if (t_min < best_ms) {
                best_ms = t_min;
                best = c;
            }
        }
    h->tuned[key] = best;
    const double tune_ms = h->stats.tune_ms + tune_total;
    h->stats = hgrms_stats_t{};  // the trials' counts are not the call's
    h->stats.tune_ms = tune_ms;
    h->stats.autotuned = 1;
    h->launch_ms.clear();
    h->launch_kind.clear();
    *out = best;
    return HGRMS_OK;
}

// One denoise with the unfused or fused-only schedule, except argument
// checks.  `dev` tells whether img is device memory.
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
    a.write_prev = 0;
    a.imgs = nullptr;
    a.nimg = 1;
    a.xb = a.yb = 16;
    a.tile_img = nullptr;
    a.bm_total = 0;
    a.img_k = nullptr;
    a.ntiles = p.tiles_x * p.tiles_y;
    a.hybrid = 0;
    a.relaunch_evals = 0;
    a.tile_eval_max = h->opt_tile_eval_max;
    a.user0 = nullptr;
    a.list_ctas = 0;
    a.bar_extra = h->opt_wait_test > 0 ? 1u : 0u;
    a.bar_spins = (unsigned)h->opt_wait_test;
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
            HG_TRY(h, p.fe->launch(a, p.tiles_x * p.tiles_y, s));
        else if (p.fused)
            HG_TRY(h, chain_coop(h, s, [&] { return hg::launch_list(beta, a, h->sms, s); }));
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
            h->launch_kind.push_back(i < (int)c.work_launches ? (p.fused ? 0 : 2) : 3);
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

namespace {

// Runs the predictor on the device-readable images of a call; returns the
// largest estimate (0 when it cannot run: no weights, or an image the
// device cannot read).
int predict_max_k(hgrms_ctx* h, const BatchImg* im, int n, int beta, float* out_max) {
    *out_max = 0.f;
    if (!h->pred[beta]) return HGRMS_OK;
    for (int i = 0; i < n; ++i)
        if (!im[i].dev) return HGRMS_OK;
    if (n > h->pred_desc_cap) {
        if (h->pred_desc) cudaFree(h->pred_desc);
        h->pred_desc = nullptr;
        h->pred_desc_cap = 0;
        HG_TRY(h, cudaMalloc(&h->pred_desc, (size_t)n * sizeof(hg::ImgDesc)));
        h->pred_desc_cap = n;
    }
    std::vector<hg::ImgDesc> t((size_t)n);
    for (int i = 0; i < n; ++i) {
        memset(&t[i], 0, sizeof(hg::ImgDesc));
        t[i].rows = im[i].rows;
        t[i].cols = im[i].cols;
        t[i].user = im[i].ptr;
    }
    HG_TRY(h, cudaMemcpyAsync(h->pred_desc, t.data(), (size_t)n * sizeof(hg::ImgDesc), cudaMemcpyHostToDevice,
                              h->stream));
    std::vector<float> kh((size_t)n);
    const int rc = hg::predictor_run(h->pred[beta], h->pred_desc, n, h->stream, kh.data(), nullptr, nullptr, nullptr);
    if (rc < 0) return rc;
    for (float v : kh) *out_max = v > *out_max ? v : *out_max;
    return HGRMS_OK;
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
    if (e == cudaSuccess) e = cudaEventCreate(&h->tune_ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&h->tune_ev[1]);
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
        if (h->stream || h->pending.active) cudaStreamSynchronize(h->stream);
        for (int i = 0; i < 3; ++i)
            if (h->canvas[i]) cudaFree(h->canvas[i]);
        if (h->ctrl) cudaFree(h->ctrl);
        if (h->bar) cudaFree(h->bar);
        if (h->tmaps) cudaFree(h->tmaps);
        if (h->tmaps_host) cudaFreeHost(h->tmaps_host);
        if (h->tmaps_ev) cudaEventDestroy(h->tmaps_ev);
        if (h->chg_maps) cudaFree(h->chg_maps);
        if (h->lists) cudaFree(h->lists);
        if (h->bitmaps) cudaFree(h->bitmaps);
        if (h->host_ctrl) cudaFreeHost(h->host_ctrl);
        if (h->d_desc) cudaFree(h->d_desc);
        if (h->host_desc) cudaFreeHost(h->host_desc);
        if (h->tile_img) cudaFree(h->tile_img);
        if (h->img_k) cudaFree(h->img_k);
        if (h->host_img_k) cudaFreeHost(h->host_img_k);
        for (cudaEvent_t e : h->events) cudaEventDestroy(e);
        for (cudaEvent_t e : h->tune_ev)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : h->coop_ev)
            if (e) cudaEventDestroy(e);
        if (h->chain_ev) {
            std::lock_guard<std::mutex> lock(g_chain_mu);
            if (h->device >= 0 && h->device < kMaxChainDevices && g_chain_last[h->device] == h->chain_ev)
                g_chain_last[h->device] = nullptr;
            cudaEventDestroy(h->chain_ev);
        }
        for (auto& g : h->graphs) cudaGraphExecDestroy(g.second);
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        for (hg::Predictor* p : h->pred) hg::predictor_free(p);
        if (h->pred_desc) cudaFree(h->pred_desc);
    }
    delete h;
}

HG_EXPORT int hgrms_denoise(hgrms_t h, uint8_t* img, int rows, int cols, int alpha, int beta, int max_k) {
    NvtxRange nr("hgrms_denoise");
    if (!h || !img) return HGRMS_EINVAL;
    if (h->pending.active) return HGRMS_EBUSY;
    int rc = check_args(rows, cols, alpha, beta, max_k);
    if (rc < 0) return rc;
    DeviceGuard g(h->device);
    uint8_t* dp = nullptr;
    const int kind = pointer_kind(img, h->device, &dp);
    if (kind < 0) return HGRMS_EINVAL;
    h->stats = hgrms_stats_t{};
    h->launch_ms.clear();
    h->launch_kind.clear();
    if (h->opt_kernel != kHybrid) return denoise_one(h, dp, rows, cols, alpha, beta, max_k, kind == 1, true);
    const BatchImg bi{dp, rows, cols, kind == 1};
    int k = 0;
    Tuning tu;
    rc = choose_tuning(h, &bi, 1, alpha, beta, max_k, &k, &tu);
    if (rc < 0) return rc;
    int forced = 0;
    h->stats.k_pred = -1.0;
    if (h->opt_predict_k) {
        float kp = 0.f;
        rc = predict_max_k(h, &bi, 1, beta, &kp);
        if (rc < 0) return rc;
        if (h->pred[beta]) {
            h->stats.k_pred = kp;
            forced = (int)std::ceil(std::min(kp, (float)max_k) / (float)tu.T);
        }
    }
    rc = run_hybrid(h, &bi, 1, alpha, beta, max_k, &k, tu, true, nullptr, forced);
    return rc < 0 ? rc : k;
}

HG_EXPORT int hgrms_denoise_async(hgrms_t h, uint8_t* img, int rows, int cols, int alpha, int beta, int max_k) {
    NvtxRange nr("hgrms_denoise_async");
    if (!h || !img) return HGRMS_EINVAL;
    if (h->pending.active) return HGRMS_EBUSY;
    int rc = check_args(rows, cols, alpha, beta, max_k);
    if (rc < 0) return rc;
    DeviceGuard g(h->device);
    uint8_t* dp = nullptr;
    if (pointer_kind(img, h->device, &dp) != 1) return HGRMS_EINVAL;  // must be device-readable
    if (h->opt_kernel != kHybrid || h->opt_autotune || h->opt_predict_k) {
        // Schedules that need the host between launches run now.
        const int k = hgrms_denoise(h, img, rows, cols, alpha, beta, max_k);
        if (k < 0) return k;
        h->pending = hgrms_ctx::PendingCall{};
        h->pending.active = true;
        h->pending.done = true;
        h->pending.result = k;
        return HGRMS_OK;
    }
    h->stats = hgrms_stats_t{};
    h->stats.k_pred = -1.0;
    h->launch_ms.clear();
    h->launch_kind.clear();
    const BatchImg bi{dp, rows, cols, true};
    int k = 0;
    Tuning tu;
    rc = choose_tuning(h, &bi, 1, alpha, beta, max_k, &k, &tu);
    if (rc < 0) return rc;
    return run_hybrid(h, &bi, 1, alpha, beta, max_k, &k, tu, true, nullptr, 0, true);
}

HG_EXPORT int hgrms_wait(hgrms_t h) {
    NvtxRange nr("hgrms_wait");
    if (!h || !h->pending.active) return HGRMS_EINVAL;
    const hgrms_ctx::PendingCall pd = h->pending;
    h->pending = hgrms_ctx::PendingCall{};
    if (pd.done) return pd.result;
    DeviceGuard g(h->device);
    HG_TRY(h, cudaStreamSynchronize(h->stream));
    int k = 0;
    const int rc = finish_hybrid(h, pd, nullptr, &k, nullptr);
    return rc < 0 ? rc : k;
}

HG_EXPORT int hgrms_denoise_batch(hgrms_t h, uint8_t* const* imgs, const int* rows, const int* cols, int n,
                                  int alpha, int beta, int max_k, int* k_out) {
    NvtxRange nr("hgrms_denoise_batch");
    if (!h || n < 0 || (n > 0 && (!imgs || !rows || !cols || !k_out))) return HGRMS_EINVAL;
    if (h->pending.active) return HGRMS_EBUSY;
    DeviceGuard g(h->device);
    std::vector<BatchImg> bi((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!imgs[i]) return HGRMS_EINVAL;
        int rc = check_args(rows[i], cols[i], alpha, beta, max_k);
        if (rc < 0) return rc;
        uint8_t* dp = nullptr;
        const int kind = pointer_kind(imgs[i], h->device, &dp);
        if (kind < 0) return HGRMS_EINVAL;
        bi[i] = BatchImg{dp, rows[i], cols[i], kind == 1};
    }
    h->launch_ms.clear();
    h->launch_kind.clear();
    if (h->opt_kernel == kHybrid && n > 0) {
        // Chunks of consecutive images, each run as one batched schedule: a
        // chunk ends before the image that would exceed the memory budget,
        // the image count of one launch or the 32-bit change-list packing.
        const int T = h->opt_passes > 0 ? h->opt_passes : default_passes(beta);
        const hg::FusedEntry* fe = find_fused(beta, T);
        if (!fe) return HGRMS_EINVAL;
        const long long budget = (long long)(h->opt_batch_mb > 0 ? h->opt_batch_mb : 8192) << 20;
        h->stats = hgrms_stats_t{};
        h->stats.k_pred = -1.0;
        int all_conv = 1;
        for (int start = 0; start < n;) {
            int end = start, mr = 1, mc = 1;
            long long bytes = 0;
            while (end < n) {
                const long long nb = hybrid_bytes(fe, rows[end], cols[end]);
                const int mr2 = rows[end] > mr ? rows[end] : mr, mc2 = cols[end] > mc ? cols[end] : mc;
                const int cnt = end - start + 1;
                const bool fits = cnt <= hg::kMaxBatchImages && bytes + nb <= budget &&
                                  bits_for(mc2 - 1) + bits_for(mr2 - 1) + (cnt > 1 ? bits_for(cnt - 1) : 0) <= 32;
                if (!fits && end > start) break;
                bytes += nb;
                mr = mr2;
                mc = mc2;
                ++end;
            }
            Tuning tu;
            int rc = choose_tuning(h, bi.data() + start, end - start, alpha, beta, max_k, k_out + start, &tu);
            if (rc < 0) return rc;
            int forced = 0;
            if (h->opt_predict_k) {
                float kp = 0.f;
                rc = predict_max_k(h, bi.data() + start, end - start, beta, &kp);
                if (rc < 0) return rc;
                if (h->pred[beta]) {
                    h->stats.k_pred = std::max(h->stats.k_pred, (double)kp);
                    forced = (int)std::ceil(std::min(kp, (float)max_k) / (float)tu.T);
                }
            }
            rc = run_hybrid(h, bi.data() + start, end - start, alpha, beta, max_k, k_out + start, tu, true, nullptr,
                            forced);
            if (rc < 0) return rc;
            start = end;
        }
        for (int i = 0; i < n; ++i) all_conv &= k_out[i] < max_k ? 1 : 0;
        h->converged = all_conv;
        return HGRMS_OK;
    }
    hgrms_stats_t acc{};
    int all_conv = 1;
    for (int i = 0; i < n; ++i) {
        h->stats = hgrms_stats_t{};
        const int k = denoise_one(h, bi[i].ptr, rows[i], cols[i], alpha, beta, max_k, bi[i].dev, true);
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

namespace hg {

// Run this handle's list-pass launches on `coop` (see hgrms_ctx::coop_stream).
int set_coop_stream(hgrms_t h, cudaStream_t coop) {
    if (!h) return HGRMS_EINVAL;
    DeviceGuard g(h->device);
    for (int i = 0; i < 2; ++i)
        if (!h->coop_ev[i]) HG_TRY(h, cudaEventCreateWithFlags(&h->coop_ev[i], cudaEventDisableTiming));
    h->coop_stream = coop;
    return HGRMS_OK;
}

}  // namespace hg

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
        case HGRMS_EAGAIN: return "request not finished yet";
        case HGRMS_EBUSY: return "an asynchronous call on this handle has not been waited for";
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
        case HGRMS_OPT_BATCH_MB:
            if (value < 0) return HGRMS_EINVAL;
            h->opt_batch_mb = value;
            return HGRMS_OK;
        case HGRMS_OPT_RELAUNCH_PPM:
            if (value < 0) return HGRMS_EINVAL;
            h->opt_relaunch_ppm = value;
            return HGRMS_OK;
        case HGRMS_OPT_PREDICT_K:
            if (value != 0 && value != 1) return HGRMS_EINVAL;
            h->opt_predict_k = value;
            return HGRMS_OK;
        case HGRMS_OPT_GRAPH:
            if (value != 0 && value != 1) return HGRMS_EINVAL;
            h->opt_graph = value;
            return HGRMS_OK;
        case HGRMS_OPT_LIST_CTAS:
            if (value < 0) return HGRMS_EINVAL;
            h->opt_list_ctas = value;
            return HGRMS_OK;
        case HGRMS_OPT_AUTOTUNE:
            if (value != 0 && value != 1) return HGRMS_EINVAL;
            h->opt_autotune = value;
            return HGRMS_OK;
        case HGRMS_OPT_TMA:
            if (value != 0 && value != 1) return HGRMS_EINVAL;
            h->opt_tma = value;
            return HGRMS_OK;
        case HGRMS_OPT_WAIT_TEST:
            if (value < 0 || value > (1 << 22)) return HGRMS_EINVAL;
            h->opt_wait_test = value;
            return HGRMS_OK;
        case HGRMS_OPT_TILE_EVAL_MAX:
            if (value < 0 || value > (1 << 20)) return HGRMS_EINVAL;
            h->opt_tile_eval_max = value;
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

HG_EXPORT int hgrms_rms(const int* sum, const int* flag, int* out, int n, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!sum || !flag || !out))) return HGRMS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = hg::launch_rms(sum, flag, out, n, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HGRMS_OK : HGRMS_ECUDA;
}

HG_EXPORT int hgrms_default_passes(int beta) {
    if (beta < 1 || beta > hg::kMaxBeta) return HGRMS_EINVAL;
    return default_passes(beta);
}

HG_EXPORT int hgrms_has_kernel(int beta, int passes) {
    return find_fused(beta, passes) != nullptr ? 1 : 0;
}

HG_EXPORT int hgrms_predictor_load(hgrms_t h, int beta, const float* weights, int n) {
    if (!h || !weights || beta < 1 || beta > hg::kMaxBeta) return HGRMS_EINVAL;
    DeviceGuard g(h->device);
    if (!h->pred[beta]) h->pred[beta] = hg::predictor_new();
    if (!h->pred[beta]) return HGRMS_ENOMEM;
    return hg::predictor_load(h->pred[beta], weights, n);
}

HG_EXPORT int hgrms_predict_k(hgrms_t h, int beta, uint8_t* const* imgs, const int* rows, const int* cols, int n,
                              float* k_hat, float* x0, float* hist, float* gap) {
    if (!h || beta < 1 || beta > hg::kMaxBeta || n < 0 || (n > 0 && (!imgs || !rows || !cols || !k_hat)))
        return HGRMS_EINVAL;
    if (!h->pred[beta]) return HGRMS_EINVAL;
    DeviceGuard g(h->device);
    std::vector<hg::ImgDesc> t((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!imgs[i] || rows[i] < 1 || cols[i] < 1 || rows[i] > 65536 || cols[i] > 65536) return HGRMS_EINVAL;
        uint8_t* dp = nullptr;
        if (pointer_kind(imgs[i], h->device, &dp) != 1) return HGRMS_EINVAL;  // must be device-readable
        memset(&t[i], 0, sizeof(hg::ImgDesc));
        t[i].rows = rows[i];
        t[i].cols = cols[i];
        t[i].user = dp;
    }
    if (n == 0) return HGRMS_OK;
    if (n > h->pred_desc_cap) {
        if (h->pred_desc) cudaFree(h->pred_desc);
        h->pred_desc = nullptr;
        h->pred_desc_cap = 0;
        HG_TRY(h, cudaMalloc(&h->pred_desc, (size_t)n * sizeof(hg::ImgDesc)));
        h->pred_desc_cap = n;
    }
    HG_TRY(h, cudaMemcpyAsync(h->pred_desc, t.data(), (size_t)n * sizeof(hg::ImgDesc), cudaMemcpyHostToDevice,
                              h->stream));
    return hg::predictor_run(h->pred[beta], h->pred_desc, n, h->stream, k_hat, x0, hist, gap);
}

HG_EXPORT int hgrms_predictor_grad(hgrms_t h, const float* weights, const float* x0, const float* hist, const float* k,
                                   int n, float* grads, float* loss) {
    if (!h || !weights || !x0 || !hist || !k || !grads || !loss) return HGRMS_EINVAL;
    DeviceGuard g(h->device);
    return hg::predictor_grad(weights, x0, hist, k, n, grads, loss, h->stream);
}

HG_EXPORT int hgrms_predictor_train(hgrms_t h, float* weights, const float* x0, const float* hist, const float* k,
                                    int n, int epochs, int batch, float lr, unsigned long long seed, float* loss) {
    if (!h || !weights || !x0 || !hist || !k) return HGRMS_EINVAL;
    DeviceGuard g(h->device);
    return hg::predictor_train(weights, x0, hist, k, n, epochs, batch, lr, seed, loss, h->stream);
}
