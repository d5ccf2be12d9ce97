// hgrms_denoise_noalloc: the fused tile path for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc or cudaFree at all: code running
// under a memory pool or arena they do not control, real-time or
// latency-critical paths where an allocation can stall or fail, and plug-ins
// embedded in hosts that own the device's memory.  This entry point takes
// every piece of scratch memory (two image canvases, the change bitmaps the
// launches pass to each other and the control block) from one file-scope
// __device__ array of fixed size, so a call allocates nothing; the caller
// passes the image (device memory) and gets it back denoised in place.
//
// The array is part of the library's device image: every GPU on which the
// library is loaded holds it until the process exits.  Host code cannot use
// the array's name as a device address, so every call asks the runtime for
// the address on the current device (cudaGetSymbolAddress, which allocates
// nothing).  The first call on a device also loads the library's device code
// there; later calls only look the address up, so a context that was reset
// and rebuilt never sees an address from before the reset.
#include <cstddef>

#include "../../include/hgrms.h"
#include "fused.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = (size_t)HGRMS_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

// Device address of the array on the current device.
cudaError_t scratch_address(uint8_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<uint8_t*>(p);
    return cudaSuccess;
}

static_assert(offsetof(hg::Ctrl, k) == 0 && offsetof(hg::Ctrl, converged) == sizeof(unsigned),
              "the group check reads k and converged as two leading words");

// Fused launches queued before the host checks whether the call has
// converged: enough for 32 passes (one group for the usual max_k <= 32).
int launches_per_check(int T) { return (32 + T - 1) / T; }

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

int fail(cudaError_t e) {
    return e == cudaErrorMemoryAllocation ? HGRMS_ENOMEM : HGRMS_ECUDA;
}

}  // namespace

#define HG_NA_TRY(call)                            \
    do {                                           \
        const cudaError_t e_ = (call);             \
        if (e_ != cudaSuccess) return fail(e_);    \
    } while (0)

extern "C" __attribute__((visibility("default"))) int hgrms_denoise_noalloc(uint8_t* img, int rows, int cols,
                                                                           int alpha, int beta, int max_k,
                                                                           void* cuda_stream) {
    if (!img || rows < 1 || cols < 1 || rows > 65536 || cols > 65536) return HGRMS_EINVAL;
    if (alpha < 0 || alpha > 255 || beta < 1 || beta > hg::kMaxBeta || max_k < 0 || max_k > 1000000)
        return HGRMS_EINVAL;
    int device = 0;
    HG_NA_TRY(cudaGetDevice(&device));
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, img) != cudaSuccess) {
        cudaGetLastError();
        return HGRMS_EINVAL;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != device)
        return HGRMS_EINVAL;  // device memory of the current device only

    // Geometry of the fused kernel (fused tile launches only).
    const int T = hg::default_passes(beta);
    const hg::FusedEntry* fe = hg::find_fused(beta, T);
    if (!fe) return HGRMS_EINVAL;
    const int tiles_x = (cols + fe->TW - 1) / fe->TW;
    const int tiles_y = (rows + fe->TH - 1) / fe->TH;
    const long long pitch = (hg::kPadX + (long long)tiles_x * fe->TW + 16 + 127) / 128 * 128;
    const long long crows = hg::kPadY + (long long)tiles_y * fe->TH + 16;
    const int map_words = (tiles_x * fe->TW + 31) / 32 + 2;
    const size_t ctrl_bytes = align256(sizeof(hg::Ctrl));
    const size_t canvas_bytes = align256((size_t)(pitch * crows));
    const size_t map_bytes = (size_t)rows * (size_t)map_words * sizeof(uint32_t);
    const size_t need = ctrl_bytes + 2 * canvas_bytes + align256(3 * map_bytes);
    if (need > kScratchBytes) return HGRMS_ETOOBIG;

    uint8_t* base = nullptr;
    HG_NA_TRY(scratch_address(&base));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int sms = 0;
    HG_NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));

    hg::Ctrl* ctrl = reinterpret_cast<hg::Ctrl*>(base);
    hg::PassArgs a;
    a.canvas[0] = base + ctrl_bytes;
    a.canvas[1] = a.canvas[0] + canvas_bytes;
    a.canvas[2] = a.canvas[0];  // the third canvas is only written for list passes, which this path has not
    a.pitch = pitch;
    a.rows = rows;
    a.cols = cols;
    a.alpha = alpha;
    a.tiles_x = tiles_x;
    a.ctrl = ctrl;
    a.chg_maps = reinterpret_cast<uint32_t*>(a.canvas[1] + canvas_bytes);
    a.map_words = map_words;
    for (int i = 0; i < 4; ++i) {
        a.lists[i] = nullptr;
        a.bitmaps[i] = nullptr;
    }
    a.list_cap = 0;
    a.bm_words = 0;
    a.write_prev = 0;
    a.bar = nullptr;
    a.imgs = nullptr;
    a.nimg = 1;
    a.xb = a.yb = 16;
    a.tile_img = nullptr;
    a.bm_total = 0;
    a.img_k = nullptr;
    a.ntiles = tiles_x * tiles_y;
    a.hybrid = 0;
    a.relaunch_evals = 0;
    a.tile_eval_max = 0;
    a.user0 = nullptr;
    a.list_ctas = 0;

    // The array keeps the previous call's contents: the control block is
    // reset by ctrl_init and change map 0 (written by the first launch) is
    // cleared here; the launches clear the other maps themselves.  Canvas
    // bytes outside the image are never read by a pixel that can change.
    HG_NA_TRY(hg::launch_copy_in(img, rows, cols, a.canvas[0], pitch, sms, s));
    HG_NA_TRY(hg::launch_ctrl_init(ctrl, (unsigned)max_k, s));
    HG_NA_TRY(cudaMemsetAsync(a.chg_maps, 0, map_bytes, s));
    // Launches after the call has converged return at once but still cost a
    // wave each, so they are queued in groups, and between groups the host
    // reads k and the converged flag (into stack memory) and stops early.
    const int launches = (max_k + T - 1) / T;
    const int group = launches_per_check(T);
    for (int done = 0; done < launches;) {
        const int n = launches - done < group ? launches - done : group;
        for (int i = 0; i < n; ++i) HG_NA_TRY(fe->launch(a, tiles_x * tiles_y, s));
        done += n;
        if (done < launches) {
            unsigned st[2] = {0u, 0u};  // Ctrl::k, Ctrl::converged
            HG_NA_TRY(cudaMemcpyAsync(st, ctrl, sizeof(st), cudaMemcpyDeviceToHost, s));
            HG_NA_TRY(cudaStreamSynchronize(s));
            if (st[1] || st[0] >= (unsigned)max_k) break;
        }
    }
    HG_NA_TRY(hg::launch_copy_out(ctrl, a.canvas, pitch, img, rows, cols, sms, s));
    unsigned k = 0;
    HG_NA_TRY(cudaMemcpyAsync(&k, &ctrl->k, sizeof(k), cudaMemcpyDeviceToHost, s));
    HG_NA_TRY(cudaStreamSynchronize(s));
    return (int)k;
}
