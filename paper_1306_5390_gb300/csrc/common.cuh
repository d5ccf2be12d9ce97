// Shared definitions of the CUDA path: canvas layout, the device control
// block that carries the iteration state (Section 2: passes repeat until no
// pixel changes, capped by the iteration factor) between launches, and the
// per-launch finalisation done by the last CTA of each launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hg {

// Canvas: every image is denoised in a padded copy ("canvas") so that tile
// loads with halos never leave the allocation.  The image's pixel (r, c)
// lives at canvas byte (kPadY + r) * pitch + kPadX + c.
constexpr int kPadX = 16;   // bytes left of the image; keeps rows 16-byte aligned
constexpr int kPadY = 16;   // rows above the image (>= any vertical tile halo)
constexpr int kMaxBeta = 7;

// Iteration state shared by the launches of one denoising call.
struct Ctrl {
    unsigned k;          // passes so far that changed at least one pixel
    unsigned converged;  // 1 once a pass changed no pixel
    unsigned cur;        // canvas holding the current image: 0 = A, 1 = B
    unsigned max_k;      // cap on k
    unsigned done;       // CTAs of the running launch that have finished
    unsigned mask;       // bit t: pass t of the running launch changed a core pixel
    unsigned work_launches;
    unsigned executed;   // passes executed by launches that did work
};

struct PassArgs {
    const uint8_t* canvas_a;  // canvas base pointers (row 0, column 0 of the canvas)
    uint8_t* canvas_b;
    long long pitch;          // canvas row pitch in bytes (multiple of 16)
    int rows, cols;           // image size
    int alpha;
    int tiles_x;              // tile grid width (fused kernel)
    Ctrl* ctrl;
    // Pixel change maps (fused kernel): three bitmaps of rows x map_words
    // 32-bit words; bit (c & 31) of word c >> 5 of row r = image pixel (r, c)
    // changed in the last pass of a launch.  Launch L writes map L % 3,
    // reads map (L + 2) % 3 and clears map (L + 1) % 3.
    uint32_t* chg_maps;
    int map_words;            // words per image row
};

// Passes the launch must run: 0 when the call has finished.
__device__ __forceinline__ int launch_passes(const Ctrl* c, int T) {
    unsigned k = __ldcg(&c->k);
    unsigned conv = __ldcg(&c->converged);
    unsigned mk = __ldcg(&c->max_k);
    if (conv || k >= mk) return 0;
    unsigned left = mk - k;
    return left < (unsigned)T ? (int)left : T;
}

// Called by thread 0 of every CTA that ran `np` passes.  `cta_mask` bit t is
// set when pass t changed a pixel of this CTA's core.  The last CTA to arrive
// folds the launch's mask into the iteration state: k grows by the number of
// leading changing passes; a pass that changed nothing means the image is a
// fixed point (every later pass is a no-op, so the buffer written by this
// launch holds the final image).
__device__ __forceinline__ void finish_launch(Ctrl* c, unsigned cta_mask, int np,
                                              unsigned nctas) {
    if (cta_mask) atomicOr(&c->mask, cta_mask);
    __threadfence();
    unsigned prev = atomicAdd(&c->done, 1u);
    if (prev == nctas - 1) {
        __threadfence();
        unsigned m = atomicExch(&c->mask, 0u);
        unsigned ones = (~m == 0u) ? 32u : (unsigned)(__ffs(~m) - 1);
        if (ones > (unsigned)np) ones = (unsigned)np;
        c->k += ones;
        if (ones < (unsigned)np) c->converged = 1u;
        c->cur ^= 1u;
        c->work_launches += 1u;
        c->executed += (unsigned)np;
        c->done = 0u;
        __threadfence();
    }
}

}  // namespace hg
