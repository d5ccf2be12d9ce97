// Shared definitions of the CUDA path: canvas layout, the device control
// block that carries the iteration state (Section 2: passes repeat until no
// pixel changes, capped by the iteration factor) between launches, and the
// per-launch finalisation done by the last CTA of each launch.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string.h>

namespace hg {

// Canvas: every image is denoised in a padded copy ("canvas") so that tile
// loads with halos never leave the allocation.  The image's pixel (r, c)
// lives at canvas byte (kPadY + r) * pitch + kPadX + c.
constexpr int kPadX = 16;   // bytes left of the image; keeps rows 16-byte aligned
constexpr int kPadY = 16;   // rows above the image (>= any vertical tile halo)
constexpr int kMaxBeta = 7;
constexpr int kMaxBatchImages = 4096;  // images per batched launch (more are split into chunks)

// Iteration state shared by the launches of one denoising call.
//
// Three canvases hold images.  `cur` holds the current image I_t.  `aux`
// holds an image that agrees with I_{t-1} wherever pass t changed nothing
// (I_{t-1} itself after a one-pass launch); a launch that writes only the
// pixels that can change (a list pass) writes into `aux`, which then holds
// I_{t+1} everywhere.
struct Ctrl {
    unsigned k;          // passes so far that changed at least one pixel
    unsigned converged;  // 1 once a pass changed no pixel
    unsigned cur;        // canvas (0..2) holding the current image
    unsigned aux;        // canvas (0..2, != cur) partnering it, see above
    unsigned max_k;      // cap on k
    unsigned done;       // CTAs of the running launch that have finished
    unsigned mask;       // bit t: pass t of the running launch changed a pixel
    unsigned work_launches;
    unsigned executed;   // passes executed by launches that did work
    unsigned list_n[4];  // entries appended to change list 0..3 (> capacity: overflow)
    unsigned error;      // 1: a bounded device wait gave up
    unsigned fused_work; // fused launches that ran passes
    unsigned dense;      // hybrid schedule: 1 = the next fused launch runs (many pixels changed)
    unsigned tile_next[2];  // tile queue of fused launch L: counter L & 1
    // Pixel evaluations the passes needed (core pixels only: a dense pass
    // counts every image pixel, a list pass the pixels it claimed), by kernel.
    unsigned long long evals_fused;
    unsigned long long evals_list;
};

// Grid barrier of the list-pass loop: two 64-bit counters on their own
// 128-byte lines (barriers alternate between them; see grid_barrier in
// list.cu).  All zero at the start of a call.
struct alignas(128) BarLine {
    unsigned long long v;
    unsigned long long pad[15];
};
struct GridBar {
    BarLine ctr[2];
};

// One image of a batch.  The images' canvases are laid out one after another
// in each of the three canvas arenas (image i's canvas starts `off` bytes into
// every arena) and their change bitmaps one after another in each bitmap
// arena (at word `bm_off`).  A single-image call uses a table of one entry.
struct alignas(16) ImgDesc {
    long long off;        // canvas offset in each arena (multiple of 128)
    long long bm_off;     // bitmap offset in words
    int pitch;            // canvas row pitch (multiple of 128)
    int rows, cols;
    int tiles_x;          // fused-kernel tile grid width
    int tile0;            // first fused-kernel tile of this image
    int bm_words;         // bitmap words per image row
    uint8_t* user;        // the caller's image if the device can read it (batches), or null
};

// A change-list entry packs (image, row, column) into 32 bits: the column in
// the low xb bits, the row in the next yb bits, the image above them (a
// single image uses xb = yb = 16).
__device__ __forceinline__ uint32_t pack_entry(unsigned img, int y, int x, int xb, int yb) {
    return (uint32_t)((unsigned long long)img << (xb + yb)) | ((uint32_t)y << xb) | (uint32_t)x;
}
__device__ __forceinline__ void unpack_entry(uint32_t e, int xb, int yb, unsigned& img, int& y, int& x) {
    x = (int)(e & ((1u << xb) - 1u));
    y = (int)((e >> xb) & ((1u << yb) - 1u));
    img = (unsigned)((unsigned long long)e >> (xb + yb));
}

// The table entry of image i, through the read-only data path.
__device__ __forceinline__ ImgDesc load_desc(const ImgDesc* t, unsigned i) {
    static_assert(sizeof(ImgDesc) == 48, "ImgDesc layout");
    const int4* p = reinterpret_cast<const int4*>(t + i);
    int4 v[3] = {__ldg(p), __ldg(p + 1), __ldg(p + 2)};
    ImgDesc d;
    memcpy(&d, v, sizeof(d));
    return d;
}

struct PassArgs {
    uint8_t* canvas[3];       // canvas base pointers (row 0, column 0 of each canvas)
    long long pitch;          // canvas row pitch in bytes (multiple of 16)
    int rows, cols;           // image size
    int alpha;
    int tiles_x;              // tile grid width (fused kernel)
    Ctrl* ctrl;
    // Pixel change maps (fused kernel launched repeatedly): three bitmaps of
    // rows x map_words 32-bit words; bit (c & 31) of word c >> 5 of row r =
    // image pixel (r, c) changed in the last pass of a launch.  Launch L
    // writes map L % 3, reads map (L + 2) % 3 and clears map (L + 1) % 3.
    // Null when unused.
    uint32_t* chg_maps;
    int map_words;            // words per image row
    // Change lists and bitmaps (list passes): changed pixels are appended,
    // packed by pack_entry, to a list (length ctrl->list_n[i]) and
    // set in the matching bitmap (rows x bm_words 32-bit words, bit c & 31 of
    // word c >> 5 of row r).  The fused launch writes set 0 with its last
    // pass; list pass t of the list-pass loop reads set t % 4, writes set
    // (t + 1) % 4 and clears bitmap (t + 3) % 4.  Null when unused.
    uint32_t* lists[4];
    unsigned list_cap;
    uint32_t* bitmaps[4];
    int bm_words;
    int write_prev;           // fused kernel: also write I_{t-1} to the third canvas
    GridBar* bar;             // list-pass loop barrier
    // Image table (hybrid schedule: fused launch + list-pass loop).  When
    // set, the fields above that describe one image (pitch, rows, cols,
    // tiles_x, bm_words) are unused: canvases and bitmaps are arenas, fused
    // tile b belongs to image tile_img[b], and list entries are packed with
    // (xb, yb).  img_k[i], when set, receives image i's k: the number of the
    // last pass that changed one of its pixels (all images run the same
    // passes, and an image that a pass leaves unchanged is at a fixed point).
    const ImgDesc* imgs;
    int nimg;
    int xb, yb;
    const int* tile_img;
    long long bm_total;       // words in one bitmap arena
    unsigned* img_k;
    int ntiles;               // fused-kernel tiles (all images)
    // Hybrid schedule: fused launch L (L = fused launches that ran before
    // it) writes change set L % 4, reads set (L + 3) % 4 and clears set
    // (L + 2) % 4.  Launches after the first run only while the previous
    // one's last pass changed so many pixels that a list pass would evaluate
    // more than relaunch_evals pixels; the list-pass loop then starts from
    // the last fused launch's set.
    int hybrid;
    long long relaunch_evals;
    // Fused kernel: a pass runs as an in-tile list pass when the previous
    // pass's changes need at most this many pixel evaluations in the tile
    // (0 = the kernel's built-in value), else as a dense pass.
    int tile_eval_max;
    // Hybrid schedule: the first fused launch reads a tile of image i from
    // the caller's image (dense rows of cols bytes; device memory or mapped
    // page-locked host memory) instead of canvas `cur`: `user0` for a single
    // image, ImgDesc::user for a batch; null = read the canvas.
    const uint8_t* user0;
    int list_ctas;            // list-pass loop CTAs (0 = as many as can be co-resident)
    // Test of the bounded barrier wait (HGRMS_OPT_WAIT_TEST): every grid
    // barrier of the list-pass loop waits for bar_extra arrivals more than
    // the launch has CTAs, and gives up after bar_spins polls (0 = the
    // built-in limit of one to two seconds).
    unsigned bar_extra = 0;
    unsigned bar_spins = 0;
    // Hybrid schedule: tensor maps for the fused kernel's tile loads by TMA,
    // kTmaMapsPerImage per image (canvas 0, 1, 2, then the caller's image),
    // each a 3-D view (16 bytes, 16-byte chunks of a row, rows) whose box is
    // one tile with its halo.  Null: tiles are read with ordinary loads.
    // tma_user: the caller's-image maps are valid (aligned device images), so
    // the first fused launch loads from them too.
    const CUtensorMap* tmaps = nullptr;
    int tma_user = 0;
};
constexpr int kTmaMapsPerImage = 4;

// The root mean square of Algorithm 2 in integers, floor(sqrt(floor(sum /
// flag))), for 0 <= sum <= flag * 255^2 (so sum < 2^24) and 2 <= flag <= 225,
// in two exact steps that need no conversion or division instruction.
//
// Quotient: floor(sum / flag) is the high word of sum * m with m = ceil(2^32
// / flag) (division by an invariant integer through multiplication, Granlund
// and Montgomery, 1994).  With e = m * flag - 2^32 < flag <= 225 and sum =
// q * flag + r, sum * m / 2^32 = q + (r + sum * e / 2^32) / flag, and sum * e
// < 2^24 * 225 < 2^32 keeps the bracket below flag.  (Also checked for every
// sum and every flag of a replaced pixel on the CPU.)
//
// Square root of q <= 255^2: q is made a float through its bit pattern (2^23
// + q has q in the low mantissa bits), rsqrtf is within 2 ulp, so q *
// rsqrtf(q) is within 10^-4 of sqrt(q); adding 1.5 * 2^23 (unit spacing)
// leaves its nearest integer in the low bits, which is floor(sqrt(q)) or one
// more, and r * r > q removes the excess.  q = 0 takes rsqrtf(1), so the
// product is 0.  Checked for every flag and quotient through hgrms_rms.
__device__ __forceinline__ int isqrt_u16(int q) {
    const float qf = __int_as_float(0x4B000000 | q) - 8388608.f;
    const float s = qf * rsqrtf(fmaxf(qf, 1.f));
    int r = __float_as_int(s + 12582912.f) - 0x4B400000;
    r -= (r * r > q) ? 1 : 0;
    return r;
}

// ceil(2^32 / d) for 2 <= d <= 2^32.
__host__ __device__ constexpr unsigned recip32(unsigned d) {
    return (unsigned)((0x100000000ull + d - 1u) / d);
}

__device__ __forceinline__ int rms_div(int sum, unsigned m) {
    return isqrt_u16((int)__umulhi((unsigned)sum, m));
}

// The root mean square of a replaced pixel of a (2B + 1)^2 window: the
// replacement test flag > pix_count - 3 leaves flag in {P - 2, P - 1, P},
// whose reciprocals are compile-time constants.
template <int B>
__device__ __forceinline__ int rms_window(int sum, int flag) {
    constexpr int P = (2 * B + 1) * (2 * B + 1);
    const unsigned m = flag == P ? recip32(P) : (flag == P - 1 ? recip32(P - 1) : recip32(P - 2));
    return rms_div(sum, m);
}

// fp16 value of an integer 0 <= v <= 255 without a conversion instruction:
// the bit pattern 0x6400 + v is the fp16 number 1024 + v, and subtracting
// 1024 is exact.
__device__ __forceinline__ __half u8_to_half(int v) {
    return __hsub(__ushort_as_half((unsigned short)(0x6400 + v)), __ushort_as_half((unsigned short)0x6400));
}

// d = prmt(a, b, sel) in the generic mode, whose selector nibbles with bit 3
// set replicate the sign bit of the chosen byte (not available through
// __byte_perm).
__device__ __forceinline__ uint32_t prmt_sign(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Warp-wide exclusive prefix sum of n; *total receives the sum.
__device__ __forceinline__ int warp_excl_scan(const int lane, const int n, int* total) {
    int incl = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    *total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - n;
}

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
// set when pass t changed a pixel of this CTA's share of the image.  The last
// CTA to arrive folds the launch's mask into the iteration state: k grows by
// the number of leading changing passes; a pass that changed nothing means
// the image is a fixed point (every later pass is a no-op, so the canvas
// written by this launch holds the final image).  new_cur / new_aux are the
// canvases the launch leaves as `cur` and `aux`.
// Returns true in the last CTA.
__device__ __forceinline__ bool finish_launch(Ctrl* c, unsigned cta_mask, int np, unsigned nctas,
                                              unsigned new_cur, unsigned new_aux) {
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
        c->cur = new_cur;
        c->aux = new_aux;
        c->work_launches += 1u;
        c->executed += (unsigned)np;
        c->done = 0u;
        __threadfence();
        return true;
    }
    return false;
}

// Appends to a global change list staged per warp in shared memory, so that
// a CTA reserves space in the global list with one atomic (same-address
// atomics from every warp of a large grid serialise in L2).
struct StagedList {
    static constexpr int kCap = 256;  // entries per warp buffer
    uint32_t* buf;                    // this warp's buffer
    int n;                            // entries in it (warp-uniform)
    unsigned total;                   // entries this warp appended since it was last reset (warp-uniform)
};

// Warp-collective: append this lane's value when `want`.  A buffer that
// cannot take another full warp is written out with a warp-level atomic
// (rare; only for CTAs with very many changes).
__device__ __forceinline__ void staged_append(StagedList& sl, uint32_t* list, unsigned* n, unsigned cap, bool want,
                                              uint32_t v, int lane) {
    const unsigned bal = __ballot_sync(0xffffffffu, want);
    if (!bal) return;
    if (sl.n > StagedList::kCap - 32) {
        __syncwarp();
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(n, (unsigned)sl.n);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int i = lane; i < sl.n; i += 32)
            if (base + i < cap) list[base + i] = sl.buf[i];
        __syncwarp();
        sl.n = 0;
    }
    if (want) sl.buf[sl.n + __popc(bal & ((1u << lane) - 1u))] = v;
    sl.n += __popc(bal);
    sl.total += (unsigned)__popc(bal);
}

// Warp-collective: append entry(b) for every set bit b of this lane's mask m
// (one warp scan for the whole warp).  A round that does not fit the buffer
// writes it out first; one larger than a whole buffer goes straight to the
// list.
template <class Entry>
__device__ __forceinline__ void staged_append_mask(StagedList& sl, uint32_t* list, unsigned* n, unsigned cap,
                                                   uint32_t m, int lane, Entry entry) {
    int total;
    const int off = warp_excl_scan(lane, __popc(m), &total);
    if (!total) return;
    if (sl.n + total > StagedList::kCap) {
        __syncwarp();
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(n, (unsigned)sl.n);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int e = lane; e < sl.n; e += 32)
            if (base + e < cap) list[base + e] = sl.buf[e];
        __syncwarp();
        sl.n = 0;
    }
    if (total > StagedList::kCap) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(n, (unsigned)total);
        unsigned pos = __shfl_sync(0xffffffffu, base, 0) + (unsigned)off;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            if (pos < cap) list[pos] = entry(b);
            ++pos;
        }
    } else {
        int pos = sl.n + off;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            sl.buf[pos++] = entry(b);
        }
        sl.n += total;
    }
    __syncwarp();
    sl.total += (unsigned)total;
}

// Block-collective (all threads): write every warp's staged entries to the
// global list with one atomic per CTA.  `counts` is shared scratch of one int
// per warp plus one; at most 32 warps.
__device__ __forceinline__ void staged_flush(StagedList& sl, uint32_t* list, unsigned* n, unsigned cap,
                                             int* counts, int nwarps) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncwarp();
    if (lane == 0) counts[warp] = sl.n;
    __syncthreads();
    if (warp == 0) {
        // Exclusive prefix of the warps' counts (nwarps <= 32).
        int total;
        const int ex = warp_excl_scan(lane, lane < nwarps ? counts[lane] : 0, &total);
        if (lane < nwarps) counts[lane] = ex;
        if (lane == 0) counts[nwarps] = total ? (int)atomicAdd(n, (unsigned)total) : 0;
    }
    __syncthreads();
    const unsigned base = (unsigned)counts[nwarps] + (unsigned)counts[warp];
    for (int i = lane; i < sl.n; i += 32)
        if (base + i < cap) list[base + i] = sl.buf[i];
    sl.n = 0;
}

}  // namespace hg
