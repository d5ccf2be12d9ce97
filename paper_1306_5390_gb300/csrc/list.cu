// List passes: passes of Algorithms 1-2 that evaluate only the pixels that
// can change, all run by one persistent (cooperative) launch.
//
// A pixel's output in pass t depends only on its (2 beta + 1)^2 window in the
// image of pass t-1, so a pixel with no changed pixel (in pass t-1) within
// beta keeps its value.  Each pass walks the list of pixels the previous
// pass changed and evaluates every pixel q within beta of one of them once,
// by the changed pixel p that "owns" q: the first changed pixel, in raster
// order, of q's window (read from the previous pass's change bitmap).  For
// beta 1 one thread takes one changed pixel p, loads its 5 x 5
// neighbourhood and evaluates the pixels of p's 3 x 3 window that p owns
// from registers.  For wider windows one thread takes one (changed
// pixel, window row) pair, decides ownership for the whole row from one
// bitmap word per window row, and queues the owned pixels in shared memory;
// the CTA then evaluates its queue with all threads, so the evaluations run
// without idle lanes.  Results go to the
// partner canvas, which already agrees with the current image at every pixel
// that is not evaluated (see Ctrl); pixels that change form the next list and
// bitmap.  When the previous list overflowed its capacity, the pass evaluates
// and writes every pixel instead.
//
// Passes are separated by a grid-wide barrier (all CTAs are co-resident, by
// cooperative launch).  Every CTA tracks k, the converged flag and the
// current canvas itself from values that are final at the barrier, so one
// barrier per pass suffices; four list/bitmap sets rotate so that each set
// is reset or cleared only while no CTA can still touch it.  Waits at the
// barrier are bounded: after one to two seconds the kernel records an error and
// returns, and the call reports HGRMS_ETIMEOUT.
#include "common.cuh"
#include "kernels.h"

namespace hg {

namespace {

constexpr int kListThreads = 512;

// Loads of the bitmaps and canvases that the previous pass wrote go through
// L1 (__ldca): nearby evaluations of one CTA read overlapping windows, and an
// L2-only load moves a whole 32-byte sector per 4-byte word.  This is
// coherent because every pass starts after the grid barrier, whose
// gpu-scope acquire (thread 0) and CTA barrier order each thread's later
// loads after every write of the previous pass - the pattern of a grid-wide
// synchronisation, after which ordinary loads observe the other CTAs' writes.
// Nothing a pass reads is written during the same pass.

// Bits [start, start + 32) of a bitmap row (outside [0, 32 * nwords): 0).
__device__ __forceinline__ uint32_t row_bits(const uint32_t* __restrict__ row, int nwords, int start) {
    const int w0 = start >= 0 ? (start >> 5) : -((31 - start) >> 5);
    const int sh = start - 32 * w0;
    const uint32_t a = (w0 >= 0 && w0 < nwords) ? __ldca(row + w0) : 0u;
    const uint32_t b = (w0 + 1 >= 0 && w0 + 1 < nwords) ? __ldca(row + w0 + 1) : 0u;
    return sh ? ((a >> sh) | (b << (32 - sh))) : a;
}

// Algorithm 2 for an interior pixel (card <= 2 is implied by flag >
// pix_count - 3 for alpha >= 1, and card is 0 for alpha = 0).  `p` points at
// the pixel in a row-major byte array with row stride `stride`.
template <int B>
__device__ __forceinline__ int eval_pixel(const uint8_t* p, long long stride, int alpha) {
    const int ip = p[0];
    int sum = 0, flag = 0;
#pragma unroll
    for (int dy = -B; dy <= B; ++dy)
#pragma unroll
        for (int dx = -B; dx <= B; ++dx) {
            const int v = p[dy * stride + dx];
            const bool open = !(v < ip + alpha + 1 && v > ip - alpha);
            sum += open ? v * v : 0;
            flag += open ? 1 : 0;
        }
    constexpr int kPixCount = (2 * B + 1) * (2 * B + 1);
    if (flag > kPixCount - 3) return rms_window<B>(sum, flag);
    return ip;
}

// Byte mask (0xFF per byte) of the bytes v_j of v with lo <= v_j <= hi, for
// kl = (256 - lo) and kh = (256 - (hi + 1)) in both 16-bit halves, 0 <= lo <=
// 256 and 0 <= hi + 1 <= 256.  The even and the odd bytes are taken apart
// into 16-bit lanes; in a lane, byte + 256 - lo lies in 0..511 and has bit 8
// set exactly when byte >= lo, and byte + 256 - (hi + 1) has it set exactly
// when byte > hi (no carry reaches the next lane).
__device__ __forceinline__ uint32_t bytes_in_range(uint32_t v, uint32_t kl, uint32_t kh) {
    const uint32_t e = v & 0x00FF00FFu, o = __byte_perm(v, 0u, 0x4341u);
    const uint32_t ce = (e + kl) & ~(e + kh);
    const uint32_t co = (o + kl) & ~(o + kh);
    return (((ce >> 8) & 0x00010001u) | (co & 0x01000100u)) * 0xFFu;
}

// Algorithm 2 for an interior pixel whose (2B + 1)^2 window is loaded as
// rows of bytes (win[r][j / 4] byte j % 4 = value at offset (r - B, j - B)),
// four values at a time: a value v is closed when ip - alpha < v <= ip +
// alpha (bytes_in_range with lo = max(ip - alpha + 1, 0), hi = min(ip +
// alpha, 255); for alpha = 0 nothing is); the open values' squares sum in
// one 4-way dot product per word and a second one with 0x01010101 counts
// the open values (255 each).  For beta 2 the fifth value of each
// row is gathered four rows to a word first.  Returns the new value (ip when
// the pixel is not replaced; card <= 2 is implied by flag > pix_count - 3
// for alpha >= 1, and card is 0 for alpha = 0).
template <int B>
__device__ __forceinline__ int eval_window(const uint32_t (&win)[2 * B + 1][(2 * B + 4) / 4], int alpha) {
    constexpr int W = 2 * B + 1, NW = (W + 3) / 4, P = W * W;
    const int ip = (int)((win[B][B / 4] >> (8 * (B % 4))) & 0xffu);
    const int lo = max(ip - alpha + 1, 0), hi = min(ip + alpha, 255);
    const uint32_t kl = 0x01000100u - (uint32_t)lo * 0x00010001u;
    const uint32_t kh = 0x01000100u - (uint32_t)(hi + 1) * 0x00010001u;
    unsigned sum = 0u, open255 = 0u;  // 255 per open value
    auto word = [&](uint32_t v, uint32_t ok) {
        const uint32_t open = ~bytes_in_range(v, kl, kh) & ok;
        sum = __dp4a(v & open, v, sum);
        open255 = __dp4a(open, 0x01010101u, open255);
    };
    if constexpr (B == 2) {
        // Values -2..1 of every row, then the values +2 of rows 0-3 in one word and of row 4.
#pragma unroll
        for (int r = 0; r < W; ++r) word(win[r][0], 0xFFFFFFFFu);
        const uint32_t t01 = __byte_perm(win[0][1], win[1][1], 0x0040u);
        const uint32_t t23 = __byte_perm(win[2][1], win[3][1], 0x0040u);
        word(__byte_perm(t01, t23, 0x5410u), 0xFFFFFFFFu);
        word(win[4][1], 0x000000FFu);
    } else {
#pragma unroll
        for (int r = 0; r < W; ++r)
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                constexpr int kLast = W - 4 * (NW - 1);  // values in the last word of a row
                const uint32_t ok = (k < NW - 1 || kLast == 4) ? 0xFFFFFFFFu : ((1u << (8 * kLast)) - 1u);
                word(win[r][k], ok);
            }
    }
    if (open255 <= 255u * (P - 3)) return ip;
    const unsigned m = open255 == 255u * P ? recip32(P) : (open255 == 255u * (P - 1) ? recip32(P - 1) : recip32(P - 2));
    return rms_div((int)sum, m);
}

// Grid-wide barrier over co-resident CTAs that also sums one count over all
// CTAs (*count: this CTA's contribution, in shared memory; *total receives
// the sum).  Barrier number b (1, 2, ...) uses counter (b & 1), a 64-bit
// word whose low half counts arrivals and whose high half accumulates the
// counts.  Each CTA arrives with one release reduction (no value returned,
// so no round trip) and polls its counter until the low half reaches the
// barrier's target; counters are never reset within a call, so the target
// of the n-th use of a counter is n * nblocks (plus `extra`, which only the
// test of the bounded wait sets: an arrival that never comes).  The high half's growth since
// this counter's previous use is this barrier's sum: a CTA can arrive at the
// next barrier of the same counter only after every CTA has passed the
// barrier in between, hence after every CTA has read this one's value.  The
// wait is bounded; returns false (for every thread of the CTA) when it gave
// up.
__device__ __forceinline__ bool grid_barrier(GridBar* b, Ctrl* c, unsigned nblocks, unsigned& nbar,
                                             const unsigned* count, unsigned (&prev_hi)[2], unsigned& total,
                                             unsigned extra, unsigned max_spins) {
    __shared__ unsigned s_total;
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        const unsigned bn = nbar + 1u;
        const unsigned par = bn & 1u;
        unsigned long long* ctr = &b->ctr[par].v;
        const unsigned long long add = 1ull + ((unsigned long long)*count << 32);
        const unsigned target = ((bn + 1u) >> 1) * nblocks + extra;  // uses of this counter so far x CTAs
        // No separate fence: the CTA barrier above orders every thread's
        // writes of this pass before thread 0's release reduction, and a
        // release is cumulative (it makes visible at gpu scope what its
        // thread has observed, here through the CTA barrier), so a CTA whose
        // acquire load sees this arrival sees those writes too.  (A fence
        // here measured 4-7 % of the list passes on 8192 x 8192.)
        asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(ctr), "l"(add) : "memory");
        unsigned spins = 0;
        unsigned long long v = 0;
        while (true) {
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
            if ((unsigned)v >= target) break;
            if (++spins > max_spins) {  // built-in limit 2^22: one to two seconds
                atomicExch(&c->error, 1u);
                ok = 0;
                break;
            }
            if (spins > 16) __nanosleep(64);
        }
        const unsigned hi = (unsigned)(v >> 32);
        s_total = ok ? hi - prev_hi[par] : 0u;
        prev_hi[par] = hi;
        nbar = bn;
    }
    ok = __syncthreads_and(ok);
    total = s_total;
    return ok != 0;
}

// W bytes of a canvas row starting at p, realigned into ((W + 3) / 4)
// words (byte j at bits 8 (j % 4) of word j / 4); reads whole aligned words,
// which the canvas padding keeps in bounds.
template <int W>
__device__ __forceinline__ void load_row_bytes(const uint8_t* p, uint32_t (&r)[(W + 3) / 4]) {
    constexpr int NW = (W + 3) / 4;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t* q = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
    const uint32_t sh = (uint32_t)(a & 3u) * 8u;
    uint32_t w[NW + 1];
#pragma unroll
    for (int i = 0; i <= NW; ++i) w[i] = __ldca(q + i);
#pragma unroll
    for (int i = 0; i < NW; ++i) r[i] = __funnelshift_r(w[i], w[i + 1], sh);
}

// Warp-collective: set the bit of `img` in the CTA's changed-image bitmap
// for every lane with `ch` (one shared atomic per distinct image).
__device__ __forceinline__ void mark_image(uint32_t* bits, bool ch, unsigned img, int lane) {
    const unsigned bal = __ballot_sync(0xffffffffu, ch);
    if (!bal) return;
    const unsigned peers = __match_any_sync(0xffffffffu, ch ? img : 0xffffffffu);
    if (ch && (int)(__ffs(peers & bal) - 1) == lane) atomicOr(bits + (img >> 5), 1u << (img & 31));
}

}  // namespace

// kBatch = false: one image, described by the launch arguments (pitch, rows,
// cols, bm_words; entries packed 16/16); true: the image table.
template <int B, bool kBatch>
__global__ void __launch_bounds__(kListThreads, 2) list_loop_kernel(PassArgs a) {
    constexpr int W = 2 * B + 1, P = W * W;
    constexpr int kWarps = kListThreads / 32;
    __shared__ int s_np;
    __shared__ unsigned s_k, s_cur, s_aux, s_maxk, s_gen, s_base;
    __shared__ unsigned s_n, s_nclr, s_app;
    __shared__ uint32_t stage_all[kWarps][StagedList::kCap];
    __shared__ int s_counts[kWarps + 1];
    __shared__ unsigned long long s_evals;
    __shared__ uint32_t s_imgbits[kBatch ? kMaxBatchImages / 32 : 1];  // images changed in this pass (by this CTA)
    __shared__ uint32_t s_queue[B == 1 ? 1 : kListThreads * W];  // pixels this CTA evaluates in the current chunk
    __shared__ int s_qn[2];  // queue lengths; chunks alternate between them
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctrl* ctrl = a.ctrl;
    if (tid == 0) {
        s_evals = 0ull;
        s_qn[0] = 0;
        s_qn[1] = 0;
        s_np = launch_passes(ctrl, 1);
        s_k = __ldcg(&ctrl->k);
        s_cur = __ldcg(&ctrl->cur);
        s_aux = __ldcg(&ctrl->aux);
        s_maxk = __ldcg(&ctrl->max_k);
        s_gen = 0u;  // barriers completed; the barrier struct is zeroed at the start of every call
        // The last fused launch wrote change set (fused launches - 1) % 4.
        s_base = (__ldcg(&ctrl->fused_work) + 3u) & 3u;
    }
    if constexpr (kBatch)
        for (int i = tid; i < kMaxBatchImages / 32; i += kListThreads) s_imgbits[i] = 0u;
    __syncthreads();
    if (s_np == 0) return;  // the fused launch already finished the call
    unsigned k = s_k, cur = s_cur, aux = s_aux, gen = s_gen;
    unsigned prev_hi[2] = {0u, 0u};  // thread 0: counts seen at the last use of each barrier counter
    const int base = (int)s_base;
    const unsigned max_k = s_maxk;
    bool converged = false, failed = false;
    int passes = 0;
    unsigned evals = 0;
    int qpar = 0;  // queue counter of the next chunk (CTA-uniform)
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
    const long long warp_base = (long long)blockIdx.x * blockDim.x + (tid & ~31);
    // The single image as a table entry (its offsets are 0).
    ImgDesc one;
    if constexpr (!kBatch) {
        one.off = 0;
        one.bm_off = 0;
        one.pitch = (int)a.pitch;
        one.rows = a.rows;
        one.cols = a.cols;
        one.tiles_x = 0;
        one.tile0 = 0;
        one.bm_words = a.bm_words;
        one.user = nullptr;
    }
    constexpr int kXb = 16, kYb = 16;
    const int xb = kBatch ? a.xb : kXb, yb = kBatch ? a.yb : kYb;
    StagedList sl{stage_all[warp], 0, 0u};
    // List lengths: n_cur = entries of the list this pass reads (appended by
    // the previous pass), n_last = those of the list the previous pass read
    // (whose bitmap this pass clears); later lengths come from the barrier.
    if (tid == 0) {
        s_n = __ldcg(&ctrl->list_n[base]);
        s_nclr = __ldcg(&ctrl->list_n[(base + 3) & 3]);
        s_app = 0u;
    }
    __syncthreads();
    unsigned n_cur = s_n, n_last = s_nclr;

    for (int t = 0; k < max_k; ++t) {
        const int si = (t + base) & 3, so = (t + base + 1) & 3, sc = (t + base + 3) & 3;
        const uint8_t* in_arena = a.canvas[cur];
        uint8_t* out_arena = a.canvas[aux];
        const uint32_t* prev = a.lists[si];
        const uint32_t* bm_prev = a.bitmaps[si];
        uint32_t* next = a.lists[so];
        uint32_t* bm_next = a.bitmaps[so];
        unsigned* nnext = &ctrl->list_n[so];
        if (tid == 0 && blockIdx.x == 0) {
            // Set (t + base + 2) % 4 is next written by pass t + 1; its list
            // was last read (to clear its bitmap) in pass t - 1.
            ctrl->list_n[(t + base + 2) & 3] = 0u;
        }
        const unsigned n = n_cur, nclr = n_last;
        // The first list entry this thread reads (beta 1: pair warp_base +
        // lane; wider windows: task tid * gridDim.x + blockIdx.x), loaded
        // before the bitmap clearing below so that the two loads overlap.
        uint32_t pk_first = 0u;
        if (n <= a.list_cap) {
            const long long i0 = (long long)tid * gridDim.x + blockIdx.x;
            const long long per = B == 1 ? 1 : W;
            if (i0 < (long long)n * per) pk_first = __ldcg(prev + (unsigned)(i0 / per));
        }
        // Clear bitmap sc (written by pass t - 2, read by pass t - 1) for pass
        // t + 2: walk its list, or clear it all if the list overflowed.
        {
            const uint32_t* clr = a.lists[sc];
            uint32_t* bm_clr = a.bitmaps[sc];
            if (nclr <= a.list_cap) {
                for (long long i = gtid; i < nclr; i += gthreads) {
                    unsigned img;
                    int y, x;
                    unpack_entry(clr[i], xb, yb, img, y, x);
                    const ImgDesc d = kBatch ? load_desc(a.imgs, img) : one;
                    bm_clr[d.bm_off + (long long)y * d.bm_words + (x >> 5)] = 0u;
                }
            } else {
                for (long long i = gtid; i < a.bm_total; i += gthreads) bm_clr[i] = 0u;
            }
        }
        if (n <= a.list_cap && B == 1) {
            // beta 1: one thread per changed pixel p.  It loads p's 5 x 5
            // neighbourhood and the previous pass's change bits of the rows
            // up to p's, and evaluates every pixel q of p's 3 x 3 window
            // that p owns (no changed pixel of q's window precedes p in
            // raster order) from those registers.  Changed pixels are dealt
            // to the CTAs in turn.
            long long i = (long long)tid * gridDim.x + blockIdx.x;
            uint32_t pk = pk_first;
            for (long long c0 = 0; c0 + blockIdx.x < (long long)n; c0 += gthreads, i += gthreads) {
                const long long inext = i + gthreads;
                const uint32_t pk_next = inext < (long long)n ? __ldcg(prev + (unsigned)inext) : 0u;
                uint32_t chm = 0u;  // bit (dy + 1) * 3 + dx + 1: q = p + (dy, dx) changed
                unsigned img = 0;
                int py = 0, px = 0;
                if (i < (long long)n) {
                    unpack_entry(pk, xb, yb, img, py, px);
                    const ImgDesc d = kBatch ? load_desc(a.imgs, img) : one;
                    const uint32_t* bmp = bm_prev + d.bm_off;
                    const uint8_t* in = in_arena + d.off + (long long)kPadY * d.pitch + kPadX;
                    uint8_t* out = out_arena + d.off + (long long)kPadY * d.pitch + kPadX;
                    // Change bits of rows py - 2 .. py, columns px - 2 .. (bit j: column px - 2 + j).
                    uint32_t rb[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const int gy = py - 2 + r;
                        rb[r] = gy >= 0 ? row_bits(bmp + (size_t)gy * d.bm_words, d.bm_words, px - 2) : 0u;
                    }
                    // Rows py - 2 .. py + 2, bytes px - 2 .. px + 2 (the canvas padding keeps them in bounds).
                    uint32_t nb[5][2];
                    const long long off = (long long)py * d.pitch + px;
#pragma unroll
                    for (int r = 0; r < 5; ++r) load_row_bytes<5>(in + off + (long long)(r - 2) * d.pitch - 2, nb[r]);
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int qy = py + dy, qx = px + dx;
                            if (qy < 1 || qy >= d.rows - 1 || qx < 1 || qx >= d.cols - 1) continue;
                            // Ownership: q's window rows above p's hold no change, and
                            // p's row none left of p (bits dx + 1 .. 1).
                            bool owner = true;
#pragma unroll
                            for (int r = dy + 1; r <= dy + 3; ++r) {
                                if (r < 2 && (rb[r] & (7u << (dx + 1)))) owner = false;
                                if (r == 2 && (rb[2] & 3u & ~((1u << (dx + 1)) - 1u))) owner = false;
                            }
                            if (!owner) continue;
                            uint32_t w3[3][1];
#pragma unroll
                            for (int r = 0; r < 3; ++r)
                                w3[r][0] = __funnelshift_r(nb[dy + 1 + r][0], nb[dy + 1 + r][1], 8 * (dx + 1));
                            const int ip = (int)((w3[1][0] >> 8) & 0xffu);
                            const int nv = eval_window<1>(w3, a.alpha);
                            ++evals;
                            out[(long long)qy * d.pitch + qx] = (uint8_t)nv;
                            if (nv != ip) {
                                chm |= 1u << ((dy + 1) * 3 + dx + 1);
                                atomicOr(bm_next + d.bm_off + (size_t)qy * d.bm_words + (qx >> 5), 1u << (qx & 31));
                            }
                        }
                }
                if (kBatch && a.img_k) mark_image(s_imgbits, chm != 0u, img, lane);
                // Append the changed pixels (one warp scan per round).
                staged_append_mask(sl, next, nnext, a.list_cap, chm, lane, [&](int bt) {
                    return pack_entry(img, py + bt / 3 - 1, px + bt % 3 - 1, xb, yb);
                });
                pk = pk_next;
            }
        } else if (n <= a.list_cap) {
            // Chunks of one task per thread: task (changed pixel p, window
            // row dy) finds the pixels q = p + (dy, dx) that p owns and
            // queues them in shared memory (phase A); the CTA then evaluates
            // its queue with every thread (phase B).  Tasks are dealt to the
            // CTAs in turn (task c0 + tid * gridDim.x + blockIdx.x of chunk
            // c0), so every CTA gets an equal share even when there are fewer
            // tasks than threads.
            const long long ntask = (long long)n * W;
            long long i = (long long)tid * gridDim.x + blockIdx.x;
            uint32_t pk = pk_first;  // later chunks' entries are loaded one chunk early
            for (long long c0 = 0; c0 + blockIdx.x < ntask; c0 += gthreads, i += gthreads) {
                const long long inext = i + gthreads;
                const uint32_t pk_next = inext < ntask ? __ldcg(prev + (unsigned)(inext / W)) : 0u;
                // Phase A.  Ownership: no changed pixel of q's window precedes
                // p in raster order.  rb[r] = the previous pass's changes in
                // row qy - B + r, columns px - 2B .. px + 2B (bit j: column
                // px - 2B + j); q = (qy, px + dx) has window columns bits
                // dx + B .. dx + 3B, its rows above py must have none and row
                // py none left of p (bits below 2B).
                unsigned own = 0u;  // bit dx + B: this task evaluates q
                unsigned img = 0;
                int py = 0, px = 0, qy = 0;
                if (i < ntask) {
                    const int dy = (int)(i % W) - B;
                    unpack_entry(pk, xb, yb, img, py, px);
                    const ImgDesc d = kBatch ? load_desc(a.imgs, img) : one;
                    qy = py + dy;
                    if (qy >= B && qy < d.rows - B) {
                        const uint32_t* bmp = bm_prev + d.bm_off;
                        uint32_t rb[2 * B + 1];
#pragma unroll
                        for (int r = 0; r <= 2 * B; ++r) {
                            const int gy = qy - B + r;
                            rb[r] = (gy <= py) ? row_bits(bmp + (size_t)gy * d.bm_words, d.bm_words, px - 2 * B) : 0u;
                        }
                        uint32_t before = 0u;
#pragma unroll
                        for (int r = 0; r <= 2 * B; ++r) {
                            const int gy = qy - B + r;
                            if (gy < py) before |= rb[r];
                            if (gy == py) before |= rb[r] & ((1u << (2 * B)) - 1u);
                        }
#pragma unroll
                        for (int dx = -B; dx <= B; ++dx) {
                            const int qx = px + dx;
                            const uint32_t wm = ((1u << W) - 1u) << (dx + B);
                            if (qx >= B && qx < d.cols - B && (before & wm) == 0u) own |= 1u << (dx + B);
                        }
                    }
                }
                {
                    // Queue the owned pixels (one shared atomic per warp).
                    const int cnt = __popc(own);
                    int incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const int wtot = __shfl_sync(0xffffffffu, incl, 31);
                    int wbase = 0;
                    if (lane == 31 && wtot) wbase = atomicAdd(&s_qn[qpar], wtot);
                    int pos = __shfl_sync(0xffffffffu, wbase, 31) + incl - cnt;
                    while (own) {
                        const int b = __ffs(own) - 1;
                        own &= own - 1u;
                        s_queue[pos++] = pack_entry(img, qy, px + b - B, xb, yb);
                    }
                }
                __syncthreads();
                // Phase B: Algorithm 2 for every queued pixel.
                const int qn = s_qn[qpar];
                // The other counter was last read before the previous chunk's
                // final barrier and is next used after this chunk's.
                if (tid == 0) s_qn[qpar ^ 1] = 0;
                for (int j0 = warp * 32; j0 < qn; j0 += kListThreads) {
                    const int j = j0 + lane;
                    bool ch = false;
                    uint32_t v = 0;
                    unsigned qimg = 0;
                    if (j < qn) {
                        int y, x;
                        unpack_entry(s_queue[j], xb, yb, qimg, y, x);
                        const ImgDesc d = kBatch ? load_desc(a.imgs, qimg) : one;
                        const uint8_t* in = in_arena + d.off + (long long)kPadY * d.pitch + kPadX;
                        constexpr int NW = (W + 3) / 4;
                        uint32_t win[W][NW];
                        const long long off = (long long)y * d.pitch + x;
#pragma unroll
                        for (int r = 0; r < W; ++r) load_row_bytes<W>(in + off + (long long)(r - B) * d.pitch - B, win[r]);
                        ++evals;
                        const int ip = (int)((win[B][B / 4] >> (8 * (B % 4))) & 0xffu);
                        const int nv = eval_window<B>(win, a.alpha);
                        out_arena[d.off + (long long)kPadY * d.pitch + kPadX + off] = (uint8_t)nv;
                        if (nv != ip) {
                            ch = true;
                            v = pack_entry(qimg, y, x, xb, yb);
                            atomicOr(bm_next + d.bm_off + (size_t)y * d.bm_words + (x >> 5), 1u << (x & 31));
                        }
                    }
                    if (kBatch && a.img_k) mark_image(s_imgbits, ch, qimg, lane);
                    staged_append(sl, next, nnext, a.list_cap, ch, v, lane);
                }
                __syncthreads();  // every thread has read the queue
                qpar ^= 1;
                pk = pk_next;
            }
        } else {
            // Previous list overflowed: evaluate and write every pixel of
            // every image.
            for (int im = 0; im < (kBatch ? a.nimg : 1); ++im) {
                const ImgDesc d = kBatch ? load_desc(a.imgs, (unsigned)im) : one;
                const uint8_t* in = in_arena + d.off + (long long)kPadY * d.pitch + kPadX;
                uint8_t* out = out_arena + d.off + (long long)kPadY * d.pitch + kPadX;
                const long long total = (long long)d.rows * d.cols;
                for (long long base = warp_base; base < total; base += gthreads) {
                    const long long i = base + lane;
                    bool ch = false;
                    uint32_t v = 0;
                    if (i < total) {
                        const int y = (int)(i / d.cols), x = (int)(i - (long long)y * d.cols);
                        const long long off = (long long)y * d.pitch + x;
                        ++evals;
                        const int ip = in[off];
                        int nv = ip;
                        if (y >= B && y < d.rows - B && x >= B && x < d.cols - B)
                            nv = eval_pixel<B>(in + off, d.pitch, a.alpha);
                        out[off] = (uint8_t)nv;
                        if (nv != ip) {
                            ch = true;
                            v = pack_entry((unsigned)im, y, x, xb, yb);
                            atomicOr(bm_next + d.bm_off + (size_t)y * d.bm_words + (x >> 5), 1u << (x & 31));
                        }
                    }
                        if (kBatch && a.img_k) mark_image(s_imgbits, ch, (unsigned)im, lane);
                    staged_append(sl, next, nnext, a.list_cap, ch, v, lane);
                }
            }
        }
        staged_flush(sl, next, nnext, a.list_cap, s_counts, kWarps);
        // Images this CTA changed in pass number k + 1 (staged_flush ends
        // with a block barrier, so every mark is in place).
        if (kBatch && a.img_k) {
            for (int w = tid; w < (a.nimg + 31) / 32; w += kListThreads) {
                uint32_t bits = s_imgbits[w];
                s_imgbits[w] = 0u;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    a.img_k[32 * w + b] = k + 1u;
                }
            }
        }
        ++passes;
        // Entries this CTA appended (every changed pixel appends one).
        if (lane == 0 && sl.total) atomicAdd(&s_app, sl.total);
        sl.total = 0u;
        unsigned appended = 0;
        if (!grid_barrier(a.bar, ctrl, gridDim.x, gen, &s_app, prev_hi, appended, a.bar_extra,
                          a.bar_spins ? a.bar_spins : (1u << 22))) {
            failed = true;
            break;
        }
        if (tid == 0) s_app = 0u;  // read by thread 0 inside the barrier only
        n_last = n_cur;
        n_cur = appended;
        if (appended == 0u) {
            converged = true;  // a fixed point: the output canvas equals the input
            break;
        }
        ++k;
        const unsigned tmp = cur;
        cur = aux;
        aux = tmp;
    }
    const unsigned ev = __reduce_add_sync(0xffffffffu, evals);
    if (lane == 0 && ev) atomicAdd(&s_evals, (unsigned long long)ev);
    __syncthreads();
    if (tid == 0) {
        if (s_evals) atomicAdd(&ctrl->evals_list, s_evals);
        if (blockIdx.x == 0 && !failed) {
            // Every CTA holds the same state; the barriers order these writes
            // after every CTA's reads of the control block.
            ctrl->k = k;
            if (converged) ctrl->converged = 1u;
            ctrl->cur = cur;
            ctrl->aux = aux;
            ctrl->work_launches += 1u;
            ctrl->executed += (unsigned)passes;
        }
    }
}

namespace {

template <int B, bool kBatch>
cudaError_t launch_loop_b(const PassArgs& a, int sms, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, list_loop_kernel<B, kBatch>, kListThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    unsigned grid = (unsigned)(sms * (per_sm < 2 ? per_sm : 2));
    if (a.list_ctas > 0 && (unsigned)a.list_ctas < grid) grid = (unsigned)a.list_ctas;
    // A cooperative launch (all CTAs co-resident), in the form that stream
    // capture into a CUDA graph accepts.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kListThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, list_loop_kernel<B, kBatch>, a);
}

template <int B>
cudaError_t launch_loop(const PassArgs& a, int sms, cudaStream_t s) {
    return a.nimg > 1 ? launch_loop_b<B, true>(a, sms, s) : launch_loop_b<B, false>(a, sms, s);
}

}  // namespace

cudaError_t launch_list(int beta, const PassArgs& a, int sms, cudaStream_t s) {
    switch (beta) {
        case 1: return launch_loop<1>(a, sms, s);
        case 2: return launch_loop<2>(a, sms, s);
        case 3: return launch_loop<3>(a, sms, s);
        case 4: return launch_loop<4>(a, sms, s);
        case 5: return launch_loop<5>(a, sms, s);
        case 6: return launch_loop<6>(a, sms, s);
        case 7: return launch_loop<7>(a, sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hg
