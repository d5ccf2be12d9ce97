// List pass: one pass of Algorithms 1-2 that evaluates only the pixels that
// can change.
//
// A pixel's output in pass t depends only on its (2 beta + 1)^2 window in the
// image of pass t-1, so a pixel with no changed pixel (in pass t-1) within
// beta keeps its value.  The kernel walks the list of pixels the previous
// pass changed; one thread takes one (changed pixel p, window offset) pair
// and evaluates q = p + offset if p "owns" q: p is the first changed pixel,
// in raster order, of q's window (read from the previous pass's change
// bitmap), so each pixel is evaluated exactly once.  Results go
// to the partner canvas, which already agrees with the current image at
// every pixel that is not evaluated (see Ctrl); pixels that change form the
// next list and bitmap.  When the previous list overflowed its capacity, the
// pass evaluates and writes every pixel instead.
#include "common.cuh"
#include "kernels.h"

namespace hg {

namespace {

// Bits [start, start + 32) of a bitmap row (outside [0, 32 * nwords): 0).
__device__ __forceinline__ uint32_t row_bits(const uint32_t* __restrict__ row, int nwords, int start) {
    const int w0 = start >= 0 ? (start >> 5) : -((31 - start) >> 5);
    const int sh = start - 32 * w0;
    const uint32_t a = (w0 >= 0 && w0 < nwords) ? __ldcg(row + w0) : 0u;
    const uint32_t b = (w0 + 1 >= 0 && w0 + 1 < nwords) ? __ldcg(row + w0 + 1) : 0u;
    return sh ? ((a >> sh) | (b << (32 - sh))) : a;
}

// Algorithm 2 for an interior pixel (card <= 2 is implied by flag >
// pix_count - 3 for alpha >= 1, and card is 0 for alpha = 0).  `p` points at
// the pixel in a row-major byte array with row stride `stride`.  sum < 2^24
// and flag <= 225, so the float quotient is exact to well under the gap to
// the next integer and its floor is floor(sum / flag); the square root is
// correctly rounded, so its floor is the integer square root (sum / flag is
// at most 255^2).
template <int B>
__device__ __forceinline__ int eval_pixel(const uint8_t* __restrict__ p, long long stride, int alpha) {
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
    if (flag > kPixCount - 3) {
        const float q = floorf(__fdiv_rn((float)sum, (float)flag));
        return (int)floorf(__fsqrt_rn(q));
    }
    return ip;
}

}  // namespace

constexpr int kListThreads = 512;

// Every pixel (the previous list overflowed): evaluate, write, record changes.
template <int B>
__device__ __forceinline__ void full_pass(const PassArgs& a, const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                          uint32_t* bm_next, uint32_t* next, unsigned* nnext, StagedList& sl,
                                          long long warp_base, long long gthreads, int lane, bool& any,
                                          unsigned& evals) {
    const long long total = (long long)a.rows * a.cols;
    for (long long base = warp_base; base < total; base += gthreads) {
        const long long i = base + lane;
        bool ch = false;
        uint32_t v = 0;
        if (i < total) {
            const int y = (int)(i / a.cols), x = (int)(i - (long long)y * a.cols);
            const long long off = (long long)y * a.pitch + x;
            ++evals;
            const int ip = in[off];
            int nv = ip;
            if (y >= B && y < a.rows - B && x >= B && x < a.cols - B) nv = eval_pixel<B>(in + off, a.pitch, a.alpha);
            out[off] = (uint8_t)nv;
            if (nv != ip) {
                ch = true;
                v = ((uint32_t)y << 16) | (uint32_t)x;
                atomicOr(bm_next + (size_t)y * a.bm_words + (x >> 5), 1u << (x & 31));
            }
        }
        any |= ch;
        staged_append(sl, next, nnext, a.list_cap, ch, v, lane);
    }
}

namespace {

// Bytes [c, c + 8 * NW) of a canvas row as NW little-endian 64-bit words
// (reads whole aligned 32-bit words; the canvas padding keeps them in bounds).
template <int NW>
__device__ __forceinline__ void load_bytes(const uint8_t* __restrict__ p, unsigned long long (&w)[NW]) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t* q = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
    const int sh = (int)(a & 3u) * 8;
    uint32_t r[2 * NW + 1];
#pragma unroll
    for (int i = 0; i < 2 * NW + 1; ++i) r[i] = __ldg(q + i);
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const uint32_t lo = __funnelshift_r(r[2 * i], r[2 * i + 1], sh);
        const uint32_t hi = __funnelshift_r(r[2 * i + 1], r[2 * i + 2], sh);
        w[i] = ((unsigned long long)hi << 32) | lo;
    }
}

}  // namespace

// Entry form (beta 1 and 2): one thread per changed pixel p.  The thread
// loads the (4 beta + 1)^2 image block around p and the change-bitmap rows
// above and at p into registers and evaluates every window pixel of p it
// owns, all with compile-time offsets.
template <int B>
__global__ void __launch_bounds__(kListThreads, 2) list_entry_kernel(PassArgs a) {
    constexpr int W = 2 * B + 1;
    constexpr int E = 4 * B + 1;         // block side
    constexpr int NW = (E + 7) / 8;      // 64-bit words per block row
    constexpr int kWarps = kListThreads / 32;
    __shared__ int s_np;
    __shared__ unsigned s_cur, s_aux, s_L, s_n, s_nclr;
    __shared__ uint32_t stage_all[kWarps][StagedList::kCap];
    __shared__ int s_counts[kWarps + 1];
    __shared__ unsigned long long s_evals;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_evals = 0ull;
        s_np = launch_passes(a.ctrl, 1);
        s_cur = __ldcg(&a.ctrl->cur);
        s_aux = __ldcg(&a.ctrl->aux);
        s_L = __ldcg(&a.ctrl->work_launches);
        s_n = __ldcg(&a.ctrl->list_n[(s_L + 2u) % 3u]);
        s_nclr = __ldcg(&a.ctrl->list_n[(s_L + 1u) % 3u]);
    }
    __syncthreads();
    if (s_np == 0) return;
    const unsigned L = s_L;
    const uint8_t* in = a.canvas[s_cur] + (long long)kPadY * a.pitch + kPadX;
    uint8_t* out = a.canvas[s_aux] + (long long)kPadY * a.pitch + kPadX;
    const uint32_t* prev = a.lists[(L + 2u) % 3u];
    const uint32_t* bm_prev = a.bitmaps[(L + 2u) % 3u];
    uint32_t* next = a.lists[L % 3u];
    uint32_t* bm_next = a.bitmaps[L % 3u];
    unsigned* nnext = &a.ctrl->list_n[L % 3u];
    const unsigned n = s_n;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
    const long long warp_base = (long long)blockIdx.x * blockDim.x + (tid & ~31);
    {
        const uint32_t* clr = a.lists[(L + 1u) % 3u];
        uint32_t* bm_clr = a.bitmaps[(L + 1u) % 3u];
        const unsigned nclr = s_nclr;
        if (nclr <= a.list_cap) {
            for (long long i = gtid; i < nclr; i += gthreads) {
                const uint32_t pk = clr[i];
                bm_clr[(size_t)(pk >> 16) * a.bm_words + ((pk & 0xffffu) >> 5)] = 0u;
            }
        } else {
            const size_t words = (size_t)a.rows * a.bm_words;
            for (size_t i = gtid; i < words; i += gthreads) bm_clr[i] = 0u;
        }
    }
    bool any = false;
    unsigned evals = 0;
    StagedList sl{stage_all[warp], 0};
    if (n > a.list_cap) full_pass<B>(a, in, out, bm_next, next, nnext, sl, warp_base, gthreads, lane, any, evals);
    const long long nent = n > a.list_cap ? 0 : (long long)n;
    for (long long base = warp_base; base < nent; base += gthreads) {
        const long long e = base + lane;
        const bool valid = e < nent;
        int py = 0, px = 0;
        unsigned long long blk[E][NW];
        uint32_t bmr[2 * B + 1];
        if (valid) {
            const uint32_t pk = __ldg(prev + e);
            py = (int)(pk >> 16);
            px = (int)(pk & 0xffffu);
            const uint8_t* b0 = in + (long long)(py - 2 * B) * a.pitch + (px - 2 * B);
#pragma unroll
            for (int r = 0; r < E; ++r) load_bytes<NW>(b0 + (long long)r * a.pitch, blk[r]);
#pragma unroll
            for (int r = 0; r <= 2 * B; ++r) {
                const int gy = py - 2 * B + r;
                bmr[r] = (gy >= 0) ? row_bits(bm_prev + (size_t)gy * a.bm_words, a.bm_words, px - 2 * B) : 0u;
            }
        }
#pragma unroll
        for (int dy = -B; dy <= B; ++dy)
#pragma unroll
            for (int dx = -B; dx <= B; ++dx) {
                const int cy = 2 * B + dy, cx = 2 * B + dx;  // block position of q
                const int y = py + dy, x = px + dx;
                bool ch = false;
                uint32_t v = 0;
                if (valid && y >= B && y < a.rows - B && x >= B && x < a.cols - B) {
                    constexpr uint32_t kWin = (1u << W) - 1u;
                    bool owner = true;
#pragma unroll
                    for (int r = cy - B; r < 2 * B; ++r)
                        if (bmr[r] & (kWin << (cx - B))) owner = false;
                    if (B - dx > 0 && (bmr[2 * B] & (kWin << (cx - B)) & ((1u << (2 * B)) - 1u))) owner = false;
                    if (owner) {
                        ++evals;
                        const int ip = (int)((blk[cy][cx >> 3] >> (8 * (cx & 7))) & 0xffu);
                        int sum = 0, flag = 0;
#pragma unroll
                        for (int ty = -B; ty <= B; ++ty)
#pragma unroll
                            for (int tx = -B; tx <= B; ++tx) {
                                const int by = cy + ty, bx = cx + tx;
                                const int t = (int)((blk[by][bx >> 3] >> (8 * (bx & 7))) & 0xffu);
                                const bool open = !(t < ip + a.alpha + 1 && t > ip - a.alpha);
                                sum += open ? t * t : 0;
                                flag += open ? 1 : 0;
                            }
                        int nv = ip;
                        if (flag > W * W - 3) {
                            const float qf = floorf(__fdiv_rn((float)sum, (float)flag));
                            nv = (int)floorf(__fsqrt_rn(qf));
                        }
                        out[(long long)y * a.pitch + x] = (uint8_t)nv;
                        if (nv != ip) {
                            ch = true;
                            v = ((uint32_t)y << 16) | (uint32_t)x;
                            atomicOr(bm_next + (size_t)y * a.bm_words + (x >> 5), 1u << (x & 31));
                        }
                    }
                }
                any |= ch;
                staged_append(sl, next, nnext, a.list_cap, ch, v, lane);
            }
    }
    staged_flush(sl, next, nnext, a.list_cap, s_counts, kWarps);
    const unsigned ev = __reduce_add_sync(0xffffffffu, evals);
    if (lane == 0 && ev) atomicAdd(&s_evals, (unsigned long long)ev);
    const int cta_any = __syncthreads_or(any);
    if (tid == 0) {
        if (s_evals) atomicAdd(&a.ctrl->evals_list, s_evals);
        finish_launch(a.ctrl, cta_any ? 1u : 0u, 1, gridDim.x, s_aux, s_cur);
    }
}


template <int B>
__global__ void __launch_bounds__(kListThreads, 2) list_kernel(PassArgs a) {
    constexpr int W = 2 * B + 1, P = W * W;
    constexpr int kWarps = kListThreads / 32;
    __shared__ int s_np;
    __shared__ unsigned s_cur, s_aux, s_L, s_n, s_nclr;
    __shared__ uint32_t stage_all[kWarps][StagedList::kCap];
    __shared__ int s_counts[kWarps + 1];
    __shared__ unsigned long long s_evals;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_evals = 0ull;
        s_np = launch_passes(a.ctrl, 1);
        s_cur = __ldcg(&a.ctrl->cur);
        s_aux = __ldcg(&a.ctrl->aux);
        s_L = __ldcg(&a.ctrl->work_launches);
        s_n = __ldcg(&a.ctrl->list_n[(s_L + 2u) % 3u]);
        s_nclr = __ldcg(&a.ctrl->list_n[(s_L + 1u) % 3u]);
    }
    __syncthreads();
    if (s_np == 0) return;
    const unsigned L = s_L;
    const uint8_t* in = a.canvas[s_cur] + (long long)kPadY * a.pitch + kPadX;
    uint8_t* out = a.canvas[s_aux] + (long long)kPadY * a.pitch + kPadX;
    const uint32_t* prev = a.lists[(L + 2u) % 3u];
    const uint32_t* bm_prev = a.bitmaps[(L + 2u) % 3u];
    uint32_t* next = a.lists[L % 3u];
    uint32_t* bm_next = a.bitmaps[L % 3u];
    unsigned* nnext = &a.ctrl->list_n[L % 3u];
    const unsigned n = s_n;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + tid;
    const long long warp_base = (long long)blockIdx.x * blockDim.x + (tid & ~31);

    // Clear the bitmap of pass L - 2 (written two launches ago, read by the
    // previous launch) for the next launch: walk its list, or clear it all if
    // the list overflowed.
    {
        const uint32_t* clr = a.lists[(L + 1u) % 3u];
        uint32_t* bm_clr = a.bitmaps[(L + 1u) % 3u];
        const unsigned nclr = s_nclr;
        if (nclr <= a.list_cap) {
            for (long long i = gtid; i < nclr; i += gthreads) {
                const uint32_t pk = clr[i];
                bm_clr[(size_t)(pk >> 16) * a.bm_words + ((pk & 0xffffu) >> 5)] = 0u;
            }
        } else {
            const size_t words = (size_t)a.rows * a.bm_words;
            for (size_t i = gtid; i < words; i += gthreads) bm_clr[i] = 0u;
        }
    }

    bool any = false;
    unsigned evals = 0;
    StagedList sl{stage_all[warp], 0};
    if (n <= a.list_cap) {
        // One thread per (changed pixel p, window offset) pair: q = p + offset
        // is evaluated by the thread of the first changed pixel of q's window
        // in raster order ("owner"), found in the previous pass's bitmap.
        const long long total = (long long)n * P;
        for (long long base = warp_base; base < total; base += gthreads) {
            const long long i = base + lane;
            bool ch = false;
            uint32_t v = 0;
            if (i < total) {
                const unsigned e = (unsigned)(i / P);
                const int o = (int)(i - (long long)e * P);
                const int dy = o / W - B, dx = o - (o / W) * W - B;
                const uint32_t pk = __ldg(prev + e);
                const int py = (int)(pk >> 16), px = (int)(pk & 0xffffu);
                const int y = py + dy, x = px + dx;
                if (y >= B && y < a.rows - B && x >= B && x < a.cols - B) {
                    bool owner = true;
                    // rows of q's window above p's row: any changed pixel there comes first
                    for (int r = y - B; r < py && owner; ++r)
                        if (row_bits(bm_prev + (size_t)r * a.bm_words, a.bm_words, x - B) & ((1u << W) - 1u))
                            owner = false;
                    // p's row: changed pixels left of p in q's window come first
                    if (owner && B - dx > 0 &&
                        (row_bits(bm_prev + (size_t)py * a.bm_words, a.bm_words, x - B) & ((1u << (B - dx)) - 1u)))
                        owner = false;
                    if (owner) {
                        ++evals;
                        const long long off = (long long)y * a.pitch + x;
                        const int ip = in[off];
                        const int nv = eval_pixel<B>(in + off, a.pitch, a.alpha);
                        out[off] = (uint8_t)nv;
                        if (nv != ip) {
                            ch = true;
                            v = ((uint32_t)y << 16) | (uint32_t)x;
                            atomicOr(bm_next + (size_t)y * a.bm_words + (x >> 5), 1u << (x & 31));
                        }
                    }
                }
            }
            any |= ch;
            staged_append(sl, next, nnext, a.list_cap, ch, v, lane);
        }
    } else {
        full_pass<B>(a, in, out, bm_next, next, nnext, sl, warp_base, gthreads, lane, any, evals);
    }
    staged_flush(sl, next, nnext, a.list_cap, s_counts, kWarps);
    const unsigned ev = __reduce_add_sync(0xffffffffu, evals);
    if (lane == 0 && ev) atomicAdd(&s_evals, (unsigned long long)ev);
    const int cta_any = __syncthreads_or(any);
    if (tid == 0) {
        if (s_evals) atomicAdd(&a.ctrl->evals_list, s_evals);
        finish_launch(a.ctrl, cta_any ? 1u : 0u, 1, gridDim.x, s_aux, s_cur);
    }
}

cudaError_t launch_list(int beta, const PassArgs& a, int sms, cudaStream_t s) {
    const unsigned grid = (unsigned)sms * 2u;
    switch (beta) {
        case 1: list_entry_kernel<1><<<grid, kListThreads, 0, s>>>(a); break;
        case 2: list_entry_kernel<2><<<grid, kListThreads, 0, s>>>(a); break;
        case 3: list_kernel<3><<<grid, kListThreads, 0, s>>>(a); break;
        case 4: list_kernel<4><<<grid, kListThreads, 0, s>>>(a); break;
        case 5: list_kernel<5><<<grid, kListThreads, 0, s>>>(a); break;
        case 6: list_kernel<6><<<grid, kListThreads, 0, s>>>(a); break;
        case 7: list_kernel<7><<<grid, kListThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hg
