// List pass: one pass of Algorithms 1-2 that evaluates only the pixels that
// can change.
//
// A pixel's output in pass t depends only on its (2 beta + 1)^2 window in the
// image of pass t-1, so a pixel with no changed pixel (in pass t-1) within
// beta keeps its value.  The kernel walks the list of pixels the previous
// pass changed; one warp takes one changed pixel p, stages the (4 beta + 1)^2
// block of the current image around p and the matching block of the
// previous pass's change bitmap in shared memory, and evaluates every pixel
// q of p's window that p "owns": p is the first changed pixel, in raster
// order, of q's window, so each pixel is evaluated exactly once.  Results go
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
// the pixel in a row-major block with row stride `stride`.
template <int B>
__device__ __forceinline__ int eval_pixel(const uint8_t* __restrict__ p, long long stride, int alpha) {
    const int ip = p[0];
    int sum = 0, flag = 0;
#pragma unroll
    for (int dy = -B; dy <= B; ++dy)
#pragma unroll
        for (int dx = -B; dx <= B; ++dx) {
            const int v = p[dy * stride + dx];
            if (!(v < ip + alpha + 1 && v > ip - alpha)) {
                sum += v * v;
                ++flag;
            }
        }
    constexpr int kPixCount = (2 * B + 1) * (2 * B + 1);
    if (flag > kPixCount - 3) return (int)floorf(__fsqrt_rn((float)(sum / flag)));
    return ip;
}

}  // namespace

template <int B>
__global__ void __launch_bounds__(256) list_kernel(PassArgs a) {
    constexpr int W = 2 * B + 1, P = W * W;
    constexpr int E = 4 * B + 1;  // staged block side
    constexpr int kWarps = 8;
    __shared__ int s_np;
    __shared__ unsigned s_cur, s_aux, s_L, s_n, s_nclr;
    __shared__ uint8_t blk_all[kWarps][E * E];
    __shared__ uint32_t bmr_all[kWarps][E];
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
        uint8_t* blk = blk_all[warp];
        uint32_t* bmr = bmr_all[warp];
        const long long nwarps = gthreads / 32;
        for (long long e = gtid / 32; e < n; e += nwarps) {
            const uint32_t pk = prev[e];
            const int py = (int)(pk >> 16), px = (int)(pk & 0xffffu);
            // Stage the image block [py - 2B, py + 2B] x [px - 2B, px + 2B]
            // (rows/columns off the image read canvas padding; only interior
            // pixels are evaluated, and their windows lie on the image).
            for (int j = lane; j < E * E; j += 32) {
                const int by = j / E, bx = j - by * E;
                blk[j] = in[(long long)(py + by - 2 * B) * a.pitch + (px + bx - 2 * B)];
            }
            if (lane < E) {
                const int gy = py + lane - 2 * B;
                bmr[lane] = (gy >= 0 && gy < a.rows)
                                ? row_bits(bm_prev + (size_t)gy * a.bm_words, a.bm_words, px - 2 * B)
                                : 0u;
            }
            __syncwarp();
            for (int base = 0; base < P; base += 32) {
                const int j = base + lane;
                bool ch = false;
                uint32_t v = 0;
                if (j < P) {
                    const int dy = j / W - B, dx = j - (j / W) * W - B;
                    const int y = py + dy, x = px + dx;
                    const int cy = 2 * B + dy, cx = 2 * B + dx;  // block coordinates of q
                    if (y >= B && y < a.rows - B && x >= B && x < a.cols - B) {
                        // p owns q unless a changed pixel before p (raster
                        // order) lies in q's window.
                        const uint32_t wm = ((1u << W) - 1u) << (cx - B);
                        bool owner = true;
#pragma unroll
                        for (int r = 0; r < W; ++r) {
                            const int by = cy - B + r;
                            if (by < 2 * B && (bmr[by] & wm)) owner = false;
                            if (by == 2 * B && (bmr[by] & wm & ((1u << (2 * B)) - 1u))) owner = false;
                        }
                        if (owner) {
                            ++evals;
                            const int ip = blk[cy * E + cx];
                            const int nv = eval_pixel<B>(blk + cy * E + cx, E, a.alpha);
                            out[(long long)y * a.pitch + x] = (uint8_t)nv;
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
            __syncwarp();
        }
    } else {
        // Previous list overflowed: evaluate and write every pixel.
        const long long total = (long long)a.rows * a.cols;
        const long long warp_base = (long long)blockIdx.x * blockDim.x + (tid & ~31);
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
    const unsigned grid = (unsigned)sms * 8u;
    switch (beta) {
        case 1: list_kernel<1><<<grid, 256, 0, s>>>(a); break;
        case 2: list_kernel<2><<<grid, 256, 0, s>>>(a); break;
        case 3: list_kernel<3><<<grid, 256, 0, s>>>(a); break;
        case 4: list_kernel<4><<<grid, 256, 0, s>>>(a); break;
        case 5: list_kernel<5><<<grid, 256, 0, s>>>(a); break;
        case 6: list_kernel<6><<<grid, 256, 0, s>>>(a); break;
        case 7: list_kernel<7><<<grid, 256, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hg
