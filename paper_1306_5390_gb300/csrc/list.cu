// List pass: one pass of Algorithms 1-2 that evaluates only the pixels that
// can change.
//
// A pixel's output in pass t depends only on its (2 beta + 1)^2 window in the
// image of pass t-1, so a pixel with no changed pixel (in pass t-1) within
// beta keeps its value.  The kernel takes the list of pixels the previous
// pass changed, visits every window position around each of them, claims
// each such pixel once (a per-pixel stamp: the first thread to swap in this
// pass's stamp evaluates it), evaluates it exactly from the current canvas
// and writes it to the partner canvas, which already agrees with the current
// image everywhere else (see Ctrl).  Pixels it changes form the next list.
// When the previous list overflowed its capacity, the pass evaluates and
// writes every pixel instead.
#include "common.cuh"
#include "kernels.h"

namespace hg {

// Algorithm 2 for an interior pixel of a byte canvas (card <= 2 is implied by
// flag > pix_count - 3 for alpha >= 1, and card is 0 for alpha = 0).
template <int B>
__device__ __forceinline__ int eval_pixel(const uint8_t* __restrict__ p, long long pitch, int alpha) {
    const int ip = p[0];
    int sum = 0, flag = 0;
#pragma unroll
    for (int dy = -B; dy <= B; ++dy)
#pragma unroll
        for (int dx = -B; dx <= B; ++dx) {
            const int v = p[dy * pitch + dx];
            if (!(v < ip + alpha + 1 && v > ip - alpha)) {
                sum += v * v;
                ++flag;
            }
        }
    constexpr int kPixCount = (2 * B + 1) * (2 * B + 1);
    if (flag > kPixCount - 3) return (int)floorf(__fsqrt_rn((float)(sum / flag)));
    return ip;
}

template <int B>
__global__ void __launch_bounds__(256) list_kernel(PassArgs a) {
    __shared__ int s_np;
    __shared__ unsigned s_cur, s_aux, s_L, s_stamp, s_n;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        s_np = launch_passes(a.ctrl, 1);
        s_cur = __ldcg(&a.ctrl->cur);
        s_aux = __ldcg(&a.ctrl->aux);
        s_L = __ldcg(&a.ctrl->work_launches);
        s_stamp = __ldcg(&a.ctrl->stamp);
        s_n = __ldcg(&a.ctrl->list_n[(s_L + 1u) & 1u]);
    }
    __syncthreads();
    if (s_np == 0) return;
    const uint8_t* in = a.canvas[s_cur] + (long long)kPadY * a.pitch + kPadX;
    uint8_t* out = a.canvas[s_aux] + (long long)kPadY * a.pitch + kPadX;
    const uint32_t* prev = a.lists[(s_L + 1u) & 1u];
    uint32_t* next = a.lists[s_L & 1u];
    unsigned* nnext = &a.ctrl->list_n[s_L & 1u];
    const unsigned stamp = s_stamp;
    const unsigned n = s_n;
    constexpr int W = 2 * B + 1, P = W * W;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    const long long warp_base = (long long)blockIdx.x * blockDim.x + (tid & ~31);
    bool any = false;
    unsigned evals = 0;
    if (n <= a.list_cap) {
        const long long total = (long long)n * P;
        for (long long base = warp_base; base < total; base += gthreads) {
            const long long i = base + lane;
            bool ch = false;
            uint32_t v = 0;
            if (i < total) {
                const unsigned e = (unsigned)(i / P);
                const int o = (int)(i - (long long)e * P);
                const uint32_t pk = prev[e];
                const int y = (int)(pk >> 16) + o / W - B;
                const int x = (int)(pk & 0xffffu) + o % W - B;
                if (y >= B && y < a.rows - B && x >= B && x < a.cols - B) {
                    const long long q = (long long)y * a.cols + x;
                    if (atomicExch(&a.stamps[q], stamp) != stamp) {
                        ++evals;
                        const long long off = (long long)y * a.pitch + x;
                        const int ip = in[off];
                        const int nv = eval_pixel<B>(in + off, a.pitch, a.alpha);
                        out[off] = (uint8_t)nv;
                        if (nv != ip) {
                            ch = true;
                            v = ((uint32_t)y << 16) | (uint32_t)x;
                        }
                    }
                }
            }
            any |= ch;
            list_append(next, nnext, a.list_cap, ch, v, lane);
        }
    } else {
        // Previous list overflowed: evaluate and write every pixel.
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
                }
            }
            any |= ch;
            list_append(next, nnext, a.list_cap, ch, v, lane);
        }
    }
    const unsigned long long ev = __reduce_add_sync(0xffffffffu, evals);
    if (lane == 0 && ev) atomicAdd(&a.ctrl->evals_list, ev);
    const int cta_any = __syncthreads_or(any);
    if (tid == 0) finish_launch(a.ctrl, cta_any ? 1u : 0u, 1, gridDim.x, s_aux, s_cur);
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
