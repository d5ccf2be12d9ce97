// Unfused one-pass kernel (one thread per pixel, global loads), canvas copy
// kernels and the control-block initialiser.
//
// The unfused kernel evaluates Algorithms 1 and 2 directly for each pixel:
// card by gathering over the window (equal to the paper's scattered
// increments, because the window and the |difference| < alpha test are
// symmetric), then flag / sum / replacement.  It is the straightforward GPU
// form of the method, kept as a second, independent device path and as the
// unfused point of comparison for the fused tile kernel.
#include "common.cuh"
#include "kernels.h"

namespace hg {

template <int B>
__global__ void __launch_bounds__(256) plain_kernel(PassArgs a) {
    __shared__ int s_np;
    __shared__ unsigned s_cur, s_aux;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid == 0) {
        s_np = launch_passes(a.ctrl, 1);
        s_cur = __ldcg(&a.ctrl->cur);
        s_aux = __ldcg(&a.ctrl->aux);
    }
    __syncthreads();
    if (s_np == 0) return;
    const uint8_t* src = a.canvas[s_cur];
    uint8_t* dst = a.canvas[s_aux];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    bool changed = false;
    if (x < a.cols && y < a.rows) {
        const long long off = (long long)(kPadY + y) * a.pitch + kPadX + x;
        const uint8_t* s = src + off;
        const int ip = *s;
        int outv = ip;
        const bool interior = x >= B && x < a.cols - B && y >= B && y < a.rows - B;
        if (interior) {
            int card = 0;
#pragma unroll
            for (int dy = -B; dy <= B; ++dy)
#pragma unroll
                for (int dx = -B; dx <= B; ++dx) {
                    const int v = s[dy * a.pitch + dx];
                    card += (v < ip + a.alpha && v > ip - a.alpha) ? 1 : 0;
                }
            if (card <= 2) {
                int sum = 0, flag = 0;
#pragma unroll
                for (int dy = -B; dy <= B; ++dy)
#pragma unroll
                    for (int dx = -B; dx <= B; ++dx) {
                        const int v = s[dy * a.pitch + dx];
                        if (!(v < ip + a.alpha + 1 && v > ip - a.alpha)) {
                            sum += v * v;
                            ++flag;
                        }
                    }
                constexpr int kPixCount = (2 * B + 1) * (2 * B + 1);
                if (flag > kPixCount - 3) outv = (int)floorf(__fsqrt_rn((float)(sum / flag)));
            }
        }
        dst[off] = (uint8_t)outv;
        changed = outv != ip;
    }
    const int any = __syncthreads_or(changed);
    if (tid == 0) finish_launch(a.ctrl, any ? 1u : 0u, 1, gridDim.x * gridDim.y, s_aux, s_cur);
}

cudaError_t launch_plain(int beta, const PassArgs& a, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((a.cols + 31) / 32, (a.rows + 7) / 8);
    switch (beta) {
        case 1: plain_kernel<1><<<grid, block, 0, s>>>(a); break;
        case 2: plain_kernel<2><<<grid, block, 0, s>>>(a); break;
        case 3: plain_kernel<3><<<grid, block, 0, s>>>(a); break;
        case 4: plain_kernel<4><<<grid, block, 0, s>>>(a); break;
        case 5: plain_kernel<5><<<grid, block, 0, s>>>(a); break;
        case 6: plain_kernel<6><<<grid, block, 0, s>>>(a); break;
        case 7: plain_kernel<7><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

__global__ void ctrl_init_kernel(Ctrl* c, unsigned max_k) {
    c->k = 0;
    c->converged = 0;
    c->cur = 0;
    c->aux = 1;
    c->max_k = max_k;
    c->done = 0;
    c->mask = 0;
    c->work_launches = 0;
    c->executed = 0;
    for (int i = 0; i < 4; ++i) c->list_n[i] = 0;
    c->error = 0;
    c->evals_fused = 0;
    c->evals_list = 0;
}

cudaError_t launch_ctrl_init(Ctrl* c, unsigned max_k, cudaStream_t s) {
    ctrl_init_kernel<<<1, 1, 0, s>>>(c, max_k);
    return cudaGetLastError();
}

// Dense user image (row r at img + r*cols) <-> canvas interior, in 16-byte
// row chunks; vector accesses when the user rows are 16-byte aligned.
__global__ void copy_in_kernel(const uint8_t* __restrict__ img, int rows, int cols,
                               uint8_t* __restrict__ canvas, long long pitch, int vec) {
    const long long chunks = (cols + 15) / 16;
    const long long total = chunks * rows;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / chunks;
        const int x = (int)(i - r * chunks) * 16;
        const uint8_t* s = img + r * cols + x;
        uint8_t* d = canvas + (kPadY + r) * pitch + kPadX + x;
        const int n = min(16, cols - x);
        if (vec && n == 16) {
            *reinterpret_cast<uint4*>(d) = __ldg(reinterpret_cast<const uint4*>(s));
        } else {
            for (int b = 0; b < n; ++b) d[b] = s[b];
        }
    }
}

__global__ void copy_out_kernel(const Ctrl* __restrict__ c, const uint8_t* __restrict__ c0,
                                const uint8_t* __restrict__ c1, const uint8_t* __restrict__ c2, long long pitch,
                                uint8_t* __restrict__ img, int rows, int cols, int vec) {
    const unsigned cur = __ldcg(&c->cur);
    const uint8_t* canvas = cur == 0 ? c0 : (cur == 1 ? c1 : c2);
    const long long chunks = (cols + 15) / 16;
    const long long total = chunks * rows;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / chunks;
        const int x = (int)(i - r * chunks) * 16;
        const uint8_t* s = canvas + (kPadY + r) * pitch + kPadX + x;
        uint8_t* d = img + r * cols + x;
        const int n = min(16, cols - x);
        if (vec && n == 16) {
            *reinterpret_cast<uint4*>(d) = *reinterpret_cast<const uint4*>(s);
        } else {
            for (int b = 0; b < n; ++b) d[b] = s[b];
        }
    }
}

static unsigned copy_grid(int rows, int cols, int sms) {
    const long long total = (long long)((cols + 15) / 16) * rows;
    long long blocks = (total + 255) / 256;
    const long long cap = (long long)sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (unsigned)blocks;
}

cudaError_t launch_copy_in(const uint8_t* img, int rows, int cols, uint8_t* canvas, long long pitch,
                           int sms, cudaStream_t s) {
    const int vec = (cols % 16 == 0) && ((reinterpret_cast<uintptr_t>(img) & 15u) == 0);
    copy_in_kernel<<<copy_grid(rows, cols, sms), 256, 0, s>>>(img, rows, cols, canvas, pitch, vec);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const Ctrl* c, uint8_t* const canvas[3], long long pitch, uint8_t* img, int rows,
                            int cols, int sms, cudaStream_t s) {
    const int vec = (cols % 16 == 0) && ((reinterpret_cast<uintptr_t>(img) & 15u) == 0);
    copy_out_kernel<<<copy_grid(rows, cols, sms), 256, 0, s>>>(c, canvas[0], canvas[1], canvas[2], pitch, img,
                                                               rows, cols, vec);
    return cudaGetLastError();
}

}  // namespace hg
