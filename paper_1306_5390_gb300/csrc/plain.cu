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
    c->fused_work = 0;
    c->dense = 0;
    c->tile_next[0] = 0;
    c->tile_next[1] = 0;
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

// Batched copy-out: grid (per-image CTAs, images); image blockIdx.y, whose
// `user` pointer is the caller's dense image (row r at user + r * cols), or
// null for an image staged by the host.

// Canvas `cur` -> dense image: one aligned 4-byte word of the destination
// per thread, gathered from the canvas; the partial words at the two ends of
// the image are written byte by byte.
__global__ void copy_out_batch_kernel(const Ctrl* __restrict__ c, const uint8_t* __restrict__ a0,
                                      const uint8_t* __restrict__ a1, const uint8_t* __restrict__ a2,
                                      const ImgDesc* __restrict__ imgs) {
    const ImgDesc d = imgs[blockIdx.y];
    if (!d.user) return;
    const unsigned cur = __ldcg(&c->cur);
    const uint8_t* canvas = (cur == 0 ? a0 : (cur == 1 ? a1 : a2)) + d.off + (long long)kPadY * d.pitch + kPadX;
    const uintptr_t ad = reinterpret_cast<uintptr_t>(d.user);
    const int m = (int)(ad & 3u);
    uint32_t* dw = reinterpret_cast<uint32_t*>(ad - (uintptr_t)m);
    const long long nbytes = (long long)d.rows * d.cols;
    const long long total = (m + nbytes + 3) / 4;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
         w += (long long)gridDim.x * blockDim.x) {
        const long long l0 = 4 * w - m;  // image byte index of the word's first byte
        long long first = l0 < 0 ? 0 : l0;
        long long r = first / d.cols;
        int col = (int)(first - r * d.cols);
        uint32_t v = 0;
        int nb = 0;
        for (int b = (int)(first - l0); b < 4 && l0 + b < nbytes; ++b) {
            v |= (uint32_t)canvas[r * d.pitch + col] << (8 * b);
            ++nb;
            if (++col == d.cols) {
                col = 0;
                ++r;
            }
        }
        if (nb == 4) {
            dw[w] = v;
        } else {
            uint8_t* db = reinterpret_cast<uint8_t*>(dw + w);
            for (int b = 0; b < 4; ++b)
                if (l0 + b >= 0 && l0 + b < nbytes) db[b] = (uint8_t)(v >> (8 * b));
        }
    }
}

// tile_img[b] = the image that fused tile b belongs to.
__global__ void tile_map_kernel(const ImgDesc* __restrict__ imgs, int nimg, int total_tiles, int* __restrict__ tile_img) {
    const int i = blockIdx.x;
    const int t0 = imgs[i].tile0;
    const int t1 = i + 1 < nimg ? imgs[i + 1].tile0 : total_tiles;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) tile_img[t] = i;
}

static unsigned batch_copy_ctas(long long max_words, int nimg, int sms) {
    long long g = (max_words + 2047) / 2048;
    const long long cap = nimg > 0 ? ((long long)sms * 16 + nimg - 1) / nimg : 1;
    const long long lim = cap > 16 ? cap : 16;
    if (g > lim) g = lim;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t launch_copy_out_batch(const Ctrl* c, uint8_t* const arena[3], const ImgDesc* imgs, int nimg,
                                  long long max_words, int sms, cudaStream_t s) {
    if (nimg <= 0) return cudaSuccess;
    copy_out_batch_kernel<<<dim3(batch_copy_ctas(max_words, nimg, sms), (unsigned)nimg), 256, 0, s>>>(
        c, arena[0], arena[1], arena[2], imgs);
    return cudaGetLastError();
}

__global__ void rms_kernel(const int* __restrict__ sum, const int* __restrict__ flag, int* __restrict__ out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = flag[i] == 1 ? isqrt_u16(sum[i]) : rms_div(sum[i], recip32((unsigned)flag[i]));
}

cudaError_t launch_rms(const int* sum, const int* flag, int* out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    rms_kernel<<<blocks, 256, 0, s>>>(sum, flag, out, n);
    return cudaGetLastError();
}

cudaError_t launch_tile_map(const ImgDesc* imgs, int nimg, int total_tiles, int* tile_img, cudaStream_t s) {
    if (nimg <= 0) return cudaSuccess;
    tile_map_kernel<<<(unsigned)nimg, 256, 0, s>>>(imgs, nimg, total_tiles, tile_img);
    return cudaGetLastError();
}

}  // namespace hg
