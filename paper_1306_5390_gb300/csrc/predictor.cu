// Learned k-predictor: a small convolutional network that estimates, from a
// 64 x 64 area-averaged copy of an image and a 16-bin histogram of its grey
// levels, how many passes (k) the method will take.  Not a method of the
// paper: its concluding section leaves choosing the iteration factor as
// future work.  The estimate only chooses a schedule; results and k are
// always those of the exact method.
//
// Network (weights from an offline fit on oracle-labelled images):
//   x0 = 64 x 64 x 1 area means / 255
//   x1..x4 = ReLU(conv3x3(x_{l-1}) + b_l), 16 channels, zero padding
//   g = mean of x4 over the 64 x 64 positions (16 values)
//   k_hat = max(0, w_h . [g, histogram] + b_h)
//
// The convolutions run on the 5th-generation tensor cores (tcgen05, BF16
// operands, FP32 accumulation in tensor memory) as implicit GEMMs: one CTA
// computes 128 output positions (two rows) x 16 channels of one image; the
// 3 x 3 taps are the K steps (K = 16 per step: the 16 input channels, or
// for the first layer the 9 taps of its single channel).  Operands sit in
// shared memory in the no-swizzle K-major layout of 8-row x 16-byte core
// matrices; one thread issues the MMAs and a commit to an mbarrier; after a
// bounded wait each warp reads its 32 accumulator rows from tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hgrms.h"
#include "kernels.h"

namespace hg {

namespace {

constexpr int kSide = 64;              // feature map side
constexpr int kPix = kSide * kSide;    // 4096 positions
constexpr int kCh = 16;                // channels
constexpr int kBins = 16;              // histogram bins
constexpr int kBlockM = 128;           // positions per CTA (MMA M)
constexpr int kTileBytes = kBlockM * 16 * 2;  // one K step of A: 128 x 16 bf16
constexpr int kBBytes = kCh * 16 * 2;         // one K step of B: 16 x 16 bf16
constexpr int kTmemCols = 32;          // smallest tensor-memory allocation

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start address, K-direction
// core-matrix stride (leading byte offset) and M/N-direction stride (stride
// byte offset), all in 16-byte units; descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 16, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kCh >> 3) << 17) |
                            ((uint32_t)(kBlockM >> 4) << 24);

// Byte offset of element (row, k) of a 16-wide K-major operand tile made of
// 8 x 8 core matrices: core matrix (row / 8, k / 8) at 256 (row / 8) +
// 128 (k / 8), rows of 16 bytes inside it.
__device__ __forceinline__ int core_off(int row, int k) {
    return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// One conv layer: in/out are [image][64][64][cin or 16] bf16; w holds the
// B operand images of the K steps (9 of 512 bytes, or 1 for the first
// layer) in shared-memory order; bias 16 floats.  Grid (32, images), 128
// threads.
__global__ void __launch_bounds__(128) conv_tc_kernel(const __nv_bfloat16* __restrict__ in, int cin,
                                                      const uint8_t* __restrict__ w, const float* __restrict__ bias,
                                                      __nv_bfloat16* __restrict__ out, unsigned* __restrict__ err) {
    __shared__ __align__(1024) uint8_t sA[9 * kTileBytes];
    __shared__ __align__(1024) uint8_t sB[9 * kBBytes];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int img = blockIdx.y;
    const int steps = cin == 1 ? 1 : 9;
    const int m = tid;                       // this thread's output position in the block
    const int py = blockIdx.x * 2 + (m >> 6), px = m & 63;
    const __nv_bfloat16* src = in + (size_t)img * kPix * cin;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // A operand: im2col rows of this block.
    if (cin == 1) {
        __align__(16) __nv_bfloat16 v[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            float x = 0.f;
            if (t < 9) {
                const int y = py + t / 3 - 1, xx = px + t % 3 - 1;
                if (y >= 0 && y < kSide && xx >= 0 && xx < kSide) x = __bfloat162float(src[y * kSide + xx]);
            }
            v[t] = __float2bfloat16_rn(x);
        }
        *reinterpret_cast<uint4*>(sA + core_off(m, 0)) = *reinterpret_cast<const uint4*>(&v[0]);
        *reinterpret_cast<uint4*>(sA + core_off(m, 8)) = *reinterpret_cast<const uint4*>(&v[8]);
    } else {
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            const int y = py + t / 3 - 1, xx = px + t % 3 - 1;
            uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
            if (y >= 0 && y < kSide && xx >= 0 && xx < kSide) {
                const uint4* p = reinterpret_cast<const uint4*>(src + (size_t)(y * kSide + xx) * kCh);
                lo = __ldg(p);
                hi = __ldg(p + 1);
            }
            uint8_t* tile = sA + t * kTileBytes;
            *reinterpret_cast<uint4*>(tile + core_off(m, 0)) = lo;
            *reinterpret_cast<uint4*>(tile + core_off(m, 8)) = hi;
        }
    }
    // B operand images.
    for (int i = tid; i < steps * kBBytes / 16; i += 128)
        reinterpret_cast<uint4*>(sB)[i] = __ldg(reinterpret_cast<const uint4*>(w) + i);
    // Shared-memory writes -> visible to the tensor core (async proxy).
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        for (int t = 0; t < steps; ++t) {
            const uint64_t ad = smem_desc(smem_u32(sA + t * kTileBytes), 128, 256);
            const uint64_t bd = smem_desc(smem_u32(sB + t * kBBytes), 128, 256);
            const uint32_t acc = t > 0 ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar)));
    }
    // Bounded wait for the MMAs (phase 0 of the mbarrier).
    uint32_t done = 0;
    for (uint32_t spins = 0; spins < (1u << 22); ++spins) {
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\nselp.u32 %0, 1, 0, q;\n}"
            : "=r"(done)
            : "r"(smem_u32(&mbar)));
        if (done) break;
    }
    if (!done) atomicExch(err, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (done) {
        // Accumulator rows 32 warp .. 32 warp + 31, columns 0..15.
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(32 * warp) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        __align__(16) __nv_bfloat16 o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(fmaxf(__uint_as_float(r[c]) + bias[c], 0.f));
        const int pos = (blockIdx.x * 2 + (m >> 6)) * kSide + (m & 63);
        uint4* dst = reinterpret_cast<uint4*>(out + ((size_t)img * kPix + pos) * kCh);
        dst[0] = *reinterpret_cast<const uint4*>(&o[0]);
        dst[1] = *reinterpret_cast<const uint4*>(&o[8]);
    }
    (void)lane;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Features of image blockIdx.y: row i = blockIdx.x of the 64 x 64 area
// means (each cell averages rows [i R / 64, max((i+1) R / 64, i R / 64 + 1))
// and the matching columns) and that row band's share of the 16-bin
// histogram (bin = value / 16, counts / pixels, added into hist).
__global__ void __launch_bounds__(256) features_kernel(const ImgDesc* __restrict__ imgs,
                                                       __nv_bfloat16* __restrict__ x0, float* __restrict__ hist,
                                                       float* __restrict__ x0f) {
    const ImgDesc d = imgs[blockIdx.y];
    const int i = blockIdx.x;
    const int r0 = (int)((long long)i * d.rows / kSide);
    const int r1 = max(r0 + 1, (int)((long long)(i + 1) * d.rows / kSide));
    __shared__ unsigned s_wh[8][kBins];  // per-warp bins
    __shared__ unsigned s_hist[kBins];
    __shared__ float s_cell[kSide];
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x < 8 * kBins) s_wh[threadIdx.x / kBins][threadIdx.x % kBins] = 0u;
    if (threadIdx.x < kSide) s_cell[threadIdx.x] = 0.f;
    __syncthreads();
    // Histogram: the rows [i R / 64, (i+1) R / 64) (each row counted once).
    const int h1 = (int)((long long)(i + 1) * d.rows / kSide);
    const uint8_t* base = d.user;
    for (long long idx = (long long)r0 * d.cols + threadIdx.x; idx < (long long)h1 * d.cols; idx += blockDim.x)
        atomicAdd(&s_wh[warp][base[idx] >> 4], 1u);
    __syncthreads();
    if (threadIdx.x < kBins) {
        unsigned t = 0;
        for (int w = 0; w < 8; ++w) t += s_wh[w][threadIdx.x];
        s_hist[threadIdx.x] = t;
    }
    // Area means of the 64 cells of this row.
    for (int j = threadIdx.x / 4; j < kSide; j += blockDim.x / 4) {
        const int c0 = (int)((long long)j * d.cols / kSide);
        const int c1 = max(c0 + 1, (int)((long long)(j + 1) * d.cols / kSide));
        float sum = 0.f;
        for (int r = r0; r < r1; ++r)
            for (int c = c0 + (threadIdx.x & 3); c < c1; c += 4) sum += (float)base[(long long)r * d.cols + c];
        sum += __shfl_xor_sync(0xffffffffu, sum, 1);
        sum += __shfl_xor_sync(0xffffffffu, sum, 2);
        if ((threadIdx.x & 3) == 0) s_cell[j] = sum / ((float)(r1 - r0) * (float)(c1 - c0) * 255.f);
    }
    __syncthreads();
    if (threadIdx.x < kSide) {
        const size_t o = (size_t)blockIdx.y * kPix + (size_t)i * kSide + threadIdx.x;
        x0[o] = __float2bfloat16_rn(s_cell[threadIdx.x]);
        if (x0f) x0f[o] = s_cell[threadIdx.x];
    }
    if (threadIdx.x < kBins && s_hist[threadIdx.x])
        atomicAdd(&hist[blockIdx.y * kBins + threadIdx.x],
                  (float)s_hist[threadIdx.x] / ((float)d.rows * (float)d.cols));
}

// k_hat of image blockIdx.x: mean of the last layer over the positions,
// then the linear head on [means, histogram].
__global__ void __launch_bounds__(256) head_kernel(const __nv_bfloat16* __restrict__ x4, const float* __restrict__ hist,
                                                   const float* __restrict__ wh, float* __restrict__ k_hat,
                                                   float* __restrict__ gap_out) {
    __shared__ float s_sum[kCh];
    if (threadIdx.x < kCh) s_sum[threadIdx.x] = 0.f;
    __syncthreads();
    float acc[kCh];
#pragma unroll
    for (int c = 0; c < kCh; ++c) acc[c] = 0.f;
    const __nv_bfloat16* x = x4 + (size_t)blockIdx.x * kPix * kCh;
    for (int p = threadIdx.x; p < kPix; p += blockDim.x)
#pragma unroll
        for (int c = 0; c < kCh; ++c) acc[c] += __bfloat162float(x[(size_t)p * kCh + c]);
#pragma unroll
    for (int c = 0; c < kCh; ++c) {
        float v = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_sum[c], v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float y = wh[2 * kCh];  // bias
        for (int c = 0; c < kCh; ++c) {
            const float g = s_sum[c] / (float)kPix;
            if (gap_out) gap_out[blockIdx.x * kCh + c] = g;
            y += wh[c] * g + wh[kCh + c] * hist[blockIdx.x * kBins + c];
        }
        k_hat[blockIdx.x] = fmaxf(y, 0.f);
    }
}

}  // namespace

// Device buffers of the predictor for up to `cap` images.
struct Predictor {
    uint8_t* w[4] = {nullptr, nullptr, nullptr, nullptr};  // B operand images per layer
    float* bias = nullptr;                                   // 4 x 16
    float* head = nullptr;                                   // 33
    __nv_bfloat16* x0 = nullptr;                             // cap x 4096
    __nv_bfloat16* act[2] = {nullptr, nullptr};              // cap x 4096 x 16, ping-pong
    float* hist = nullptr;                                   // cap x 16
    float* khat = nullptr;                                   // cap
    unsigned* err = nullptr;
    int cap = 0;
    bool loaded = false;
};

Predictor* predictor_new() { return new Predictor(); }

void predictor_free(Predictor* p) {
    if (!p) return;
    for (int l = 0; l < 4; ++l) cudaFree(p->w[l]);
    cudaFree(p->bias);
    cudaFree(p->head);
    cudaFree(p->x0);
    cudaFree(p->act[0]);
    cudaFree(p->act[1]);
    cudaFree(p->hist);
    cudaFree(p->khat);
    cudaFree(p->err);
    delete p;
}

// Host: B operand image of one K step: element (n = output channel, k) at
// core_off(n, k), bf16.
static void pack_b(const float* wl, int cin, int step, uint16_t* dst) {
    for (int n = 0; n < kCh; ++n)
        for (int k = 0; k < 16; ++k) {
            float v = 0.f;
            if (cin == 1) {
                if (k < 9) v = wl[(k * 1 + 0) * kCh + n];  // tap k, channel 0
            } else {
                v = wl[(step * kCh + k) * kCh + n];  // tap step, input channel k
            }
            uint32_t u;
            memcpy(&u, &v, 4);
            const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
            const int off = (n >> 3) * 256 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
            dst[off / 2] = (uint16_t)(r >> 16);
        }
}

// weights: layer l (0..3) as [tap 0..8][cin][16] floats (cin = 1 for l = 0,
// else 16), then 4 x 16 biases, then the head: 16 weights on the channel
// means, 16 on the histogram, 1 bias.
int predictor_load(Predictor* p, const float* weights, int n) {
    const int need = 9 * 1 * 16 + 3 * 9 * 16 * 16 + 4 * 16 + 33;
    if (n != need) return HGRMS_EINVAL;
    const float* q = weights;
    for (int l = 0; l < 4; ++l) {
        const int cin = l == 0 ? 1 : 16;
        const int steps = l == 0 ? 1 : 9;
        uint16_t img[9 * kBBytes / 2];
        memset(img, 0, sizeof(img));
        for (int s = 0; s < steps; ++s) pack_b(q, cin, s, img + s * kBBytes / 2);
        if (!p->w[l] && cudaMalloc(&p->w[l], 9 * kBBytes) != cudaSuccess) return HGRMS_ENOMEM;
        if (cudaMemcpy(p->w[l], img, 9 * kBBytes, cudaMemcpyHostToDevice) != cudaSuccess) return HGRMS_ECUDA;
        q += 9 * cin * 16;
    }
    if (!p->bias && cudaMalloc(&p->bias, 64 * sizeof(float)) != cudaSuccess) return HGRMS_ENOMEM;
    if (!p->head && cudaMalloc(&p->head, 33 * sizeof(float)) != cudaSuccess) return HGRMS_ENOMEM;
    if (!p->err && cudaMalloc(&p->err, sizeof(unsigned)) != cudaSuccess) return HGRMS_ENOMEM;
    if (cudaMemcpy(p->bias, q, 64 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return HGRMS_ECUDA;
    q += 64;
    if (cudaMemcpy(p->head, q, 33 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return HGRMS_ECUDA;
    p->loaded = true;
    return HGRMS_OK;
}

static int predictor_reserve(Predictor* p, int n) {
    if (n <= p->cap) return HGRMS_OK;
    cudaFree(p->x0);
    cudaFree(p->act[0]);
    cudaFree(p->act[1]);
    cudaFree(p->hist);
    cudaFree(p->khat);
    p->x0 = nullptr;
    p->act[0] = p->act[1] = nullptr;
    p->hist = p->khat = nullptr;
    p->cap = 0;
    if (cudaMalloc(&p->x0, (size_t)n * kPix * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&p->act[0], (size_t)n * kPix * kCh * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&p->act[1], (size_t)n * kPix * kCh * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&p->hist, (size_t)n * kBins * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->khat, (size_t)n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return HGRMS_ENOMEM;
    }
    p->cap = n;
    return HGRMS_OK;
}

// Features and network for n images described by the device table `imgs`
// (their `user` pointers: device-readable image bytes).  k_hat (host, n
// floats) receives the estimates; x0_host / gap_host (optional, host) the
// area means and the last layer's channel means, for tests.
int predictor_run(Predictor* p, const ImgDesc* imgs, int n, cudaStream_t s, float* k_hat, float* x0_host,
                  float* hist_host, float* gap_host) {
    if (!p->loaded) return HGRMS_EINVAL;
    if (n <= 0) return HGRMS_OK;
    int rc = predictor_reserve(p, n);
    if (rc < 0) return rc;
    float* x0f = nullptr;
    float* gap = nullptr;
    if (x0_host && cudaMalloc(&x0f, (size_t)n * kPix * sizeof(float)) != cudaSuccess) return HGRMS_ENOMEM;
    if (gap_host && cudaMalloc(&gap, (size_t)n * kCh * sizeof(float)) != cudaSuccess) {
        cudaFree(x0f);
        return HGRMS_ENOMEM;
    }
    cudaError_t e = cudaMemsetAsync(p->hist, 0, (size_t)n * kBins * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->err, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        features_kernel<<<dim3(kSide, (unsigned)n), 256, 0, s>>>(imgs, p->x0, p->hist, x0f);
        e = cudaGetLastError();
    }
    const __nv_bfloat16* in = p->x0;
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        __nv_bfloat16* out = p->act[l & 1];
        conv_tc_kernel<<<dim3(kPix / kBlockM, (unsigned)n), 128, 0, s>>>(in, l == 0 ? 1 : kCh, p->w[l],
                                                                          p->bias + 16 * l, out, p->err);
        e = cudaGetLastError();
        in = out;
    }
    if (e == cudaSuccess) {
        head_kernel<<<(unsigned)n, 256, 0, s>>>(in, p->hist, p->head, p->khat, gap);
        e = cudaGetLastError();
    }
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(k_hat, p->khat, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, p->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && x0_host)
        e = cudaMemcpyAsync(x0_host, x0f, (size_t)n * kPix * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && hist_host)
        e = cudaMemcpyAsync(hist_host, p->hist, (size_t)n * kBins * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && gap_host)
        e = cudaMemcpyAsync(gap_host, gap, (size_t)n * kCh * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(x0f);
    cudaFree(gap);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? HGRMS_ENOMEM : HGRMS_ECUDA;
    return err ? HGRMS_ETIMEOUT : HGRMS_OK;
}

}  // namespace hg
