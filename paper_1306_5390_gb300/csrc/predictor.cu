// Learned k-predictor: a small convolutional network that estimates, from a
// 64 x 64 area-averaged copy of an image and a 16-bin histogram of its grey
// levels, how many passes (k) the method will take.  Not a method of the
// paper: its concluding section leaves choosing the iteration factor as
// future work.  The estimate only chooses a schedule; results and k are
// always those of the exact method.
//
// Network (weights from an offline fit on seeded synthetic images labelled
// with k by this library's exact denoiser; a sample of the labels is checked
// against the CPU oracle by the tests):
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
#include <string.h>

#include <utility>
#include <vector>

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
//
// With mask != null the kernel computes the gradient of a layer's input
// instead (back-propagation through a 16-channel convolution): `in` is the
// gradient of the layer's output, the taps' offsets are negated, w holds the
// transposed weights (output channel = the layer's input channel), and the
// result is multiplied by (mask > 0), the ReLU of the layer's input.
__global__ void __launch_bounds__(128) conv_tc_kernel(const __nv_bfloat16* __restrict__ in, int cin,
                                                      const uint8_t* __restrict__ w, const float* __restrict__ bias,
                                                      __nv_bfloat16* __restrict__ out, unsigned* __restrict__ err,
                                                      const __nv_bfloat16* __restrict__ mask = nullptr) {
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
        const int sgn = mask ? -1 : 1;
#pragma unroll 1
        for (int t = 0; t < 9; ++t) {
            const int y = py + sgn * (t / 3 - 1), xx = px + sgn * (t % 3 - 1);
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
        const int pos = (blockIdx.x * 2 + (m >> 6)) * kSide + (m & 63);
        if (mask) {
            const __nv_bfloat16* mk = mask + ((size_t)img * kPix + pos) * kCh;
#pragma unroll
            for (int c = 0; c < 16; ++c)
                o[c] = __float2bfloat16_rn(__bfloat162float(mk[c]) > 0.f ? __uint_as_float(r[c]) : 0.f);
        } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(fmaxf(__uint_as_float(r[c]) + bias[c], 0.f));
        }
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

// Weight and bias gradients of one conv layer (back-propagation):
//   dW[tap][ci][co] += sum over positions p of X[p + off(tap)][ci] dY[p][co]
//   db[co]          += sum over p of dY[p][co]
// for image blockIdx.x, as GEMMs on the tensor cores: M = 128 rows
// (tap, ci) - taps 0..7 x 16 channels in group 0 and tap 8 in group 1, or
// the 9 taps of a 1-channel input in group 0 - N = 16 output channels,
// K = positions, 64 per chunk (4 K steps), accumulated in tensor memory
// over the 64 chunks of the image.  The operands are transposed into the
// K-major layout while they are written to shared memory.  128 threads.
__global__ void __launch_bounds__(128) conv_wgrad_tc_kernel(const __nv_bfloat16* __restrict__ X, int cin,
                                                            const __nv_bfloat16* __restrict__ dY,
                                                            float* __restrict__ dW, float* __restrict__ db,
                                                            unsigned* __restrict__ err) {
    constexpr int kChunk = 64, kSteps = kChunk / 16;
    __shared__ __align__(1024) uint8_t sA[2][kSteps][kTileBytes];
    __shared__ __align__(1024) uint8_t sB[kSteps][kBBytes];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float s_db[kCh];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int img = blockIdx.x;
    const int groups = cin == 1 ? 1 : 2;
    const __nv_bfloat16* x = X + (size_t)img * kPix * cin;
    const __nv_bfloat16* dy = dY + (size_t)img * kPix * kCh;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < kCh) s_db[tid] = 0.f;
    // Rows that no (tap, channel) fills stay zero for the whole kernel.
    for (int i = tid; i < (int)(sizeof(sA) / 16); i += 128) reinterpret_cast<uint4*>(&sA[0][0][0])[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    float dbl[kCh];
#pragma unroll
    for (int c = 0; c < kCh; ++c) dbl[c] = 0.f;
    bool ok = true;
    for (int chunk = 0; chunk < kPix / kChunk && ok; ++chunk) {
        // Fill: thread t handles position k = t & 63 of the chunk; the two
        // halves of the block split the taps.
        const int k = tid & 63, half = tid >> 6;
        const int p = chunk * kChunk + k;
        const int py = p >> 6, px = p & 63;
        const int step = k >> 4, kk = k & 15;
        for (int t = half; t < 9; t += 2) {
            const int y = py + t / 3 - 1, xx = px + t % 3 - 1;
            const bool in_img = y >= 0 && y < kSide && xx >= 0 && xx < kSide;
            if (cin == 1) {
                const float v = in_img ? __bfloat162float(x[y * kSide + xx]) : 0.f;
                *reinterpret_cast<__nv_bfloat16*>(&sA[0][step][core_off(t, kk)]) = __float2bfloat16_rn(v);
            } else {
                __align__(16) __nv_bfloat16 v[16];
                if (in_img) {
                    const uint4* q = reinterpret_cast<const uint4*>(x + (size_t)(y * kSide + xx) * kCh);
                    *reinterpret_cast<uint4*>(&v[0]) = __ldg(q);
                    *reinterpret_cast<uint4*>(&v[8]) = __ldg(q + 1);
                } else {
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
                }
                const int g = t >> 3, row0 = (t & 7) * 16;
#pragma unroll
                for (int c = 0; c < 16; ++c) *reinterpret_cast<__nv_bfloat16*>(&sA[g][step][core_off(row0 + c, kk)]) = v[c];
            }
        }
        if (half == 0) {
            __align__(16) __nv_bfloat16 v[16];
            const uint4* q = reinterpret_cast<const uint4*>(dy + (size_t)p * kCh);
            *reinterpret_cast<uint4*>(&v[0]) = __ldg(q);
            *reinterpret_cast<uint4*>(&v[8]) = __ldg(q + 1);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                *reinterpret_cast<__nv_bfloat16*>(&sB[step][core_off(c, kk)]) = v[c];
                dbl[c] += __bfloat162float(v[c]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            for (int g = 0; g < groups; ++g)
                for (int st = 0; st < kSteps; ++st) {
                    const uint64_t ad = smem_desc(smem_u32(&sA[g][st][0]), 128, 256);
                    const uint64_t bd = smem_desc(smem_u32(&sB[st][0]), 128, 256);
                    const uint32_t acc = (chunk > 0 || st > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + 16u * g),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        // The next fill overwrites the operands: wait for these MMAs.
        uint32_t done = 0;
        for (uint32_t spins = 0; spins < (1u << 22); ++spins) {
            asm volatile(
                "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}"
                : "=r"(done)
                : "r"(smem_u32(&mbar)), "r"((uint32_t)(chunk & 1)));
            if (done) break;
        }
        if (!done) {
            atomicExch(err, 1u);
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        ok = __syncthreads_and(ok);
    }
    if (ok) {
        for (int g = 0; g < groups; ++g) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)(32 * warp) << 16) + 16u * g));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            const int row = 32 * warp + (tid & 31);
            int tap, ci;
            if (cin == 1) {
                tap = row;
                ci = 0;
            } else {
                tap = g * 8 + (row >> 4);
                ci = row & 15;
            }
            if (tap < 9 && (cin == 16 || row < 9) && (g == 0 || row < 16)) {
#pragma unroll
                for (int c = 0; c < kCh; ++c) atomicAdd(&dW[(tap * cin + ci) * kCh + c], __uint_as_float(r[c]));
            }
        }
    }
    if (tid < 64) {
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            float v = dbl[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((tid & 31) == 0) atomicAdd(&s_db[c], v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid < kCh) atomicAdd(&db[tid], s_db[tid]);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Training head of image blockIdx.x: y = w . [means of x4, hist] + b (no
// ReLU while fitting), loss term (y - k)^2 / n, its gradient g = 2 (y - k) / n
// added into the head's gradients, and dgap[c] = g w[c] / 4096 for the
// backward pass.
__global__ void __launch_bounds__(256) train_head_kernel(const __nv_bfloat16* __restrict__ x4,
                                                         const float* __restrict__ hist, const float* __restrict__ k,
                                                         const float* __restrict__ wh, int n, float* __restrict__ gwh,
                                                         float* __restrict__ dgap, float* __restrict__ loss) {
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
        const float* hb = hist + blockIdx.x * kBins;
        float y = wh[2 * kCh];
        for (int c = 0; c < kCh; ++c) y += wh[c] * (s_sum[c] / (float)kPix) + wh[kCh + c] * hb[c];
        const float e = y - k[blockIdx.x];
        atomicAdd(loss, e * e / (float)n);
        const float g = 2.f * e / (float)n;
        for (int c = 0; c < kCh; ++c) {
            atomicAdd(&gwh[c], g * (s_sum[c] / (float)kPix));
            atomicAdd(&gwh[kCh + c], g * hb[c]);
            dgap[blockIdx.x * kCh + c] = g * wh[c] / (float)kPix;
        }
        atomicAdd(&gwh[2 * kCh], g);
    }
}

// Gradient of the last layer's output: dgap broadcast over the positions,
// times the ReLU of that output.
__global__ void train_dx4_kernel(const __nv_bfloat16* __restrict__ x4, const float* __restrict__ dgap, int n,
                                 __nv_bfloat16* __restrict__ dx4) {
    const size_t total = (size_t)n * kPix * kCh;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t img = i / ((size_t)kPix * kCh);
        const int c = (int)(i % kCh);
        dx4[i] = __float2bfloat16_rn(__bfloat162float(x4[i]) > 0.f ? dgap[img * kCh + c] : 0.f);
    }
}

// Adam step on the parameter vector (gradients g): m, v moments, step t.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    w[i] -= lr * mh / (sqrtf(vh) + eps);
}

// x0 (bf16) of the selected images: out[b] = in[idx[b]].
__global__ void gather_kernel(const __nv_bfloat16* __restrict__ in, const float* __restrict__ hist_in,
                              const float* __restrict__ k_in, const int* __restrict__ idx, int n,
                              __nv_bfloat16* __restrict__ out, float* __restrict__ hist_out, float* __restrict__ k_out) {
    const int b = blockIdx.x;
    if (b >= n) return;
    const int j = idx[b];
    for (int p = threadIdx.x; p < kPix; p += blockDim.x) out[(size_t)b * kPix + p] = in[(size_t)j * kPix + p];
    if (threadIdx.x < kBins) hist_out[b * kBins + threadIdx.x] = hist_in[j * kBins + threadIdx.x];
    if (threadIdx.x == 0) k_out[b] = k_in[j];
}

// Parameter vector (hgrms_predictor_load's order) -> the B operand images
// of the four layers for the forward pass (element (n = output channel,
// k = input channel or, for layer 1, tap)) and of layers 2..4 for the
// backward pass through their input (element (n = input channel, k =
// output channel)), bf16, rounded to nearest even.
__global__ void pack_kernel(const float* __restrict__ wv, uint8_t* __restrict__ fwd0, uint8_t* __restrict__ fwd1,
                            uint8_t* __restrict__ fwd2, uint8_t* __restrict__ fwd3, uint8_t* __restrict__ bwd1,
                            uint8_t* __restrict__ bwd2, uint8_t* __restrict__ bwd3) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 7 x 9 steps x 256 elements
    if (i >= 7 * 9 * 256) return;
    const int which = i / (9 * 256), rem = i % (9 * 256);
    const int step = rem / 256, n = (rem % 256) / 16, k = rem % 16;
    float v = 0.f;
    uint8_t* dst;
    if (which == 0) {  // layer 1 forward: one step, k = tap
        if (step != 0) return;
        if (k < 9) v = wv[k * kCh + n];
        dst = fwd0;
    } else if (which <= 3) {  // layers 2..4 forward
        const float* wl = wv + 144 + (which - 1) * 2304;
        v = wl[(step * kCh + k) * kCh + n];
        dst = which == 1 ? fwd1 : (which == 2 ? fwd2 : fwd3);
    } else {  // layers 2..4 backward through the input
        const float* wl = wv + 144 + (which - 4) * 2304;
        v = wl[(step * kCh + n) * kCh + k];
        dst = which == 4 ? bwd1 : (which == 5 ? bwd2 : bwd3);
    }
    *reinterpret_cast<__nv_bfloat16*>(dst + step * kBBytes + core_off(n, k)) = __float2bfloat16_rn(v);
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

namespace hg {

namespace {

constexpr int kNW = 144 + 3 * 2304 + 64 + 33;  // parameters
constexpr int kBiasOff = 144 + 3 * 2304;
constexpr int kHeadOff = kBiasOff + 64;

// Device state of a fit.
struct Trainer {
    int n = 0, batch = 0;
    __nv_bfloat16* x0 = nullptr;  // n x 4096
    float* hist = nullptr;        // n x 16
    float* k = nullptr;           // n
    __nv_bfloat16* xb = nullptr;  // batch x 4096
    float* hb = nullptr;
    float* kb = nullptr;
    int* idx = nullptr;
    __nv_bfloat16* act[4] = {};   // batch x 4096 x 16
    __nv_bfloat16* grad[2] = {};  // batch x 4096 x 16
    float* dgap = nullptr;
    float* w = nullptr;           // parameters
    float* g = nullptr;           // gradients
    float* m = nullptr;
    float* v = nullptr;
    float* loss = nullptr;
    unsigned* err = nullptr;
    uint8_t* fwd[4] = {};
    uint8_t* bwd[4] = {};

    ~Trainer() {
        cudaFree(x0); cudaFree(hist); cudaFree(k); cudaFree(xb); cudaFree(hb); cudaFree(kb); cudaFree(idx);
        for (auto* a : act) cudaFree(a);
        for (auto* a : grad) cudaFree(a);
        cudaFree(dgap); cudaFree(w); cudaFree(g); cudaFree(m); cudaFree(v); cudaFree(loss); cudaFree(err);
        for (auto* a : fwd) cudaFree(a);
        for (auto* a : bwd) cudaFree(a);
    }
};

uint16_t to_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

int trainer_init(Trainer& t, const float* x0, const float* hist, const float* k, int n, int batch,
                 const float* weights, cudaStream_t s) {
    t.n = n;
    t.batch = batch;
    const size_t act = (size_t)batch * kPix * kCh * sizeof(__nv_bfloat16);
    bool ok = cudaMalloc(&t.x0, (size_t)n * kPix * 2) == cudaSuccess &&
              cudaMalloc(&t.hist, (size_t)n * kBins * 4) == cudaSuccess && cudaMalloc(&t.k, (size_t)n * 4) == cudaSuccess &&
              cudaMalloc(&t.xb, (size_t)batch * kPix * 2) == cudaSuccess &&
              cudaMalloc(&t.hb, (size_t)batch * kBins * 4) == cudaSuccess &&
              cudaMalloc(&t.kb, (size_t)batch * 4) == cudaSuccess && cudaMalloc(&t.idx, (size_t)batch * 4) == cudaSuccess &&
              cudaMalloc(&t.dgap, (size_t)batch * kCh * 4) == cudaSuccess && cudaMalloc(&t.w, kNW * 4) == cudaSuccess &&
              cudaMalloc(&t.g, kNW * 4) == cudaSuccess && cudaMalloc(&t.m, kNW * 4) == cudaSuccess &&
              cudaMalloc(&t.v, kNW * 4) == cudaSuccess && cudaMalloc(&t.loss, 4) == cudaSuccess &&
              cudaMalloc(&t.err, 4) == cudaSuccess;
    for (int i = 0; i < 4 && ok; ++i) ok = cudaMalloc(&t.act[i], act) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i) ok = cudaMalloc(&t.grad[i], act) == cudaSuccess;
    for (int i = 0; i < 4 && ok; ++i)
        ok = cudaMalloc(&t.fwd[i], 9 * kBBytes) == cudaSuccess && cudaMalloc(&t.bwd[i], 9 * kBBytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return HGRMS_ENOMEM;
    }
    std::vector<uint16_t> xh((size_t)n * kPix);
    for (size_t i = 0; i < xh.size(); ++i) xh[i] = to_bf16(x0[i]);
    cudaError_t e = cudaMemcpyAsync(t.x0, xh.data(), xh.size() * 2, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.hist, hist, (size_t)n * kBins * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.k, k, (size_t)n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.w, weights, kNW * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t.m, 0, kNW * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t.v, 0, kNW * 4, s);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
        e = cudaMemsetAsync(t.fwd[i], 0, 9 * kBBytes, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(t.bwd[i], 0, 9 * kBBytes, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(t.err, 0, 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // xh goes out of scope
    return e == cudaSuccess ? HGRMS_OK : HGRMS_ECUDA;
}

cudaError_t trainer_pack(Trainer& t, cudaStream_t s) {
    pack_kernel<<<(7 * 9 * 256 + 255) / 256, 256, 0, s>>>(t.w, t.fwd[0], t.fwd[1], t.fwd[2], t.fwd[3], t.bwd[1],
                                                          t.bwd[2], t.bwd[3]);
    return cudaGetLastError();
}

// Gradient of the mean squared k error over the images idx_host[0..nb) into
// t.g (and their loss into t.loss): forward through the tensor-core layers,
// then back through them.
cudaError_t trainer_grad(Trainer& t, const int* idx_host, int nb, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(t.idx, idx_host, (size_t)nb * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t.g, 0, kNW * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t.loss, 0, 4, s);
    if (e != cudaSuccess) return e;
    gather_kernel<<<nb, 256, 0, s>>>(t.x0, t.hist, t.k, t.idx, nb, t.xb, t.hb, t.kb);
    const __nv_bfloat16* in = t.xb;
    for (int l = 0; l < 4; ++l) {
        conv_tc_kernel<<<dim3(kPix / kBlockM, nb), 128, 0, s>>>(in, l == 0 ? 1 : kCh, t.fwd[l], t.w + kBiasOff + 16 * l,
                                                                t.act[l], t.err);
        in = t.act[l];
    }
    train_head_kernel<<<nb, 256, 0, s>>>(t.act[3], t.hb, t.kb, t.w + kHeadOff, nb, t.g + kHeadOff, t.dgap, t.loss);
    train_dx4_kernel<<<256, 256, 0, s>>>(t.act[3], t.dgap, nb, t.grad[0]);
    int cur = 0;
    const int woff[4] = {0, 144, 144 + 2304, 144 + 2 * 2304};
    for (int l = 3; l >= 0; --l) {
        const __nv_bfloat16* X = l == 0 ? t.xb : t.act[l - 1];
        conv_wgrad_tc_kernel<<<nb, 128, 0, s>>>(X, l == 0 ? 1 : kCh, t.grad[cur], t.g + woff[l],
                                                t.g + kBiasOff + 16 * l, t.err);
        if (l > 0) {
            conv_tc_kernel<<<dim3(kPix / kBlockM, nb), 128, 0, s>>>(t.grad[cur], kCh, t.bwd[l], nullptr,
                                                                    t.grad[cur ^ 1], t.err, t.act[l - 1]);
            cur ^= 1;
        }
    }
    return cudaGetLastError();
}

}  // namespace

int predictor_grad(const float* weights, const float* x0, const float* hist, const float* k, int n, float* grads,
                   float* loss, cudaStream_t s) {
    if (n < 1 || n > 4096) return HGRMS_EINVAL;
    Trainer t;
    int rc = trainer_init(t, x0, hist, k, n, n, weights, s);
    if (rc < 0) return rc;
    std::vector<int> idx((size_t)n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    cudaError_t e = trainer_pack(t, s);
    if (e == cudaSuccess) e = trainer_grad(t, idx.data(), n, s);
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(grads, t.g, kNW * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, t.loss, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, t.err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return HGRMS_ECUDA;
    return err ? HGRMS_ETIMEOUT : HGRMS_OK;
}

int predictor_train(float* weights, const float* x0, const float* hist, const float* k, int n, int epochs, int batch,
                    float lr, unsigned long long seed, float* loss_out, cudaStream_t s) {
    if (n < 1 || batch < 1 || batch > 4096 || epochs < 0 || !(lr > 0.f)) return HGRMS_EINVAL;
    if (batch > n) batch = n;
    Trainer t;
    int rc = trainer_init(t, x0, hist, k, n, batch, weights, s);
    if (rc < 0) return rc;
    std::vector<int> perm((size_t)n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    unsigned long long st = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto next = [&st]() {  // 64-bit LCG, high bits
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        return (uint32_t)(st >> 33);
    };
    cudaError_t e = trainer_pack(t, s);
    int step = 0;
    double last = 0.0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[next() % (uint32_t)(i + 1)]);
        double ep_loss = 0.0;
        int batches = 0;
        const float lr_ep = ep >= (3 * epochs) / 4 ? lr / 3.f : lr;
        for (int b0 = 0; b0 + batch <= n && e == cudaSuccess; b0 += batch) {
            e = trainer_grad(t, perm.data() + b0, batch, s);
            if (e != cudaSuccess) break;
            ++step;
            adam_kernel<<<(kNW + 255) / 256, 256, 0, s>>>(t.w, t.g, t.m, t.v, kNW, lr_ep, 0.9f, 0.999f, 1e-8f, step);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = trainer_pack(t, s);
            float l = 0.f;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&l, t.loss, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            ep_loss += l;
            ++batches;
        }
        last = batches ? ep_loss / batches : 0.0;
    }
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(weights, t.w, kNW * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, t.err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return HGRMS_ECUDA;
    if (loss_out) *loss_out = (float)last;
    return err ? HGRMS_ETIMEOUT : HGRMS_OK;
}

}  // namespace hg
