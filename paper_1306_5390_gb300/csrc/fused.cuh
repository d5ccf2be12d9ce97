// Fused multi-pass tile kernel: T consecutive passes of the P-HGRMS stencil
// pair (Algorithm 1, cardinality; Algorithm 2, root-mean-square replacement)
// on one shared-memory tile per CTA.
//
// Mathematical basis (all derived from Algorithms 1-2; see also the oracle):
//  * One pass reads only the (2 beta + 1)^2 window of each pixel, so T passes
//    on a core tile need a halo of T*beta pixels; the halo is recomputed
//    redundantly by neighbouring tiles and gives bit-identical values.
//  * Border band: a pixel closer than beta to an image edge can never be
//    replaced (too few of its window positions are on the image for flag to
//    exceed pix_count - 3), and every other pixel has its whole window on
//    the image.  So the stencil needs no bounds tests; pixels in the band and
//    pixels outside the image simply keep their value.
//  * Interior decision: with pix_count = (2 beta + 1)^2 and flag = pix_count
//    minus the number of "closed" window pixels (I[p]-alpha < I[n] <=
//    I[p]+alpha, p itself closed when alpha >= 1), "flag > pix_count - 3"
//    is "at most one closed neighbour besides p", and it implies card <= 2.
//    The kernel counts closed neighbours for every pixel with packed fp16
//    arithmetic and runs the exact scalar definition only for pixels with at
//    most one closed neighbour (for alpha = 0 nothing is closed, so every
//    interior pixel takes the exact path).
//
// Packed closed-neighbour test.  Pixel values are stored in shared memory as
// fp16 (exact for 0..255), two pixels per 32-bit word.  For a centre value
// c and neighbour v, closed <=> -alpha < v - c <= alpha <=> |v - (c + 0.5)|
// < alpha.  With e = v - (c + 0.5) (a half-integer, exact in fp16) the value
// sat(2 alpha - 2|e|) is exactly 1 when closed and exactly 0 otherwise (the
// argument is an odd integer), so one subtract, one fused multiply-add with
// saturation and one add count two pixels' neighbours.  A count of 0 or 1 is
// an fp16 bit pattern with bit 14 clear; 2 and above have it set.
#pragma once

#include <cuda_fp16.h>
#include "common.cuh"

namespace hg {

template <int B, int T>
struct FusedGeo {
    static constexpr int kThreads = 256;
    static constexpr int kWarps = kThreads / 32;
    static constexpr int kRows = 8;                  // output rows per thread per pass
    static constexpr int TW = 240;                   // core tile width (pixels)
    static constexpr int RN = kRows * kWarps;        // rows computed per pass (64)
    static constexpr int TH = RN - 2 * (T - 1) * B;  // core tile height
    static constexpr int H = T * B;                  // vertical halo
    static constexpr int SH = TH + 2 * H;            // tile rows in shared memory
    static constexpr int SW = TW + 2 * kPadX;        // tile columns (fp16 values)
    static constexpr int SWW = SW / 2;               // 32-bit words per tile row
    static constexpr int R0 = H - (T - 1) * B;       // first computed row
    static constexpr int C0 = kPadX - 8;             // first computed column
    static constexpr size_t kSmem = 2ull * SH * SW * sizeof(__half);
    // Lanes 0..31 cover columns [C0, C0 + 256): results within T*beta of
    // those edges may use wrong horizontal neighbours, so T*beta <= 8 keeps
    // the core [kPadX, kPadX + TW) exact after T passes.
    static_assert(T * B <= 8, "fused halo exceeds the computed margin");
    static_assert(TH >= 16, "tile too short");
    static_assert(C0 + 8 * 32 == kPadX + TW + 8, "strip layout");
};

__device__ __forceinline__ __half2 u2h(uint32_t x) {
    __half2 h;
    *reinterpret_cast<uint32_t*>(&h) = x;
    return h;
}
__device__ __forceinline__ uint32_t h2u(__half2 h) {
    return *reinterpret_cast<uint32_t*>(&h);
}

// Four bytes of word w selected by `sel` (0x4140: bytes 0,1; 0x4342: bytes
// 2,3) -> an fp16 pair of their values: 0x64 in the high byte makes the
// fp16 number 1024 + byte, and subtracting 1024 is exact.
__device__ __forceinline__ uint32_t bytes_to_h2(uint32_t w, uint32_t sel) {
    const __half2 k1024 = __float2half2_rn(1024.f);
    return h2u(__hsub2(u2h(__byte_perm(w, 0x64646464u, sel)), k1024));
}
// Two fp16 pairs holding integers 0..255 -> four bytes.
__device__ __forceinline__ uint32_t h2_to_bytes(uint32_t a, uint32_t b) {
    const __half2 k1024 = __float2half2_rn(1024.f);
    uint32_t ab = h2u(__hadd2(u2h(a), k1024));
    uint32_t bb = h2u(__hadd2(u2h(b), k1024));
    return __byte_perm(ab, bb, 0x6420);
}

// One tile row as seen by one thread: fp16 pairs starting at pixel offsets
// -B .. 6+B relative to the thread's 8-pixel strip.
template <int B>
struct Row {
    static constexpr int WB = (B + 1) / 2;  // words needed beyond each side of the strip
    static constexpr int NP = 7 + 2 * B;
    uint32_t p[NP];
};

// Load one row: the strip's four words with one 16-byte shared load, the
// neighbouring words from the adjacent lanes (lane 0 / lane 31 get their own
// words, which only affects pixels outside the exact region), and the
// odd-offset pairs by byte permutation.
template <int B>
__device__ __forceinline__ void load_row(const uint32_t* __restrict__ rowp, Row<B>& r) {
    constexpr int WB = Row<B>::WB;
    const uint4 c = *reinterpret_cast<const uint4*>(rowp);
    const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
    uint32_t w[4 + 2 * WB];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[WB + i] = cw[i];
#pragma unroll
    for (int i = 0; i < WB; ++i) {
        w[WB - 1 - i] = __shfl_up_sync(0xffffffffu, cw[3 - i], 1);
        w[WB + 4 + i] = __shfl_down_sync(0xffffffffu, cw[i], 1);
    }
#pragma unroll
    for (int o = -B; o <= 6 + B; ++o) {
        if ((o & 1) == 0)
            r.p[o + B] = w[WB + o / 2];
        else
            r.p[o + B] = __byte_perm(w[WB + (o - 1) / 2], w[WB + (o + 1) / 2], 0x5432);
    }
}

// Add row `dy`'s closed neighbours to the counts of the strip's 8 pixels.
template <int B>
__device__ __forceinline__ void count_row(const Row<B>& rr, const int dy, const __half2 (&cp)[4],
                                          const __half2 two_a, __half2 (&cnt)[4]) {
    const __half2 m2 = __float2half2_rn(-2.f);
#pragma unroll
    for (int dx = -B; dx <= B; ++dx) {
        if (dy == 0 && dx == 0) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __half2 e = __hsub2(u2h(rr.p[2 * j + dx + B]), cp[j]);
            const __half2 f = __hfma2_sat(__habs2(e), m2, two_a);
            cnt[j] = __hadd2(cnt[j], f);
        }
    }
}

// Exact Algorithm 2 for one interior pixel at tile position (y, x): returns
// the replacement value, or -1 when the pixel is not replaced.  Values are
// integers below 2^24, so float arithmetic is exact; floor(sum / flag) is
// exact because a non-integer quotient is at least 1/flag from the next
// integer, far above float rounding at these magnitudes, and the square
// root is correctly rounded (floor of it is exact for arguments <= 65025).
template <int B, int SW>
__device__ __noinline__ int exact_replacement(const __half* __restrict__ in, int y, int x, int alpha) {
    const float ip = __half2float(in[y * SW + x]);
    const float hi = ip + (float)alpha + 1.f;
    const float lo = ip - (float)alpha;
    float sum = 0.f;
    int flag = 0;
#pragma unroll
    for (int dy = -B; dy <= B; ++dy)
#pragma unroll
        for (int dx = -B; dx <= B; ++dx) {
            const float v = __half2float(in[(y + dy) * SW + x + dx]);
            if (!(v < hi && v > lo)) {
                sum = fmaf(v, v, sum);
                ++flag;
            }
        }
    constexpr int kPixCount = (2 * B + 1) * (2 * B + 1);
    if (flag > kPixCount - 3) {
        const float q = floorf(__fdiv_rn(sum, (float)flag));
        return (int)floorf(__fsqrt_rn(q));
    }
    return -1;
}

// One pass over this thread's strip: 8 columns x 8 rows starting at tile row
// ys and word ws.  Writes the strip to `out`; returns whether a core pixel
// changed.
template <int B, int T>
__device__ __forceinline__ bool pass_strip(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                           const int ys, const int ws, const __half2 two_a,
                                           const int x0, const int y0, const int rows, const int cols,
                                           const int alpha) {
    using G = FusedGeo<B, T>;
    constexpr bool kRing = (B <= 2);
    const __half2 half_ = __float2half2_rn(0.5f);
    bool changed = false;
    Row<B> win[kRing ? 2 * B + 1 : 1];
    if constexpr (kRing) {
#pragma unroll
        for (int d = 0; d < 2 * B; ++d) load_row<B>(in + (ys - B + d) * G::SWW + ws, win[d + 1]);
    }
#pragma unroll
    for (int r = 0; r < G::kRows; ++r) {
        const int y = ys + r;
        __half2 cp[4], cnt[4];
        uint4 centre;
        if constexpr (kRing) {
#pragma unroll
            for (int d = 0; d < 2 * B; ++d) win[d] = win[d + 1];
            load_row<B>(in + (y + B) * G::SWW + ws, win[2 * B]);
            const Row<B>& c = win[B];
            centre = make_uint4(c.p[B], c.p[B + 2], c.p[B + 4], c.p[B + 6]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cp[j] = __hadd2(u2h(c.p[2 * j + B]), half_);
                cnt[j] = __float2half2_rn(0.f);
            }
#pragma unroll
            for (int dy = -B; dy <= B; ++dy) count_row<B>(win[dy + B], dy, cp, two_a, cnt);
        } else {
            Row<B>& rr = win[0];
            load_row<B>(in + y * G::SWW + ws, rr);
            centre = make_uint4(rr.p[B], rr.p[B + 2], rr.p[B + 4], rr.p[B + 6]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cp[j] = __hadd2(u2h(rr.p[2 * j + B]), half_);
                cnt[j] = __float2half2_rn(0.f);
            }
            count_row<B>(rr, 0, cp, two_a, cnt);
#pragma unroll
            for (int dy = -B; dy <= B; ++dy) {
                if (dy == 0) continue;
                load_row<B>(in + (y + dy) * G::SWW + ws, rr);
                count_row<B>(rr, dy, cp, two_a, cnt);
            }
        }
        *reinterpret_cast<uint4*>(out + y * G::SWW + ws) = centre;
        const uint32_t all = h2u(cnt[0]) & h2u(cnt[1]) & h2u(cnt[2]) & h2u(cnt[3]);
        if ((all & 0x40004000u) != 0x40004000u) {
            const __half* hin = reinterpret_cast<const __half*>(in);
            __half* hout = reinterpret_cast<__half*>(out);
            const int gy = y0 + y - G::H;
            const bool row_interior = gy >= B && gy < rows - B;
            const bool row_core = y >= G::H && y < G::H + G::TH;
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    if ((h2u(cnt[j]) >> (16 * hh)) & 0x4000u) continue;
                    const int x = 2 * ws + 2 * j + hh;
                    const int gx = x0 + x - kPadX;
                    if (!row_interior || gx < B || gx >= cols - B) continue;
                    const int v = exact_replacement<B, G::SW>(hin, y, x, alpha);
                    if (v < 0) continue;
                    const __half hv = __int2half_rn(v);
                    hout[y * G::SW + x] = hv;
                    if (row_core && x >= kPadX && x < kPadX + G::TW &&
                        __half_as_ushort(hv) != __half_as_ushort(hin[y * G::SW + x]))
                        changed = true;
                }
        }
    }
    return changed;
}

template <int B, int T>
__global__ void __launch_bounds__(256, (B == 1 ? 3 : 2))
fused_kernel(PassArgs a) {
    using G = FusedGeo<B, T>;
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_np;
    __shared__ unsigned s_cur;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_np = launch_passes(a.ctrl, T);
        s_cur = __ldcg(&a.ctrl->cur);
    }
    __syncthreads();
    const int np = s_np;
    if (np == 0) return;
    const uint8_t* src = s_cur ? a.canvas_b : a.canvas_a;
    uint8_t* dst = s_cur ? const_cast<uint8_t*>(a.canvas_a) : a.canvas_b;
    const int tx = blockIdx.x % a.tiles_x;
    const int ty = blockIdx.x / a.tiles_x;
    const int x0 = tx * G::TW, y0 = ty * G::TH;
    uint32_t* buf0 = smem;
    uint32_t* buf1 = smem + G::SH * G::SWW;

    // Tile with halo: image rows [y0 - H, y0 + TH + H), columns [x0 - 16,
    // x0 + TW + 16); always inside the canvas.  Bytes -> fp16 pairs.
    {
        const uint8_t* base = src + (long long)(kPadY + y0 - G::H) * a.pitch + x0;
        constexpr int CH = G::SW / 16;
        for (int i = tid; i < G::SH * CH; i += G::kThreads) {
            const int r = i / CH, c = i - r * CH;
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(base + (long long)r * a.pitch + c * 16));
            uint4 lo, hi;
            lo.x = bytes_to_h2(v.x, 0x4140u); lo.y = bytes_to_h2(v.x, 0x4342u);
            lo.z = bytes_to_h2(v.y, 0x4140u); lo.w = bytes_to_h2(v.y, 0x4342u);
            hi.x = bytes_to_h2(v.z, 0x4140u); hi.y = bytes_to_h2(v.z, 0x4342u);
            hi.z = bytes_to_h2(v.w, 0x4140u); hi.w = bytes_to_h2(v.w, 0x4342u);
            uint4* d = reinterpret_cast<uint4*>(buf0 + r * G::SWW + c * 8);
            d[0] = lo;
            d[1] = hi;
        }
    }
    __syncthreads();

    unsigned cta_mask = 0;
    const __half2 two_a = __float2half2_rn(2.f * (float)a.alpha);
    const int ys = G::R0 + warp * G::kRows;
    const int ws = G::C0 / 2 + 4 * lane;
    for (int t = 0; t < np; ++t) {
        const uint32_t* in = (t & 1) ? buf1 : buf0;
        uint32_t* out = (t & 1) ? buf0 : buf1;
        const bool ch = pass_strip<B, T>(in, out, ys, ws, two_a, x0, y0, a.rows, a.cols, a.alpha);
        if (__syncthreads_or(ch)) cta_mask |= 1u << t;
    }
    const uint32_t* fin = (np & 1) ? buf1 : buf0;

    // Core -> canvas bytes.
    {
        uint8_t* base = dst + (long long)(kPadY + y0) * a.pitch + kPadX + x0;
        constexpr int CH = G::TW / 16;
        for (int i = tid; i < G::TH * CH; i += G::kThreads) {
            const int r = i / CH, c = i - r * CH;
            const uint4* s = reinterpret_cast<const uint4*>(fin + (G::H + r) * G::SWW + kPadX / 2 + c * 8);
            const uint4 p = s[0], q = s[1];
            uint4 o;
            o.x = h2_to_bytes(p.x, p.y);
            o.y = h2_to_bytes(p.z, p.w);
            o.z = h2_to_bytes(q.x, q.y);
            o.w = h2_to_bytes(q.z, q.w);
            *reinterpret_cast<uint4*>(base + (long long)r * a.pitch + c * 16) = o;
        }
    }
    if (tid == 0) finish_launch(a.ctrl, cta_mask, np, gridDim.x);
}

// Host-side description of one compiled (beta, T) instance.
struct FusedEntry {
    int beta, T, TH, TW;
    size_t smem;
    cudaError_t (*launch)(const PassArgs&, int tiles_y, cudaStream_t);
};

template <int B, int T>
cudaError_t launch_fused(const PassArgs& a, int tiles_y, cudaStream_t s) {
    using G = FusedGeo<B, T>;
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<B, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::kSmem);
    if (e != cudaSuccess) return e;
    fused_kernel<B, T><<<(unsigned)(a.tiles_x * tiles_y), G::kThreads, G::kSmem, s>>>(a);
    return cudaGetLastError();
}

template <int B, int T>
constexpr FusedEntry fused_entry() {
    using G = FusedGeo<B, T>;
    return FusedEntry{B, T, G::TH, G::TW, G::kSmem, &launch_fused<B, T>};
}

}  // namespace hg
