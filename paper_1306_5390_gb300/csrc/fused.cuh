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
//  * Locality of change: a pixel's output in pass t depends only on its
//    window in the image of pass t-1.  If no pixel within beta of p changed
//    in pass t-1, p's output in pass t equals its output in pass t-1, i.e.
//    its current value.  With two ping-pong buffers, the buffer written by
//    pass t already holds pass t-2's values, which equal pass t-1's at every
//    pixel that did not change in pass t-1.  So once few pixels change, a
//    pass only evaluates the windows around the pixels the previous pass
//    changed (a "list pass"); every other pixel is already correct in both
//    buffers.  Between launches the changed pixels of a launch's last pass
//    travel in a global bitmap, one bit per pixel.
//
// Packed closed-neighbour test.  Pixel values are stored in shared memory as
// fp16 (exact for 0..255), two pixels per 32-bit word.  For a centre value
// c and neighbour v, closed <=> -alpha < v - c <= alpha <=> |v - (c + 0.5)|
// < alpha.  With e = v - (c + 0.5) (a half-integer, exact in fp16) the value
// sat(2 alpha - 2|e|) is exactly 1 when closed and exactly +0 otherwise (the
// argument is an odd integer), so one subtract and one fused multiply-add
// with saturation test two pixels against one neighbour each.
//
// Counting on the integer pipe (beta <= 3).  The two fp16 instructions above
// run on the FMA pipe; the 0/1 results are summed as 32-bit integers instead
// of with a third fp16 add (bit patterns 0x0000 / 0x3C00 per half, two
// results per three-input add), which moves a third of the per-neighbour
// work to the ALU pipe.  After K_lo and K_hi closed neighbours (K <= 48 for
// beta <= 3; wider windows keep an fp16 running count) the low half holds 15360 K_lo mod 2^16 and
// the high half 15360 K_hi + c (mod 2^16), c = floor(15360 K_lo / 2^16) <= 11
// being the carry out of the low half.  Since 15360 = 1024 * 15 and 47 * 15 =
// 1 (mod 64), multiplying the word by 47 leaves 1024 (K_lo mod 64) in the
// low half and 1024 (K_hi mod 64) + r, r < 1024, in the high half, so byte 1
// of the product is 4 K_lo and byte 3 is 4 K_hi + (0..2): "at most one
// closed neighbour" is "byte & 0xF8 == 0" for both.

// Work layout: a pass computes rows [R0, R0 + RN) (RN = 64, or 128 for the
// tall instances of beta 1 and 2) and columns [8, 264).  In a dense pass warp w walks the rows
// [R0 + rw, R0 + rw + r) of its band (r = 4 for beta 1, else 8) with a register ring
// of the 2 beta + 1 window rows, lane l owning the 8 pixels at columns
// [8 + 8l, 16 + 8l); candidate pixels (at most one closed neighbour) are
// appended to a per-warp list and evaluated exactly, one per lane.  A list
// pass spreads (changed pixel, window offset) pairs over all threads.
#pragma once

#include <cuda_fp16.h>
#include "common.cuh"

namespace hg {

template <int B, int T, int RN_ = 64>
struct FusedGeo {
    // Rows computed per pass: 64 (two CTAs per SM) or 128 (one CTA per SM
    // with twice the threads: the T*beta halo rows above and below are a
    // smaller share of the work, measured 7 % faster for beta 1 and 4 % for
    // beta 2 on large images; small images get fewer, longer tiles).  beta 1
    // uses warps of 4-row bands (twice the resident warps at the same shared
    // memory); wider windows need more registers per thread and use warps of
    // 8-row bands.
    static constexpr int RN = RN_;
    static_assert(RN == 64 || RN == 128, "tile rows");
    static constexpr int kMinBlocks = RN == 64 ? 2 : 1;  // resident CTAs per SM
    static constexpr int kThreads = (B == 1 ? 512 : 256) * (RN / 64);
    static constexpr int kWarps = kThreads / 32;
    static constexpr int kRows = RN / kWarps;        // rows per warp band (dense passes)
    static constexpr int TW = 240;                   // core tile width (pixels)
    static constexpr int TH = RN - 2 * (T - 1) * B;  // core tile height
    static constexpr int H = T * B;                  // vertical halo
    static constexpr int SH = TH + 2 * H;            // tile rows in shared memory (= RN + 2B)
    static constexpr int SW = TW + 2 * kPadX;        // tile columns (fp16 values)
    static constexpr int SWW = SW / 2;               // 32-bit words per tile row
    static constexpr int R0 = H - (T - 1) * B;       // first computed row (= B)
    static constexpr int C0 = kPadX - 8;             // first computed column
    static constexpr int CN = 256;                   // computed columns
    static constexpr int P = (2 * B + 1) * (2 * B + 1);
    // Band rows per candidate append (at most 256 candidates per row): beta 2
    // appends every 4 rows (measured faster than 2), the others every 2, which
    // keeps the lists small enough for the TMA staging buffer.
    static constexpr int kAppendRows = B == 2 ? 4 : 2;
    // beta 3: dense passes count in stages (band_dense2; for beta 2 the
    // single-stage count measured faster); the second half of a warp's
    // candidate buffer then holds its work list of unsettled pixel pairs (at
    // most 4 per lane and row of a kAppendRows-row group).
    static constexpr bool kStaged = B == 3 && kRows == 8;
    static constexpr int kCandCap = kAppendRows * 256;  // per-warp candidate list
    static constexpr int kCandLimit = kStaged ? kCandCap / 2 : kCandCap;
    // Changed pixels kept per pass: a list pass needs at most eval_max /
    // (2 beta + 1)^2 of them at the built-in switch points (455 for beta 1,
    // 82 for beta 2, 84 for beta 3); a longer list makes the next pass dense.
    static constexpr int kListCap = B == 1 ? 1024 : 448;
    static constexpr int kListEvalMax = 2048;        // default: list-pass evaluations above which a pass runs dense
    static constexpr int kMarkWords = (SH * SW + 31) / 32;
    // shared memory layout (bytes)
    static constexpr size_t kBufBytes = (size_t)SH * SW * sizeof(__half);
    static constexpr size_t kCandOff = 2 * kBufBytes;
    static constexpr size_t kListOff = kCandOff + (size_t)kWarps * kCandCap * sizeof(uint16_t);
    static constexpr size_t kMarkOff = kListOff + 2ull * kListCap * sizeof(uint16_t);
    static constexpr size_t kCntOff = kMarkOff + 2ull * kMarkWords * sizeof(uint32_t);
    static constexpr size_t kSmemBase = kCntOff + 8 * sizeof(int);
    // TMA staging buffer: the next tile with its halo, as bytes (SH rows of SW
    // bytes), loaded while the current tile computes.  Only when the resident
    // CTAs per SM still fit (the SM's 228 KB, less 1 KB reserved per CTA and
    // the static shared variables; at most 227 KB per CTA).
    static constexpr size_t kStaticSmem = 192;  // the kernel's static shared variables (128 bytes) and slack
    static constexpr size_t kStageOff = (kSmemBase + 127) / 128 * 128;
    static constexpr size_t kStageBytes = ((size_t)SH * SW + 127) / 128 * 128;
    static constexpr bool kTma = kMinBlocks * (kStageOff + kStageBytes + 1024 + kStaticSmem) <= 233472 &&
                                 kStageOff + kStageBytes + kStaticSmem <= 232448;
    static constexpr size_t kSmem = kTma ? kStageOff + kStageBytes : kSmemBase;
    // Lanes 0..31 cover columns [C0, C0 + 256): results within T*beta of
    // those edges may use wrong horizontal neighbours, so T*beta <= 8 keeps
    // the core [kPadX, kPadX + TW) exact after T passes.
    static_assert(T * B <= 8, "fused halo exceeds the computed margin");
    static_assert(SW == 17 * 16 && SH <= 256, "TMA box: 17 chunks of 16 bytes by SH rows");
    static_assert(TH >= 16, "tile too short");
    static_assert(SH * SW < 65536, "pixel index encoding");
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

// One tile row as seen by one segment: fp16 pairs starting at pixel offsets
// -B .. 6+B relative to the segment's first pixel.
template <int B>
struct Row {
    static constexpr int WB = (B + 1) / 2;  // words needed beyond each side of the segment
    static constexpr int NP = 7 + 2 * B;
    uint32_t p[NP];
};

template <int B>
__device__ __forceinline__ void make_pairs(const uint32_t (&w)[4 + 2 * Row<B>::WB], Row<B>& r) {
    constexpr int WB = Row<B>::WB;
#pragma unroll
    for (int o = -B; o <= 6 + B; ++o) {
        if ((o & 1) == 0)
            r.p[o + B] = w[WB + o / 2];
        else
            r.p[o + B] = __byte_perm(w[WB + (o - 1) / 2], w[WB + (o + 1) / 2], 0x5432);
    }
}

// Dense form: the segment's four words with one 16-byte shared load, the
// neighbouring words from the adjacent lanes (lane 0 / lane 31 get their own
// words, which only affects pixels outside the exact region).
template <int B>
__device__ __forceinline__ void load_row_shfl(const uint32_t* __restrict__ rowp, Row<B>& r) {
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
    make_pairs<B>(w, r);
}

// Running closed-neighbour count of a segment's 8 pixels.  For beta <= 3
// (at most 48 neighbours, so K mod 64 is K) acc[j] sums the 0/1 results of
// pixels 2j, 2j + 1 as integers (see the header), two results per add, the
// first of each pair waiting in pend.  Wider windows keep the count in fp16
// (exact up to 2048): h[j] = h[j] + result.
template <int B>
struct Count {
    static constexpr bool kInt = (2 * B + 1) * (2 * B + 1) - 1 < 64;
    uint32_t acc[4];
    uint32_t pend[4];
    int n;  // results so far (a compile-time constant after unrolling)
};

// Add row `dy`'s closed neighbours to the counts of the segment's 8 pixels.
template <int B>
__device__ __forceinline__ void count_row(const Row<B>& rr, const int dy, const __half2 (&cp)[4],
                                          const __half2 two_a, Count<B>& c) {
    const __half2 m2 = __float2half2_rn(-2.f);
#pragma unroll
    for (int dx = -B; dx <= B; ++dx) {
        if (dy == 0 && dx == 0) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __half2 e = __hsub2(u2h(rr.p[2 * j + dx + B]), cp[j]);
            const __half2 f = __hfma2_sat(__habs2(e), m2, two_a);
            if constexpr (Count<B>::kInt) {
                if (c.n & 1)
                    c.acc[j] += c.pend[j] + h2u(f);
                else
                    c.pend[j] = h2u(f);
            } else {
                c.acc[j] = h2u(__hadd2(u2h(c.acc[j]), f));
            }
        }
        ++c.n;
    }
}

template <int B>
__device__ __forceinline__ void centre_setup(const Row<B>& c, __half2 (&cp)[4], Count<B>& cnt, uint4& centre) {
    const __half2 half_ = __float2half2_rn(0.5f);
    centre = make_uint4(c.p[B], c.p[B + 2], c.p[B + 4], c.p[B + 6]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        cp[j] = __hadd2(u2h(c.p[2 * j + B]), half_);
        cnt.acc[j] = 0u;  // also fp16 +0
    }
    cnt.n = 0;
}

// Bit 7 of each byte: the pixel has two or more closed neighbours.  Bytes
// are pixels 4i .. 4i + 3 for the pair (acc[2i], acc[2i + 1]).  Integer
// counts: each byte is 4 K (+ 0..2), see the header.  fp16 counts: the high
// byte of a count of 0 or 1 has bit 6 clear, of 2 and above set.
template <int B>
__device__ __forceinline__ uint32_t not_candidate_bits(const uint32_t acc_a, const uint32_t acc_b) {
    if constexpr (Count<B>::kInt) {
        const uint32_t q = __byte_perm(acc_a * 47u, acc_b * 47u, 0x7531);
        return (((q & 0x78787878u) + 0x7F7F7F7Fu) | q) & 0x80808080u;  // byte & 0xF8 != 0
    } else {
        return (__byte_perm(acc_a, acc_b, 0x7531) << 1) & 0x80808080u;
    }
}

// 8-bit mask (pixel i -> bit i) of the pixels with at most one closed
// neighbour, from the two words of not_candidate_bits.
__device__ __forceinline__ uint32_t candidate_mask(const uint32_t na, const uint32_t nb) {
    const uint32_t ma = ((~na >> 7) & 0x01010101u) * 0x01020408u >> 24;
    const uint32_t mb = ((~nb >> 7) & 0x01010101u) * 0x01020408u >> 24;
    return (ma & 0xFu) | ((mb & 0xFu) << 4);
}

// Exact Algorithm 2 for one interior pixel at tile index q = y * SW + x, in
// packed arithmetic: returns the replacement value, or -1 when the pixel is
// not replaced.  cp holds c + 1/2 (c: the pixel's value) and na holds -alpha, in
// both halves.
//
// Each window row is read as the B + 1 words that hold its 2B + 1 fp16
// values.  They hold 2B + 2 halves; the one outside the window (the first
// when the row starts at an odd column, else the last) is masked off, as are
// the padding bytes of a last byte word that takes a single fp16 word.
//  * Closed test: for a value v, g = |v - (c + 1/2)| - alpha is negative
//    exactly when c - alpha < v <= c + alpha (v and c integers, |g| never
//    0), so a byte permute that replicates the sign bits of the halves' high
//    bytes gives 0xFF for a closed value and 0x00 for an open one.  For alpha
//    = 0 every value is open, the pixel itself included.
//  * Values as bytes: the fp16 number 1024 + v has v as its low byte.
//  * With four values and their masks in one word each, the open values'
//    squares sum in one 4-way integer dot product, and a second one with
//    0x01010101 counts the open values (255 per open value).
template <int B, int SW>
__device__ __forceinline__ int exact_packed(const uint32_t* __restrict__ w32, int q, __half2 cp, __half2 na) {
    constexpr int SWW = SW / 2;
    constexpr int NW = B + 1;         // fp16 words per window row
    constexpr int NB = (NW + 1) / 2;  // byte words per window row
    // q = y * SW + x; the window's first value of row y + dy is half q - B +
    // dy * SW, i.e. (SW even) word ((q - B) >> 1) + dy * SWW, at the parity of q - B.
    const int h0 = q - B;
    const bool odd = (h0 & 1) != 0;
    // Bytes of the row that are window values (bit pattern per byte word).
    constexpr uint32_t kLastPad = (NW & 1) ? 0x0000FFFFu : 0xFFFFFFFFu;  // a last word of two bytes
    const uint32_t first_ok = odd ? 0xFFFFFF00u : 0xFFFFFFFFu;
    const uint32_t last_ok = odd ? kLastPad : (kLastPad >> 8);
    const __half2 k1024 = __float2half2_rn(1024.f);
    int sum = 0, open255 = 0;  // sum of the open values' squares; 255 per open value
#pragma unroll
    for (int dy = -B; dy <= B; ++dy) {
        const uint32_t* row = w32 + (h0 >> 1) + dy * SWW;
        uint32_t w[NW];
#pragma unroll
        for (int i = 0; i < NW; ++i) w[i] = row[i];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const uint32_t a = w[2 * k];
            const uint32_t b = (2 * k + 1 < NW) ? w[2 * k + 1] : 0u;
            const uint32_t ga = h2u(__hadd2(__habs2(__hsub2(u2h(a), cp)), na));
            const uint32_t gb = h2u(__hadd2(__habs2(__hsub2(u2h(b), cp)), na));
            const uint32_t vb = __byte_perm(h2u(__hadd2(u2h(a), k1024)), h2u(__hadd2(u2h(b), k1024)), 0x6420u);
            const uint32_t closed = prmt_sign(ga, gb, 0xFDB9u);
            uint32_t ok = 0xFFFFFFFFu;
            if (k == 0) ok &= first_ok;
            if (k == NB - 1) ok &= last_ok;
            const uint32_t open = ~closed & ok;
            sum = (int)__dp4a(vb & open, vb, (unsigned)sum);
            open255 = (int)__dp4a(open, 0x01010101u, (unsigned)open255);
        }
    }
    // flag = open255 / 255; replaced when flag > P - 3, and then flag is
    // P - 2, P - 1 or P, whose reciprocals are constants.
    constexpr int P = (2 * B + 1) * (2 * B + 1);
    if (open255 <= 255 * (P - 3)) return -1;
    const unsigned m = open255 == 255 * P ? recip32(P) : (open255 == 255 * (P - 1) ? recip32(P - 1) : recip32(P - 2));
    return rms_div(sum, m);
}

// Image columns [gx0, gx0 + 16) of row gy of a dense caller image (rows x
// cols bytes, row stride cols), 0 outside the image.  Reads only aligned
// words that hold image bytes: one 16-byte load when aligned, else four or
// five 4-byte loads realigned by funnel shifts, and single bytes for chunks
// that cross a column edge of the image.
__device__ __forceinline__ uint4 load_user_chunk(const uint8_t* __restrict__ user, int rows, int cols, int gy,
                                                 int gx0) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gy < 0 || gy >= rows) return v;
    const uint8_t* rowp = user + (long long)gy * cols;
    if (gx0 >= 0 && gx0 + 16 <= cols) {
        const uintptr_t ad = reinterpret_cast<uintptr_t>(rowp + gx0);
        if ((ad & 15u) == 0) return __ldg(reinterpret_cast<const uint4*>(ad));
        const uint32_t* q = reinterpret_cast<const uint32_t*>(ad & ~uintptr_t(3));
        const uint32_t sh = (uint32_t)(ad & 3u) * 8u;
        const uint32_t w0 = __ldg(q), w1 = __ldg(q + 1), w2 = __ldg(q + 2), w3 = __ldg(q + 3);
        const uint32_t w4 = sh ? __ldg(q + 4) : 0u;
        v.x = __funnelshift_r(w0, w1, sh);
        v.y = __funnelshift_r(w1, w2, sh);
        v.z = __funnelshift_r(w2, w3, sh);
        v.w = __funnelshift_r(w3, w4, sh);
        return v;
    }
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        const int gx = gx0 + b;
        if (gx >= 0 && gx < cols) w[b >> 2] |= (uint32_t)rowp[gx] << (8 * (b & 3));
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Per-pass context shared by the helpers below.
template <int B, int T, int RN>
struct PassCtx {
    using G = FusedGeo<B, T, RN>;
    const uint32_t* in;
    uint32_t* out;
    uint16_t* cand;      // this warp's candidate list (dense passes)
    int ncand;           // entries in the list (warp-uniform)
    uint16_t* list;      // changed pixels of this pass (index y * SW + x)
    int* nlist;          // its counter (may exceed kListCap: overflow)
    unsigned evals;      // core pixels this thread evaluated in list passes
    int x0, y0, rows, cols, alpha;
    // Tile positions of the image pixels at least beta from every edge (the
    // only ones that can change): ylo <= y < yhi, xlo <= x < xhi.
    int ylo, yhi, xlo, xhi;
    bool all_interior;   // every computed position of the tile is interior
    __half2 na;          // -alpha in both halves (exact_packed)
    bool changed_core;   // this lane saw a core pixel change
};

template <int B, int T, int RN>
__device__ __forceinline__ bool interior(const PassCtx<B, T, RN>& c, int y, int x) {
    return y >= c.ylo && y < c.yhi && x >= c.xlo && x < c.xhi;
}

__device__ __forceinline__ bool in_core_px(int y, int x, int H, int TH, int TW) {
    return y >= H && y < H + TH && x >= kPadX && x < kPadX + TW;
}

// Evaluate and clear the warp's candidate list (dense passes): replaced
// pixels are written to the output buffer and recorded as changed.
template <int B, int T, int RN>
__device__ __forceinline__ void flush_candidates(PassCtx<B, T, RN>& c, const int lane) {
    using G = FusedGeo<B, T, RN>;
    __syncwarp();
    const __half* hin = reinterpret_cast<const __half*>(c.in);
    __half* hout = reinterpret_cast<__half*>(c.out);
    for (int base = 0; base < c.ncand; base += 32) {
        const int i = base + lane;
        bool ch = false;
        uint32_t q = 0;
        if (i < c.ncand) {
            q = c.cand[i];
            bool inner = c.all_interior;
            if (!inner) {
                const int y = (int)(q / G::SW), x = (int)(q - (uint32_t)y * G::SW);
                inner = interior(c, y, x);
            }
            if (inner) {
                const __half old = hin[q];
                const int v = exact_packed<B, G::SW>(c.in, (int)q, __half2half2(__hadd(old, __float2half(0.5f))), c.na);
                if (v >= 0) {
                    const __half hv = u8_to_half(v);
                    if (__half_as_ushort(hv) != __half_as_ushort(old)) {
                        hout[q] = hv;
                        ch = true;
                        // Whether a core pixel changed: decoded until this lane has seen one.
                        if (!c.changed_core) {
                            const int y = (int)(q / G::SW), x = (int)(q - (uint32_t)y * G::SW);
                            c.changed_core = in_core_px(y, x, G::H, G::TH, G::TW);
                        }
                    }
                }
            }
        }
        // record the changed pixels (one shared atomic per warp)
        const uint32_t bal = __ballot_sync(0xffffffffu, ch);
        if (bal) {
            int pos = 0;
            if (lane == 0) pos = atomicAdd(c.nlist, __popc(bal));
            pos = __shfl_sync(0xffffffffu, pos, 0) + __popc(bal & ((1u << lane) - 1u));
            if (ch && pos < G::kListCap) c.list[pos] = (uint16_t)q;
        }
    }
    __syncwarp();
    c.ncand = 0;
}

// Append candidate bits (bit 8r + i: row ys + r, pixel x + i) to the warp list.
template <int B, int T, int RN>
__device__ __forceinline__ void append_bits(PassCtx<B, T, RN>& c, const int lane, uint32_t m, const int ys,
                                            const int x) {
    using G = FusedGeo<B, T, RN>;
    if (!__any_sync(0xffffffffu, m != 0u)) return;
    int total;
    const int off0 = warp_excl_scan(lane, __popc(m), &total);
    if (c.ncand + total > G::kCandLimit) flush_candidates<B, T, RN>(c, lane);
    int off = c.ncand + off0;
    while (m) {
        const int b = __ffs(m) - 1;
        c.cand[off++] = (uint16_t)((ys + (b >> 3)) * G::SW + x + (b & 7));
        m &= m - 1;
    }
    c.ncand += total;
}

// Dense pass over the warp's 8-row band: every pixel's closed neighbours are
// counted with the packed test; candidates go to the warp list.
template <int B, int T, int RN>
__device__ __forceinline__ void band_dense(PassCtx<B, T, RN>& c, const int ys, const int ws, const int lane,
                                           const __half2 two_a) {
    using G = FusedGeo<B, T, RN>;
    constexpr bool kRing = (B <= 2);
    Row<B> win[kRing ? 2 * B + 1 : 1];
    unsigned long long m64 = 0ull;
    if constexpr (kRing) {
#pragma unroll
        for (int d = 0; d < 2 * B; ++d) load_row_shfl<B>(c.in + (ys - B + d) * G::SWW + ws, win[d + 1]);
    }
#pragma unroll
    for (int r = 0; r < G::kRows; ++r) {
        const int y = ys + r;
        __half2 cp[4];
        Count<B> cnt;
        uint4 centre;
        if constexpr (kRing) {
#pragma unroll
            for (int d = 0; d < 2 * B; ++d) win[d] = win[d + 1];
            load_row_shfl<B>(c.in + (y + B) * G::SWW + ws, win[2 * B]);
            centre_setup<B>(win[B], cp, cnt, centre);
#pragma unroll
            for (int dy = -B; dy <= B; ++dy) count_row<B>(win[dy + B], dy, cp, two_a, cnt);
        } else {
            Row<B>& rr = win[0];
            load_row_shfl<B>(c.in + y * G::SWW + ws, rr);
            centre_setup<B>(rr, cp, cnt, centre);
            count_row<B>(rr, 0, cp, two_a, cnt);
#pragma unroll
            for (int dy = -B; dy <= B; ++dy) {
                if (dy == 0) continue;
                load_row_shfl<B>(c.in + (y + dy) * G::SWW + ws, rr);
                count_row<B>(rr, dy, cp, two_a, cnt);
            }
        }
        *reinterpret_cast<uint4*>(c.out + y * G::SWW + ws) = centre;
        const uint32_t na = not_candidate_bits<B>(cnt.acc[0], cnt.acc[1]);
        const uint32_t nb = not_candidate_bits<B>(cnt.acc[2], cnt.acc[3]);
        if ((na & nb) != 0x80808080u) m64 |= (unsigned long long)candidate_mask(na, nb) << (8 * r);
    }
    constexpr int kA = G::kAppendRows;  // rows per append (kA * 256 candidates at most)
    constexpr unsigned long long kAMask = (1ull << (8 * kA)) - 1ull;
#pragma unroll
    for (int g = 0; g < G::kRows / kA; ++g)
        append_bits<B, T, RN>(c, lane, (uint32_t)((m64 >> (8 * kA * g)) & kAMask), ys + kA * g, 2 * ws);
}

// ---- Symmetric count (beta 1 and 2) --------------------------------------
// The dense passes only need to know which pixels have at most one closed
// neighbour.  Algorithm 1's own test, |I_n - I_p| < alpha, implies the closed
// test of Algorithm 2 (I_p - alpha < I_n <= I_p + alpha), so a pixel with at
// most one closed neighbour has at most one neighbour passing it: counting
// with it keeps every candidate (the few extra ones, whose neighbours differ
// by exactly alpha, the exact evaluation turns away).  And it is symmetric,
// so each unordered pair of pixels is tested once and the result counts for
// both.  Row y tests its "forward" pairs - (0, dx) for dx = 1..B and (dy, dx)
// for dy = 1..B, dx = -B..B - and adds each result to row y's counts and,
// moved by dx pixels, to row y + dy's.  One fp16x2 test covers a pixel pair:
// sat(2 alpha - 1 - 2 |v_n - v_p|) is 1 for |v_n - v_p| <= alpha - 1 and +0
// otherwise (exact integers in fp16; for alpha = 0 it is always 0).

// Results R[j] (first endpoints: pixels 2j, 2j + 1 of the lane's segment)
// moved by DX pixels: word j of the result covers second endpoints 2j + DX,
// 2j + 1 + DX.  Words that cross into the neighbouring lane's segment come by
// shuffle (lanes 0 and 31 get wrong values there, which only reach pixels
// within B of the computed region's edge, outside the exact region).
template <int DX>
__device__ __forceinline__ void shifted_words(const uint32_t (&r)[4], uint32_t (&s)[4]) {
    static_assert(DX >= -2 && DX <= 2, "beta <= 2");
    if constexpr (DX == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) s[j] = r[j];
    } else if constexpr (DX == 2) {
        const uint32_t nb = __shfl_up_sync(0xffffffffu, r[3], 1);
        s[0] = nb; s[1] = r[0]; s[2] = r[1]; s[3] = r[2];
    } else if constexpr (DX == -2) {
        const uint32_t nb = __shfl_down_sync(0xffffffffu, r[0], 1);
        s[0] = r[1]; s[1] = r[2]; s[2] = r[3]; s[3] = nb;
    } else if constexpr (DX == 1) {
        const uint32_t nb = __shfl_up_sync(0xffffffffu, r[3], 1);
        s[0] = __byte_perm(nb, r[0], 0x5432);
        s[1] = __byte_perm(r[0], r[1], 0x5432);
        s[2] = __byte_perm(r[1], r[2], 0x5432);
        s[3] = __byte_perm(r[2], r[3], 0x5432);
    } else {  // DX == -1
        const uint32_t nb = __shfl_down_sync(0xffffffffu, r[0], 1);
        s[0] = __byte_perm(r[0], r[1], 0x5432);
        s[1] = __byte_perm(r[1], r[2], 0x5432);
        s[2] = __byte_perm(r[2], r[3], 0x5432);
        s[3] = __byte_perm(r[3], nb, 0x5432);
    }
}

// One forward direction (DY, DX) of row y: test it, add the results to the
// counts of row y (when y is in the band: TO_Y) and of row y + DY (TO_YD).
template <int B, int DY, int DX, bool TO_Y, bool TO_YD>
__device__ __forceinline__ void sym_dir(const Row<B>& ry, const Row<B>& ryd, const __half2 lim,
                                        uint32_t (&ky)[4], uint32_t (&kyd)[4]) {
    if constexpr (TO_Y || TO_YD) {
        const __half2 m2 = __float2half2_rn(-2.f);
        uint32_t r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __half2 e = __hsub2(u2h(ryd.p[2 * j + DX + B]), u2h(ry.p[2 * j + B]));
            r[j] = h2u(__hfma2_sat(__habs2(e), m2, lim));
        }
        if constexpr (TO_Y) {
#pragma unroll
            for (int j = 0; j < 4; ++j) ky[j] += r[j];
        }
        if constexpr (TO_YD) {
            uint32_t sh[4];
            shifted_words<DX>(r, sh);
#pragma unroll
            for (int j = 0; j < 4; ++j) kyd[j] += sh[j];
        }
    }
}

// All forward directions of band row R (R < 0: a row above the band, whose
// own counts are not needed).
template <int B, int T, int RN, int R>
__device__ __forceinline__ void sym_row(const Row<B> (&win)[B + 1], const __half2 lim, uint32_t (&k)[B + 1][4]) {
    constexpr int kRows = FusedGeo<B, T, RN>::kRows;
    constexpr bool kIn = R >= 0;
    // same row: both endpoints in row y
    sym_dir<B, 0, 1, kIn, kIn>(win[0], win[0], lim, k[0], k[0]);
    if constexpr (B == 2) sym_dir<B, 0, 2, kIn, kIn>(win[0], win[0], lim, k[0], k[0]);
    // rows below: second endpoint in row y + dy (only when that row is in the band)
    constexpr bool d1 = R + 1 >= 0 && R + 1 < kRows;
    sym_dir<B, 1, -1, kIn, d1>(win[0], win[1], lim, k[0], k[1]);
    sym_dir<B, 1, 0, kIn, d1>(win[0], win[1], lim, k[0], k[1]);
    sym_dir<B, 1, 1, kIn, d1>(win[0], win[1], lim, k[0], k[1]);
    if constexpr (B == 2) {
        sym_dir<B, 1, -2, kIn, d1>(win[0], win[1], lim, k[0], k[1]);
        sym_dir<B, 1, 2, kIn, d1>(win[0], win[1], lim, k[0], k[1]);
        constexpr bool d2 = R + 2 >= 0 && R + 2 < kRows;
        sym_dir<B, 2, -2, kIn, d2>(win[0], win[2], lim, k[0], k[B]);
        sym_dir<B, 2, -1, kIn, d2>(win[0], win[2], lim, k[0], k[B]);
        sym_dir<B, 2, 0, kIn, d2>(win[0], win[2], lim, k[0], k[B]);
        sym_dir<B, 2, 1, kIn, d2>(win[0], win[2], lim, k[0], k[B]);
        sym_dir<B, 2, 2, kIn, d2>(win[0], win[2], lim, k[0], k[B]);
    }
}

template <int B, int T, int RN, int R>
__device__ __forceinline__ void sym_band_row(PassCtx<B, T, RN>& c, const int ys, const int ws, const __half2 lim,
                                             Row<B> (&win)[B + 1], uint32_t (&k)[B + 1][4],
                                             unsigned long long& m64) {
    using G = FusedGeo<B, T, RN>;
    if constexpr (R < G::kRows) {
        // win[i] holds row ys + R + i.
        sym_row<B, T, RN, R>(win, lim, k);
        if constexpr (R >= 0) {
            const uint4 centre = make_uint4(win[0].p[B], win[0].p[B + 2], win[0].p[B + 4], win[0].p[B + 6]);
            *reinterpret_cast<uint4*>(c.out + (ys + R) * G::SWW + ws) = centre;
            const uint32_t na = not_candidate_bits<B>(k[0][0], k[0][1]);
            const uint32_t nb = not_candidate_bits<B>(k[0][2], k[0][3]);
            if ((na & nb) != 0x80808080u) m64 |= (unsigned long long)candidate_mask(na, nb) << (8 * R);
        }
        // Next row: counts and window move up one row.
#pragma unroll
        for (int i = 0; i < B; ++i) {
#pragma unroll
            for (int j = 0; j < 4; ++j) k[i][j] = k[i + 1][j];
            win[i] = win[i + 1];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) k[B][j] = 0u;
        if constexpr (R + 1 < G::kRows) load_row_shfl<B>(c.in + (ys + R + 1 + B) * G::SWW + ws, win[B]);
        sym_band_row<B, T, RN, R + 1>(c, ys, ws, lim, win, k, m64);
    }
}

// Dense pass over the warp's band with the symmetric count (beta 1, 2).
template <int B, int T, int RN>
__device__ __forceinline__ void band_dense_sym(PassCtx<B, T, RN>& c, const int ys, const int ws, const int lane) {
    using G = FusedGeo<B, T, RN>;
    static_assert(B == 1 || B == 2, "symmetric count for beta 1 and 2");
    const __half2 lim = __float2half2_rn(2.f * (float)c.alpha - 1.f);
    Row<B> win[B + 1];
    uint32_t k[B + 1][4];
#pragma unroll
    for (int i = 0; i <= B; ++i) {
        load_row_shfl<B>(c.in + (ys - B + i) * G::SWW + ws, win[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) k[i][j] = 0u;
    }
    unsigned long long m64 = 0ull;
    sym_band_row<B, T, RN, -B>(c, ys, ws, lim, win, k, m64);
    constexpr int kA = G::kAppendRows;
    constexpr unsigned long long kAMask = (1ull << (8 * kA)) - 1ull;
#pragma unroll
    for (int g = 0; g < G::kRows / kA; ++g)
        append_bits<B, T, RN>(c, lane, (uint32_t)((m64 >> (8 * kA * g)) & kAMask), ys + kA * g, 2 * ws);
}

// Closed-neighbour count of one pixel pair (the fp16 pair at word xw of
// tile row y) over the window positions at Chebyshev distance exactly D,
// summed as integers (see the header): 16 results for D = 2, 24 for D = 3.
template <int D, int SWW>
__device__ __forceinline__ uint32_t ring_count(const uint32_t* __restrict__ in, const int y, const int xw,
                                               const __half2 cp, const __half2 two_a) {
    constexpr int WB = (D + 1) / 2;
    const __half2 m2 = __float2half2_rn(-2.f);
    uint32_t acc = 0u, pend = 0u;
    int n = 0;
#pragma unroll
    for (int dy = -D; dy <= D; ++dy) {
        const uint32_t* row = in + (y + dy) * SWW + xw;
        uint32_t w[2 * WB + 1];
#pragma unroll
        for (int k = 0; k <= 2 * WB; ++k) w[k] = row[k - WB];
#pragma unroll
        for (int dx = -D; dx <= D; ++dx) {
            if (dy > -D && dy < D && dx > -D && dx < D) continue;
            const uint32_t pw = (dx & 1) ? __byte_perm(w[WB + (dx - 1) / 2], w[WB + (dx + 1) / 2], 0x5432)
                                         : w[WB + dx / 2];
            const __half2 e = __hsub2(u2h(pw), cp);
            const uint32_t f = h2u(__hfma2_sat(__habs2(e), m2, two_a));
            if (n & 1)
                acc += pend + f;
            else
                pend = f;
            ++n;
        }
    }
    if (n & 1) acc += pend;
    return acc;
}

// Dense pass over the warp's 8-row band in stages (beta 3), in groups of
// kAppendRows rows.  Stage one counts every pixel's closed neighbours in the
// inner 3 x 3 ring, packed as in band_dense; a pixel with two or more already
// has too many to be a candidate.  The other pixels' pairs go to a per-warp
// work list (row, lane, pair and the pixels' state: not settled, one closed
// neighbour so far); stage two counts the ring at distance 2 for them, one
// pair per lane, and keeps (compacted in place) only the pairs with a pixel
// still not settled; stage three counts the ring at distance 3 for those.
// Pixels with at most one closed neighbour in all are candidates.
template <int B, int T, int RN>
__device__ __forceinline__ void band_dense2(PassCtx<B, T, RN>& c, const int ys, const int ws, const int lane,
                                            const __half2 two_a) {
    using G = FusedGeo<B, T, RN>;
    constexpr int kHalf = G::kAppendRows;  // rows per group (its work list fits half the buffer)
    uint16_t* items = c.cand + G::kCandCap / 2;
    Row<1> win[3];
    load_row_shfl<1>(c.in + (ys - 1) * G::SWW + ws, win[1]);
    load_row_shfl<1>(c.in + ys * G::SWW + ws, win[2]);
#pragma unroll
    for (int h = 0; h < G::kRows / kHalf; ++h) {
        // Stage one.  U: pixels not settled (8 bits per row), K: those of
        // them with one closed neighbour in the inner ring.
        uint32_t U = 0u, K = 0u;
#pragma unroll
        for (int rr = 0; rr < kHalf; ++rr) {
            const int y = ys + h * kHalf + rr;
            win[0] = win[1];
            win[1] = win[2];
            load_row_shfl<1>(c.in + (y + 1) * G::SWW + ws, win[2]);
            __half2 cp[4];
            Count<1> cnt;
            uint4 centre;
            centre_setup<1>(win[1], cp, cnt, centre);
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) count_row<1>(win[dy + 1], dy, cp, two_a, cnt);
            *reinterpret_cast<uint4*>(c.out + y * G::SWW + ws) = centre;
            // Bytes 4 K (+ 0..2) of the four pixels of each word (see the header).
            const uint32_t qa = __byte_perm(cnt.acc[0] * 47u, cnt.acc[1] * 47u, 0x7531);
            const uint32_t qb = __byte_perm(cnt.acc[2] * 47u, cnt.acc[3] * 47u, 0x7531);
            const uint32_t na = (((qa & 0x78787878u) + 0x7F7F7F7Fu) | qa) & 0x80808080u;  // K >= 2
            const uint32_t nb = (((qb & 0x78787878u) + 0x7F7F7F7Fu) | qb) & 0x80808080u;
            const uint32_t u8 = candidate_mask(na, nb);
            const uint32_t ka = ((qa >> 2) & 0x01010101u) * 0x01020408u >> 24;
            const uint32_t kb = ((qb >> 2) & 0x01010101u) * 0x01020408u >> 24;
            const uint32_t k8 = ((ka & 0xFu) | ((kb & 0xFu) << 4)) & u8;
            U |= u8 << (8 * rr);
            K |= k8 << (8 * rr);
        }
        // Work list: pair j of row rr when one of its pixels is not settled.
        uint32_t im = 0u;
#pragma unroll
        for (int rr = 0; rr < kHalf; ++rr)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if ((U >> (8 * rr + 2 * j)) & 3u) im |= 1u << (4 * rr + j);
        if (!__any_sync(0xffffffffu, im != 0u)) continue;
        int total;
        int pos = warp_excl_scan(lane, __popc(im), &total);
        while (im) {
            const int b = __ffs(im) - 1;
            im &= im - 1u;
            const int rr = b >> 2, j = b & 3;
            const uint32_t fl = ((U >> (8 * rr + 2 * j)) & 3u) | (((K >> (8 * rr + 2 * j)) & 3u) << 2);
            items[pos++] = (uint16_t)((h * kHalf + rr) | (lane << 3) | (j << 8) | (fl << 10));
        }
        __syncwarp();
        // Stage two (beta 3): the ring at distance 2 for every item; an item
        // whose pixels are all settled by then leaves the list, the others
        // are compacted (in place) and stage three counts their ring at
        // distance 3.  fl: bits 0-1 the pair's unsettled pixels, bits 2-3
        // those with one closed neighbour so far.
        int total2 = 0;
        for (int base = 0; base < total; base += 32) {
            const int i = base + lane;
            uint32_t e = 0u, keep = 0u;
            if (i < total) {
                e = items[i];
                const int y = ys + (int)(e & 7u);
                const int xw = ws - 4 * lane + 4 * (int)((e >> 3) & 31u) + (int)((e >> 8) & 3u);
                const uint32_t fl = e >> 10;
                const __half2 cpair = __hadd2(u2h(c.in[y * G::SWW + xw]), __float2half2_rn(0.5f));
                const uint32_t z = ring_count<2, G::SWW>(c.in, y, xw, cpair, two_a) * 47u;
                const uint32_t blo = (z >> 8) & 0xFFu, bhi = z >> 24;  // 4 K (+ 0..2), K <= 16
                uint32_t fl2 = 0u;
                // Still at most one closed neighbour: stays; K so far = 1 when either count had one.
                if ((fl & 1u) && blo < (((fl >> 2) & 1u) ? 4u : 8u)) fl2 |= 1u | ((((fl >> 2) & 1u) | (blo >= 4u ? 1u : 0u)) << 2);
                if ((fl & 2u) && bhi < (((fl >> 3) & 1u) ? 4u : 8u)) fl2 |= 2u | ((((fl >> 3) & 1u) | (bhi >= 4u ? 1u : 0u)) << 3);
                if (fl2) keep = (e & 0x3FFu) | (fl2 << 10);
            }
            __syncwarp();  // every lane has read its item before the compacted ones are written
            const unsigned bal = __ballot_sync(0xffffffffu, keep != 0u);
            if (keep) items[total2 + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)keep;
            total2 += __popc(bal);
        }
        __syncwarp();
        // Stage three.
        for (int base = 0; base < total2; base += 32) {
            const int i = base + lane;
            uint32_t cb = 0u;  // bit h: pixel 2 xw + h is a candidate
            int q0 = 0;
            if (i < total2) {
                const uint32_t e = items[i];
                const int y = ys + (int)(e & 7u);
                const int xw = ws - 4 * lane + 4 * (int)((e >> 3) & 31u) + (int)((e >> 8) & 3u);
                const uint32_t fl = e >> 10;
                const __half2 cpair = __hadd2(u2h(c.in[y * G::SWW + xw]), __float2half2_rn(0.5f));
                const uint32_t z = ring_count<3, G::SWW>(c.in, y, xw, cpair, two_a) * 47u;
                const uint32_t blo = (z >> 8) & 0xFFu, bhi = z >> 24;  // 4 K_outer (+ 0..2)
                // At most one closed neighbour in all.
                if ((fl & 1u) && blo < (((fl >> 2) & 1u) ? 4u : 8u)) cb |= 1u;
                if ((fl & 2u) && bhi < (((fl >> 3) & 1u) ? 4u : 8u)) cb |= 2u;
                q0 = y * G::SW + 2 * xw;
            }
            // Append the candidates (one shared counter update per warp).
            if (__any_sync(0xffffffffu, cb != 0u)) {
                int tot2;
                const int off = warp_excl_scan(lane, __popc(cb), &tot2);
                if (c.ncand + tot2 > G::kCandLimit) flush_candidates<B, T, RN>(c, lane);
                int o = c.ncand + off;
                if (cb & 1u) c.cand[o++] = (uint16_t)q0;
                if (cb & 2u) c.cand[o++] = (uint16_t)(q0 + 1);
                c.ncand += tot2;
            }
        }
        __syncwarp();
    }
}

// List pass: only pixels within beta of a pixel that changed in the
// previous pass can change now.  Each (changed pixel, window offset) pair
// claims its pixel in the mark bitmap; the claimer evaluates it exactly
// (Algorithm 2) from `in` and writes it to `out`.
template <int B, int T, int RN>
__device__ __forceinline__ void list_pass(PassCtx<B, T, RN>& c, const uint16_t* prev, const int nprev, uint32_t* mark,
                                          const int tid) {
    using G = FusedGeo<B, T, RN>;
    const __half* hin = reinterpret_cast<const __half*>(c.in);
    __half* hout = reinterpret_cast<__half*>(c.out);
    const int npairs = nprev * G::P;
    for (int i = tid; i < npairs; i += G::kThreads) {
        const int e = i / G::P;
        const int o = i - e * G::P;
        const int dy = o / (2 * B + 1) - B, dx = o % (2 * B + 1) - B;
        const int p = prev[e];
        const int py = p / G::SW;
        const int y = py + dy, x = p - py * G::SW + dx;
        if (y < G::R0 || y >= G::R0 + G::RN || x < G::C0 || x >= G::C0 + G::CN) continue;
        const int q = y * G::SW + x;
        const uint32_t bit = 1u << (q & 31);
        if (atomicOr(&mark[q >> 5], bit) & bit) continue;  // someone else evaluates q
        if (in_core_px(y, x, G::H, G::TH, G::TW)) ++c.evals;
        const __half old = hin[q];
        __half nv = old;
        if (interior(c, y, x)) {
            const int v = exact_packed<B, G::SW>(c.in, q, __half2half2(__hadd(old, __float2half(0.5f))), c.na);
            if (v >= 0) nv = u8_to_half(v);
        }
        hout[q] = nv;
        if (__half_as_ushort(nv) != __half_as_ushort(old)) {
            const int pos = atomicAdd(c.nlist, 1);
            if (pos < G::kListCap) c.list[pos] = (uint16_t)q;
            if (in_core_px(y, x, G::H, G::TH, G::TW)) c.changed_core = true;
        }
    }
}

// ---- Tile loads by TMA --------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* m) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32addr(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Thread 0: announce `bytes` of transfer on the mbarrier and start the tile
// load (box origin: byte 0, 16-byte chunk `chunk`, row `row` of the map; a
// box partly outside the tensor reads zeros there).
__device__ __forceinline__ void tma_tile_load(void* dst, const CUtensorMap* map, int chunk, int row, uint64_t* m,
                                              unsigned bytes) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
    // The staging buffer's previous contents were read by ordinary loads.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32addr(m)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32addr(dst)),
        "l"(map), "r"(0), "r"(chunk), "r"(row), "r"(smem_u32addr(m))
        : "memory");
}
// Bounded wait for phase `parity` of the mbarrier (every thread).
__device__ __forceinline__ bool mbar_wait(uint64_t* m, unsigned parity) {
    for (unsigned spins = 0; spins < (1u << 22); ++spins) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(smem_u32addr(m)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Persistent: each CTA takes tiles from a queue (one counter per launch in
// the control block) until none are left, so a launch whose work is done, or
// that the hybrid schedule skips, costs one short wave.  With tensor maps,
// thread 0 takes the next tile from the queue as soon as the current one is
// in shared memory and starts its TMA load into the staging buffer, so the
// load runs while the current tile computes.
template <int B, int T, int RN>
__global__ void __launch_bounds__(FusedGeo<B, T, RN>::kThreads, FusedGeo<B, T, RN>::kMinBlocks)
fused_kernel(PassArgs a) {
    using G = FusedGeo<B, T, RN>;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int s_np, s_tile, s_staged;
    __shared__ unsigned s_cur, s_aux, s_launch, s_k, s_img, s_nclr, s_nin;
    __shared__ ImgDesc s_d;
    __shared__ const uint8_t* s_user;
    __shared__ __align__(8) uint64_t s_mbar;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    Ctrl* ctrl = a.ctrl;
    if (tid == 0) {
        int np = launch_passes(ctrl, T);
        // Every launch that did work before this one was a fused launch.
        const unsigned L = __ldcg(&ctrl->work_launches);
        if (a.hybrid && L > 0 && __ldcg(&ctrl->dense) == 0u) np = 0;  // few changes left: the list passes take over
        s_np = np;
        s_cur = __ldcg(&ctrl->cur);
        s_aux = __ldcg(&ctrl->aux);
        s_launch = L;
        s_k = __ldcg(&ctrl->k);
        s_nclr = a.hybrid ? __ldcg(&ctrl->list_n[(L + 2) & 3]) : 0u;
        s_nin = a.hybrid ? __ldcg(&ctrl->list_n[(L + 3) & 3]) : 0u;
    }
    __syncthreads();
    const int np = s_np;
    if (np == 0) return;
    const unsigned L = s_launch;
    const unsigned cur = s_cur, aux = s_aux, third = 3u - s_cur - s_aux;
    uint32_t* buf0 = reinterpret_cast<uint32_t*>(smem);
    uint32_t* buf1 = reinterpret_cast<uint32_t*>(smem + G::kBufBytes);
    uint16_t* cand = reinterpret_cast<uint16_t*>(smem + G::kCandOff) + warp * G::kCandCap;
    uint16_t* lists = reinterpret_cast<uint16_t*>(smem + G::kListOff);  // 2 lists: pass t uses t & 1
    uint32_t* marks = reinterpret_cast<uint32_t*>(smem + G::kMarkOff);  // 2 bitmaps: pass t uses t & 1
    int* s_cnt = reinterpret_cast<int*>(smem + G::kCntOff);             // list counters, pass t uses t % 3
    // Single-image pixel change maps (fused-only schedule).
    const bool use_maps = a.chg_maps != nullptr;
    const size_t map_size = use_maps ? (size_t)a.rows * (size_t)a.map_words : 0;
    uint32_t* map_out = use_maps ? a.chg_maps + (size_t)(L % 3u) * map_size : nullptr;
    const uint32_t* map_in = use_maps ? a.chg_maps + (size_t)((L + 2u) % 3u) * map_size : nullptr;
    uint32_t* map_clr = use_maps ? a.chg_maps + (size_t)((L + 1u) % 3u) * map_size : nullptr;
    // Change sets of the hybrid schedule.
    const int set_out = (int)(L & 3u), set_in = (int)((L + 3u) & 3u), set_clr = (int)((L + 2u) & 3u);

    // Launch-wide clearing, shared by all CTAs: the map the next launch
    // writes, or the change set the next launch writes (its bitmap, by
    // walking its list, or all of it after an overflow).
    {
        const size_t gt = (size_t)gridDim.x * G::kThreads, gi = (size_t)blockIdx.x * G::kThreads + tid;
        for (size_t i = gi; i < map_size; i += gt) map_clr[i] = 0u;  // map_size is 0 without maps
        if (a.hybrid) {
            uint32_t* bm = a.bitmaps[set_clr];
            const unsigned nclr = s_nclr;
            if (nclr <= a.list_cap) {
                const uint32_t* lst = a.lists[set_clr];
                for (size_t i = gi; i < nclr; i += gt) {
                    unsigned im;
                    int y, x;
                    unpack_entry(__ldcg(lst + i), a.xb, a.yb, im, y, x);
                    const ImgDesc d = load_desc(a.imgs, im);
                    bm[d.bm_off + (long long)y * d.bm_words + (x >> 5)] = 0u;
                }
            } else {
                for (size_t i = gi; i < (size_t)a.bm_total; i += gt) bm[i] = 0u;
            }
        }
    }

    unsigned cta_mask = 0;          // passes that changed a core pixel of any of this CTA's tiles
    unsigned long long dense_px = 0;  // thread 0: core pixels of the dense passes
    const __half2 two_a = __float2half2_rn(2.f * (float)a.alpha);
    const int ys = G::R0 + warp * G::kRows;
    const int ws = G::C0 / 2 + 4 * lane;
    PassCtx<B, T, RN> c;
    c.cand = cand;
    c.ncand = 0;
    c.alpha = a.alpha;
    c.na = __float2half2_rn(-(float)a.alpha);
    c.evals = 0;
    unsigned* queue = &ctrl->tile_next[L & 1u];
    const int eval_max = a.tile_eval_max > 0 ? a.tile_eval_max : G::kListEvalMax;
    uint8_t* stage = smem + G::kStageOff;
    // Thread 0: take the next tile from the queue, publish its image and
    // source, and start its TMA load into the staging buffer when a tensor
    // map covers it (s_staged).
    auto take_next = [&]() {
        const int t = (int)atomicAdd(queue, 1u);
        s_tile = t;
        s_staged = 0;
        if (t >= a.ntiles) return;
        // The tile's image: from the image table, else the single image
        // described by the arguments.
        ImgDesc d;
        unsigned img = 0;
        if (a.imgs) {
            img = (unsigned)__ldg(a.tile_img + t);
            d = load_desc(a.imgs, img);
        } else {
            d.off = 0;
            d.bm_off = 0;
            d.pitch = (int)a.pitch;
            d.rows = a.rows;
            d.cols = a.cols;
            d.tiles_x = a.tiles_x;
            d.tile0 = 0;
            d.bm_words = a.bm_words;
            d.user = nullptr;
        }
        s_d = d;
        s_img = img;
        // The first launch of the hybrid schedule reads the caller's image.
        const uint8_t* user = (a.hybrid && L == 0) ? (a.nimg > 1 ? d.user : a.user0) : nullptr;
        s_user = user;
        if constexpr (G::kTma) {
            if (a.tmaps && (!user || a.tma_user) && (smem_u32addr(stage) & 127u) == 0) {
                const int tile = t - d.tile0;
                const int x0 = (tile % d.tiles_x) * G::TW, y0 = (tile / d.tiles_x) * G::TH;
                // Box origin: canvas column x0 (image column x0 - 16) and the
                // first halo row; in the caller's image, the same pixels.
                const CUtensorMap* map = a.tmaps + (size_t)img * kTmaMapsPerImage + (user ? 3u : cur);
                tma_tile_load(stage, map, user ? x0 / 16 - 1 : x0 / 16, user ? y0 - G::H : kPadY + y0 - G::H,
                              &s_mbar, (unsigned)(G::SH * G::SW));
                s_staged = 1;
            }
        }
    };
    if (tid == 0) {
        if constexpr (G::kTma) {
            if (a.tmaps) mbar_init(&s_mbar);
        }
        take_next();
    }
    __syncthreads();
    unsigned tma_waits = 0;  // TMA loads waited for (the mbarrier's phase)
    for (;;) {
        if (s_tile >= a.ntiles) break;
        const unsigned img = s_img;
        const long long pitch = s_d.pitch, coff = s_d.off, bm_off = s_d.bm_off;
        const int rows = s_d.rows, cols = s_d.cols, bm_words = s_d.bm_words;
        const uint8_t* src = a.canvas[cur] + coff;
        uint8_t* dst = a.canvas[aux] + coff;
        const int tile = s_tile - s_d.tile0;
        const int tx = tile % s_d.tiles_x;
        const int ty = tile / s_d.tiles_x;
        const int x0 = tx * G::TW, y0 = ty * G::TH;
        const bool staged = s_staged != 0;
        const uint8_t* user = s_user;

        // Tile with halo: image rows [y0 - H, y0 + TH + H), columns [x0 - 16,
        // x0 + TW + 16); always inside the canvas.  Bytes -> fp16 pairs, into
        // both buffers (a list pass leaves unevaluated pixels as they are in
        // its output buffer, so that buffer must start equal to the input).
        bool tma_failed = false;
        {
            const uint8_t* base = src + (long long)(kPadY + y0 - G::H) * pitch + x0;
            constexpr int CH = G::SW / 16;
            auto load_chunk = [&](int i) -> uint4 {
                const int r = i / CH, cc = i - r * CH;
                return user ? load_user_chunk(user, rows, cols, y0 - G::H + r, x0 - kPadX + cc * 16)
                            : __ldg(reinterpret_cast<const uint4*>(base + (long long)r * pitch + cc * 16));
            };
            auto store_chunk = [&](int i, const uint4 v) {
                const int r = i / CH, cc = i - r * CH;
                uint4 lo, hi;
                lo.x = bytes_to_h2(v.x, 0x4140u); lo.y = bytes_to_h2(v.x, 0x4342u);
                lo.z = bytes_to_h2(v.y, 0x4140u); lo.w = bytes_to_h2(v.y, 0x4342u);
                hi.x = bytes_to_h2(v.z, 0x4140u); hi.y = bytes_to_h2(v.z, 0x4342u);
                hi.z = bytes_to_h2(v.w, 0x4140u); hi.w = bytes_to_h2(v.w, 0x4342u);
                uint4* d0 = reinterpret_cast<uint4*>(buf0 + r * G::SWW + cc * 8);
                uint4* d1 = reinterpret_cast<uint4*>(buf1 + r * G::SWW + cc * 8);
                d0[0] = lo;
                d0[1] = hi;
                d1[0] = lo;
                d1[1] = hi;
            };
            if (staged) {
                // The TMA load started when the previous tile was set up
                // (SH rows of SW bytes, dense).  A wait that gives up records
                // the error, waits once more for the load to land and stops
                // this CTA's work.
                if (!mbar_wait(&s_mbar, tma_waits & 1u)) {
                    tma_failed = true;
                    if (tid == 0) atomicExch(&ctrl->error, 1u);
                    mbar_wait(&s_mbar, tma_waits & 1u);
                }
                ++tma_waits;
                for (int i = tid; i < G::SH * CH; i += G::kThreads)
                    store_chunk(i, *reinterpret_cast<const uint4*>(stage + i * 16));
            } else if constexpr (B >= 2) {
                // beta >= 2 (4-5 chunks per thread): every chunk of this
                // thread is loaded before any is converted, so that the
                // loads are in flight together (measured faster; for beta 1,
                // 2-3 chunks per thread, the plain loop is).
                constexpr int kIt = (G::SH * CH + G::kThreads - 1) / G::kThreads;
                uint4 vv[kIt];
#pragma unroll
                for (int it = 0; it < kIt; ++it) {
                    const int i = tid + it * G::kThreads;
                    if (i < G::SH * CH) vv[it] = load_chunk(i);
                }
#pragma unroll
                for (int it = 0; it < kIt; ++it) {
                    const int i = tid + it * G::kThreads;
                    if (i < G::SH * CH) store_chunk(i, vv[it]);
                }
            } else {
                for (int i = tid; i < G::SH * CH; i += G::kThreads) store_chunk(i, load_chunk(i));
            }
            for (int i = tid; i < 2 * G::kMarkWords; i += G::kThreads) marks[i] = 0u;
            if (tid < 8) s_cnt[tid] = 0;
        }
        if (__syncthreads_or(tma_failed)) break;
        // The staging buffer is free again: start the next tile's load.  (Every
        // thread has copied this tile's description into registers above.)
        if (tid == 0) take_next();
        // Pass 0's "previous pass": the pixels the previous launch's last
        // pass changed (its map or change bitmap), listed in list 1 / counter
        // 2.  A change set that overflowed lacks some of its bits: pass 0 is
        // then a dense pass.
        const bool from_map = L > 0 && (use_maps || (a.hybrid && s_nin <= a.list_cap));
        if (from_map) {
            const uint32_t* mp = use_maps ? map_in : a.bitmaps[set_in] + bm_off;
            const int mw = use_maps ? a.map_words : bm_words;
            const int wlo = (x0 - kPadX) >> 5;  // floor division (x0 - 16 >= -16)
            const int nw = ((x0 + G::TW + kPadX - 1) >> 5) - wlo + 1;
            for (int i = tid; i < G::SH * nw; i += G::kThreads) {
                const int y = i / nw, w = wlo + (i - y * nw);
                const int gy = y0 - G::H + y;
                if (gy < 0 || gy >= rows || w < 0 || w >= mw) continue;
                uint32_t bits = __ldcg(mp + (size_t)gy * mw + w);
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int x = 32 * w + b - x0 + kPadX;
                    if (x < 0 || x >= G::SW) continue;
                    const int pos = atomicAdd(&s_cnt[2], 1);
                    if (pos < G::kListCap) lists[G::kListCap + pos] = (uint16_t)(y * G::SW + x);
                }
            }
            __syncthreads();
        }

        unsigned tile_mask = 0;
        c.x0 = x0;
        c.y0 = y0;
        c.rows = rows;
        c.cols = cols;
        c.ylo = B + G::H - y0;           // gy = y0 + y - H >= B
        c.yhi = rows - B + G::H - y0;    // gy < rows - B
        c.xlo = B + kPadX - x0;          // gx = x0 + x - kPadX >= B
        c.xhi = cols - B + kPadX - x0;   // gx < cols - B
        c.all_interior = c.ylo <= G::R0 && c.yhi >= G::R0 + G::RN && c.xlo <= G::C0 && c.xhi >= G::C0 + G::CN;
        int dense_passes = 0;
        for (int t = 0; t < np; ++t) {
            c.in = (t & 1) ? buf1 : buf0;
            c.out = (t & 1) ? buf0 : buf1;
            c.list = lists + (t & 1) * G::kListCap;
            c.nlist = &s_cnt[t % 3];
            const uint16_t* prev = lists + ((t + 1) & 1) * G::kListCap;
            const int nprev = s_cnt[(t + 2) % 3];
            c.changed_core = false;
            // Counter (t + 1) % 3 was last read at the start of pass t - 1;
            // bitmap (t + 1) & 1 was last used in pass t - 1.
            if (tid == 0) s_cnt[(t + 1) % 3] = 0;
            uint32_t* mark_next = marks + ((t + 1) & 1) * G::kMarkWords;
            for (int i = tid; i < G::kMarkWords; i += G::kThreads) mark_next[i] = 0u;
            const bool dense = (t == 0 && !from_map) || nprev > G::kListCap || nprev * G::P > eval_max;
            if (dense) {
                ++dense_passes;
                if constexpr (G::kStaged)
                    band_dense2<B, T, RN>(c, ys, ws, lane, two_a);
                else if constexpr (B <= 2)
                    band_dense_sym<B, T, RN>(c, ys, ws, lane);
                else
                    band_dense<B, T, RN>(c, ys, ws, lane, two_a);
                flush_candidates<B, T, RN>(c, lane);
            } else {
                list_pass<B, T, RN>(c, prev, nprev, marks + (t & 1) * G::kMarkWords, tid);
            }
            if (__syncthreads_or(c.changed_core)) tile_mask |= 1u << t;
        }
        const uint32_t* fin = (np & 1) ? buf1 : buf0;  // I_np
        const uint32_t* pen = (np & 1) ? buf0 : buf1;  // I_(np-1) (the loaded tile when np == 1)

        // Core -> canvas bytes (and I_(np-1) -> the third canvas when asked).
        {
            const long long off = (long long)(kPadY + y0) * pitch + kPadX + x0;
            uint8_t* base = dst + off;
            uint8_t* base_prev = a.canvas[third] + coff + off;
            constexpr int CH = G::TW / 16;
            for (int i = tid; i < G::TH * CH; i += G::kThreads) {
                const int r = i / CH, cc = i - r * CH;
                const int so = (G::H + r) * G::SWW + kPadX / 2 + cc * 8;
                const uint4* s = reinterpret_cast<const uint4*>(fin + so);
                const uint4 p = s[0], q = s[1];
                uint4 o;
                o.x = h2_to_bytes(p.x, p.y);
                o.y = h2_to_bytes(p.z, p.w);
                o.z = h2_to_bytes(q.x, q.y);
                o.w = h2_to_bytes(q.z, q.w);
                *reinterpret_cast<uint4*>(base + (long long)r * pitch + cc * 16) = o;
                if (a.write_prev) {
                    const uint4* s2 = reinterpret_cast<const uint4*>(pen + so);
                    const uint4 p2 = s2[0], q2 = s2[1];
                    o.x = h2_to_bytes(p2.x, p2.y);
                    o.y = h2_to_bytes(p2.z, p2.w);
                    o.z = h2_to_bytes(q2.x, q2.y);
                    o.w = h2_to_bytes(q2.z, q2.w);
                    *reinterpret_cast<uint4*>(base_prev + (long long)r * pitch + cc * 16) = o;
                }
            }
        }
        const int nlast = s_cnt[(np - 1) % 3];
        const uint16_t* last = lists + ((np - 1) & 1) * G::kListCap;
        // The last pass's changed core pixels -> this launch's change set
        // (one global atomic per tile); an overflowed tile list marks the
        // set as overflowed, so the next pass evaluates every pixel.
        if (a.hybrid) {
            uint32_t* glist = a.lists[set_out];
            unsigned* gn = &ctrl->list_n[set_out];
            uint32_t* gbm = a.bitmaps[set_out];
            int* s_sel = s_cnt + 4;  // [0]: core entries, [1]: global base
            if (nlast <= G::kListCap) {
                // Compact the core entries to the front of `cand` (free now).
                uint32_t* sel = reinterpret_cast<uint32_t*>(smem + G::kCandOff);
                for (int i = tid; i < nlast; i += G::kThreads) {
                    const int q = last[i];
                    const int y = q / G::SW, x = q - y * G::SW;
                    const int gy = y0 + y - G::H, gx = x0 + x - kPadX;
                    if (in_core_px(y, x, G::H, G::TH, G::TW) && gy < rows && gx < cols) {
                        sel[atomicAdd(&s_sel[0], 1)] = pack_entry(img, gy, gx, a.xb, a.yb);
                        atomicOr(gbm + bm_off + (size_t)gy * bm_words + (gx >> 5), 1u << (gx & 31));
                    }
                }
                __syncthreads();
                const int nsel = s_sel[0];
                if (tid == 0) s_sel[1] = nsel ? (int)atomicAdd(gn, (unsigned)nsel) : 0;
                __syncthreads();
                const unsigned gbase = (unsigned)s_sel[1];
                for (int i = tid; i < nsel; i += G::kThreads)
                    if (gbase + i < a.list_cap) glist[gbase + i] = sel[i];
            } else if (tid == 0) {
                atomicAdd(gn, a.list_cap + 1u);  // overflow: the next pass evaluates every pixel
            }
        }
        // The last pass's changed core pixels -> this launch's map (all core
        // pixels when the list overflowed: a superset is always safe).
        if (use_maps) {
            if (nlast <= G::kListCap) {
                for (int i = tid; i < nlast; i += G::kThreads) {
                    const int q = last[i];
                    const int y = q / G::SW, x = q - y * G::SW;
                    if (!in_core_px(y, x, G::H, G::TH, G::TW)) continue;
                    const int gy = y0 + y - G::H, gx = x0 + x - kPadX;
                    if (gy >= rows || gx >= cols) continue;
                    atomicOr(map_out + (size_t)gy * a.map_words + (gx >> 5), 1u << (gx & 31));
                }
            } else {
                for (int r = tid; r < G::TH; r += G::kThreads) {
                    const int gy = y0 + r;
                    if (gy >= rows) break;
                    uint32_t* row = map_out + (size_t)gy * a.map_words;
                    for (int gx = x0; gx < x0 + G::TW; gx += 32 - (gx & 31)) {
                        const int n = min(32 - (gx & 31), x0 + G::TW - gx);
                        const uint32_t m = (n == 32 ? 0xffffffffu : ((1u << n) - 1u)) << (gx & 31);
                        atomicOr(row + (gx >> 5), m);
                    }
                }
            }
        }
        if (tid == 0) {
            // Dense passes evaluate every core pixel on the image.
            const int ch = min(G::TH, rows - y0), cw = min(G::TW, cols - x0);
            dense_px += (unsigned long long)dense_passes * (unsigned long long)(ch * cw);
            // Image k: the image changed in passes 1 .. (highest set bit).
            if (a.img_k && tile_mask) atomicMax(a.img_k + img, s_k + 32u - (unsigned)__clz(tile_mask));
        }
        cta_mask |= tile_mask;
        __syncthreads();  // the next tile reuses shared memory
    }
    // Work accounting (one global atomic per CTA).
    {
        __shared__ unsigned long long s_ev;
        if (tid == 0) s_ev = dense_px;
        __syncthreads();
        const unsigned ev = __reduce_add_sync(0xffffffffu, c.evals);
        if (lane == 0 && ev) atomicAdd(&s_ev, (unsigned long long)ev);
        __syncthreads();
        if (tid == 0 && s_ev) atomicAdd(&ctrl->evals_fused, s_ev);
    }
    if (tid == 0) {
        const bool last_cta = finish_launch(ctrl, cta_mask, np, gridDim.x, aux, a.write_prev ? third : cur);
        if (last_cta) {
            ctrl->fused_work += 1u;
            ctrl->tile_next[(L + 1u) & 1u] = 0u;  // the queue of the next fused launch
            if (a.hybrid) {
                ctrl->list_n[set_clr] = 0u;  // cleared above; every CTA has read its count
                // Would a list pass evaluate more than relaunch_evals pixels?
                const unsigned long long nout = ctrl->list_n[set_out];
                ctrl->dense = (nout > a.list_cap || nout * (unsigned long long)G::P > (unsigned long long)a.relaunch_evals)
                                  ? 1u : 0u;
            }
            __threadfence();
        }
    }
}

// Host-side description of one compiled (beta, T, tile rows) instance.
struct FusedEntry {
    int beta, T, TH, TW;
    int RN;    // rows computed per pass (64, or 128 for the tall tiles of large images)
    int SH;    // tile rows with the halo (the TMA box height)
    bool tma;  // the kernel stages tiles by TMA when given tensor maps
    size_t smem;
    cudaError_t (*launch)(const PassArgs&, int ctas, cudaStream_t);  // one CTA per tile
};

template <int B, int T, int RN>
cudaError_t launch_fused(const PassArgs& a, int ctas, cudaStream_t s) {
    using G = FusedGeo<B, T, RN>;
    // Per device: resident CTAs per SM and SM count (set up on first use).
    constexpr int kMaxDev = 64;
    static int occ[kMaxDev] = {};
    static int sms[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    if (occ[dev] == 0) {
        e = cudaFuncSetAttribute(fused_kernel<B, T, RN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::kSmem);
        int n = 0, o = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fused_kernel<B, T, RN>, G::kThreads, G::kSmem);
        if (e != cudaSuccess) return e;
        if (o < 1) return cudaErrorInvalidConfiguration;
        sms[dev] = n;
        occ[dev] = o;
    }
    const long long cap = (long long)sms[dev] * occ[dev];
    const unsigned grid = (unsigned)(ctas < cap ? (ctas > 0 ? ctas : 1) : cap);
    fused_kernel<B, T, RN><<<grid, G::kThreads, G::kSmem, s>>>(a);
    return cudaGetLastError();
}

template <int B, int T, int RN = 64>
constexpr FusedEntry fused_entry() {
    using G = FusedGeo<B, T, RN>;
    return FusedEntry{B, T, G::TH, G::TW, RN, G::SH, G::kTma, G::kSmem, &launch_fused<B, T, RN>};
}

}  // namespace hg
