/*
 * CPU oracle for the P-HGRMS salt-and-pepper denoiser (TEST INFRASTRUCTURE).
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this code.  The CUDA library never links, includes or calls it;
 * the two implementations share no source.
 *
 * It is plain, slow, single-threaded C written from the paper:
 *   - Algorithm 1 (findIsolatedPixels): the cardinality matrix C, one count
 *     per pixel of the alpha-similar pixels in its beta window.
 *   - Algorithm 2 (removeNoise): for a pixel with C <= 2, count the "open"
 *     neighbours (flag) and the sum of their squares; if flag exceeds
 *     pix_count - 3, the pixel becomes the root mean square of those
 *     neighbours in a temporary image I'.
 *   - Section 2: I' starts as a copy of I, is copied back after every pass, and
 *     passes repeat until no noise remains, the count of passes being capped
 *     by the iteration factor k.
 *
 * Two forms are given.  hgo_literal_* follow the printed algorithms step by
 * step (C built by scattered increments into the neighbour, Algorithm 1;
 * Algorithm 2 over that matrix; explicit copy-back).  hgo_pass/hgo_denoise use
 * the gather form of Algorithm 1 (each pixel counts its own similar
 * neighbours), which equals the scatter form because both the window and the
 * |difference| < alpha test are symmetric.  The tests pin one against the
 * other.
 *
 * Readings of passages that are ambiguous or garbled in the paper:
 *   window   rows r-beta .. r+beta and columns c-beta .. c+beta inclusive, a
 *            (2 beta + 1)^2 window (Algorithm 2 bounds its loops with "<
 *            i+beta+1"; Algorithm 1's "to r+beta+1" is read the same way).
 *   card     C[n] += 1 for each in-image neighbour n of p with
 *            I[p]-alpha < I[n] < I[p]+alpha; every count is exact (the
 *            printed update is garbled and unsynchronised; a lost update is
 *            a race, not part of the method).  C is zeroed before each pass.
 *   open     n is open for p when NOT (I[n] < I[p]+alpha+1 and
 *            I[n] > I[p]-alpha), compared in int (no uint8 wrap-around).
 *   pix_count counts every window position, on or off the image.
 *   replace  flag > pix_count - 3 (strict), value floor(sqrt(floor(sum/flag)))
 *            in integers: the paper's pseudo-code prints sum/flag but the
 *            method is a root mean square (title, Section 2 prose).
 *   I'       pixels that are not replaced keep their value (I' = I at the
 *            start of each pass, because of the copy-back).
 *   stop     after the first pass that changes no pixel (a fixed point;
 *            later passes would change nothing), or once max_k passes that
 *            changed pixels have run.  k = number of passes that changed at
 *            least one pixel.  With max_k = 5 this is the paper's fixed k = 5.
 *
 * Images are uint8, row-major, I[r*cols + c].
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define HGO_EXPORT __attribute__((visibility("default")))

/* floor(sqrt(x)) by bisection on r with r*r <= x (exact for any uint32). */
HGO_EXPORT uint32_t hgo_isqrt(uint32_t x)
{
    uint64_t lo = 0, hi = 65536; /* invariant: lo*lo <= x < hi*hi */
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) / 2;
        if (mid * mid <= (uint64_t)x) lo = mid; else hi = mid;
    }
    return (uint32_t)lo;
}

static int in_image(long i, long j, int rows, int cols)
{
    return i >= 0 && i < rows && j >= 0 && j < cols;
}

/* ---------------------------------------------------------------------- */
/* Literal form of Algorithm 1: every pixel p adds one to the count of each   */
/* in-image window neighbour n that is alpha-similar to it.  card is zeroed   */
/* first.                                                                     */
HGO_EXPORT void hgo_literal_find_isolated(const uint8_t* image, int32_t* card,
                                          int rows, int cols, int alpha, int beta)
{
    memset(card, 0, sizeof(int32_t) * (size_t)rows * (size_t)cols);
    for (long r = 0; r < rows; ++r)
        for (long c = 0; c < cols; ++c) {
            int ip = image[r * cols + c];
            for (long i = r - beta; i < r + beta + 1; ++i)
                for (long j = c - beta; j < c + beta + 1; ++j)
                    if (i < rows && i >= 0 && j < cols && j >= 0) {
                        int in = image[i * cols + j];
                        if (in < ip + alpha && in > ip - alpha)
                            card[i * cols + j] += 1;
                    }
        }
}

/* Literal form of Algorithm 2 over a cardinality matrix.  temp must hold a  */
/* copy of image on entry (the copy-back of Section 2); only replaced pixels */
/* are written.  Returns the number of pixels whose value changed.           */
HGO_EXPORT long hgo_literal_remove_noise(const uint8_t* image, uint8_t* temp,
                                         const int32_t* card, int rows, int cols,
                                         int alpha, int beta)
{
    long changed = 0;
    for (long i = 0; i < rows; ++i)
        for (long j = 0; j < cols; ++j) {
            long sum = 0;
            int pix_count = 0;
            int flag = 0;
            int ip = image[i * cols + j];
            if (card[i * cols + j] <= 2) {
                for (long i1 = i - beta; i1 < i + beta + 1; ++i1)
                    for (long j1 = j - beta; j1 < j + beta + 1; ++j1) {
                        pix_count = pix_count + 1;
                        if (i1 < rows && i1 >= 0 && j1 < cols && j1 >= 0) {
                            int in = image[i1 * cols + j1];
                            if (!(in < ip + alpha + 1 && in > ip - alpha)) {
                                sum = sum + (long)in * in;
                                flag = flag + 1;
                            }
                        }
                    }
                if (flag > pix_count - 3) {
                    uint8_t v = (uint8_t)hgo_isqrt((uint32_t)(sum / flag));
                    if (v != image[i * cols + j]) ++changed;
                    temp[i * cols + j] = v;
                }
            }
        }
    return changed;
}

/* Literal driver: Algorithm 1, Algorithm 2 into I', copy I' back to I,      */
/* repeated; same stopping rule and return value as hgo_denoise.             */
HGO_EXPORT int hgo_literal_denoise(uint8_t* image, int rows, int cols, int alpha,
                                   int beta, int max_k, int* converged)
{
    size_t n = (size_t)rows * (size_t)cols;
    int32_t* card = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
    uint8_t* temp = (uint8_t*)malloc(n ? n : 1);
    int k = 0, conv = 0;
    if (!card || !temp) { free(card); free(temp); return -1; }
    while (k < max_k) {
        hgo_literal_find_isolated(image, card, rows, cols, alpha, beta);
        memcpy(temp, image, n);
        long changed = hgo_literal_remove_noise(image, temp, card, rows, cols,
                                                alpha, beta);
        memcpy(image, temp, n);
        if (changed == 0) { conv = 1; break; }
        ++k;
    }
    if (converged) *converged = conv;
    free(card);
    free(temp);
    return k;
}

/* ---------------------------------------------------------------------- */
/* Gather form of Algorithm 1 for one pixel: the number of in-image window   */
/* positions n with |I[n] - I[p]| < alpha (p itself included).               */
static int card_of(const uint8_t* in, int rows, int cols, long r, long c,
                   int alpha, int beta)
{
    int ip = in[r * cols + c];
    int card = 0;
    for (long i = r - beta; i <= r + beta; ++i)
        for (long j = c - beta; j <= c + beta; ++j)
            if (in_image(i, j, rows, cols)) {
                int d = (int)in[i * cols + j] - ip;
                if (d < alpha && d > -alpha) ++card;
            }
    return card;
}

HGO_EXPORT void hgo_card(const uint8_t* in, int32_t* card, int rows, int cols,
                         int alpha, int beta)
{
    for (long r = 0; r < rows; ++r)
        for (long c = 0; c < cols; ++c)
            card[r * cols + c] = card_of(in, rows, cols, r, c, alpha, beta);
}

/* One pass (Algorithm 1 in gather form, then Algorithm 2) from in to out    */
/* (in != out).  Returns the number of pixels with out != in.                */
HGO_EXPORT long hgo_pass(const uint8_t* in, uint8_t* out, int rows, int cols,
                         int alpha, int beta)
{
    long changed = 0;
    for (long r = 0; r < rows; ++r)
        for (long c = 0; c < cols; ++c) {
            int ip = in[r * cols + c];
            out[r * cols + c] = (uint8_t)ip;
            if (card_of(in, rows, cols, r, c, alpha, beta) > 2) continue;
            long sum = 0;
            int flag = 0, pix_count = 0;
            for (long i = r - beta; i <= r + beta; ++i)
                for (long j = c - beta; j <= c + beta; ++j) {
                    ++pix_count; /* off-image positions are counted too */
                    if (!in_image(i, j, rows, cols)) continue;
                    int v = in[i * cols + j];
                    int closed = (v < ip + alpha + 1) && (v > ip - alpha);
                    if (!closed) {
                        sum += (long)v * v;
                        ++flag;
                    }
                }
            if (flag > pix_count - 3) {
                out[r * cols + c] = (uint8_t)hgo_isqrt((uint32_t)(sum / flag));
                if (out[r * cols + c] != ip) ++changed;
            }
        }
    return changed;
}

/* Iterate passes in place on image.  Returns k (passes that changed at     */
/* least one pixel, at most max_k), or -1 if memory runs out.  *converged   */
/* is 1 when the loop ended on a pass that changed nothing.  If changes_out */
/* is not NULL it receives the changed-pixel count of every pass run (at     */
/* most max_k + 1 entries).                                                 */
HGO_EXPORT int hgo_denoise(uint8_t* image, int rows, int cols, int alpha,
                           int beta, int max_k, int* converged, long* changes_out)
{
    size_t n = (size_t)rows * (size_t)cols;
    uint8_t* other = (uint8_t*)malloc(n ? n : 1);
    uint8_t *src = image, *dst = other;
    int k = 0, conv = 0, npass = 0;
    if (!other) return -1;
    while (k < max_k) {
        long changed = hgo_pass(src, dst, rows, cols, alpha, beta);
        if (changes_out) changes_out[npass] = changed;
        ++npass;
        if (changed == 0) { conv = 1; break; }
        ++k;
        uint8_t* t = src; src = dst; dst = t;
    }
    if (src != image) memcpy(image, src, n);
    if (converged) *converged = conv;
    free(other);
    return k;
}

/* Peak signal-to-noise ratio in dB of b against reference a (8-bit peak).  */
/* Returns INFINITY when the images are identical.                          */
HGO_EXPORT double hgo_psnr(const uint8_t* a, const uint8_t* b, long n)
{
    double se = 0.0;
    for (long i = 0; i < n; ++i) {
        double d = (double)a[i] - (double)b[i];
        se += d * d;
    }
    if (se == 0.0) return INFINITY;
    double mse = se / (double)n;
    return 10.0 * log10(255.0 * 255.0 / mse);
}
