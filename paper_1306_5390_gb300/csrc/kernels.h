// Internal declarations shared by the runtime and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace hg {

struct FusedEntry;
extern const FusedEntry kFusedB1[];
extern const int kFusedB1Count;
extern const FusedEntry kFusedB2[];
extern const int kFusedB2Count;
extern const FusedEntry kFusedB3[];
extern const int kFusedB3Count;

// Compiled fused kernel for (beta, passes per launch, rows computed per
// pass), or null; the built-in passes per launch for beta.
const FusedEntry* find_fused(int beta, int T, int rn = 64);
int default_passes(int beta);

cudaError_t launch_plain(int beta, const PassArgs& a, cudaStream_t s);
cudaError_t launch_ctrl_init(Ctrl* c, unsigned max_k, cudaStream_t s);
cudaError_t launch_copy_in(const uint8_t* img, int rows, int cols, uint8_t* canvas, long long pitch,
                           int sms, cudaStream_t s);
cudaError_t launch_copy_out(const Ctrl* c, uint8_t* const canvas[3], long long pitch, uint8_t* img, int rows,
                            int cols, int sms, cudaStream_t s);
cudaError_t launch_list(int beta, const PassArgs& a, int sms, cudaStream_t s);
// Batched forms (image table on the device; max_words = the largest image's
// rows * cols / 4, rounded up, sizes the grid).
cudaError_t launch_copy_out_batch(const Ctrl* c, uint8_t* const arena[3], const ImgDesc* imgs, int nimg,
                                  long long max_words, int sms, cudaStream_t s);
cudaError_t launch_tile_map(const ImgDesc* imgs, int nimg, int total_tiles, int* tile_img, cudaStream_t s);
// out[i] = floor(sqrt(floor(sum[i] / flag[i]))) by the kernels' integer root mean square (rms_div).
cudaError_t launch_rms(const int* sum, const int* flag, int* out, int n, cudaStream_t s);

}  // namespace hg

struct hgrms_ctx;
namespace hg {
// Run the handle's list-pass launches on `coop`, a stream shared by handles
// whose work overlaps (null: the handle's own stream).
int set_coop_stream(hgrms_ctx* h, cudaStream_t coop);

// Learned k-predictor (predictor.cu).
struct Predictor;
Predictor* predictor_new();
void predictor_free(Predictor* p);
int predictor_load(Predictor* p, const float* weights, int n);
int predictor_run(Predictor* p, const ImgDesc* imgs, int n, cudaStream_t s, float* k_hat, float* x0_host,
                  float* hist_host, float* gap_host);
int predictor_grad(const float* weights, const float* x0, const float* hist, const float* k, int n, float* grads,
                   float* loss, cudaStream_t s);
int predictor_train(float* weights, const float* x0, const float* hist, const float* k, int n, int epochs, int batch,
                    float lr, unsigned long long seed, float* loss_out, cudaStream_t s);

}  // namespace hg
