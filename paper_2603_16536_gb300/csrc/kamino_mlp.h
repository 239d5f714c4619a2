// Internal declarations of the warm-start MLP kernels (kamino_mlp.cu); not part of the ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kamino_internal.h"

namespace kamino {
namespace mlp {

enum { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_BIAS_F32 = 2, EPI_GELU_BWD = 3 };

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16 *A;
    long sam, sak;                 // A(m, k) = A[m sam + k sak]
    const __nv_bfloat16 *B;
    long sbk, sbn;                 // B(k, n) = B[k sbk + n sbn]
    int epi;
    const float *bias;             // [N]
    float *Cf;                     // FP32 output (pre-activation, output layer, gradient)
    long ldcf;
    __nv_bfloat16 *Cb;             // BF16 output (activation, back-propagated gradient)
    long ldcb;
    const float *Zin;              // pre-activation for EPI_GELU_BWD
    long ldz;
};

template <typename T>
struct FeatureArgs {
    ModelView<T> m;
    const T *q, *u, *tau;
    const T *cache;                // the state's impulse cache (the previous step's solution)
    const int *worlds;
    int count, din, nact, dout;
    float *out;                    // [count][din]
};

cudaError_t gemm(const GemmArgs &g, cudaStream_t s);
cudaError_t colsum(const float *X, int rows, int cols, long ld, float *out, cudaStream_t s);
cudaError_t normalize_rows(const float *Xraw, int dim, const int *rows, int batch, const float *mean,
                           const float *inv_std, __nv_bfloat16 *out, cudaStream_t s);
cudaError_t loss_grad(const float *Y, const float *Traw, int dout, const int *rows, int batch,
                      const float *ymean, const float *yinv, __nv_bfloat16 *dY, float *dYf, float *loss,
                      cudaStream_t s);
cudaError_t denormalize(const float *Y, int rows, int dout, const float *ymean, const float *yinv, float *out,
                        cudaStream_t s);
cudaError_t adam(float *p, const float *g, float *m1, float *m2, int n, float lr, float b1, float b2, float eps,
                 float c1, float c2, __nv_bfloat16 *pb, const unsigned char *is_weight, cudaStream_t s);
cudaError_t to_bf16(const float *p, __nv_bfloat16 *pb, int n, cudaStream_t s);
cudaError_t colstats(const float *X, long rows, int cols, float *mean, float *inv_std, cudaStream_t s);
template <typename T>
cudaError_t features(const FeatureArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t targets(const int4 *world_a, const int *worlds, int count, int dout, const T *cache, float *out,
                    cudaStream_t s);
template <typename T>
cudaError_t warm_write(const int4 *world_a, const int *worlds, int count, int dout, const float *Y,
                       const float *ymean, const float *yinv, T *warm, cudaStream_t s);

// Read-only view of a network's parameters and normalisation (defined with the network's host code).
struct NetView {
    int din, dout, hidden, layers, max_batch;
    int device;                     // the device that holds the network's arrays
    const float *P;                 // FP32 master parameters
    const __nv_bfloat16 *PB;        // BF16 copy of the weight matrices (same offsets)
    long woff[8], boff[8];          // per layer offsets of W_l and b_l
    const float *xmean, *xinv, *ymean, *yinv;
};
bool net_view(const struct kamino_mlp_s *net, NetView *out);

}  // namespace mlp

// Sets the calling thread's kamino_last_error message and returns `s`.
kamino_status report_error(kamino_status s, const char *msg);

}  // namespace kamino
