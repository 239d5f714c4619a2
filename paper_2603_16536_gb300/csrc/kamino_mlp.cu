// Learned warm start for PADMM: a small MLP per world type maps the state, the actuation and the
// contact geometry of a world to initial constraint impulses (the warm start of Alg. 1,
// Sec. 4.1, written into the state's external warm-start buffer).  The network has L hidden
// layers of width H with GELU, BF16 weights and activations, FP32 accumulation; it is trained on
// the GPU by the kernels below (forward, backward, Adam) on impulses the solver itself converged.
//
// GEMMs use the warp-level tensor-core instruction mma.sync m16n8k16 (BF16 in, FP32 accumulate):
// the layers are at most a few hundred wide, so one 64x64 CTA tile per output block with fused
// epilogues (bias, GELU, GELU derivative) is enough; the step kernel is where the time goes.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kamino_device.cuh"
#include "kamino_internal.h"
#include "kamino_mlp.h"

namespace kamino {
namespace mlp {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, GEMM_THREADS = 128, PAD = 8;

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// C(m, n) = sum_k A(m, k) B(k, n) with A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn]
// (BF16), then the epilogue.  64 x 64 tile per CTA, 4 warps of 32 x 32.
__global__ void __launch_bounds__(GEMM_THREADS) gemm_kernel(const GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        for (int q = 0; q < (BM * BK) / GEMM_THREADS; ++q) {
            const int idx = tid + GEMM_THREADS * q;
            int m, k;
            if (g.sak == 1) { k = idx % BK; m = idx / BK; } else { m = idx % BM; k = idx / BM; }
            const int gm = m0 + m, gk = k0 + k;
            As[m][k] = (gm < g.M && gk < g.K) ? g.A[(long)gm * g.sam + (long)gk * g.sak] : zero;
        }
        for (int q = 0; q < (BN * BK) / GEMM_THREADS; ++q) {
            const int idx = tid + GEMM_THREADS * q;
            int n, k;
            if (g.sbn == 1) { n = idx % BN; k = idx / BN; } else { k = idx % BK; n = idx / BK; }
            const int gn = n0 + n, gk = k0 + k;
            Bs[n][k] = (gn < g.N && gk < g.K) ? g.B[(long)gk * g.sbk + (long)gn * g.sbn] : zero;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int r = wm + 16 * a + gq;
                af[a][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * tq]);
                af[a][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * tq]);
                af[a][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * tq + 8]);
                af[a][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int cn = wn + 8 * b + gq;
                bf[b][0] = *reinterpret_cast<const uint32_t *>(&Bs[cn][kk + 2 * tq]);
                bf[b][1] = *reinterpret_cast<const uint32_t *>(&Bs[cn][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) mma16816(acc[a][b], af[a], bf[b]);
        }
        __syncthreads();
    }
    // epilogue: c0, c1 at (row gq, cols 2 tq, 2 tq + 1); c2, c3 at row gq + 8
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + wm + 16 * a + gq + (c >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * b + 2 * tq + (c & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[a][b][c];
                switch (g.epi) {
                    case EPI_F32:
                        g.Cf[(long)m * g.ldcf + n] = v;
                        break;
                    case EPI_BIAS_F32:
                        g.Cf[(long)m * g.ldcf + n] = v + g.bias[n];
                        break;
                    case EPI_BIAS_GELU: {
                        const float z = v + g.bias[n];
                        if (g.Cf) g.Cf[(long)m * g.ldcf + n] = z;
                        g.Cb[(long)m * g.ldcb + n] = __float2bfloat16(gelu(z));
                        break;
                    }
                    case EPI_GELU_BWD: {
                        const float dz = v * gelu_grad(g.Zin[(long)m * g.ldz + n]);
                        g.Cf[(long)m * g.ldcf + n] = dz;
                        g.Cb[(long)m * g.ldcb + n] = __float2bfloat16(dz);
                        break;
                    }
                }
            }
}

// Column sums of an FP32 matrix [rows][cols] (bias gradients): one warp per column.
__global__ void colsum_kernel(const float *X, int rows, int cols, long ld, float *out) {
    const int col = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (col >= cols) return;
    float s = 0.0f;
    for (int r = lane; r < rows; r += 32) s += X[(long)r * ld + col];
    s = dev::warp_sum(s);
    if (lane == 0) out[col] = s;
}

// Gather rows of the raw feature matrix, normalise them and round to BF16.
__global__ void normalize_rows_kernel(const float *Xraw, int dim, const int *rows, int batch, const float *mean,
                                      const float *inv_std, __nv_bfloat16 *out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)batch * dim) return;
    const int b = (int)(e / dim), f = (int)(e - (long)b * dim);
    const long r = rows ? rows[b] : b;
    out[e] = __float2bfloat16((Xraw[r * dim + f] - mean[f]) * inv_std[f]);
}

// Normalised targets, squared error and dL/dy = 2 (y - t) / (batch * dout) as BF16.
__global__ void loss_grad_kernel(const float *Y, const float *Traw, int dout, const int *rows, int batch,
                                 const float *ymean, const float *yinv, __nv_bfloat16 *dY, float *dYf, float *loss) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    float sq = 0.0f;
    if (e < (long)batch * dout) {
        const int b = (int)(e / dout), o = (int)(e - (long)b * dout);
        const long r = rows ? rows[b] : b;
        const float t = (Traw[r * dout + o] - ymean[o]) * yinv[o];
        const float d = Y[e] - t;
        const float scale = 2.0f / ((float)batch * (float)dout);
        dY[e] = __float2bfloat16(d * scale);
        dYf[e] = d * scale;
        sq = d * d / ((float)batch * (float)dout);
    }
    sq = dev::warp_sum(sq);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, sq);
}

// Adam on FP32 master parameters; refreshes the BF16 copies of the weight matrices.
__global__ void adam_kernel(float *p, const float *gr, float *m1, float *m2, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16 *pb, const unsigned char *is_weight) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gv = gr[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gv;
    const float v = b2 * m2[i] + (1.0f - b2) * gv * gv;
    m1[i] = a;
    m2[i] = v;
    const float np = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    p[i] = np;
    if (is_weight[i]) pb[i] = __float2bfloat16(np);
}

__global__ void to_bf16_kernel(const float *p, __nv_bfloat16 *pb, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16(p[i]);
}

// Column mean and 1/std over `rows` rows (two passes, FP64 sums); std floored at 1e-6.
__global__ void colstats_kernel(const float *X, long rows, int cols, float *mean, float *inv_std) {
    const int col = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (col >= cols) return;
    double s = 0.0;
    for (long r = lane; r < rows; r += 32) s += X[r * cols + col];
    s = dev::warp_sum(s);
    const double mu = s / (double)rows;
    double q = 0.0;
    for (long r = lane; r < rows; r += 32) {
        const double d = X[r * cols + col] - mu;
        q += d * d;
    }
    q = dev::warp_sum(q);
    if (lane == 0) {
        const double sd = sqrt(q / (double)rows);
        mean[col] = (float)mu;
        inv_std[col] = (float)(1.0 / (sd > 1e-6 ? sd : 1e-6));
    }
}

// Features of one world: per body (r - r_root, q, v, w) [13], root height [1], actuation
// [n_act], per contact candidate (signed distance, terrain normal) [4].
template <typename T>
__global__ void features_kernel(const FeatureArgs<T> a) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)a.count * a.din) return;
    const int wi = (int)(e / a.din), f = (int)(e - (long)wi * a.din);
    const int w = a.worlds[wi];
    const int4 wa = a.m.world_a[w], wb = a.m.world_b[w];
    const int b0 = wa.x, c0 = wa.z, nb = wb.x, nc = wb.z;
    float v = 0.0f;
    if (f < 13 * nb) {
        const int b = f / 13, k = f - 13 * (f / 13);
        if (k < 3) v = (float)(a.q[7 * (long)(b0 + b) + k] - a.q[7 * (long)b0 + k]);
        else if (k < 7) v = (float)a.q[7 * (long)(b0 + b) + k];
        else v = (float)a.u[6 * (long)(b0 + b) + (k - 7)];
    } else if (f == 13 * nb) {
        v = (float)a.q[7 * (long)b0 + 2];
    } else if (f < 13 * nb + 1 + a.nact) {
        const int k = f - 13 * nb - 1;
        v = a.tau ? (float)a.tau[(long)w * a.m.n_act_max + k] : 0.0f;
    } else if (f < 13 * nb + 1 + a.nact + 4 * nc) {
        const int k = f - 13 * nb - 1 - a.nact;
        const int c = k / 4, comp = k - 4 * (k / 4);
        if (a.m.terrain_kind != KAMINO_TERRAIN_NONE) {
            const int body = a.m.contact_body[c0 + c];
            const T *qb = a.q + 7 * (long)(b0 + body);
            double R[9], p[3], n[3];
            double qq[4] = {(double)qb[3], (double)qb[4], (double)qb[5], (double)qb[6]};
            const double inv = 1.0 / sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
            for (int t = 0; t < 4; ++t) qq[t] *= inv;
            dev::quat_rot(qq, R);
            const double *cp = a.m.contact_point + 3 * (long)(c0 + c);
            dev::matvec3(R, cp, p);
            for (int t = 0; t < 3; ++t) p[t] += (double)qb[t];
            const double phi = dev::terrain(a.m, p, n);
            v = comp == 0 ? (float)phi : (float)n[comp - 1];
        }
    } else {
        const int k = f - 13 * nb - 1 - a.nact - 4 * nc;    // impulse cache, joint rows then candidates
        if (a.cache && k < a.dout) v = (float)a.cache[wa.w + k];
    }
    a.out[e] = v;
}

// Impulses of the converged step (the state's cache) as training targets.
template <typename T>
__global__ void targets_kernel(const int4 *world_a, const int *worlds, int count, int dout, const T *cache,
                               float *out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)count * dout) return;
    const int wi = (int)(e / dout), o = (int)(e - (long)wi * dout);
    out[e] = (float)cache[world_a[worlds[wi]].w + o];
}

// De-normalised network output [rows][dout].
__global__ void denormalize_kernel(const float *Y, int rows, int dout, const float *ymean, const float *yinv,
                                   float *out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)rows * dout) return;
    const int o = (int)(e % dout);
    out[e] = Y[e] / yinv[o] + ymean[o];
}

// De-normalised network output -> the state's external warm-start buffer (cache layout).
template <typename T>
__global__ void warm_write_kernel(const int4 *world_a, const int *worlds, int count, int dout, const float *Y,
                                  const float *ymean, const float *yinv, T *warm) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)count * dout) return;
    const int wi = (int)(e / dout), o = (int)(e - (long)wi * dout);
    warm[world_a[worlds[wi]].w + o] = (T)(Y[e] / yinv[o] + ymean[o]);
}

inline unsigned blocks(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t gemm(const GemmArgs &g, cudaStream_t s) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
    gemm_kernel<<<grid, GEMM_THREADS, 0, s>>>(g);
    return cudaGetLastError();
}
cudaError_t colsum(const float *X, int rows, int cols, long ld, float *out, cudaStream_t s) {
    colsum_kernel<<<blocks(cols, 8), 256, 0, s>>>(X, rows, cols, ld, out);
    return cudaGetLastError();
}
cudaError_t normalize_rows(const float *Xraw, int dim, const int *rows, int batch, const float *mean, const float *inv,
                           __nv_bfloat16 *out, cudaStream_t s) {
    normalize_rows_kernel<<<blocks((long)batch * dim, 256), 256, 0, s>>>(Xraw, dim, rows, batch, mean, inv, out);
    return cudaGetLastError();
}
cudaError_t loss_grad(const float *Y, const float *Traw, int dout, const int *rows, int batch, const float *ymean,
                      const float *yinv, __nv_bfloat16 *dY, float *dYf, float *loss, cudaStream_t s) {
    loss_grad_kernel<<<blocks((long)batch * dout, 256), 256, 0, s>>>(Y, Traw, dout, rows, batch, ymean, yinv, dY, dYf,
                                                                      loss);
    return cudaGetLastError();
}
cudaError_t adam(float *p, const float *gr, float *m1, float *m2, int n, float lr, float b1, float b2, float eps,
                 float c1, float c2, __nv_bfloat16 *pb, const unsigned char *is_weight, cudaStream_t s) {
    adam_kernel<<<blocks(n, 256), 256, 0, s>>>(p, gr, m1, m2, n, lr, b1, b2, eps, c1, c2, pb, is_weight);
    return cudaGetLastError();
}
cudaError_t denormalize(const float *Y, int rows, int dout, const float *ymean, const float *yinv, float *out,
                        cudaStream_t s) {
    denormalize_kernel<<<blocks((long)rows * dout, 256), 256, 0, s>>>(Y, rows, dout, ymean, yinv, out);
    return cudaGetLastError();
}
cudaError_t to_bf16(const float *p, __nv_bfloat16 *pb, int n, cudaStream_t s) {
    to_bf16_kernel<<<blocks(n, 256), 256, 0, s>>>(p, pb, n);
    return cudaGetLastError();
}
cudaError_t colstats(const float *X, long rows, int cols, float *mean, float *inv, cudaStream_t s) {
    colstats_kernel<<<blocks(cols, 8), 256, 0, s>>>(X, rows, cols, mean, inv);
    return cudaGetLastError();
}
template <typename T>
cudaError_t features(const FeatureArgs<T> &a, cudaStream_t s) {
    features_kernel<T><<<blocks((long)a.count * a.din, 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
template <typename T>
cudaError_t targets(const int4 *world_a, const int *worlds, int count, int dout, const T *cache, float *out,
                    cudaStream_t s) {
    targets_kernel<T><<<blocks((long)count * dout, 256), 256, 0, s>>>(world_a, worlds, count, dout, cache, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t warm_write(const int4 *world_a, const int *worlds, int count, int dout, const float *Y, const float *ymean,
                       const float *yinv, T *warm, cudaStream_t s) {
    warm_write_kernel<T><<<blocks((long)count * dout, 256), 256, 0, s>>>(world_a, worlds, count, dout, Y, ymean, yinv,
                                                                           warm);
    return cudaGetLastError();
}

template cudaError_t features<float>(const FeatureArgs<float> &, cudaStream_t);
template cudaError_t features<double>(const FeatureArgs<double> &, cudaStream_t);
template cudaError_t targets<float>(const int4 *, const int *, int, int, const float *, float *, cudaStream_t);
template cudaError_t targets<double>(const int4 *, const int *, int, int, const double *, float *, cudaStream_t);
template cudaError_t warm_write<float>(const int4 *, const int *, int, int, const float *, const float *,
                                       const float *, float *, cudaStream_t);
template cudaError_t warm_write<double>(const int4 *, const int *, int, int, const float *, const float *,
                                        const float *, double *, cudaStream_t);

}  // namespace mlp
}  // namespace kamino
