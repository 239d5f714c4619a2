// Small device helpers shared by the step kernel and the warm-start kernels: 3-vector and
// rotation algebra, warp reductions, the contact-frame basis and the terrain query.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "kamino_internal.h"

namespace kamino {
namespace dev {

// ----------------------------------------------------------------------------- small math
template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void cross3(const T *a, const T *b, T *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename T>
__device__ __forceinline__ T dot3(const T *a, const T *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// rotation matrix (row-major) of the unit quaternion (x, y, z, w)
template <typename T>
__device__ __forceinline__ void quat_rot(const T *q, T *R) {
    const T x = q[0], y = q[1], z = q[2], w = q[3];
    R[0] = T(1) - T(2) * (y * y + z * z); R[1] = T(2) * (x * y - z * w); R[2] = T(2) * (x * z + y * w);
    R[3] = T(2) * (x * y + z * w); R[4] = T(1) - T(2) * (x * x + z * z); R[5] = T(2) * (y * z - x * w);
    R[6] = T(2) * (x * z - y * w); R[7] = T(2) * (y * z + x * w); R[8] = T(1) - T(2) * (x * x + y * y);
}
template <typename T>
__device__ __forceinline__ void matvec3(const T *R, const T *v, T *o) {
    o[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    o[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    o[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}
template <typename T>
__device__ __forceinline__ void matTvec3(const T *R, const T *v, T *o) {
    o[0] = R[0] * v[0] + R[3] * v[1] + R[6] * v[2];
    o[1] = R[1] * v[0] + R[4] * v[1] + R[7] * v[2];
    o[2] = R[2] * v[0] + R[5] * v[1] + R[8] * v[2];
}
template <typename T>
__device__ __forceinline__ void matmul3(const T *A, const T *B, T *C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}
// symmetric 3x3 stored (xx, yy, zz, xy, xz, yz) times v
template <typename T>
__device__ __forceinline__ void symvec3(const T *S, const T *v, T *o) {
    o[0] = S[0] * v[0] + S[3] * v[1] + S[4] * v[2];
    o[1] = S[3] * v[0] + S[1] * v[1] + S[5] * v[2];
    o[2] = S[4] * v[0] + S[5] * v[1] + S[2] * v[2];
}

// the same product with the vector and the result in FP64 (S in any precision)
template <typename T>
__device__ __forceinline__ void symvec3d(const T *S, const double *v, double *o) {
    const double s0 = S[0], s1 = S[1], s2 = S[2], s3 = S[3], s4 = S[4], s5 = S[5];
    o[0] = s0 * v[0] + s3 * v[1] + s4 * v[2];
    o[1] = s3 * v[0] + s1 * v[1] + s5 * v[2];
    o[2] = s4 * v[0] + s5 * v[1] + s2 * v[2];
}

// Pose advanced along a twist for a time h (Sec. 3, FP64): r + h v and exp(h w) (x) q, with w in
// the world frame (hence the left product) and the result renormalised.  q = (r[3], quat xyzw[4]).
__device__ __forceinline__ void pose_advance(const double *q, const double *v, const double *w, double h,
                                             double *out) {
    const double th[3] = {h * w[0], h * w[1], h * w[2]};
    const double ang = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
    double dq[4];
    if (ang > 0.0) {
        const double s = sin(0.5 * ang) / ang;
        dq[0] = s * th[0]; dq[1] = s * th[1]; dq[2] = s * th[2]; dq[3] = cos(0.5 * ang);
    } else {
        dq[0] = dq[1] = dq[2] = 0.0; dq[3] = 1.0;
    }
    const double qx = q[3], qy = q[4], qz = q[5], qw = q[6];
    const double qn[4] = {dq[3] * qx + dq[0] * qw + dq[1] * qz - dq[2] * qy,
                          dq[3] * qy - dq[0] * qz + dq[1] * qw + dq[2] * qx,
                          dq[3] * qz + dq[0] * qy - dq[1] * qx + dq[2] * qw,
                          dq[3] * qw - dq[0] * qx - dq[1] * qy - dq[2] * qz};
    const double nrm = 1.0 / sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    for (int k = 0; k < 3; ++k) out[k] = q[k] + h * v[k];
    for (int k = 0; k < 4; ++k) out[3 + k] = qn[k] * nrm;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Duff et al. 2017 branchless orthonormal basis: (t1, t2, n) right-handed
template <typename T>
__device__ __forceinline__ void onb(const T *n, T *t1, T *t2) {
    const T sign = n[2] >= T(0) ? T(1) : T(-1);
    const T a = T(-1) / (sign + n[2]);
    const T b = n[0] * n[1] * a;
    t1[0] = T(1) + sign * n[0] * n[0] * a; t1[1] = sign * b; t1[2] = -sign * n[0];
    t2[0] = b; t2[1] = sign + n[1] * n[1] * a; t2[2] = -n[1];
}

// Signed distance of p to the terrain and the terrain normal there (FP64).  Plane: z = 0.
// Heightfield: cells split along the (i, j)-(i+1, j+1) diagonal; (x, y) clamped into the grid.
template <typename T>
__device__ __forceinline__ double terrain(const ModelView<T> &m, const double *p, double *n) {
    if (m.terrain_kind == KAMINO_TERRAIN_PLANE) {
        n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
        return p[2];
    }
    const double h = m.hf_cell;
    double gx = (p[0] - m.hf_x0) / h, gy = (p[1] - m.hf_y0) / h;
    gx = fmin(fmax(gx, 0.0), (double)(m.hf_nx - 1));
    gy = fmin(fmax(gy, 0.0), (double)(m.hf_ny - 1));
    const int i = min((int)floor(gx), m.hf_nx - 2);
    const int j = min((int)floor(gy), m.hf_ny - 2);
    const double fx = gx - i, fy = gy - j;
    const double *H = m.hf_heights;
    const double h00 = H[j * m.hf_nx + i], h11 = H[(j + 1) * m.hf_nx + i + 1];
    double e1[3], e2[3];
    if (fx >= fy) {   // vertices (i,j), (i+1,j), (i+1,j+1)
        const double h10 = H[j * m.hf_nx + i + 1];
        e1[0] = h; e1[1] = 0.0; e1[2] = h10 - h00;
        e2[0] = h; e2[1] = h; e2[2] = h11 - h00;
    } else {          // vertices (i,j), (i+1,j+1), (i,j+1)
        const double h01 = H[(j + 1) * m.hf_nx + i];
        e1[0] = h; e1[1] = h; e1[2] = h11 - h00;
        e2[0] = 0.0; e2[1] = h; e2[2] = h01 - h00;
    }
    cross3(e1, e2, n);
    const double inv = 1.0 / sqrt(dot3(n, n));
    n[0] *= inv; n[1] *= inv; n[2] *= inv;
    const double q[3] = {(gx - i) * h, (gy - j) * h, p[2] - h00};
    return dot3(q, n);
}

}  // namespace dev
}  // namespace kamino
