// Fused per-world constrained forward-dynamics step for sm_103a (Kamino, arXiv 2603.16536).
//
// One CTA (256 threads) owns one world for the whole step and keeps its working set on chip
// (shared memory, and for worlds of up to 256 padded rows the matrix in tensor memory); nothing
// but the state, the inputs and the impulse cache touches HBM.
//
//   1  body kinematics: R(q), world inverse inertia, M^-1 (Sec. 3, Eq. 1)
//   2  joint rows (incl. loop closures) with Baumgarte bias; actuation as J_d^T tau (Sec. 3)
//   3  contacts against the terrain, compacted in candidate order, rows (t1, t2, n) (Sec. 3)
//   4  u_free = u + dt M^-1 h (gyroscopic + gravity + actuation); v_f = J u_free + v* (Eq. 4)
//   5  D = J M^-1 J^T from the two 1x6 blocks of every row (block-sparse), Jacobi scaling
//      P = diag(D)^-1/2 with a shared tangential scale per contact (Sec. 4.1), packed lower
//      storage of A = P D P + (eta + rho) I
//   6  warm start (cached or external impulses)                          (Sec. 4.1)
//   7  regularised factorisation, computed once per step (Sec. 4: A is constant across the
//      iterations).  The paper factorises with block-Cholesky and runs a backward-forward
//      pass every iteration; here A^-1 is formed once by a blocked symmetric sweep
//      (Gauss-Jordan on the SPD matrix, panels of NB columns, rank-NB updates on the tensor
//      cores in the mixed mode), so every iteration's solve is one fully parallel matrix-vector
//      product instead of two length-m dependency chains, made exact by one refinement step
//      against the matrix-free residual (the fixed point is that of the exact solve).
//   8  Proximal-ADMM (Alg. 1): De Saxce correction, solve, cone projection, dual update,
//      Nesterov with adaptive restart, infinity-norm residuals, early exit
//   9  lambda = P y; u+ = u_free + M^-1 J^T lambda; r+ = r + dt v+, q+ = exp(dt w+) q (Sec. 3);
//      impulse cache (warm start of the next step) and the per-world report.
//
// Every loop is bounded (N_max iterations at most); there are no inter-CTA waits.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kamino_device.cuh"
#include "kamino_internal.h"

namespace kamino {
namespace {
using namespace dev;

// A group of `size` threads (a multiple of 32) that owns one world.  `bar` is the named barrier it
// synchronises on: 0 with size == blockDim.x is the CTA barrier; groups inside a CTA use ids 1..8.
struct Group {
    int tid, size, bar;
    __device__ __forceinline__ int lane() const { return tid & 31; }
    __device__ __forceinline__ int warp() const { return tid >> 5; }
    __device__ __forceinline__ int warps() const { return size >> 5; }
    __device__ __forceinline__ void sync() const {
        if (size == 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(size) : "memory");
    }
};

// packed lower-triangular, column-major storage of a symmetric mp x mp matrix
__device__ __forceinline__ int col_start(int j, int mp) { return j * mp - (j * (j - 1)) / 2; }
__device__ __forceinline__ int pidx(int i, int j, int mp) {  // requires i >= j
    return col_start(j, mp) + (i - j);
}
__device__ __forceinline__ int sidx(int i, int j, int mp) { return i >= j ? pidx(i, j, mp) : pidx(j, i, mp); }

template <typename T>
__device__ __forceinline__ void put_row(int *rbody, T *rJ, double *rvs, int row, int ba, int bb, const double *Ja,
                                        const double *Jb, double vstar) {
    rbody[2 * row] = ba;
    rbody[2 * row + 1] = bb;
    T *J = rJ + 12 * row;
    for (int k = 0; k < 6; ++k) { J[k] = T(Ja[k]); J[6 + k] = T(Jb[k]); }
    rvs[row] = vstar;
}

// Joint rows of one joint (Sec. 3): positional rows along world axes, angular rows along the
// parent frame's axes; returns the actuation wrench (J_d^T value) for parent and child.  All
// position-level quantities (anchors, frame axes, errors f) are formed in FP64 from the stored
// pose, then J and the bias are rounded to T.
template <typename T>
__device__ void joint_rows(int type, int par, int ch, const double *fr, const double *bq, const double *bRd, int row0,
                           double kbias, int *rbody, T *rJ, double *rvs, bool actuated, T value, T *wr) {
    double rA[3] = {0.0, 0.0, 0.0}, RA[9] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0};
    if (par >= 0) {
        for (int k = 0; k < 3; ++k) rA[k] = bq[7 * par + k];
        for (int k = 0; k < 9; ++k) RA[k] = bRd[9 * par + k];
    }
    const double rB[3] = {bq[7 * ch], bq[7 * ch + 1], bq[7 * ch + 2]};
    const double *RB = bRd + 9 * ch;
    double cA[3], cB[3], pA[3], pB[3], QA[9], QB[9], FA[9], FB[9];
    matvec3(RA, fr, cA);
    matvec3(RB, fr + 7, cB);
    for (int k = 0; k < 3; ++k) { pA[k] = rA[k] + cA[k]; pB[k] = rB[k] + cB[k]; }
    quat_rot(fr + 3, QA);
    quat_rot(fr + 10, QB);
    matmul3(RA, QA, FA);
    matmul3(RB, QB, FB);
    double a[3][3], b[3][3];   // a[k] = k-th axis of the parent-side frame (column k)
    for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) { a[k][r] = FA[3 * r + k]; b[k][r] = FB[3 * r + k]; }
    const double dp[3] = {pB[0] - pA[0], pB[1] - pA[1], pB[2] - pA[2]};
    double Ja[6], Jb[6], t[3];
    int row = row0;
    const bool positional = (type == KAMINO_JOINT_REVOLUTE || type == KAMINO_JOINT_UNIVERSAL ||
                             type == KAMINO_JOINT_SPHERICAL || type == KAMINO_JOINT_FIXED);
    if (positional) {
        for (int k = 0; k < 3; ++k) {
            const double e[3] = {double(k == 0), double(k == 1), double(k == 2)};
            cross3(cA, e, t);
            Ja[0] = -e[0]; Ja[1] = -e[1]; Ja[2] = -e[2]; Ja[3] = -t[0]; Ja[4] = -t[1]; Ja[5] = -t[2];
            cross3(cB, e, t);
            Jb[0] = e[0]; Jb[1] = e[1]; Jb[2] = e[2]; Jb[3] = t[0]; Jb[4] = t[1]; Jb[5] = t[2];
            put_row(rbody, rJ, rvs, row++, par, ch, Ja, Jb, kbias * dp[k]);
        }
    }
    if (type == KAMINO_JOINT_REVOLUTE) {
        double err[3];
        cross3(a[2], b[2], err);
        for (int k = 0; k < 2; ++k) {
            for (int r = 0; r < 3; ++r) { Ja[r] = 0.0; Jb[r] = 0.0; Ja[3 + r] = -a[k][r]; Jb[3 + r] = a[k][r]; }
            put_row(rbody, rJ, rvs, row++, par, ch, Ja, Jb, kbias * dot3(a[k], err));
        }
    } else if (type == KAMINO_JOINT_PRISMATIC) {
        const double lever[3] = {pB[0] - rA[0], pB[1] - rA[1], pB[2] - rA[2]};
        for (int k = 0; k < 2; ++k) {
            cross3(lever, a[k], t);
            Ja[0] = -a[k][0]; Ja[1] = -a[k][1]; Ja[2] = -a[k][2]; Ja[3] = -t[0]; Ja[4] = -t[1]; Ja[5] = -t[2];
            cross3(cB, a[k], t);
            Jb[0] = a[k][0]; Jb[1] = a[k][1]; Jb[2] = a[k][2]; Jb[3] = t[0]; Jb[4] = t[1]; Jb[5] = t[2];
            put_row(rbody, rJ, rvs, row++, par, ch, Ja, Jb, kbias * dot3(a[k], dp));
        }
    }
    if (type == KAMINO_JOINT_PRISMATIC || type == KAMINO_JOINT_FIXED) {
        double err[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 3; ++i) {
            cross3(a[i], b[i], t);
            err[0] += 0.5 * t[0]; err[1] += 0.5 * t[1]; err[2] += 0.5 * t[2];
        }
        for (int k = 0; k < 3; ++k) {
            for (int r = 0; r < 3; ++r) { Ja[r] = 0.0; Jb[r] = 0.0; Ja[3 + r] = -a[k][r]; Jb[3 + r] = a[k][r]; }
            put_row(rbody, rJ, rvs, row++, par, ch, Ja, Jb, kbias * dot3(a[k], err));
        }
    }
    if (type == KAMINO_JOINT_UNIVERSAL) {
        double n[3];
        cross3(a[0], b[1], n);
        for (int r = 0; r < 3; ++r) { Ja[r] = 0.0; Jb[r] = 0.0; Ja[3 + r] = n[r]; Jb[3 + r] = -n[r]; }
        put_row(rbody, rJ, rvs, row++, par, ch, Ja, Jb, kbias * dot3(a[0], b[1]));
    }
    for (int k = 0; k < 12; ++k) wr[k] = T(0);
    if (actuated) {
        const double v = (double)value;
        if (type == KAMINO_JOINT_REVOLUTE) {
            for (int r = 0; r < 3; ++r) { wr[3 + r] = T(-v * a[2][r]); wr[9 + r] = T(v * a[2][r]); }
        } else if (type == KAMINO_JOINT_PRISMATIC) {
            const double lever[3] = {pB[0] - rA[0], pB[1] - rA[1], pB[2] - rA[2]};
            cross3(lever, a[2], t);
            for (int r = 0; r < 3; ++r) { wr[r] = T(-v * a[2][r]); wr[3 + r] = T(-v * t[r]); }
            cross3(cB, a[2], t);
            for (int r = 0; r < 3; ++r) { wr[6 + r] = T(v * a[2][r]); wr[9 + r] = T(v * t[r]); }
        }
    }
}

// The joint coordinate d(q) and its row J_d (J_d u = d-dot) of a revolute or prismatic joint
// (Sec. 3, the coordinate drives and limits act on), in FP64: for a revolute the angle of the child
// frame's e1 about the hinge a3, measured from a1 towards a2, d = atan2(a2.b1, a1.b1),
// J_d = [0, -a3 | 0, a3]; for a prismatic the slide d = a3.(p_B - p_A),
// J_d = [-a3, -(p_B - r_A) x a3 | a3, c_B x a3].
__device__ void joint_coordinate(int type, int par, int ch, const double *fr, const double *bq, const double *bRd,
                                 double *d, double *Ja, double *Jb) {
    double rA[3] = {0.0, 0.0, 0.0}, RA[9] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0};
    if (par >= 0) {
        for (int k = 0; k < 3; ++k) rA[k] = bq[7 * par + k];
        for (int k = 0; k < 9; ++k) RA[k] = bRd[9 * par + k];
    }
    const double *RB = bRd + 9 * ch;
    double QA[9], QB[9], FA[9], FB[9], cA[3], cB[3];
    quat_rot(fr + 3, QA);
    quat_rot(fr + 10, QB);
    matmul3(RA, QA, FA);
    matmul3(RB, QB, FB);
    const double a1[3] = {FA[0], FA[3], FA[6]}, a2[3] = {FA[1], FA[4], FA[7]}, a3[3] = {FA[2], FA[5], FA[8]};
    for (int k = 0; k < 6; ++k) { Ja[k] = 0.0; Jb[k] = 0.0; }
    if (type == KAMINO_JOINT_REVOLUTE) {
        const double b1[3] = {FB[0], FB[3], FB[6]};
        *d = atan2(dot3(a2, b1), dot3(a1, b1));
        for (int k = 0; k < 3; ++k) { Ja[3 + k] = -a3[k]; Jb[3 + k] = a3[k]; }
    } else {
        matvec3(RA, fr, cA);
        matvec3(RB, fr + 7, cB);
        double pA[3], pB[3], lev[3], t[3];
        for (int k = 0; k < 3; ++k) {
            pA[k] = rA[k] + cA[k];
            pB[k] = bq[7 * ch + k] + cB[k];
            lev[k] = pB[k] - rA[k];
        }
        const double dp[3] = {pB[0] - pA[0], pB[1] - pA[1], pB[2] - pA[2]};
        *d = dot3(a3, dp);
        cross3(lev, a3, t);
        for (int k = 0; k < 3; ++k) { Ja[k] = -a3[k]; Ja[3 + k] = -t[k]; }
        cross3(cB, a3, t);
        for (int k = 0; k < 3; ++k) { Jb[k] = a3[k]; Jb[3 + k] = t[k]; }
    }
}

// Group-wide reductions of (max, max, max, sum) of non-negative values; every thread gets the
// results.  The scratch is
// double-buffered by `phase` so consecutive calls need only the one barrier inside.
template <typename T>
__device__ __forceinline__ void group_reduce4(T &a, T &b, T &c, T &d, T *red, int phase, const Group &g) {
    const int lane = g.lane(), warp = g.warp(), nw = g.warps();
    if constexpr (sizeof(T) == 4) {
        // a, b, c are maxima of absolute values: as unsigned integers their bit patterns order like
        // the floats, so one redux.sync each
        a = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(a)));
        b = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(b)));
        c = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(c)));
    } else {
        a = warp_max(a); b = warp_max(b); c = warp_max(c);
    }
    d = warp_sum(d);
    T *r = red + phase * 4 * kWarps;
    if (lane == 0) { r[warp] = a; r[kWarps + warp] = b; r[2 * kWarps + warp] = c; r[3 * kWarps + warp] = d; }
    g.sync();
    a = r[0]; b = r[kWarps]; c = r[2 * kWarps]; d = r[3 * kWarps];
    for (int k = 1; k < nw; ++k) {
        a = fmax(a, r[k]); b = fmax(b, r[kWarps + k]); c = fmax(c, r[2 * kWarps + k]); d += r[3 * kWarps + k];
    }
}

// Six consecutive words at an 8-byte aligned shared-memory address (a row block of J, 12 r + 6 side,
// or a per-body 6-vector): three 8-byte loads in FP32.
template <typename T>
__device__ __forceinline__ void load6(const T *p, T (&v)[6]) {
    if constexpr (sizeof(T) == 4) {
        const float2 *q = reinterpret_cast<const float2 *>(p);
        const float2 a = q[0], b = q[1], c = q[2];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = p[k];
    }
}

// 16 consecutive values from a 16-byte aligned shared-memory address (vector loads).
__device__ __forceinline__ void load16(const float *p, float (&v)[16]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 t = q[k];
        v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    }
}
__device__ __forceinline__ void load16(const double *p, double (&v)[16]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double2 t = q[k];
        v[2 * k] = t.x; v[2 * k + 1] = t.y;
    }
}

// Sum over the 32 lanes of v[c], delivered to lane c (recursive halving: 16 + 8 + 4 + 2 + 1
// shuffles; at each level a lane keeps the half of its values whose index has its lane bit).
template <typename T>
__device__ __forceinline__ T transpose_reduce32(T (&v)[32], int lane) {
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const T send = up ? v[k] : v[k + h];
            const T keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

// y = S x for a symmetric S in packed lower column-major storage (mp x mp).  The lower triangle is
// cut into 32 x 32 tiles (I >= J) dealt round-robin to the warps of the group.  In a tile, lane l
// owns row 32I + l: every element S(i, j) is read once from shared memory (consecutive lanes read
// consecutive addresses) and used twice, for y_i += S_ij x_j in a register and for
// y_j += S_ij x_i in a per-column register that one transpose-reduction per tile sums over the
// lanes.  Per-warp partial rows (`partial`, [warps][mp]) are summed at the end, so the result does
// not depend on scheduling.
template <typename T>
__device__ void symv_packed(const T *S, int mp, const T *x, T *y, T *partial, const Group &g) {
    const int lane = g.lane(), warp = g.warp(), nw = g.warps();
    T *part = partial + warp * mp;
    for (int i = lane; i < mp; i += 32) part[i] = T(0);
    __syncwarp();
    const int nt = (mp + 31) >> 5;
    const int ntiles = nt * (nt + 1) / 2;
    for (int t = warp; t < ntiles; t += nw) {
        int I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (I * (I + 1) / 2 > t) --I;
        while ((I + 1) * (I + 2) / 2 <= t) ++I;
        const int J = t - I * (I + 1) / 2;
        const int i = 32 * I + lane;
        const bool rowok = i < mp;
        const T xi = rowok ? x[i] : T(0);
        T rowacc = T(0);
        T col[32];
        int j = 32 * J;
        int cs = col_start(j, mp) - j;     // S(i, j) = S[cs + i] for i >= j
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            T s = T(0), xj = T(0);
            if (j < mp) {
                xj = x[j];
                if (rowok && i >= j) s = S[cs + i];
                cs += mp - j - 1;
            }
            rowacc = fma(s, xj, rowacc);
            col[c] = i > j ? s * xi : T(0);
            ++j;
        }
        const T csum = transpose_reduce32(col, lane);
        if (rowok) part[i] += rowacc;
        __syncwarp();
        const int jc = 32 * J + lane;
        if (jc < mp) part[jc] += csum;
        __syncwarp();
    }
    g.sync();
    for (int i = g.tid; i < mp; i += g.size) {
        T acc = T(0);
        for (int w = 0; w < nw; ++w) acc += partial[w * mp + i];
        y[i] = acc;
    }
    g.sync();
}

// ----------------------------------------------------------------------------- BF16 tiles of S
// Mixed precision (KAMINO_MIXED).  After the sweep, S = -A^-1 is re-stored as BF16 16 x 16 tiles of its lower triangle (tile (I, J),
// I >= J, at index J nt - J (J - 1) / 2 + (I - J); diagonal tiles hold both triangles), in place at
// the start of the packed FP32 region: one column block at a time is staged in the X scratch
// (all of its FP32 words are read before any of its tiles is written, and a block's tiles end
// before the next block's FP32 words begin).  Inside a tile, row r is 32 bytes; its two 16-byte
// halves swap places when bit 2 of r is set, so the 8 row addresses of an ldmatrix phase fall on
// distinct banks.
__device__ __forceinline__ int tile_index(int I, int J, int nt) { return J * nt - (J * (J - 1)) / 2 + (I - J); }
__device__ __forceinline__ int tile_byte(int r, int c) { return r * 32 + (((c >> 3) ^ ((r >> 2) & 1)) << 4) + ((c & 7) << 1); }

template <typename T>
__device__ void pack_bf16_tiles(T *A, int mp, T *X, const Group &g) {
    const int nt = mp / 16;
    unsigned char *base = reinterpret_cast<unsigned char *>(A);
    for (int J = 0; J < nt; ++J) {
        const int j0 = 16 * J, rows = mp - j0;
        for (int e = g.tid; e < rows * 16; e += g.size) {
            const int i = j0 + e / 16, j = j0 + (e & 15);
            X[e] = A[sidx(i, j, mp)];
        }
        g.sync();
        for (int e = g.tid; e < rows * 16; e += g.size) {
            const int i = j0 + e / 16, c = e & 15;
            const int I = i >> 4;
            __nv_bfloat16 *dst = reinterpret_cast<__nv_bfloat16 *>(base + 512 * tile_index(I, J, nt) +
                                                                   tile_byte(i & 15, c));
            *dst = __float2bfloat16((float)X[e]);
        }
        g.sync();
    }
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&a)[4], const void *p) {
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&a)[4], const void *p) {
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]) : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// y = S c on tensor cores.  c comes split into c_hi = bf16(c) and c_lo = bf16(c - c_hi), which form
// columns 0 and 1 of the mma's B operand, so the vector keeps ~16 significant bits; S is BF16 and
// the products accumulate in FP32.  Warp w owns the output row blocks I = w, w + warps, ...; it
// runs two of them at a time (four independent accumulator chains, one B fragment per column
// block shared by both).  For J <= I it reads tile (I, J), for J > I the transpose of tile (J, I)
// (ldmatrix .trans), so each row block is one chain of mma without any cross-warp reduction.
template <typename T>
__device__ void apply_bf16_tiles(const T *A, int mp, const __nv_bfloat16 *chi, const __nv_bfloat16 *clo, T *y,
                                 const Group &g) {
    const unsigned char *base = reinterpret_cast<const unsigned char *>(A);
    const int nt = mp / 16, lane = g.lane(), gq = lane >> 2, tq = lane & 3, nw = g.warps();
    const int q = lane >> 3, rr = lane & 7;
    // per-lane row / 16-byte half inside a tile for the normal and the transposed loads
    const int rn = rr + 8 * (q & 1), hn = q >> 1;
    const int rt = rr + 8 * (q >> 1), ht = q & 1;
    const int offn = rn * 32 + ((hn ^ ((rn >> 2) & 1)) << 4);
    const int offt = rt * 32 + ((ht ^ ((rt >> 2) & 1)) << 4);
    const __nv_bfloat16 *vec = gq == 0 ? chi : clo;
    for (int I0 = g.warp(); I0 < nt; I0 += 2 * nw) {
        const int I1 = I0 + nw;
        const bool two = I1 < nt;
        float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
        float q0[4] = {0.f, 0.f, 0.f, 0.f}, q1[4] = {0.f, 0.f, 0.f, 0.f};
        for (int J = 0; J < nt; ++J) {
            const int k0 = 16 * J + 2 * tq;
            uint32_t b0 = 0u, b1 = 0u;
            if (gq < 2) {
                b0 = *reinterpret_cast<const uint32_t *>(vec + k0);
                b1 = *reinterpret_cast<const uint32_t *>(vec + k0 + 8);
            }
            uint32_t t0[4];
            if (J <= I0) ldsm_x4(t0, base + 512 * tile_index(I0, J, nt) + offn);
            else ldsm_x4_trans(t0, base + 512 * tile_index(J, I0, nt) + offt);
            if (two) {
                uint32_t t1[4];
                if (J <= I1) ldsm_x4(t1, base + 512 * tile_index(I1, J, nt) + offn);
                else ldsm_x4_trans(t1, base + 512 * tile_index(J, I1, nt) + offt);
                if (J & 1) mma_bf16(q1, t1, b0, b1);
                else mma_bf16(q0, t1, b0, b1);
            }
            if (J & 1) mma_bf16(p1, t0, b0, b1);
            else mma_bf16(p0, t0, b0, b1);
        }
        if (tq == 0) {
            y[16 * I0 + gq] = T((p0[0] + p0[1]) + (p1[0] + p1[1]));
            y[16 * I0 + gq + 8] = T((p0[2] + p0[3]) + (p1[2] + p1[3]));
            if (two) {
                y[16 * I1 + gq] = T((q0[0] + q0[1]) + (q1[0] + q1[1]));
                y[16 * I1 + gq + 8] = T((q0[2] + q0[3]) + (q1[2] + q1[3]));
            }
        }
    }
    g.sync();
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ----------------------------------------------------------------------------- tensor memory
// The swept inverse can live in tensor memory (TMEM, 512 columns x 128 lanes of 32 bits per SM)
// for the whole PADMM loop: row r of S = -A^-1 sits in lane r mod 128 of chunk r / 128, chunk ch at
// columns 256 ch ... 256 ch + mp - 1 (FP32, mp <= 256).  Warp w may only touch lanes
// 32 (w mod 4) ... + 31, so warps 0-3 own chunk 0 and warps 4-7 chunk 1; every warp reads back
// exactly the rows it wrote.  Used only by the one-world-per-CTA kernel when the world's shared
// memory keeps a second CTA off the SM, so the allocation never waits for another CTA.
constexpr int kTmemCols = 512;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t t, const uint32_t (&v)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(t), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
                    "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t t, uint32_t (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(t) : "memory");
}

// Rows of S (packed lower FP32 in shared memory) into tensor memory; zero beyond mp.
__device__ void tmem_store_inverse(const float *A, int mp, uint32_t tbase, const Group &g) {
    const int warp = g.warp(), lane = g.lane();
    const int ch = warp >> 2;
    const int row = 128 * ch + 32 * (warp & 3) + lane;
    if (128 * ch < mp) {
        const uint32_t t = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * ch);
        for (int j0 = 0; j0 < mp; j0 += 16) {
            uint32_t v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = __float_as_uint(row < mp ? A[sidx(row, j0 + q, mp)] : 0.0f);
            tmem_st16(t + (uint32_t)j0, v);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
}

// y = S c with S in tensor memory: lane = row, 32 columns per load, c broadcast from shared memory,
// four FP32 partial sums.
__device__ __forceinline__ void fma16(const uint32_t (&v)[16], const float *c, float &a0, float &a1, float &a2,
                                      float &a3) {
    const float4 *cp = reinterpret_cast<const float4 *>(c);
#pragma unroll
    for (int q = 0; q < 16; q += 4) {
        const float4 cc = cp[q / 4];
        a0 = fmaf(__uint_as_float(v[q]), cc.x, a0);
        a1 = fmaf(__uint_as_float(v[q + 1]), cc.y, a1);
        a2 = fmaf(__uint_as_float(v[q + 2]), cc.z, a2);
        a3 = fmaf(__uint_as_float(v[q + 3]), cc.w, a3);
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t t, uint32_t (&v)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(t) : "memory");
}

// Waits for this thread's outstanding tensor-memory loads; the registers of the block about to be
// used are tied to the wait, so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&v)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
                   "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]),
                   "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :: "memory");
}

// 32 columns of a row against c (broadcast float4 loads from shared memory), as packed FP32 FMAs on
// two pairs of partial sums: (a0.x, a0.y, a1.x, a1.y) collect the columns 0, 1, 2, 3 mod 4.
__device__ __forceinline__ void ffma32(const uint32_t (&v)[32], const float *c, float2 &a0, float2 &a1) {
    const float4 *cp = reinterpret_cast<const float4 *>(c);
#pragma unroll
    for (int q = 0; q < 32; q += 4) {
        const float4 cc = cp[q / 4];
        a0 = __ffma2_rn(make_float2(__uint_as_float(v[q]), __uint_as_float(v[q + 1])), make_float2(cc.x, cc.y), a0);
        a1 = __ffma2_rn(make_float2(__uint_as_float(v[q + 2]), __uint_as_float(v[q + 3])), make_float2(cc.z, cc.w), a1);
    }
}

// y = S c with S in tensor memory: lane = row, 32 columns per load, c broadcast from shared memory,
// packed FP32 FMAs on four partial sums.
__device__ void tmem_matvec(uint32_t tbase, int mp, const float *c, float *y, const Group &g) {
    const int warp = g.warp(), lane = g.lane();
    const int ch = warp >> 2;
    const int row = 128 * ch + 32 * (warp & 3) + lane;
    if (128 * ch < mp) {
        const uint32_t t = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(256 * ch);
        float2 a0 = make_float2(0.0f, 0.0f), a1 = make_float2(0.0f, 0.0f);
        const int nblk = mp >> 5;                              // whole blocks of 32 columns
        for (int k = 0; k < nblk; ++k) {
            uint32_t v[32];
            tmem_ld32(t + (uint32_t)(32 * k), v);
            tmem_wait_ld32(v);
            ffma32(v, c + 32 * k, a0, a1);
        }
        if (mp & 16) {                                         // mp = 16 mod 32
            uint32_t v[16];
            tmem_ld16(t + (uint32_t)(32 * nblk), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float b0 = a0.x, b1 = a0.y, b2 = a1.x, b3 = a1.y;
            fma16(v, c + 32 * nblk, b0, b1, b2, b3);
            a0 = make_float2(b0, b1);
            a1 = make_float2(b2, b3);
        }
        if (row < mp) y[row] = (a0.x + a0.y) + (a1.x + a1.y);
    }
    g.sync();
}

// In-place blocked sweep of a symmetric positive definite matrix in packed lower storage:
// sweeping every pivot turns A into -A^-1.  Per panel K of NB columns: PT = A(:, K)^T, the NB x NB
// pivot block inverted by an unblocked sweep on one warp, TT = (A(:, K) A_KK^-1)^T, the rank-NB
// update A(i, j) -= T(i, :) P(j, :)^T for i, j outside K, then A(:, K) = T and A_KK = -A_KK^-1.
// The panels are stored transposed ([NB][ld], ld = panel_ld(mp)) so that lanes walking
// consecutive rows read consecutive words.  The update runs in strips of 32 rows x 16 columns per
// warp: on FP32 lanes (lane = row, 16 accumulators, the panel row of P read as broadcast float4
// loads), or with `tc` on tensor cores, as 8 mma.m16n8k8 TF32 products per strip with FP32
// accumulation (the mixed-precision mode, whose inverse is stored in BF16 afterwards); ld is 8
// words off a multiple of 32 so that the fragment loads of the four k-rows fall on distinct banks.
template <typename T, int NB>
__device__ void sweep_inverse(T *A, int mp, T *X, bool tc, const Group &g) {
    const int ld = panel_ld(mp);
    T *PT = X;                   // [NB][ld] old panel, transposed
    T *TT = X + NB * ld;         // [NB][ld]
    T *Dm = X + 2 * NB * ld;     // [NB][NB]
    const int tid = g.tid, nthr = g.size, lane = g.lane(), warp = g.warp(), nw = g.warps();
    const int nrb = (mp + 31) / 32;      // 32-row blocks
    const int ncb = mp / 16 + (mp % 16 ? 1 : 0);
    for (int k0 = 0; k0 < mp; k0 += NB) {
        for (int i = tid; i < mp; i += nthr) {
#pragma unroll
            for (int u = 0; u < NB; ++u) PT[u * ld + i] = A[sidx(i, k0 + u, mp)];
        }
        g.sync();
        // -- pivot block inverse by an unblocked sweep on one warp, in registers: lane l holds row
        // l / LR, columns (l % LR) * CPL ... + CPL - 1 of the NB x NB block; the pivot row, column and
        // value of every step come by shuffles (result negated at the end)
        if (warp == 0) {
            constexpr int LR = 32 / NB, CPL = NB / LR;
            const int ri = lane / LR, h = lane % LR;
            T v[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) v[c] = PT[(h * CPL + c) * ld + k0 + ri];
#pragma unroll
            for (int pv = 0; pv < NB; ++pv) {
                const T d = T(1) / __shfl_sync(0xffffffffu, v[pv % CPL], pv * LR + pv / CPL);
                const T aip = __shfl_sync(0xffffffffu, v[pv % CPL], ri * LR + pv / CPL);
                T apj[CPL];
#pragma unroll
                for (int c = 0; c < CPL; ++c) apj[c] = __shfl_sync(0xffffffffu, v[c], pv * LR + h);
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int j = h * CPL + c;
                    if (ri == pv) v[c] = j == pv ? -d : apj[c] * d;
                    else if (j == pv) v[c] = aip * d;
                    else v[c] -= aip * apj[c] * d;
                }
            }
#pragma unroll
            for (int c = 0; c < CPL; ++c) Dm[ri * NB + h * CPL + c] = -v[c];   // = A_KK^-1 (symmetric)
        }
        g.sync();
        // -- TT[t][i] = sum_u P(i, u) Dinv(u, t) for rows outside K (zero on K)
        for (int i = tid; i < mp; i += nthr) {
            T acc[NB];
#pragma unroll
            for (int t = 0; t < NB; ++t) acc[t] = T(0);
            if (i < k0 || i >= k0 + NB) {
#pragma unroll
                for (int u = 0; u < NB; ++u) {
                    const T pv = PT[u * ld + i];
#pragma unroll
                    for (int t = 0; t < NB; ++t) acc[t] = fma(pv, Dm[u * NB + t], acc[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < NB; ++t) TT[t * ld + i] = acc[t];
        }
        g.sync();
        // -- rank-NB update of the lower triangle outside K: strips (row block R, column block C)
        const int kc0 = k0 / 16, kc1 = (k0 + NB + 15) / 16;
        for (int R = 0, strip = 0; R < nrb; ++R) {
            const int cmax = min(ncb, 2 * R + 2);
            for (int C = 0; C < cmax; ++C, ++strip) {
                if (strip % nw != warp) continue;
                if (NB == 16 && C >= kc0 && C < kc1) continue;    // the pivot columns
                if constexpr (sizeof(T) == 4) {
                    if (tc) {
                        const int gq = lane >> 2, tq = lane & 3;
                        float acc[2][2][4];
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
#pragma unroll
                        for (int ks = 0; ks < NB / 8; ++ks) {
                            const T *t0 = TT + (8 * ks + tq) * ld, *t1 = t0 + 4 * ld;
                            const T *p0 = PT + (8 * ks + tq) * ld, *p1 = p0 + 4 * ld;
                            uint32_t af[2][4], bf[2][2];
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt) {
                                const int i0 = 32 * R + 16 * mt + gq;
                                af[mt][0] = tf32_bits(i0 < mp ? t0[i0] : 0.0f);
                                af[mt][1] = tf32_bits(i0 + 8 < mp ? t0[i0 + 8] : 0.0f);
                                af[mt][2] = tf32_bits(i0 < mp ? t1[i0] : 0.0f);
                                af[mt][3] = tf32_bits(i0 + 8 < mp ? t1[i0 + 8] : 0.0f);
                            }
#pragma unroll
                            for (int nt = 0; nt < 2; ++nt) {
                                const int j0 = 16 * C + 8 * nt + gq;
                                bf[nt][0] = tf32_bits(j0 < mp ? p0[j0] : 0.0f);
                                bf[nt][1] = tf32_bits(j0 < mp ? p1[j0] : 0.0f);
                            }
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                for (int nt = 0; nt < 2; ++nt) mma_tf32(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
                        }
                        const int r0 = 32 * R, c0 = 16 * C;
                        const bool plain = r0 >= c0 + 15 && r0 + 31 < mp && (r0 >= k0 + NB || r0 + 31 < k0) &&
                                           (c0 >= k0 + NB || c0 + 15 < k0);
                        if (plain) {
                            // every (i, j) of the strip is a lower-triangle element outside K
                            int cs[2][2];
#pragma unroll
                            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                                for (int b = 0; b < 2; ++b) {
                                    const int j = c0 + 8 * nt + 2 * tq + b;
                                    cs[nt][b] = col_start(j, mp) - j;
                                }
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        A[cs[nt][e & 1] + r0 + 16 * mt + gq + (e >> 1) * 8] -= acc[mt][nt][e];
                        } else {
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                                    for (int e = 0; e < 4; ++e) {
                                        const int i = r0 + 16 * mt + gq + (e >> 1) * 8;
                                        const int j = c0 + 8 * nt + 2 * tq + (e & 1);
                                        if (i < mp && j <= i && (i < k0 || i >= k0 + NB) && (j < k0 || j >= k0 + NB))
                                            A[col_start(j, mp) + i - j] -= acc[mt][nt][e];
                                    }
                        }
                        continue;
                    }
                }
                const int i = 32 * R + lane;
                const bool rowin = i < mp && (i < k0 || i >= k0 + NB);
                T acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = T(0);
#pragma unroll 4
                for (int u = 0; u < NB; ++u) {
                    const T tv = rowin ? TT[u * ld + i] : T(0);
                    T pr[16];
                    load16(PT + u * ld + 16 * C, pr);   // broadcast: every lane reads the same words
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc[c] = fma(tv, pr[c], acc[c]);
                }
                if (rowin) {
                    int j = 16 * C;
                    T *colp = A + col_start(j, mp) - j;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        if (j < mp && j <= i && (j < k0 || j >= k0 + NB)) colp[i] -= acc[c];
                        colp += mp - j - 1;
                        ++j;
                    }
                }
            }
        }
        g.sync();
        // -- write back the swept panel
        for (int i = tid; i < mp; i += nthr) {
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                const int j = k0 + t;
                if (i >= k0 && i < k0 + NB) {
                    if (i >= j) A[pidx(i, j, mp)] = -Dm[(i - k0) * NB + t];
                } else {
                    A[sidx(i, j, mp)] = TT[t * ld + i];
                }
            }
        }
        g.sync();
    }
}

// ----------------------------------------------------------------------------- sweep in tensor memory
// Mixed precision, panel width 16, worlds of up to 256 padded rows run by a whole CTA: the full
// square matrix lives in tensor memory for the whole sweep (row r in lane r mod 128 of column block
// 256 (r / 128), as the PADMM loop reads it afterwards), so the rank-16 update of every panel is
// four tcgen05 TF32 products accumulated straight into it (M = 128 rows, N = mp, K = 8, two K
// steps per row chunk) and no element is read back and rewritten by the lanes.  Per panel K:
//   P = A(:, K) (tcgen05.ld of the column block, lane = row) into shared memory, K-major;
//   A_KK^-1 in one warp's registers; T = P A_KK^-1, stored negated (zero on the rows of K);
//   one thread issues D += (-T) P^T and commits to an mbarrier;
//   column block K := T (A_KK^-1 on K), row block K := T^T (the warp that owns the lanes of K).
// Both triangles are kept, so the panels are read without index mapping.  The operands' shared-
// memory layout is the tensor cores' K-major one: 8-row x 16-byte core matrices, word (r, k) at
// 128 (r / 8) + 32 (k / 4) + 4 (r mod 8) + k mod 4, rows padded with zeros to 256.
__device__ __forceinline__ int kmaj(int r, int k) { return 128 * (r >> 3) + 32 * (k >> 2) + 4 * (r & 7) + (k & 3); }
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address / 16
    d |= (uint64_t)(128u >> 4) << 16;                           // K-direction core matrices 128 B apart
    d |= (uint64_t)(512u >> 4) << 32;                           // 8-row groups 512 B apart
    d |= (uint64_t)1 << 46;                                     // descriptor version (tcgen05), no swizzle
    return d;
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int n = 0; n < (1 << 22); ++n) {                       // bounded (~10 ms)
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// Returns false (uniformly over the CTA) when the tensor cores' completion did not arrive within two
// bounded waits; the world is then abandoned (KAMINO_WORLD_TIMEOUT) and its state left unchanged.
__device__ bool sweep_inverse_tmem(const float *A, int mp, float *X, uint32_t tbase, int *misc, const Group &g) {
    constexpr int NB = 16;
    float *PT = X;                 // K-major [256 rows][16]: the panel P
    float *TN = X + 256 * 16;      // K-major [256 rows][16]: -T
    float *Dm = X + 2 * 256 * 16;  // [16][16]: A_KK^-1
    const int tid = g.tid, nthr = g.size, lane = g.lane(), warp = g.warp();
    const int ch = warp >> 2, q = warp & 3;
    const int row = 128 * ch + 32 * q + lane;                 // the matrix row of this lane
    const bool has_rows = 128 * ch < mp;                        // warp-uniform
    const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + 256u * ch;
    const uint32_t mbar = smem_addr(misc + 4);
    const int nch = mp > 128 ? 2 : 1;
    // the assembled matrix (packed lower, shared memory) into tensor memory, both triangles
    if (has_rows) {
        for (int j0 = 0; j0 < mp; j0 += 16) {
            uint32_t v[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) v[c] = __float_as_uint(row < mp ? A[sidx(row, j0 + c, mp)] : 0.0f);
            tmem_st16(trow + (uint32_t)j0, v);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    for (int e = tid; e < 2 * 256 * 16; e += nthr) X[e] = 0.0f;   // padding rows stay zero
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before();
    g.sync();
    tmem_fence_after();
    // kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both K-major, N / 8 at
    // bits 17-22, M / 16 at bits 24-28
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(mp >> 3) << 17) | ((128u >> 4) << 24);
    int panel = 0;
    for (int k0 = 0; k0 < mp; k0 += NB, ++panel) {
        // -- P = A(:, K): column block K of every row
        if (has_rows) {
            uint32_t v[16];
            tmem_ld16(trow + (uint32_t)k0, v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < mp) {
#pragma unroll
                for (int c = 0; c < 16; c += 4)
                    *reinterpret_cast<float4 *>(PT + kmaj(row, c)) =
                        make_float4(__uint_as_float(v[c]), __uint_as_float(v[c + 1]), __uint_as_float(v[c + 2]),
                                    __uint_as_float(v[c + 3]));
            }
        }
        g.sync();
        // -- A_KK^-1 by an unblocked sweep in one warp's registers (as in sweep_inverse), while the
        // warp that owns the previous pivot rows writes the rest of their row block (deferred from
        // the previous panel: -T of that panel is still in TN, and this panel's products, which
        // touch every column, are issued only after the next barrier)
        const int wprev = k0 > 0 ? 4 * ((k0 - NB) >> 7) + (((k0 - NB) & 127) >> 5) : -1;
        if (k0 > 0 && warp == wprev) {
            const int kp = k0 - NB;                                  // the previous panel
            const int r0 = kp - (128 * ch + 32 * q);
            const bool mine = lane >= r0 && lane < r0 + NB;
            for (int j0 = 0; j0 < mp; j0 += 16) {
                if (j0 == kp || j0 == k0) continue;                 // written with that panel / before
                uint32_t v[16];
                tmem_ld16(trow + (uint32_t)j0, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (mine) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = __float_as_uint(-TN[kmaj(j0 + c, lane - r0)]);
                }
                tmem_st16(trow + (uint32_t)j0, v);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        if (warp == (wprev == 0 ? 1 : 0)) {
            constexpr int LR = 32 / NB, CPL = NB / LR;
            const int ri = lane / LR, h = lane % LR;
            float v[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) v[c] = PT[kmaj(k0 + ri, h * CPL + c)];
#pragma unroll
            for (int pv = 0; pv < NB; ++pv) {
                const float d = __frcp_rn(__shfl_sync(0xffffffffu, v[pv % CPL], pv * LR + pv / CPL));
                const float aip = __shfl_sync(0xffffffffu, v[pv % CPL], ri * LR + pv / CPL);
                float apj[CPL];
#pragma unroll
                for (int c = 0; c < CPL; ++c) apj[c] = __shfl_sync(0xffffffffu, v[c], pv * LR + h);
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int j = h * CPL + c;
                    if (ri == pv) v[c] = j == pv ? -d : apj[c] * d;
                    else if (j == pv) v[c] = aip * d;
                    else v[c] -= aip * apj[c] * d;
                }
            }
#pragma unroll
            for (int c = 0; c < CPL; ++c) Dm[ri * NB + h * CPL + c] = -v[c];
        }
        tmem_fence_before();
        g.sync();
        tmem_fence_after();
        // -- -T = -P A_KK^-1 outside K (zero on K)
        for (int i = tid; i < mp; i += nthr) {
            float acc[NB];
#pragma unroll
            for (int t = 0; t < NB; ++t) acc[t] = 0.0f;
            if (i < k0 || i >= k0 + NB) {
#pragma unroll
                for (int u = 0; u < NB; ++u) {
                    const float pv = PT[kmaj(i, u)];
#pragma unroll
                    for (int t = 0; t < NB; ++t) acc[t] = fmaf(pv, Dm[u * NB + t], acc[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < NB; t += 4)
                *reinterpret_cast<float4 *>(TN + kmaj(i, t)) = make_float4(-acc[t], -acc[t + 1], -acc[t + 2], -acc[t + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // P and -T visible to the tensor cores
        tmem_fence_before();
        g.sync();
        // -- A += (-T) P^T on the tensor cores, accumulated in place
        if (tid == 0) {
            tmem_fence_after();
            for (int c = 0; c < nch; ++c)
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t da = smem_desc_kmajor(smem_addr(TN) + 8192u * c + 256u * ks);
                    const uint64_t db = smem_desc_kmajor(smem_addr(PT) + 256u * ks);
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                                 :: "r"(tbase + 256u * c), "l"(da), "l"(db), "r"(idesc), "r"(1u) : "memory");
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mbar) : "memory");
        }
        bool ok = mbar_wait(mbar, (uint32_t)(panel & 1));
        if (!ok) ok = mbar_wait(mbar, (uint32_t)(panel & 1));  // a second bounded wait for the products
        if (__syncthreads_or(!ok)) {                            // whole-CTA group: a uniform decision
            if (tid == 0) misc[1] |= 2;
            tmem_fence_after();
            return false;
        }
        tmem_fence_after();
        // -- column block K := T on the rows outside K, A_KK^-1 negated on K (every warp, its rows)
        if (has_rows) {
            uint32_t v[16];
            const bool inK = row >= k0 && row < k0 + NB;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float x = 0.0f;
                if (row < mp) x = inK ? -Dm[(row - k0) * NB + c] : -TN[kmaj(row, c)];
                v[c] = __float_as_uint(x);
            }
            tmem_st16(trow + (uint32_t)k0, v);
        }
        // -- row block K := T^T outside K (the warp that owns the lanes of K; they lie in one warp):
        // now only the next panel's column block, which its panel copy reads; the rest during the
        // next pivot inversion.  The last panel writes every column here.
        if (warp == 4 * (k0 >> 7) + ((k0 & 127) >> 5)) {
            const int r0 = k0 - (128 * ch + 32 * q);             // first lane of K in this warp
            const bool mine = lane >= r0 && lane < r0 + NB;
            const bool last = k0 + NB >= mp;
            for (int j0 = 0; j0 < mp; j0 += 16) {
                if (j0 == k0 || (!last && j0 != k0 + NB)) continue;
                uint32_t v[16];
                tmem_ld16(trow + (uint32_t)j0, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (mine) {
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = __float_as_uint(-TN[kmaj(j0 + c, lane - r0)]);
                }
                tmem_st16(trow + (uint32_t)j0, v);
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tmem_fence_before();
        g.sync();
        tmem_fence_after();
    }
    return true;
}

// ----------------------------------------------------------------------------- PADMM owner phases
// FP64 iterates of the refinement end game (x, y, z, y^, z^ and the new y, z of an iteration across
// its reduction barrier: 7 mp doubles) in shared memory that is
// dead during the PADMM loop: the packed matrix region once the inverse lives in tensor memory, the
// part of that region the BF16 tiles leave free, else the sweep scratch past the mat-vec partials
// and the FP64 refinement vectors.  nullptr when none has room (the iterates then stay in FP32).
template <typename T>
__device__ __forceinline__ double *fp64_iterates(unsigned char *smem, const Layout &L, bool in_tmem, bool bf16_tiles,
                                                 int mp, int nb, T *X) {
    if constexpr (sizeof(T) != 4) {
        return nullptr;
    } else {
        const size_t need = (size_t)7 * mp * sizeof(double);
        const size_t a_bytes = L.red - L.A;
        if (in_tmem && need <= a_bytes) return reinterpret_cast<double *>(smem + L.A);
        if (bf16_tiles) {
            const int nt = mp / 16;
            const size_t tiles = align_up((size_t)nt * (nt + 1) / 2 * 512, 16);
            if (tiles + need <= a_bytes) return reinterpret_cast<double *>(smem + L.A + tiles);
        }
        const size_t used = ((size_t)kWarps * mp + 2 * (size_t)mp + 12 * (size_t)nb) * sizeof(float);
        if (used + need <= L.A - L.X) return reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(X) + used);
        return nullptr;
    }
}

// The owners' slots: slot j = tid + s * group size of a thread holds unit slot_unit(j).  Joint rows
// keep slot = unit; the contacts start at slot `cslot0`, the first warp boundary after the joint
// rows when the slots have room (else right after them), so that no warp mixes the two kinds of
// unit and their different owner phases.  Returns a value >= nunits for an empty slot.
__device__ __forceinline__ int slot_unit(int j, int nbil, int cslot0) {
    return j < nbil ? j : j >= cslot0 ? nbil + (j - cslot0) : 0x3fffffff;
}

// |(a, b)| in the iteration's precision: in FP32 from the hardware reciprocal square root (a few
// ulp, no slow path), in FP64 the rounded square root.
template <typename V>
__device__ __forceinline__ V hypot2(V a, V b) {
    const V s = a * a + b * b;
    if constexpr (sizeof(V) == 4) return s > 0.0f ? s * rsqrtf(s) : 0.0f;
    else return sqrt(s);
}

// Projection of v onto the Coulomb cone {|y_t| <= mu y_n} (Sec. 3), `mui` = 1 / (1 + mu^2): the three
// cases of the closed form (inside: v; in the polar cone: 0; else onto the cone's surface) as
// selects, so that the lanes of a warp do not diverge over them.  FP32 divides by the hardware
// reciprocal.
template <typename V>
__device__ __forceinline__ void cone_project(const V (&v)[3], V mu, V mui, V (&y)[3]) {
    const V tn = hypot2(v[0], v[1]);
    const bool inside = tn <= mu * v[2], polar = mu * tn <= -v[2];
    const V nn = (mu * tn + v[2]) * mui;
    V sc;
    if constexpr (sizeof(V) == 4) sc = __fdividef(mu * nn, tn);
    else sc = mu * nn / tn;
    // tn > 0 whenever neither case holds, so the quotient is used only where it is finite
    y[0] = inside ? v[0] : polar ? V(0) : sc * v[0];
    y[1] = inside ? v[1] : polar ? V(0) : sc * v[1];
    y[2] = inside ? v[2] : polar ? V(0) : nn;
}

// Owner phase of a PADMM iteration (Alg. 1) for the units of this thread, with the iterates of type
// V (T, or FP64 in the refinement end game): x^i = x^{i-1} + xn (the refined x-step),
// y^i = Pi_K(x^i - z^/rho) (identity on joint rows, the Coulomb cone on contacts),
// z^i = z^ - rho (x^i - y^i), and this thread's terms of the residuals r_p = ||x - y||,
// r_d = ||eta (x^i - x^{i-1}) + rho (y^i - y^)||, r_c = |y_k . z_k| and of Nesterov's combined
// residual.  The new iterates stay in registers; x^i and P x^i go to shared memory at once.
template <typename V, typename T, int S>
__device__ __forceinline__ void owner_update(const Group &g, int nunits, int nfix, int nbil, V *x, const T *xn, const V *yh,
                                             const V *zh, const T *mut, const T *mui, const T *p, T *wv, T eta_, T rho_,
                                             T irho_, V (&xnew)[S][3], V (&ynew)[S][3], V (&znew)[S][3], T &lrp,
                                             T &lrd, T &lrc, T &lc, int cslot0) {
    const V eta = V(eta_), rho = V(rho_), irho = V(irho_);
#pragma unroll
    for (int sl = 0; sl < S; ++sl)
#pragma unroll
        for (int t = 0; t < 3; ++t) xnew[sl][t] = ynew[sl][t] = znew[sl][t] = V(0);
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = slot_unit(g.tid + sl * g.size, nbil, cslot0);
        if (u >= nunits) continue;
        if (u < nbil) {
            // joint and drive rows: the identity; joint-limit rows (u >= nfix): the ray R+ (Sec. 3)
            const V xv = x[u] + V(xn[u]);
            V yv = xv - zh[u] * irho;
            if (u >= nfix) yv = fmax(yv, V(0));
            const V zv = zh[u] - rho * (xv - yv);
            lrp = fmax(lrp, T(fabs(xv - yv)));
            lrd = fmax(lrd, T(fabs(eta * (xv - x[u]) + rho * (yv - yh[u]))));
            lc += T((zv - zh[u]) * (zv - zh[u]) * irho + rho * (yv - yh[u]) * (yv - yh[u]));
            if (u >= nfix) lrc = fmax(lrc, T(fabs(yv * zv)));
            xnew[sl][0] = xv; ynew[sl][0] = yv; znew[sl][0] = zv;
            x[u] = xv;
            wv[u] = T(V(p[u]) * xv);
        } else {
            const int k = u - nbil, r0 = nbil + 3 * k;
            const V mu = V(mut[k]);
            V v[3], yv[3], xv[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                xv[t] = x[r0 + t] + V(xn[r0 + t]);
                v[t] = xv[t] - zh[r0 + t] * irho;
            }
            cone_project<V>(v, mu, V(mui[k]), yv);
            V ydz = V(0);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const V zv = zh[r0 + t] - rho * (xv[t] - yv[t]);
                lrp = fmax(lrp, T(fabs(xv[t] - yv[t])));
                lrd = fmax(lrd, T(fabs(eta * (xv[t] - x[r0 + t]) + rho * (yv[t] - yh[r0 + t]))));
                lc += T((zv - zh[r0 + t]) * (zv - zh[r0 + t]) * irho + rho * (yv[t] - yh[r0 + t]) * (yv[t] - yh[r0 + t]));
                ydz += yv[t] * zv;
                xnew[sl][t] = xv[t]; ynew[sl][t] = yv[t]; znew[sl][t] = zv;
            }
            lrc = fmax(lrc, T(fabs(ydz)));
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                x[r0 + t] = xv[t];
                wv[r0 + t] = T(V(p[r0 + t]) * xv[t]);
            }
        }
    }
}

// The rows of this thread's units from registers into a row vector and back.
template <int S>
__device__ __forceinline__ void stash_rows(const Group &g, int nunits, int nbil, const double (&v)[S][3], double *dst,
                                           int cslot0) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = slot_unit(g.tid + sl * g.size, nbil, cslot0);
        if (u >= nunits) continue;
        const int r0 = u < nbil ? u : nbil + 3 * (u - nbil), cnt = u < nbil ? 1 : 3;
        for (int t = 0; t < cnt; ++t) dst[r0 + t] = v[sl][t];
    }
}
template <int S>
__device__ __forceinline__ void unstash_rows(const Group &g, int nunits, int nbil, const double *src, double (&v)[S][3],
                                             int cslot0) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = slot_unit(g.tid + sl * g.size, nbil, cslot0);
#pragma unroll
        for (int t = 0; t < 3; ++t) v[sl][t] = 0.0;
        if (u >= nunits) continue;
        const int r0 = u < nbil ? u : nbil + 3 * (u - nbil), cnt = u < nbil ? 1 : 3;
        for (int t = 0; t < cnt; ++t) v[sl][t] = src[r0 + t];
    }
}

// Commit of a PADMM iteration by the owners: Nesterov's extrapolation (or restart) of (y, z) into
// (y^, z^) (Sec. 4.1), the new y, z, y^, z^, and the next iteration's right-hand side
// b = v_f + Gamma(z^) - eta x - rho y^ - z^ (in FP64 from the FP64 v_f when `hp`).  `init64`, when
// set, is the FP64 iterate block (x, y, z, y^, z^ of mp each) that takes over from this commit on.
// With `lag` the next iteration does not evaluate the refinement residual: the owners store its
// correction's right-hand side c = b^{i+1} - b^i directly (in bb, or as the BF16 hi / lo split when
// chi is set), which is b^{i+1} + A x^i when x^i solved A x = -b^i exactly.  `bprev` carries this
// thread's b from commit to commit (FP32 path).
template <typename V, typename T, int S>
__device__ __forceinline__ void owner_commit(const Group &g, int nunits, int nbil, V *y, V *z, V *yh, V *zh,
                                             const double *vfd, const T (&vfo)[S][3], const T *mut, T eta_, T rho_,
                                             bool nesterov, bool restart, T beta_, const V (&xnew)[S][3],
                                             const V (&ynew)[S][3], const V (&znew)[S][3], bool hp, T *bb, double *bbd,
                                             double *init64, int mp, bool lag, T (&bprev)[S][3],
                                             __nv_bfloat16 *chi, __nv_bfloat16 *clo, int cslot0) {
    const V beta_n = V(beta_);
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = slot_unit(g.tid + sl * g.size, nbil, cslot0);
        if (u >= nunits) continue;
        const int r0 = u < nbil ? u : nbil + 3 * (u - nbil);
        const int cnt = u < nbil ? 1 : 3;
        // all loads first and every new value kept in registers: the vectors share one
        // shared-memory buffer, so a value stored and read back would wait for the store
        V yo[3], zo[3], yhv[3], zhv[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const bool on = t < cnt;
            yo[t] = on ? y[r0 + t] : V(0);
            zo[t] = on ? z[r0 + t] : V(0);
        }
        const T mu = cnt == 3 ? mut[u - nbil] : T(0);
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const V yv = ynew[sl][t], zv = znew[sl][t];
            if (!nesterov) { yhv[t] = yv; zhv[t] = zv; }
            else if (restart) { yhv[t] = yo[t]; zhv[t] = zo[t]; }
            else { yhv[t] = yv + beta_n * (yv - yo[t]); zhv[t] = zv + beta_n * (zv - zo[t]); }
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t >= cnt) break;
            const int r = r0 + t;
            yh[r] = yhv[t]; zh[r] = zhv[t];
            y[r] = ynew[sl][t]; z[r] = znew[sl][t];
        }
        if (init64) {
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (t >= cnt) break;
                const int r = r0 + t;
                init64[r] = (double)xnew[sl][t];
                init64[mp + r] = (double)ynew[sl][t];
                init64[2 * mp + r] = (double)znew[sl][t];
                init64[3 * mp + r] = (double)yhv[t];
                init64[4 * mp + r] = (double)zhv[t];
            }
        }
        if (hp) {
            const double z0 = (double)zhv[0], z1 = (double)zhv[1];
            const double sd = cnt == 3 ? (double)mu * sqrt(z0 * z0 + z1 * z1) : 0.0;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (t >= cnt) break;
                bbd[r0 + t] = vfd[r0 + t] + (t == 2 ? sd : 0.0) - (double)eta_ * (double)xnew[sl][t] -
                              (double)rho_ * (double)yhv[t] - (double)zhv[t];
            }
        } else {
            const V eta = V(eta_), rho = V(rho_);
            const V sv = cnt == 3 ? V(mu) * hypot2(zhv[0], zhv[1]) : V(0);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (t >= cnt) break;
                const T bn = T(V(vfo[sl][t]) + (t == 2 ? sv : V(0)) - eta * xnew[sl][t] - rho * yhv[t] - zhv[t]);
                if (!lag) {
                    bb[r0 + t] = bn;
                } else if (chi == nullptr) {
                    bb[r0 + t] = bn - bprev[sl][t];
                } else {
                    const float v = (float)(bn - bprev[sl][t]);
                    const __nv_bfloat16 h = __float2bfloat16(v);
                    chi[r0 + t] = h;
                    clo[r0 + t] = __float2bfloat16(v - __bfloat162float(h));
                }
                bprev[sl][t] = bn;
            }
        }
    }
}

// ----------------------------------------------------------------------------- NCP residual
// What the natural-map residual of a world needs (shared memory, built by phases 1-5).
template <typename T>
struct NcpWorld {
    int nb, nfix, nbil, nact;
    const int *bro, *brow, *rbody;
    const T *rJ, *p, *mut, *bminv, *bIinv, *bufree;
    const double *rvs;
};

// u+ = u_free + M^-1 J^T P y in FP64 into fd (6 per body); y from `yfin` (FP64) when set, else `y`.
// Thread per (body, component) for J^T lambda, then thread per body; ends without a barrier.
// Returns true when a velocity this thread formed is not finite.
template <typename T>
__device__ bool ncp_velocities(const NcpWorld<T> &c, const Group &g, const double *yfin, const T *y, double *fd) {
    const int tid = g.tid, nthr = g.size;
    for (int t = tid; t < 6 * c.nb; t += nthr) {
        const int i = t / 6, k = t - 6 * (t / 6);
        double f = 0.0;
        for (int e = c.bro[i]; e < c.bro[i + 1]; ++e) {
            const int code = c.brow[e], r = code >> 1;
            const double yr = yfin ? yfin[r] : (double)y[r];
            f = fma((double)c.rJ[6 * code + k], (double)c.p[r] * yr, f);   // 12 r + 6 side + k
        }
        fd[t] = f;
    }
    g.sync();
    // each thread reads and writes only its body's words
    bool bad = false;
    for (int i = tid; i < c.nb; i += nthr) {
        double f[6];
        for (int k = 0; k < 6; ++k) f[k] = fd[6 * i + k];
        double dw[3];
        symvec3d(c.bIinv + 6 * i, f + 3, dw);
        for (int k = 0; k < 3; ++k) {
            fd[6 * i + k] = (double)c.bufree[6 * i + k] + (double)c.bminv[i] * f[k];
            fd[6 * i + 3 + k] = (double)c.bufree[6 * i + 3 + k] + dw[k];
        }
        for (int k = 0; k < 6; ++k) bad |= !isfinite(fd[6 * i + k]);
    }
    return bad;
}

// Natural-map NCP residual of (lambda, u+) on the complementarity blocks (Eq. 3), scaled units, with
// u+ in fd (after a barrier that follows ncp_velocities): with v~ = P (J u+ + v*) and
// lambda~ = P^-1 lambda = y, max_k || lambda~_k - Pi_K(lambda~_k - (v~_k + Gamma(v~_k))) ||_inf over the
// contacts; a joint-limit row (0 <= lambda ⟂ g >= 0) adds |lambda~ - max(lambda~ - v~, 0)|.  Every
// thread gets the group's value (one reduction, buffer `phase`).
template <typename T>
__device__ T ncp_natural_map(const NcpWorld<T> &c, const Group &g, const double *yfin, const T *y, const double *fd,
                             T *red, int phase) {
    const int tid = g.tid, nthr = g.size;
    T lncp = T(0);
    for (int r = c.nfix + tid; r < c.nbil; r += nthr) {
        const int sa = c.rbody[2 * r], sb = c.rbody[2 * r + 1];
        double v = c.rvs[r];
        for (int q = 0; q < 6; ++q) {
            if (sa >= 0) v = fma((double)c.rJ[12 * r + q], fd[6 * sa + q], v);
            v = fma((double)c.rJ[12 * r + 6 + q], fd[6 * sb + q], v);
        }
        const double vs = (double)c.p[r] * v, ls = yfin ? yfin[r] : (double)y[r];
        lncp = fmax(lncp, T(fabs(ls - fmax(ls - vs, 0.0))));
    }
    for (int k = tid; k < c.nact; k += nthr) {
        const int r0 = c.nbil + 3 * k;
        double vs[3], ls[3];
        for (int t = 0; t < 3; ++t) {
            const int r = r0 + t, sa = c.rbody[2 * r], sb = c.rbody[2 * r + 1];
            double v = c.rvs[r];
            for (int q = 0; q < 6; ++q) {
                if (sa >= 0) v = fma((double)c.rJ[12 * r + q], fd[6 * sa + q], v);
                v = fma((double)c.rJ[12 * r + 6 + q], fd[6 * sb + q], v);
            }
            vs[t] = (double)c.p[r] * v;
            ls[t] = yfin ? yfin[r] : (double)y[r];
        }
        const double mu = (double)c.mut[k];
        const double s[3] = {ls[0] - vs[0], ls[1] - vs[1], ls[2] - (vs[2] + mu * sqrt(vs[0] * vs[0] + vs[1] * vs[1]))};
        const double tn = sqrt(s[0] * s[0] + s[1] * s[1]);
        double pr[3];
        if (tn <= mu * s[2]) {
            pr[0] = s[0]; pr[1] = s[1]; pr[2] = s[2];
        } else if (mu * tn <= -s[2]) {
            pr[0] = pr[1] = pr[2] = 0.0;
        } else {
            const double nn = (mu * tn + s[2]) / (1.0 + mu * mu);
            pr[0] = mu * nn * s[0] / tn; pr[1] = mu * nn * s[1] / tn; pr[2] = nn;
        }
        for (int t = 0; t < 3; ++t) lncp = fmax(lncp, T(fabs(ls[t] - pr[t])));
    }
    T d0 = T(0), d1 = T(0), d2 = T(0);
    group_reduce4(lncp, d0, d1, d2, red, phase, g);
    return lncp;
}

// Per-body row lists for the matrix-free products: bro[i] .. bro[i+1] index brow, whose entries are
// 2 r + side for every row r that has body i on that side (side 0: A, side 1: B).
__device__ void body_row_lists(const Group &g, int nb, int m, const int *rbody, int *bro, int *brow) {
    const int tid = g.tid, nthr = g.size;
    for (int i = tid; i < nb; i += nthr) {
        int cnt = 0;
        for (int r = 0; r < m; ++r) cnt += (rbody[2 * r] == i) + (rbody[2 * r + 1] == i);
        bro[i + 1] = cnt;
    }
    g.sync();
    if (tid == 0) {
        bro[0] = 0;
        for (int i = 0; i < nb; ++i) bro[i + 1] += bro[i];
    }
    g.sync();
    for (int i = tid; i < nb; i += nthr) {
        int e = bro[i];
        for (int r = 0; r < m; ++r) {
            if (rbody[2 * r] == i) brow[e++] = 2 * r;
            if (rbody[2 * r + 1] == i) brow[e++] = 2 * r + 1;
        }
    }
}

// ----------------------------------------------------------------------------- sparse formulation
// Sec. 5.1: the Delassus matrix is never formed.  A v = P (J M^-1 J^T + R) P v + (eta + rho) v is
// applied from the rows: the owners of the units publish w = P v, LB lanes per body gather
// g_b = M_b^-1 sum_r J_rb^T w_r, and every owner forms (A v)_r = p_r J_r (g_A, g_B) +
// (eta + rho + p_r^2 R_r) v_r for its own rows (the scaling by P is folded into the publication and
// the row product, which is what pre-scaled P J and M^-1 J^T P rows save).  Each x-step of Alg. 1
// runs k Conjugate Residual iterations on A x = -b from the previous x; every PADMM and CR vector of a
// unit stays in its owner's registers and only w and g go through shared memory, so one application
// of A costs two barriers and one CR iteration three (the dot products of one reduction).

// Group-wide sums of three values (fixed order, so the result does not depend on scheduling),
// double-buffered by `phase` like group_reduce4.
template <typename V>
__device__ __forceinline__ void group_sum3(V &a, V &b, V &c, V *red, int phase, const Group &g) {
    const int lane = g.lane(), warp = g.warp(), nw = g.warps();
    a = warp_sum(a); b = warp_sum(b); c = warp_sum(c);
    V *r = red + phase * 4 * kWarps;
    if (lane == 0) { r[warp] = a; r[kWarps + warp] = b; r[2 * kWarps + warp] = c; }
    g.sync();
    a = r[0]; b = r[kWarps]; c = r[2 * kWarps];
    for (int k = 1; k < nw; ++k) { a += r[k]; b += r[kWarps + k]; c += r[2 * kWarps + k]; }
}

// What the sparse x-step needs of the world (shared memory, built by phases 1-5).
template <typename T>
struct CrWorld {
    int nunits, nfix, nbil, nb, LB;
    const int *bro, *brow, *rbody;
    const T *rJ, *p, *rreg, *bminv, *bIinv, *mut, *mui;
    const double *vfd;
    T shift, eta, rho;
    int ncp_stop;              // converged also requires the natural-map residual below tol
    NcpWorld<T> ncw;
    double *yout, *fd;         // FP64 y for the NCP check and phase 9; FP64 scratch (6 nb)
};

// The PADMM iterates of this thread's units, in registers: slot [s][t] is row t of unit
// tid + s * group size (a joint row uses t = 0 only); Ax = A x, b the next right-hand side.
template <typename V, int S>
struct CrIterates {
    V x[S][3], y[S][3], z[S][3], yh[S][3], zh[S][3], b[S][3], Ax[S][3];
};

__device__ __forceinline__ void unit_rows(int u, int nbil, int &r0, int &cnt) {
    r0 = u < nbil ? u : nbil + 3 * (u - nbil);
    cnt = u < nbil ? 1 : 3;
}

// out = A v for the rows of this thread's units (zero on unused slots).  Two barriers; w and g may be
// reused by the next call at once.
template <typename V, typename T, int S>
__device__ __forceinline__ void cr_apply(const CrWorld<T> &c, const Group &g, const V (&v)[S][3], V (&out)[S][3],
                                         V *w, V *gb) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = g.tid + sl * g.size;
        if (u >= c.nunits) continue;
        int r0, cnt;
        unit_rows(u, c.nbil, r0, cnt);
        for (int t = 0; t < cnt; ++t) w[r0 + t] = V(c.p[r0 + t]) * v[sl][t];
    }
    g.sync();
    const int nthr = g.size, tid = g.tid, LB = c.LB;
    for (int base = 0; base < c.nb * LB; base += nthr) {
        if (base + (tid & ~31) >= c.nb * LB) continue;          // the whole warp is past the bodies
        const int t = base + tid, body = t / LB, sub = t - body * LB;
        const bool on = t < c.nb * LB;
        V f[6] = {V(0), V(0), V(0), V(0), V(0), V(0)};
        if (on) {
            for (int e = c.bro[body] + sub; e < c.bro[body + 1]; e += LB) {
                const int code = c.brow[e];
                const V wr = w[code >> 1];
                const T *J = c.rJ + 6 * code;                     // 12 r + 6 side
#pragma unroll
                for (int k = 0; k < 6; ++k) f[k] = fma(V(J[k]), wr, f[k]);
            }
        }
        for (int o = LB >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
        }
        if (on && sub == 0) {
            const V mi = V(c.bminv[body]);
            const T *Si = c.bIinv + 6 * body;
            const V s0 = V(Si[0]), s1 = V(Si[1]), s2 = V(Si[2]), s3 = V(Si[3]), s4 = V(Si[4]), s5 = V(Si[5]);
            V *o = gb + 6 * body;
            o[0] = mi * f[0]; o[1] = mi * f[1]; o[2] = mi * f[2];
            o[3] = s0 * f[3] + s3 * f[4] + s4 * f[5];
            o[4] = s3 * f[3] + s1 * f[4] + s5 * f[5];
            o[5] = s4 * f[3] + s5 * f[4] + s2 * f[5];
        }
    }
    g.sync();
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = g.tid + sl * g.size;
#pragma unroll
        for (int t = 0; t < 3; ++t) out[sl][t] = V(0);
        if (u >= c.nunits) continue;
        int r0, cnt;
        unit_rows(u, c.nbil, r0, cnt);
        for (int t = 0; t < cnt; ++t) {
            const int r = r0 + t, sa = c.rbody[2 * r], sb = c.rbody[2 * r + 1];
            const T *J = c.rJ + 12 * r;
            V acc = V(0);
            if (sa >= 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) acc = fma(V(J[k]), gb[6 * sa + k], acc);
            }
            if (sb >= 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) acc = fma(V(J[6 + k]), gb[6 * sb + k], acc);
            }
            const V pr = V(c.p[r]);
            out[sl][t] = pr * acc + (V(c.shift) + pr * pr * V(c.rreg[r])) * v[sl][t];
        }
    }
}

// b = v_f + Gamma(z^) - eta x - rho y^ - z^ for this thread's units (Alg. 1's right-hand side).
template <typename V, typename T, int S>
__device__ __forceinline__ void cr_rhs(const CrWorld<T> &c, const Group &g, CrIterates<V, S> &I) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = g.tid + sl * g.size;
        if (u >= c.nunits) continue;
        int r0, cnt;
        unit_rows(u, c.nbil, r0, cnt);
        const V s = cnt == 3 ? V(c.mut[u - c.nbil]) * sqrt(I.zh[sl][0] * I.zh[sl][0] + I.zh[sl][1] * I.zh[sl][1]) : V(0);
        for (int t = 0; t < cnt; ++t)
            I.b[sl][t] = V(c.vfd[r0 + t]) + (t == 2 ? s : V(0)) - V(c.eta) * I.x[sl][t] - V(c.rho) * I.yh[sl][t] -
                         I.zh[sl][t];
    }
}

// Nesterov state of Alg. 1 (Sec. 4.1), kept in FP64 whatever the iterates' type.
struct CrMomentum {
    double a, c_prev;
};

// PADMM iterations it ... iters with the sparse x-step (k CR iterations).  Returns true when it stopped
// because `switch64` is set and r_p, r_d fell below KAMINO_REFINE64_BELOW (the caller continues in
// FP64); `it` is then the next iteration.  Otherwise `it` is the last iteration run.
template <typename V, typename T, int S>
__device__ bool cr_padmm(const CrWorld<T> &c, const Group &g, CrIterates<V, S> &I, V *w, V *gb, V *red, int &ph,
                         int &it, int iters, int k, double tol, bool nesterov, CrMomentum &mom, double &rp, double &rd,
                         double &rc, bool &converged, bool switch64) {
    const V eta = V(c.eta), rho = V(c.rho), irho = V(1) / V(c.rho);
    for (; it <= iters; ++it) {
        V xprev[S][3], r[S][3], pd[S][3], Ap[S][3], Ar[S][3];
        // -- x-step: CR on A x = -b from x^{i-1}: r0 = -b - A x^{i-1}
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                xprev[sl][t] = I.x[sl][t];
                r[sl][t] = -I.b[sl][t] - I.Ax[sl][t];
            }
        cr_apply<V, T, S>(c, g, r, Ar, w, gb);
        V s0 = V(0), s1 = V(0), s2 = V(0);
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                pd[sl][t] = r[sl][t];
                Ap[sl][t] = Ar[sl][t];
                s0 = fma(r[sl][t], Ar[sl][t], s0);
                s1 = fma(Ar[sl][t], Ar[sl][t], s1);
            }
        group_sum3<V>(s0, s1, s2, red, ph++ & 1, g);
        V rAr = s0, ApAp = s1;
        for (int j = 0; j < k; ++j) {
            if (!(rAr > V(0)) || !(ApAp > V(0))) break;           // the residual vanished (uniform)
            const V alpha = rAr / ApAp;
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    I.x[sl][t] = fma(alpha, pd[sl][t], I.x[sl][t]);
                    r[sl][t] = fma(-alpha, Ap[sl][t], r[sl][t]);
                }
            if (j == k - 1) break;
            cr_apply<V, T, S>(c, g, r, Ar, w, gb);
            s0 = s1 = s2 = V(0);
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    s0 = fma(r[sl][t], Ar[sl][t], s0);
                    s1 = fma(Ar[sl][t], Ar[sl][t], s1);
                    s2 = fma(Ar[sl][t], Ap[sl][t], s2);
                }
            group_sum3<V>(s0, s1, s2, red, ph++ & 1, g);
            // beta = (r', A r') / (r, A r); A p' = A r' + beta A p, so
            // (A p', A p') = (A r', A r') + 2 beta (A r', A p) + beta^2 (A p, A p)
            const V beta = s0 / rAr;
            rAr = s0;
            ApAp = s1 + V(2) * beta * s2 + beta * beta * ApAp;
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    pd[sl][t] = fma(beta, pd[sl][t], r[sl][t]);
                    Ap[sl][t] = fma(beta, Ap[sl][t], Ar[sl][t]);
                }
        }
        // -- A x^i, evaluated (not carried by the recurrence): the x-step's residual A x + b enters the
        // dual residual, and it is the next iteration's starting residual
        cr_apply<V, T, S>(c, g, I.x, I.Ax, w, gb);
        // -- owners: y^i = Pi_K(x^i - z^/rho), z^i = z^ - rho (x^i - y^i), residual terms
        V lrp = V(0), lrd = V(0), lrc = V(0), lc = V(0);
        V yn[S][3], zn[S][3];
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
            const int u = g.tid + sl * g.size;
#pragma unroll
            for (int t = 0; t < 3; ++t) yn[sl][t] = zn[sl][t] = V(0);
            if (u >= c.nunits) continue;
            if (u < c.nbil) {
                const V xv = I.x[sl][0];
                V yv = xv - I.zh[sl][0] * irho;
                if (u >= c.nfix) yv = fmax(yv, V(0));             // joint-limit rows: the ray R+
                const V zv = I.zh[sl][0] - rho * (xv - yv);
                const V lin = I.Ax[sl][0] + I.b[sl][0];
                lrp = fmax(lrp, fabs(xv - yv));
                lrd = fmax(lrd, fabs(eta * (xv - xprev[sl][0]) + rho * (yv - I.yh[sl][0]) - lin));
                lc += (zv - I.zh[sl][0]) * (zv - I.zh[sl][0]) * irho + rho * (yv - I.yh[sl][0]) * (yv - I.yh[sl][0]);
                if (u >= c.nfix) lrc = fmax(lrc, fabs(yv * zv));
                yn[sl][0] = yv;
                zn[sl][0] = zv;
            } else {
                const int kc = u - c.nbil;
                const V mu = V(c.mut[kc]);
                V v[3], yv[3];
#pragma unroll
                for (int t = 0; t < 3; ++t) v[t] = I.x[sl][t] - I.zh[sl][t] * irho;
                const V tn = sqrt(v[0] * v[0] + v[1] * v[1]);
                if (tn <= mu * v[2]) {
                    yv[0] = v[0]; yv[1] = v[1]; yv[2] = v[2];
                } else if (mu * tn <= -v[2]) {
                    yv[0] = yv[1] = yv[2] = V(0);
                } else {
                    const V nn = (mu * tn + v[2]) * V(c.mui[kc]);
                    const V sc = mu * nn / tn;
                    yv[0] = sc * v[0]; yv[1] = sc * v[1]; yv[2] = nn;
                }
                V ydz = V(0);
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const V xv = I.x[sl][t];
                    const V zv = I.zh[sl][t] - rho * (xv - yv[t]);
                    const V lin = I.Ax[sl][t] + I.b[sl][t];
                    lrp = fmax(lrp, fabs(xv - yv[t]));
                    lrd = fmax(lrd, fabs(eta * (xv - xprev[sl][t]) + rho * (yv[t] - I.yh[sl][t]) - lin));
                    lc += (zv - I.zh[sl][t]) * (zv - I.zh[sl][t]) * irho + rho * (yv[t] - I.yh[sl][t]) * (yv[t] - I.yh[sl][t]);
                    ydz += yv[t] * zv;
                    yn[sl][t] = yv[t];
                    zn[sl][t] = zv;
                }
                lrc = fmax(lrc, fabs(ydz));
            }
        }
        group_reduce4<V>(lrp, lrd, lrc, lc, red, ph++ & 1, g);
        rp = (double)lrp; rd = (double)lrd; rc = (double)lrc;
        converged = rp < tol && rd < tol && rc < tol;
        // -- Nesterov with adaptive restart (uniform decision), commit, next right-hand side
        double beta_n = 0.0;
        bool restart = false;
        if (nesterov) {
            if ((double)lc < 0.999 * mom.c_prev) {
                const double an = 0.5 * (1.0 + sqrt(1.0 + 4.0 * mom.a * mom.a));
                beta_n = (mom.a - 1.0) / an;
                mom.a = an;
                mom.c_prev = (double)lc;
            } else {
                restart = true;
                mom.a = 1.0;
                mom.c_prev = mom.c_prev / 0.999;
            }
        }
        const V bn = V(beta_n);
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const V yv = yn[sl][t], zv = zn[sl][t];
                if (!nesterov) { I.yh[sl][t] = yv; I.zh[sl][t] = zv; }
                else if (restart) { I.yh[sl][t] = I.y[sl][t]; I.zh[sl][t] = I.z[sl][t]; }
                else { I.yh[sl][t] = yv + bn * (yv - I.y[sl][t]); I.zh[sl][t] = zv + bn * (zv - I.z[sl][t]); }
                I.y[sl][t] = yv;
                I.z[sl][t] = zv;
            }
        cr_rhs<V, T, S>(c, g, I);
        if (converged) return false;
        if (switch64 && fmax(rp, rd) < KAMINO_REFINE64_BELOW) { ++it; return true; }
    }
    it = iters;
    return false;
}

// ncp_stop in the sparse formulation: the natural-map residual of the iterates' (lambda, u+) on the
// complementarity blocks, with y published to c.yout (FP64); true when it is below tol.
template <typename V, typename T, int S>
__device__ bool cr_ncp_ok(const CrWorld<T> &c, const Group &g, const CrIterates<V, S> &I, V *red, int &ph,
                          double tol) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = g.tid + sl * g.size;
        if (u >= c.nunits) continue;
        int r0, cnt;
        unit_rows(u, c.nbil, r0, cnt);
        for (int t = 0; t < cnt; ++t) c.yout[r0 + t] = (double)I.y[sl][t];
    }
    g.sync();
    ncp_velocities(c.ncw, g, c.yout, static_cast<const T *>(nullptr), c.fd);
    g.sync();
    return (double)ncp_natural_map(c.ncw, g, c.yout, static_cast<const T *>(nullptr), c.fd,
                                   reinterpret_cast<T *>(red), ph++ & 1) < tol;
}

// ncp_stop at tolerances of 1e-6 and above: the natural-map residual of ncp_natural_map evaluated in
// the iteration's own precision with the loop's machinery instead of FP64 (whose rate on this part
// makes the FP64 check cost more than an iteration): the owners publish w = P y, LB lanes per body
// gather M^-1 J^T w into fb, and the owners of the limit rows and contacts form
// v~ = v~_f + P J (M^-1 J^T P y) on their rows and the natural map.  Two barriers and one reduction;
// y from y64 when set.  The caller compares with a margin below tol for the FP32 rounding of v~.
// With `ust` set (the stall exit), also u+ = u_free + M^-1 J^T P y per body: `du` gets the largest
// change against the u+ stored in `ust` by the previous check, `umax` the largest |u+|, and `ust`
// the new u+.
template <typename T, int S>
__device__ T ncp_check_fast(const Group &g, int nunits, int nfix, int nbil, int nb, int LB, const int *bro,
                            const int *brow, const int *rbody, const T *rJ, const T *p, const T *mut,
                            const T *bminv, const T *bIinv, const double *vfd, const T *y, const double *y64,
                            T *w, T *fb, T *red, int phase, const T *bufree = nullptr, T *ust = nullptr,
                            T *du = nullptr, T *umax = nullptr) {
    const int tid = g.tid, nthr = g.size;
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = tid + sl * nthr;
        if (u >= nunits) continue;
        int r0, cnt;
        unit_rows(u, nbil, r0, cnt);
        for (int t = 0; t < cnt; ++t) w[r0 + t] = p[r0 + t] * (y64 ? T(y64[r0 + t]) : y[r0 + t]);
    }
    g.sync();
    for (int base = 0; base < nb * LB; base += nthr) {
        if (base + (tid & ~31) >= nb * LB) continue;
        const int t = base + tid, body = t / LB, sub = t - body * LB;
        const bool on = t < nb * LB;
        T f[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        if (on) {
            for (int e = bro[body] + sub; e < bro[body + 1]; e += LB) {
                const int code = brow[e];
                const T wr = w[code >> 1];
                const T *J = rJ + 6 * code;
#pragma unroll
                for (int k = 0; k < 6; ++k) f[k] = fma(J[k], wr, f[k]);
            }
        }
        for (int o = LB >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
        }
        if (on && sub == 0) {
            const T mi = bminv[body];
            for (int k = 0; k < 3; ++k) fb[6 * body + k] = mi * f[k];
            symvec3(bIinv + 6 * body, f + 3, fb + 6 * body + 3);
        }
    }
    g.sync();
    T lncp = T(0), ldu = T(0), lum = T(0);
    if (ust != nullptr) {
        for (int i = tid; i < nb; i += nthr)
            for (int k = 0; k < 6; ++k) {
                const T uk = bufree[6 * i + k] + fb[6 * i + k];
                ldu = fmax(ldu, fabs(uk - ust[6 * i + k]));
                lum = fmax(lum, fabs(uk));
                ust[6 * i + k] = uk;
            }
    }
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        const int u = tid + sl * nthr;
        if (u >= nunits || u < nfix) continue;
        int r0, cnt;
        unit_rows(u, nbil, r0, cnt);
        T vs[3], ls[3];
        for (int t = 0; t < cnt; ++t) {
            const int r = r0 + t, sa = rbody[2 * r], sb = rbody[2 * r + 1];
            const T *J = rJ + 12 * r;
            T acc = T(0);
            if (sa >= 0) for (int k = 0; k < 6; ++k) acc = fma(J[k], fb[6 * sa + k], acc);
            if (sb >= 0) for (int k = 0; k < 6; ++k) acc = fma(J[6 + k], fb[6 * sb + k], acc);
            vs[t] = T(vfd[r]) + p[r] * acc;
            ls[t] = y64 ? T(y64[r]) : y[r];
        }
        if (cnt == 1) {                       // joint-limit row: 0 <= lambda ⟂ v >= 0
            lncp = fmax(lncp, fabs(ls[0] - fmax(ls[0] - vs[0], T(0))));
            continue;
        }
        const T mu = mut[u - nbil];
        const T sv[3] = {ls[0] - vs[0], ls[1] - vs[1], ls[2] - (vs[2] + mu * sqrt(vs[0] * vs[0] + vs[1] * vs[1]))};
        const T tn = sqrt(sv[0] * sv[0] + sv[1] * sv[1]);
        T pr[3];
        if (tn <= mu * sv[2]) {
            pr[0] = sv[0]; pr[1] = sv[1]; pr[2] = sv[2];
        } else if (mu * tn <= -sv[2]) {
            pr[0] = pr[1] = pr[2] = T(0);
        } else {
            const T nn = (mu * tn + sv[2]) / (T(1) + mu * mu);
            pr[0] = mu * nn * sv[0] / tn; pr[1] = mu * nn * sv[1] / tn; pr[2] = nn;
        }
        for (int t = 0; t < 3; ++t) lncp = fmax(lncp, fabs(ls[t] - pr[t]));
    }
    T d2 = T(0);
    group_reduce4(lncp, ldu, lum, d2, red, phase, g);
    if (du) *du = ldu;
    if (umax) *umax = lum;
    return lncp;
}

// ----------------------------------------------------------------------------- the step kernel
// S: PADMM units per thread (units <= S * group size).  tbase: tensor-memory columns of the CTA
// (tm_cta: allocated by the kernel, whole-CTA group) that hold the inverse of worlds of up to 256
// padded rows.
template <typename T, int NB, int S, bool CR>
__device__ void world_step(const StepArgs<T> &a, int w, unsigned char *smem, const Group &g, uint32_t tbase,
                           bool tm_cta) {
    const int tid = g.tid, lane = g.lane(), warp = g.warp(), nthr = g.size, nwarps = g.warps();
    const ModelView<T> &M = a.m;
    const int4 wa = M.world_a[w], wb = M.world_b[w];
    const int b0 = wa.x, j0 = wa.y, c0 = wa.z, k0 = wa.w;
    const int nb = wb.x, nj = wb.y, nc = wb.z, nfix = wb.w;
    const int nlc = M.world_c ? M.world_c[w].x : 0;       // joint-limit candidates
    const Layout L = make_layout<T>(a.nb_max, a.nj_max, a.nc_max, a.mp_max, NB, a.nl_max, !CR);
    double *bq = (double *)(smem + L.bq);
    T *bu = (T *)(smem + L.bu), *bI = (T *)(smem + L.bI);
    double *bRd = (double *)(smem + L.bRd);
    T *bIinv = (T *)(smem + L.bIinv), *bminv = (T *)(smem + L.bminv), *bufree = (T *)(smem + L.bufree);
    T *jwr = (T *)(smem + L.jwr);
    int *cid = (int *)(smem + L.cid), *cslot = (int *)(smem + L.cslot), *rbody = (int *)(smem + L.rbody);
    T *rJ = (T *)(smem + L.rJ);
    double *rvs = (double *)(smem + L.rvs), *vfd = (double *)(smem + L.vfd), *lgap = (double *)(smem + L.lgap);
    T *rreg = (T *)(smem + L.rreg), *lJ = (T *)(smem + L.lJ);
    int *lrank = (int *)(smem + L.lrank), *lcid = (int *)(smem + L.lcid);
    T *p = (T *)(smem + L.p), *x = (T *)(smem + L.x), *xn = (T *)(smem + L.xn);
    T *y = (T *)(smem + L.y), *z = (T *)(smem + L.z), *yh = (T *)(smem + L.yh), *zh = (T *)(smem + L.zh);
    T *bb = (T *)(smem + L.b), *mut = (T *)(smem + L.mut), *X = (T *)(smem + L.X), *A = (T *)(smem + L.A);
    T *mui = (T *)(smem + L.mui);
    T *red = (T *)(smem + L.red);
    int *misc = (int *)(smem + L.misc);
    T *wv = (T *)(smem + L.wv), *fb = (T *)(smem + L.fb);
    int *bro = (int *)(smem + L.bro), *brow = (int *)(smem + L.brow);
    const T dt = a.dt, kbias = a.beta / a.dt;
    const double dtd = (double)a.dt, kbiasd = (double)a.beta / (double)a.dt;
    if (tid == 0) misc[1] = 0;   // failure bits of this world: 1 non-finite result, 2 tensor-core timeout
    for (int r = tid; r < a.mp_max; r += nthr) rreg[r] = T(0);
    // ---- 1. body kinematics
    for (int i = tid; i < nb; i += nthr) {
        const T *gq = a.body_q + 7 * (size_t)(b0 + i);
        const T *gu = a.body_u + 6 * (size_t)(b0 + i);
        double pose[7] = {(double)gq[0], (double)gq[1], (double)gq[2], (double)gq[3], (double)gq[4], (double)gq[5],
                          (double)gq[6]};
        const double qn = 1.0 / sqrt(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
        for (int k = 3; k < 7; ++k) pose[k] *= qn;
        if (a.midpoint) {
            // Moreau-Jean (Sec. 3): the step is evaluated at the half-step pose q_m = q (+) (dt/2) u-
            const double v[3] = {(double)gu[0], (double)gu[1], (double)gu[2]};
            const double om[3] = {(double)gu[3], (double)gu[4], (double)gu[5]};
            double pm[7];
            pose_advance(pose, v, om, 0.5 * dtd, pm);
            for (int k = 0; k < 7; ++k) pose[k] = pm[k];
        }
        for (int k = 0; k < 7; ++k) bq[7 * i + k] = pose[k];
        const double *qd = pose + 3;
        for (int k = 0; k < 6; ++k) bu[6 * i + k] = gu[k];
        double Rd[9];
        quat_rot(qd, Rd);
        T R[9];
        for (int k = 0; k < 9; ++k) { bRd[9 * i + k] = Rd[k]; R[k] = T(Rd[k]); }
        const T m = M.body_mass[b0 + i];
        T inv[3];
        for (int k = 0; k < 3; ++k) {
            const T Ik = M.body_inertia[3 * (size_t)(b0 + i) + k];
            bI[3 * i + k] = Ik;
            inv[k] = T(1) / Ik;
        }
        // R diag(1/I) R^T, symmetric (xx, yy, zz, xy, xz, yz)
        T *Sw = bIinv + 6 * i;
        const int rr[6] = {0, 1, 2, 0, 0, 1}, cc[6] = {0, 1, 2, 1, 2, 2};
        for (int k = 0; k < 6; ++k) {
            const int r = rr[k], c = cc[k];
            Sw[k] = R[3 * r] * inv[0] * R[3 * c] + R[3 * r + 1] * inv[1] * R[3 * c + 1] + R[3 * r + 2] * inv[2] * R[3 * c + 2];
        }
        bminv[i] = T(1) / m;
    }
    g.sync();

    // ---- 2. joint rows and actuation wrenches (thread per joint), then the joint-space dynamics:
    // a drive row per driven joint, the gap of every joint-limit candidate; 3. contacts (last warp,
    // concurrently with the joints unless limit rows must be placed first)
    for (int j = tid; j < nj; j += nthr) {
        const int4 meta = M.joint_meta[j0 + j];
        const double *dyn = M.joint_dyn ? M.joint_dyn + 8 * (size_t)(j0 + j) : nullptr;
        const bool pd = dyn != nullptr && dyn[0] == 1.0;         // the actuation is this drive's target
        const bool act = meta.w >= 0 && a.tau != nullptr && !pd;
        const T val = act ? a.tau[(size_t)w * M.n_act_max + meta.w] : T(0);
        const double *fr = M.joint_frames + 14 * (size_t)(j0 + j);
        joint_rows(meta.x, meta.y, meta.z, fr, bq, bRd, M.joint_row[j0 + j], kbiasd, rbody, rJ, rvs, act, val,
                   jwr + 12 * j);
        const int drow = M.joint_drow ? M.joint_drow[j0 + j] : -1;
        int ls = M.joint_lslot ? M.joint_lslot[j0 + j] : -1;
        if (drow >= 0 || ls >= 0) {
            double d, Ja[6], Jb[6];
            joint_coordinate(meta.x, meta.y, meta.z, fr, bq, bRd, &d, Ja, Jb);
            if (drow >= 0) {
                // implicit PD, armature and damping as one regularised row (Sec. 3, Eq. 2's R and v*):
                // lambda = I_a (d'- - d'+) + dt Kp (target - d - dt d'+) - dt (Kd + b) d'+
                double ddot = 0.0;
                for (int k = 0; k < 6; ++k) {
                    ddot += Jb[k] * (double)bu[6 * meta.z + k];
                    if (meta.y >= 0) ddot += Ja[k] * (double)bu[6 * meta.y + k];
                }
                const double kp = pd ? dyn[1] : 0.0, kd = pd ? dyn[2] : 0.0, arm = dyn[3], damp = dyn[4];
                const double target = (pd && a.tau != nullptr && meta.w >= 0)
                                          ? (double)a.tau[(size_t)w * M.n_act_max + meta.w] : d;
                const double C = arm + dtd * dtd * kp + dtd * (kd + damp);
                put_row(rbody, rJ, rvs, drow, meta.y, meta.z, Ja, Jb, -(arm * ddot + dtd * kp * (target - d)) / C);
                rreg[drow] = T(1.0 / C);
            }
            if (ls >= 0) {
                // unilateral rows g = d - lower >= 0 and g = upper - d >= 0 on the joint coordinate
                for (int side = 0; side < 2; ++side) {
                    const double bound = dyn[5 + side];
                    if (!isfinite(bound)) continue;
                    const double sg = side == 0 ? 1.0 : -1.0;
                    lgap[ls] = sg * (d - bound);
                    for (int k = 0; k < 6; ++k) { lJ[12 * ls + k] = T(sg * Ja[k]); lJ[12 * ls + 6 + k] = T(sg * Jb[k]); }
                    lrank[ls] = j;
                    ++ls;
                }
            }
        }
    }
    int nbil = nfix;                 // rows before the contacts: fixed rows, then the active limits
    if (nlc > 0) {
        g.sync();
        if (warp == 0) {             // active limit candidates (gap below the margin), in candidate order
            int count = 0;
            for (int cb = 0; cb < nlc; cb += 32) {
                const int s = cb + lane;
                const double gap = s < nlc ? lgap[s] : 0.0;
                const bool active = s < nlc && gap < (double)a.margin;
                const unsigned mask = __ballot_sync(0xffffffffu, active);
                const int rank = count + __popc(mask & ((1u << lane) - 1u));
                if (active) {
                    const int4 meta = M.joint_meta[j0 + lrank[s]];
                    double Ja[6], Jb[6];
                    for (int k = 0; k < 6; ++k) { Ja[k] = (double)lJ[12 * s + k]; Jb[k] = (double)lJ[12 * s + 6 + k]; }
                    // the gap may close within the step (g/dt while g > 0); a violation goes at
                    // Baumgarte's rate (beta g/dt), as a contact's normal row
                    put_row(rbody, rJ, rvs, nfix + rank, meta.y, meta.z, Ja, Jb, gap > 0.0 ? gap / dtd : kbiasd * gap);
                    lcid[rank] = s;
                }
                if (s < nlc) lrank[s] = active ? rank : -1;
                count += __popc(mask);
            }
            if (lane == 0) misc[5] = count;
        }
        g.sync();
        nbil = nfix + misc[5];
    }
    if (warp == nwarps - 1) {
        int count = 0;
        for (int cb = 0; cb < nc; cb += 32) {
            const int c = cb + lane;
            bool active = false;
            double pw[3], n[3], phi = 0.0, rb[3];
            int body = 0;
            if (c < nc && M.terrain_kind != KAMINO_TERRAIN_NONE) {
                body = M.contact_body[c0 + c];
                const double *cp = M.contact_point + 3 * (size_t)(c0 + c);
                double wc[3];
                matvec3(bRd + 9 * body, cp, wc);
                for (int k = 0; k < 3; ++k) { rb[k] = bq[7 * body + k]; pw[k] = rb[k] + wc[k]; }
                phi = terrain(M, pw, n);
                active = phi < (double)a.margin;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, active);
            const int rank = count + __popc(mask & ((1u << lane) - 1u));
            if (c < nc) cslot[c] = active ? rank : -1;
            if (active) {
                cid[rank] = c;
                double t1[3], t2[3], lev[3], Ja[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, Jb[6], cr[3];
                onb(n, t1, t2);
                for (int k = 0; k < 3; ++k) lev[k] = pw[k] - rb[k];
                const double *dirs[3] = {t1, t2, n};
                const int row0 = nbil + 3 * rank;
                for (int d = 0; d < 3; ++d) {
                    cross3(lev, dirs[d], cr);
                    for (int k = 0; k < 3; ++k) { Jb[k] = dirs[d][k]; Jb[3 + k] = cr[k]; }
                    const double vs = d < 2 ? 0.0 : (phi > 0.0 ? phi / dtd : kbiasd * phi);
                    put_row(rbody, rJ, rvs, row0 + d, -1, body, Ja, Jb, vs);
                }
            }
            count += __popc(mask);
        }
        if (lane == 0) misc[0] = count;
    }
    g.sync();
    const int nact = misc[0];
    const int m = nbil + 3 * nact;
    const int mp = ((m + 15) / 16) * 16;
    const int nunits = nbil + nact;

    // ---- 4. u_free = u + dt M^-1 h
    for (int i = tid; i < nb; i += nthr) {
        T f[3] = {M.gx * (T(1) / bminv[i]), M.gy * (T(1) / bminv[i]), M.gz * (T(1) / bminv[i])};
        T tq[3] = {T(0), T(0), T(0)};
        for (int j = 0; j < nj; ++j) {
            const int4 meta = M.joint_meta[j0 + j];
            if (meta.w < 0 || a.tau == nullptr) continue;
            const T *wr = jwr + 12 * j;
            if (meta.y == i) for (int k = 0; k < 3; ++k) { f[k] += wr[k]; tq[k] += wr[3 + k]; }
            if (meta.z == i) for (int k = 0; k < 3; ++k) { f[k] += wr[6 + k]; tq[k] += wr[9 + k]; }
        }
        // gyroscopic: -w x (I_w w), I_w w = R (I o (R^T w))
        const T *om = bu + 6 * i + 3;
        T wbody[3], Iw[3], Iww[3], gy[3];
        T Ri[9];
        for (int k = 0; k < 9; ++k) Ri[k] = T(bRd[9 * i + k]);
        matTvec3(Ri, om, wbody);
        for (int k = 0; k < 3; ++k) Iw[k] = bI[3 * i + k] * wbody[k];
        matvec3(Ri, Iw, Iww);
        cross3(om, Iww, gy);
        for (int k = 0; k < 3; ++k) tq[k] -= gy[k];
        T dw[3];
        symvec3(bIinv + 6 * i, tq, dw);
        for (int k = 0; k < 3; ++k) {
            bufree[6 * i + k] = bu[6 * i + k] + dt * bminv[i] * f[k];
            bufree[6 * i + 3 + k] = bu[6 * i + 3 + k] + dt * dw[k];
        }
    }
    g.sync();

    // ---- 5a. per row: M^-1 J^T blocks (into X), diag(D), v_f
    T *MJ = X;
    for (int r = tid; r < m; r += nthr) {
        const int ba = rbody[2 * r], bbd = rbody[2 * r + 1];
        const T *J = rJ + 12 * r;
        T d = T(0);
        double v = rvs[r];       // v_f in FP64 (see the layout): J u_free + v*
        for (int s = 0; s < 2; ++s) {
            const int body = s == 0 ? ba : bbd;
            T *o = MJ + 12 * r + 6 * s;
            if (body < 0) { for (int k = 0; k < 6; ++k) o[k] = T(0); continue; }
            const T *Js = J + 6 * s;
            for (int k = 0; k < 3; ++k) o[k] = bminv[body] * Js[k];
            symvec3(bIinv + 6 * body, Js + 3, o + 3);
            for (int k = 0; k < 6; ++k) { d += Js[k] * o[k]; v = fma((double)Js[k], (double)bufree[6 * body + k], v); }
        }
        x[r] = d + rreg[r];      // diag(D + R) of Eq. 4, temporarily
        vfd[r] = v;
    }
    g.sync();
    // ---- 5b. Jacobi scaling (tangent rows of a contact share one scale), scaled mu, scaled v_f
    for (int r = tid; r < mp; r += nthr) {
        T pr = T(1);
        if (r < m && a.precond) {
            if (r < nbil) {
                pr = rsq(x[r]);
            } else {
                const int k = (r - nbil) / 3, t = (r - nbil) % 3;
                const int rt = nbil + 3 * k;
                pr = t < 2 ? rsq(T(0.5) * (x[rt] + x[rt + 1])) : rsq(x[r]);
            }
        }
        p[r] = pr;
    }
    g.sync();
    for (int r = tid; r < mp; r += nthr) {
        vfd[r] = r < m ? (double)p[r] * vfd[r] : 0.0;
        if constexpr (!CR) bb[r] = T(0);
    }
    for (int k = tid; k < nact; k += nthr) {
        const int rt = nbil + 3 * k;
        mut[k] = M.world_mu[w] * p[rt + 2] / p[rt];
        mui[k] = T(1) / (T(1) + mut[k] * mut[k]);
    }
    const NcpWorld<T> ncw{nb, nfix, nbil, nact, bro, brow, rbody, rJ, p, mut, bminv, bIinv, bufree, rvs};
    double *yfin = nullptr;   // the final y in FP64 when the iterates ended in FP64 (or the sparse formulation)
    double *fd = nullptr;     // FP64 scratch of 6 nb words for phase 9
    T rp = T(INFINITY), rd = T(INFINITY), rc = T(INFINITY);
    int it = 0;
    bool converged = false, stalled = false;
    if constexpr (CR) {
        // ---- 5c'-8'. Sparse formulation (Sec. 5.1): no matrix, no factorisation; Alg. 1 with every
        // x-step k Conjugate Residual iterations on the matrix-free operator (see cr_padmm)
        g.sync();
        body_row_lists(g, nb, m, rbody, bro, brow);
        int LB = 8;               // lanes per body in the gather: a power of two with LB * nb <= group size
        while (LB > 1 && LB * nb > nthr) LB >>= 1;
        // the assembly scratch X is dead: the final y (FP64), then w and g, both sized for FP64
        double *y64c = reinterpret_cast<double *>(X);
        double *wbuf = y64c + a.mp_max;
        double *gbuf = wbuf + a.mp_max;
        const CrWorld<T> cw{nunits, nfix, nbil, nb, LB, bro, brow, rbody, rJ, p, rreg, bminv, bIinv, mut, mui,
                            vfd, T(a.eta + a.rho), a.eta, a.rho, a.ncp_stop, ncw, y64c, gbuf};
        // ---- 6'. warm start in the owners' registers: x0 = y0 = P^-1 lambda0, z0 = v0 + Gamma(v0),
        // v0 = A x0 - (eta + rho) x0 + v~_f
        CrIterates<T, S> I;
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
#pragma unroll
            for (int t = 0; t < 3; ++t)
                I.x[sl][t] = I.y[sl][t] = I.z[sl][t] = I.yh[sl][t] = I.zh[sl][t] = I.b[sl][t] = I.Ax[sl][t] = T(0);
        const bool warm = a.warm_mode != KAMINO_WARM_COLD;
        const T *src = !warm ? nullptr : a.warm_mode == KAMINO_WARM_EXTERNAL ? a.warm : a.cache;
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
            const int u = tid + sl * nthr;
            if (u >= nunits || src == nullptr) continue;
            int r0, cnt;
            unit_rows(u, nbil, r0, cnt);
            for (int t = 0; t < cnt; ++t) {   // cache layout: fixed rows, limit candidates, 3 per contact candidate
                const int r = r0 + t;
                T l0;
                if (r < nfix) l0 = src[k0 + r];
                else if (r < nbil) l0 = src[k0 + nfix + lcid[r - nfix]];
                else l0 = src[k0 + nfix + nlc + 3 * cid[u - nbil] + t];
                I.x[sl][t] = l0 / p[r];
            }
        }
        if (warm) {
            cr_apply<T, T, S>(cw, g, I.x, I.Ax, reinterpret_cast<T *>(wbuf), reinterpret_cast<T *>(gbuf));
            const T shift = T(a.eta + a.rho);
#pragma unroll
            for (int sl = 0; sl < S; ++sl) {
                const int u = tid + sl * nthr;
                if (u >= nunits) continue;
                int r0, cnt;
                unit_rows(u, nbil, r0, cnt);
                T v0[3] = {T(0), T(0), T(0)};
                for (int t = 0; t < cnt; ++t) v0[t] = I.Ax[sl][t] - shift * I.x[sl][t] + T(vfd[r0 + t]);
                for (int t = 0; t < cnt; ++t) I.z[sl][t] = v0[t];
                if (cnt == 3) I.z[sl][2] += mut[u - nbil] * sqrt(v0[0] * v0[0] + v0[1] * v0[1]);
            }
        }
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                I.y[sl][t] = I.yh[sl][t] = I.x[sl][t];
                I.zh[sl][t] = I.z[sl][t];
            }
        cr_rhs<T, T, S>(cw, g, I);
        // ---- 8'. Alg. 1, then (refine64, tolerances below KAMINO_REFINE64_BELOW) the same iterations
        // in FP64 from the moment r_p and r_d fall below that level
        CrMomentum mom{1.0, (double)INFINITY};
        int ph = 0;
        double rpd = INFINITY, rdd = INFINITY, rcd = INFINITY;
        it = 1;
        const bool use64 = sizeof(T) == 4 && a.refine64 && a.tol < T(KAMINO_REFINE64_BELOW);
        bool sw = false;
        for (;;) {   // the iterations, then (ncp_stop) the natural-map check, resumed if it fails
            sw = cr_padmm<T, T, S>(cw, g, I, reinterpret_cast<T *>(wbuf), reinterpret_cast<T *>(gbuf),
                                   reinterpret_cast<T *>(red), ph, it, a.iters, a.cr_iters, (double)a.tol,
                                   a.nesterov != 0, mom, rpd, rdd, rcd, converged, use64);
            if (sw || !(converged && a.ncp_stop)) break;
            converged = cr_ncp_ok<T, T, S>(cw, g, I, reinterpret_cast<T *>(red), ph, (double)a.tol);
            if (converged || it >= a.iters) break;
            ++it;
        }
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (sw) {
                CrIterates<double, S> D;
#pragma unroll
                for (int sl = 0; sl < S; ++sl)
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        D.x[sl][t] = I.x[sl][t]; D.y[sl][t] = I.y[sl][t]; D.z[sl][t] = I.z[sl][t];
                        D.yh[sl][t] = I.yh[sl][t]; D.zh[sl][t] = I.zh[sl][t]; D.b[sl][t] = 0.0;
                    }
                cr_rhs<double, T, S>(cw, g, D);                      // from the FP64 v_f
                cr_apply<double, T, S>(cw, g, D.x, D.Ax, wbuf, gbuf);
                for (;;) {
                    cr_padmm<double, T, S>(cw, g, D, wbuf, gbuf, reinterpret_cast<double *>(red), ph, it, a.iters,
                                           a.cr_iters, (double)a.tol, a.nesterov != 0, mom, rpd, rdd, rcd, converged,
                                           false);
                    if (!(converged && a.ncp_stop)) break;
                    converged = cr_ncp_ok<double, T, S>(cw, g, D, reinterpret_cast<double *>(red), ph, (double)a.tol);
                    if (converged || it >= a.iters) break;
                    ++it;
                }
#pragma unroll
                for (int sl = 0; sl < S; ++sl) {
                    const int u = tid + sl * nthr;
                    if (u >= nunits) continue;
                    int r0, cnt;
                    unit_rows(u, nbil, r0, cnt);
                    for (int t = 0; t < cnt; ++t) y64c[r0 + t] = D.y[sl][t];
                }
                done = true;
            }
        }
        if (!done) {
#pragma unroll
            for (int sl = 0; sl < S; ++sl) {
                const int u = tid + sl * nthr;
                if (u >= nunits) continue;
                int r0, cnt;
                unit_rows(u, nbil, r0, cnt);
                for (int t = 0; t < cnt; ++t) y64c[r0 + t] = (double)I.y[sl][t];
            }
        }
        rp = T(rpd); rd = T(rdd); rc = T(rcd);
        yfin = y64c;
        fd = gbuf;
    } else {
        // ---- 5c. A = P (D + R) P + (eta + rho) I in packed storage (identity on the padding rows)
        const T shift = a.eta + a.rho;
        for (int j = warp; j < mp; j += nwarps) {
            T *col = A + col_start(j, mp) - j;
            const int ja = j < m ? rbody[2 * j] : -2, jb = j < m ? rbody[2 * j + 1] : -2;
            for (int i = j + lane; i < mp; i += 32) {
                T v;
                if (i >= m || j >= m) {
                    v = i == j ? T(1) : T(0);
                } else {
                    const int ia = rbody[2 * i], ib = rbody[2 * i + 1];
                    const T *Ji = rJ + 12 * i;
                    const T *Mj = MJ + 12 * j;
                    T s = T(0);
                    if (ia >= 0 && ia == ja) for (int k = 0; k < 6; ++k) s += Ji[k] * Mj[k];
                    if (ia >= 0 && ia == jb) for (int k = 0; k < 6; ++k) s += Ji[k] * Mj[6 + k];
                    if (ib == ja) for (int k = 0; k < 6; ++k) s += Ji[6 + k] * Mj[k];
                    if (ib == jb) for (int k = 0; k < 6; ++k) s += Ji[6 + k] * Mj[6 + k];
                    v = p[i] * p[j] * s + (i == j ? shift + p[i] * p[i] * rreg[i] : T(0));
                }
                col[i] = v;
            }
        }
        g.sync();

        // ---- 6. warm start: x0 = y0 = P^-1 lambda0, z0 = v0 + Gamma(v0), v0 = D~ x0 + v~_f
        const bool warm = a.warm_mode != KAMINO_WARM_COLD;
        for (int r = tid; r < mp; r += nthr) {
            T l0 = T(0);
            if (warm && r < m) {
                const T *src = a.warm_mode == KAMINO_WARM_EXTERNAL ? a.warm : a.cache;
                if (src) {   // cache layout: fixed rows, limit candidates, 3 per contact candidate
                    if (r < nfix) l0 = src[k0 + r];
                    else if (r < nbil) l0 = src[k0 + nfix + lcid[r - nfix]];
                    else {
                        const int k = (r - nbil) / 3, t = (r - nbil) % 3;
                        l0 = src[k0 + nfix + nlc + 3 * cid[k] + t];
                    }
                }
            }
            x[r] = l0 / p[r];
        }
        g.sync();
        if (warm) {
            symv_packed(A, mp, x, xn, X, g);          // xn = A x0 = D~ x0 + (eta + rho) x0
            for (int u = tid; u < nunits; u += nthr) {
                if (u < nbil) {
                    const T v0 = xn[u] - shift * x[u] + T(vfd[u]);
                    z[u] = v0;
                } else {
                    const int r0 = nbil + 3 * (u - nbil);
                    T v0[3];
                    for (int t = 0; t < 3; ++t) v0[t] = xn[r0 + t] - shift * x[r0 + t] + T(vfd[r0 + t]);
                    z[r0] = v0[0]; z[r0 + 1] = v0[1];
                    z[r0 + 2] = v0[2] + mut[u - nbil] * sqrt(v0[0] * v0[0] + v0[1] * v0[1]);
                }
            }
            g.sync();   // z of a contact is written by the unit's owner and read below row by row
        }
        for (int r = tid; r < mp; r += nthr) {
            if (!warm || r >= m) z[r] = T(0);
            y[r] = x[r]; yh[r] = x[r]; zh[r] = z[r];
        }
        g.sync();

        // ---- 7. A <- -A^-1 (blocked sweep): in tensor memory (mixed mode, whole CTA, mp <= 256), else
        // on the packed triangle in shared memory, then stored into tensor memory (FP32 mode, whole
        // CTA) or re-stored as BF16 tiles (mixed mode otherwise); per-body row lists for the
        // matrix-free products
        const bool tm = tm_cta && mp <= 256;
        bool in_tmem = false;                 // the inverse is already in tensor memory
        if constexpr (sizeof(T) == 4 && NB == 16) {
            // the two K-major panels (256 rows x 16) and the pivot block must fit the scratch X
            if (tm && a.mixed && L.A - L.X >= (size_t)(2 * 256 * 16 + 256) * sizeof(float)) {
                if (!sweep_inverse_tmem(A, mp, X, tbase, misc, g)) {
                    // the tensor cores did not complete: report the world, leave its state as it was
                    if (tid == 0) {
                        kamino_residual rep{};
                        rep.iterations = 0;
                        rep.status = KAMINO_WORLD_NOT_CONVERGED | KAMINO_WORLD_TIMEOUT;
                        rep.num_rows = m;
                        rep.num_contacts = nact;
                        rep.r_primal = rep.r_dual = rep.r_compl = rep.r_ncp = INFINITY;
                        a.res[w] = rep;
                    }
                    g.sync();
                    return;
                }
                in_tmem = true;
            }
        }
        if (!in_tmem) sweep_inverse<T, NB>(A, mp, X, a.mixed != 0, g);
        if constexpr (sizeof(T) == 4) {
            if (tm && !in_tmem) tmem_store_inverse(A, mp, tbase, g);
        }
        if (a.mixed && !tm) pack_bf16_tiles(A, mp, X, g);
        body_row_lists(g, nb, m, rbody, bro, brow);

        // ---- 8. Proximal-ADMM (Alg. 1).  The linear solve of every iteration is one step of
        // iterative refinement from the previous x:  x^i = x^{i-1} - A^-1 (b + A x^{i-1}), with A x
        // evaluated matrix-free from the rows (P J M^-1 J^T P x + (eta + rho) x) and A^-1 the swept
        // inverse.  At a fixed point A x = -b holds to the accuracy of the matrix-free product, so the
        // inverse's own rounding (which the nearly singular D~ would amplify) does not move the
        // solution.  With refine64, once r_p and r_d fall below KAMINO_REFINE64_BELOW the refinement
        // end game runs in FP64: the right-hand side b (from the FP64 v_f), the per-body velocities
        // M^-1 J^T P x and the residual b + A x are formed in FP64, and the iterates x, y, z, y^, z^
        // themselves are kept in FP64 (in shared memory that is dead during the loop), as in iterative
        // refinement whose solution is accumulated in the higher precision: an FP32 iterate cannot hold
        // the solution of these mechanisms closer than ~1e-4 in u+ (u+ is a small difference of large
        // joint impulses through light bodies).  The correction S (b + A x) stays on the FP32 / BF16
        // inverse.
        //
        // Unit u (a joint row, or the three rows of a contact) belongs to thread u mod group size for
        // the whole solve: only its owner writes its x, b, y, z, y^, z^ (the residual rows read x and b
        // row by row after a barrier), so an iteration has four barriers (after the per-body gather,
        // after the residual rows, after the mat-vec, and the residual reduction, which also publishes
        // x, P x and b).
        const T eta = a.eta, rho = a.rho, irho = T(1) / a.rho;
        double *bbd = reinterpret_cast<double *>(X + kWarps * mp);   // FP32 worlds only (make_layout)
        double *gbd = bbd + mp;
        __nv_bfloat16 *chi = reinterpret_cast<__nv_bfloat16 *>(X), *clo = chi + mp;   // mixed: split c
        // the FP64 end game only matters below the FP32 residual floor, i.e. for tolerances under the
        // switch level
        const bool use64 = sizeof(T) == 4 && a.refine64 && a.tol < T(KAMINO_REFINE64_BELOW);
        double *x64 = nullptr;
        if (use64) x64 = fp64_iterates(smem, L, tm, a.mixed && !tm, mp, nb, X);
        double *y64 = x64 + mp, *z64 = x64 + 2 * mp, *yh64 = x64 + 3 * mp, *zh64 = x64 + 4 * mp;
        double *yn64 = x64 + 5 * mp, *zn64 = x64 + 6 * mp;
        bool hp = false;     // b of the coming iteration is the FP64 one; set once, uniform over the group
        bool hpv = false;    // the iterates live in the FP64 vectors (from the commit after hp is set)
        bool x_in64 = false; // the last owner update wrote x to the FP64 vector
        int LB = 8;          // lanes per body in the gather: a power of two with LB * nb <= group size
        while (LB > 1 && LB * nb > nthr) LB >>= 1;
        // Loop invariants in registers, so that an iteration's loads depend on nothing but the
        // iterates: the row codes of this gather lane (when one pass covers the bodies and the lane
        // has at most kGatherRows rows; gcnt < 0 otherwise) and, for the residual row r = tid, its
        // bodies, its scaling and its diagonal shift + p^2 R.
        constexpr int kGatherRows = 6;
        int gcode[kGatherRows];
        int gcnt = -1;
        g.sync();            // the row lists are complete (each body's list is written by one thread)
        if (nb * LB <= nthr) {
            const int body = tid / LB, sub = tid - body * LB;
            const int e0 = tid < nb * LB ? bro[body] + sub : 0, e1 = tid < nb * LB ? bro[body + 1] : 0;
            const int n = e1 > e0 ? (e1 - e0 + LB - 1) / LB : 0;
#pragma unroll
            for (int k = 0; k < kGatherRows; ++k) gcode[k] = k < n ? brow[e0 + k * LB] : 0;
            gcnt = n <= kGatherRows ? n : -1;
        }
        int rsa = -1, rsb = -1;
        T rpr = T(0), rdiag = T(0);
        if (tid < m) {
            rsa = rbody[2 * tid];
            rsb = rbody[2 * tid + 1];
            rpr = p[tid];
            rdiag = shift + p[tid] * p[tid] * rreg[tid];
        }
        T acc_a = T(1), c_prev = T(INFINITY);
        // v_f of the owner's rows in the iteration's precision, in registers for the whole loop (the
        // conversion from the FP64 v_f would otherwise run on the slow FP64 pipe every iteration)
        // contacts owned from the first warp boundary after the joint rows when the slots have room
        const int cslot0 = ((nbil + 31) & ~31) + (nunits - nbil) <= S * nthr ? ((nbil + 31) & ~31) : nbil;
        T vfo[S][3];
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
            const int u = slot_unit(tid + sl * nthr, nbil, cslot0);
            const int r0 = u < nbil ? u : nbil + 3 * (u - nbil), cnt = u >= nunits ? 0 : u < nbil ? 1 : 3;
#pragma unroll
            for (int t = 0; t < 3; ++t) vfo[sl][t] = t < cnt ? T(vfd[r0 + t]) : T(0);
        }
        // b = v_f + Gamma(z^) - eta x - rho y^ - z^ and w = P x for the first iteration (by the owners)
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
            const int u = slot_unit(tid + sl * nthr, nbil, cslot0);
            if (u >= nunits) continue;
            if (u < nbil) {
                bb[u] = T(vfd[u]) - eta * x[u] - rho * yh[u] - zh[u];
                wv[u] = p[u] * x[u];
            } else {
                const int r0 = nbil + 3 * (u - nbil);
                const T s = mut[u - nbil] * sqrt(zh[r0] * zh[r0] + zh[r0 + 1] * zh[r0 + 1]);
                for (int t = 0; t < 3; ++t) {
                    bb[r0 + t] = T(vfd[r0 + t]) + (t == 2 ? s : T(0)) - eta * x[r0 + t] - rho * yh[r0 + t] - zh[r0 + t];
                    wv[r0 + t] = p[r0 + t] * x[r0 + t];
                }
            }
        }
        if (a.mixed && !tm) {
            for (int r = m + tid; r < mp; r += nthr) {
                chi[r] = __float2bfloat16(0.0f);
                clo[r] = __float2bfloat16(0.0f);
            }
        }
        // this thread's b of the coming iteration (its own rows, written just above), for the
        // iterations that take c = b^i - b^{i-1} (residual_every > 1)
        T bprev[S][3];
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
            const int u = slot_unit(tid + sl * nthr, nbil, cslot0);
            const int r0 = u < nbil ? u : nbil + 3 * (u - nbil), cnt = u >= nunits ? 0 : u < nbil ? 1 : 3;
#pragma unroll
            for (int t = 0; t < 3; ++t) bprev[sl][t] = t < cnt ? bb[r0 + t] : T(0);
        }
        // BF16 inverse tiles (mixed mode outside tensor memory) are lagged 4 iterations at most: their
        // larger error, accumulated over a longer lag, costs short solves iterations
        const int kres = a.mixed && !tm ? min(a.residual_every, 4) : a.residual_every;
        bool lagged = false;     // this iteration takes c = b^i - b^{i-1} (stored by the last commit)
        g.sync();
        // The iterations run until Sec. 4.1's test passes; with ncp_stop the natural-map check follows
        // outside the loop (kept out of the loop body, which it would otherwise make slower) and the
        // iterations resume if it fails.
        it = 1;
        bool stall_due = false, stall_prev = false;
        T *ust = (T *)(smem + L.ust);
        for (;;) {
        for (; it <= a.iters; ++it) {
            if (lagged) {
                // c = b^i - b^{i-1} was stored by the owners' commit: publish it to the mat-vec
                g.sync();
            } else {
            // [8a] per body: g_b = M_b^-1 sum over the body's rows r of J_rb^T (P x)_r; LB lanes per
            // body take its rows round-robin, then a shuffle reduction
            for (int base = 0; base < nb * LB; base += nthr) {
                if (base + (tid & ~31) >= nb * LB) continue;          // the whole warp is past the bodies
                const int t = base + tid, body = t / LB, sub = t - body * LB;
                const bool on = t < nb * LB;
                if (hp) {
                    double f[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                    if (on) {
                        for (int e = bro[body] + sub; e < bro[body + 1]; e += LB) {
                            const int code = brow[e], r = code >> 1;
                            const double w = (double)p[r] * (x_in64 ? x64[r] : (double)x[r]);
                            const T *J = rJ + 6 * code;                 // 12 r + 6 side
    #pragma unroll
                            for (int k = 0; k < 6; ++k) f[k] = fma((double)J[k], w, f[k]);
                        }
                    }
                    for (int o = LB >> 1; o > 0; o >>= 1) {
    #pragma unroll
                        for (int k = 0; k < 6; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
                    }
                    if (on && sub == 0) {
                        const double mi = bminv[body];
                        for (int k = 0; k < 3; ++k) gbd[6 * body + k] = mi * f[k];
                        symvec3d(bIinv + 6 * body, f + 3, gbd + 6 * body + 3);
                    }
                } else {
                    T f[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                    if (gcnt >= 0) {
    #pragma unroll
                        for (int q = 0; q < kGatherRows; ++q) {
                            if (q >= gcnt) break;
                            const int code = gcode[q];
                            const T w = wv[code >> 1];
                            T Jv[6];
                            load6(rJ + 6 * code, Jv);
    #pragma unroll
                            for (int k = 0; k < 6; ++k) f[k] = fma(Jv[k], w, f[k]);
                        }
                    } else if (on) {
                        for (int e = bro[body] + sub; e < bro[body + 1]; e += LB) {
                            const int code = brow[e];
                            const T w = wv[code >> 1];
                            T Jv[6];
                            load6(rJ + 6 * code, Jv);
    #pragma unroll
                            for (int k = 0; k < 6; ++k) f[k] = fma(Jv[k], w, f[k]);
                        }
                    }
                    for (int o = LB >> 1; o > 0; o >>= 1) {
    #pragma unroll
                        for (int k = 0; k < 6; ++k) f[k] += __shfl_xor_sync(0xffffffffu, f[k], o);
                    }
                    if (on && sub == 0) {
                        const T mi = bminv[body];
                        for (int k = 0; k < 3; ++k) fb[6 * body + k] = mi * f[k];
                        symvec3(bIinv + 6 * body, f + 3, fb + 6 * body + 3);
                    }
                }
            }
            g.sync();
            // [8b] thread r: c_r = b_r + p_r J_r (g_A, g_B) + (eta + rho) x_r (b_r and x_r were written by
            // the row's owner before the last barrier), stored as the BF16 hi / lo split (mixed, inverse
            // in shared memory) or in bb (tensor-memory, FP32 and FP64 mat-vecs)
            for (int r = tid; r < m; r += nthr) {
                const bool own = r == tid;
                const int sa = own ? rsa : rbody[2 * r], sb = own ? rsb : rbody[2 * r + 1];
                const T *J = rJ + 12 * r;
                T c;
                if (hp) {
                    double acc = 0.0;
                    if (sa >= 0) {
    #pragma unroll
                        for (int k = 0; k < 6; ++k) acc = fma((double)J[k], gbd[6 * sa + k], acc);
                    }
                    if (sb >= 0) {
    #pragma unroll
                        for (int k = 0; k < 6; ++k) acc = fma((double)J[6 + k], gbd[6 * sb + k], acc);
                    }
                    const double xr = x_in64 ? x64[r] : (double)x[r];
                    c = T(bbd[r] + (double)p[r] * acc + ((double)shift + (double)p[r] * (double)p[r] * (double)rreg[r]) * xr);
                } else {
                    T acc = T(0), Jv[6], gv[6];
                    if (sa >= 0) {
                        load6(J, Jv);
                        load6(fb + 6 * sa, gv);
    #pragma unroll
                        for (int k = 0; k < 6; ++k) acc = fma(Jv[k], gv[k], acc);
                    }
                    if (sb >= 0) {
                        load6(J + 6, Jv);
                        load6(fb + 6 * sb, gv);
    #pragma unroll
                        for (int k = 0; k < 6; ++k) acc = fma(Jv[k], gv[k], acc);
                    }
                    c = own ? bb[r] + rpr * acc + rdiag * x[r] : bb[r] + p[r] * acc + (shift + p[r] * p[r] * rreg[r]) * x[r];
                }
                if (a.mixed && !tm) {
                    const float v = (float)c;
                    const __nv_bfloat16 h = __float2bfloat16(v);
                    chi[r] = h;
                    clo[r] = __float2bfloat16(v - __bfloat162float(h));
                } else {
                    bb[r] = c;
                }
            }
            g.sync();
            }
            // [8c] correction: xn = S c with S = -A^-1, so x^i = x^{i-1} + xn (ends with a barrier)
            bool done_c = false;
            if constexpr (sizeof(T) == 4) {
                if (tm) { tmem_matvec(tbase, mp, bb, xn, g); done_c = true; }
            }
            if (!done_c) {
                if (a.mixed) apply_bf16_tiles(A, mp, chi, clo, xn, g);
                else symv_packed(A, mp, bb, xn, X, g);
            }
            // [8d] owners: x^i, y^i = Pi_K(x^i - z^/rho), z^i = z^ - rho (x^i - y^i), residual terms; x and
            // P x go to shared memory at once (the reduction's barrier publishes them for [8a])
            T lrp = T(0), lrd = T(0), lrc = T(0), lc = T(0);
            T xnT[S][3], ynT[S][3], znT[S][3];          // units tid + s * group size
            if (hpv) {
                // the new FP64 iterates wait for the commit in shared memory (x^i in x, y^i and z^i in
                // the two spare vectors), not in registers across the reduction
                double xnD[S][3], ynD[S][3], znD[S][3];
                owner_update<double, T, S>(g, nunits, nfix, nbil, x64, xn, yh64, zh64, mut, mui, p, wv, eta, rho, irho, xnD, ynD,
                                           znD, lrp, lrd, lrc, lc, cslot0);
                stash_rows<S>(g, nunits, nbil, ynD, yn64, cslot0);
                stash_rows<S>(g, nunits, nbil, znD, zn64, cslot0);
            } else {
                owner_update<T, T, S>(g, nunits, nfix, nbil, x, xn, yh, zh, mut, mui, p, wv, eta, rho, irho, xnT, ynT, znT, lrp,
                                      lrd, lrc, lc, cslot0);
            }
            x_in64 = hpv;
            // Nesterov's next coefficients and the next iteration's kind depend on nothing the
            // reduction returns: formed before it
            const T an_next = T(0.5) * (T(1) + sqrt(T(1) + T(4) * acc_a * acc_a));
            const T beta_next = (acc_a - T(1)) / an_next;
            const bool lag_due = kres > 1 && it % kres != 0;
            group_reduce4(lrp, lrd, lrc, lc, red, it & 1, g);
            rp = lrp; rd = lrd; rc = lrc;
            converged = rp < a.tol && rd < a.tol && rc < a.tol;
            hp = use64 && (hp || fmax(rp, rd) < T(KAMINO_REFINE64_BELOW));
            // Nesterov with adaptive restart (uniform decision), then the owners commit y, z, y^, z^ and
            // form the next iteration's b (in FP64 once hp is set)
            T beta_n = T(0);
            bool restart = false;
            if (a.nesterov) {
                if (lc < T(0.999) * c_prev) {
                    beta_n = beta_next;
                    acc_a = an_next;
                    c_prev = lc;
                } else {
                    restart = true;
                    acc_a = T(1);
                    c_prev = c_prev / T(0.999);
                }
            }
            // the next iteration evaluates the refinement residual in iterations 1, K+1, 2K+1, ... and
            // throughout the FP64 end game; the others take c = b^{i+1} - b^i
            lagged = lag_due && !hp;
            if (hpv) {
                double xnD[S][3], ynD[S][3], znD[S][3];
                unstash_rows<S>(g, nunits, nbil, x64, xnD, cslot0);
                unstash_rows<S>(g, nunits, nbil, yn64, ynD, cslot0);
                unstash_rows<S>(g, nunits, nbil, zn64, znD, cslot0);
                owner_commit<double, T, S>(g, nunits, nbil, y64, z64, yh64, zh64, vfd, vfo, mut, eta, rho, a.nesterov != 0,
                                           restart, beta_n, xnD, ynD, znD, true, bb, bbd, nullptr, mp, false, bprev,
                                           nullptr, nullptr, cslot0);
            } else {
                // the iterates move to the FP64 vectors at this commit once the end game has started
                double *init = hp && x64 != nullptr ? x64 : nullptr;
                owner_commit<T, T, S>(g, nunits, nbil, y, z, yh, zh, vfd, vfo, mut, eta, rho, a.nesterov != 0, restart,
                                      beta_n, xnT, ynT, znT, hp, bb, bbd, init, mp, lagged, bprev,
                                      a.mixed && !tm ? chi : nullptr, clo, cslot0);
                hpv = init != nullptr;
            }
            if (converged) break;
            if (a.stall_window > 0 && it % a.stall_window == 0) {
                if (rp < a.tol && rc < a.tol) { stall_due = true; break; }
                stall_prev = false;
            }
        }
        if (stall_due) {
            // the stall exit: r_p and r_c are below tol, r_d is not.  Stop when the natural map is
            // below tol and u+ moved by less than tol (relative) since the check stall_window
            // iterations ago: r_d then sits on the floor of the redundant rows (readings 15, 17)
            stall_due = false;
            g.sync();
            T du = T(0), umax = T(0);
            const T r = ncp_check_fast<T, S>(g, nunits, nfix, nbil, nb, LB, bro, brow, rbody, rJ, p, mut, bminv,
                                             bIinv, vfd, y, hpv ? y64 : nullptr, xn, fb, red, (it + 1) & 1, bufree,
                                             ust, &du, &umax);
            const T gdt = dt * sqrt(M.gx * M.gx + M.gy * M.gy + M.gz * M.gz);
            if (stall_prev && r < T(0.8) * a.tol && du < a.tol * fmax(umax, gdt)) {
                converged = true;
                stalled = true;
                break;
            }
            stall_prev = true;
            if (it >= a.iters) break;
            ++it;
            continue;
        }
        if (!(converged && a.ncp_stop)) break;
        if (a.tol >= T(1e-6)) {
            // ncp_stop: the natural-map residual of the committed (lambda, u+) on the complementarity
            // blocks must be below tol too; in the iteration's precision, with a margin of 20 % for
            // its rounding of v~ (~1e-6 here), so that phase 9's FP64 report stays below tol
            g.sync();
            converged = ncp_check_fast<T, S>(g, nunits, nfix, nbil, nb, LB, bro, brow, rbody, rJ, p, mut, bminv,
                                             bIinv, vfd, y, hpv ? y64 : nullptr, xn, fb, red, (it + 1) & 1) <
                        T(0.8) * a.tol;
        } else {
            // tighter tolerances: in FP64 (the scratch of the refinement end game is free here)
            double *fdl = sizeof(T) == 8 ? reinterpret_cast<double *>(fb) : gbd;
            g.sync();
            ncp_velocities(ncw, g, hpv ? y64 : nullptr, y, fdl);
            g.sync();
            converged = ncp_natural_map(ncw, g, hpv ? y64 : nullptr, y, fdl, red, (it + 1) & 1) < a.tol;
        }
        if (converged) break;
        ++it;
        }
        if (it > a.iters) it = a.iters;
        yfin = hpv ? y64 : nullptr;
        fd = sizeof(T) == 8 ? reinterpret_cast<double *>(fb) : gbd;
    }
    g.sync();

    // ---- 9. lambda = P y; u+ = u_free + M^-1 J^T lambda; integrate; cache; report.  Formed in
    // FP64 (once per step): u+ is a small difference of large joint impulses through light bodies,
    // and the pose update adds a small increment to the stored pose.
    for (int r = tid; r < m; r += nthr) xn[r] = T((double)p[r] * (yfin ? yfin[r] : (double)y[r]));
    // u+ into FP64 scratch (the per-body FP64 velocities of the refinement for FP32 worlds, the
    // per-body force words for FP64 worlds), then the natural-map NCP residual of (lambda, u+)
    if (ncp_velocities(ncw, g, yfin, y, fd)) atomicOr(misc + 1, 1);
    g.sync();
    const bool world_bad = (misc[1] & 1) != 0;
    const T lncp = ncp_natural_map(ncw, g, yfin, y, fd, red, (it + 1) & 1);
    // poses and twists (a non-finite world keeps its state and cache; its report says so)
    for (int i = tid; i < nb && !world_bad; i += nthr) {
        // semi-implicit Euler: q+ = q (+) dt u+; Moreau-Jean: q+ = q_m (+) (dt/2) u+ (Sec. 3)
        const double *up = fd + 6 * i;
        double qp[7];
        pose_advance(bq + 7 * i, up, up + 3, a.midpoint ? 0.5 * dtd : dtd, qp);
        T *gq = a.body_q + 7 * (size_t)(b0 + i);
        T *gu = a.body_u + 6 * (size_t)(b0 + i);
        for (int k = 0; k < 7; ++k) gq[k] = T(qp[k]);
        for (int k = 0; k < 6; ++k) gu[k] = T(up[k]);
    }
    // impulse cache: fixed rows, then one per joint-limit candidate and 3 per contact candidate
    // (zero for candidates that were not active)
    if (!world_bad) {
        for (int r = tid; r < nfix; r += nthr) a.cache[k0 + r] = xn[r];
        for (int e = tid; e < nlc; e += nthr) a.cache[k0 + nfix + e] = lrank[e] >= 0 ? xn[nfix + lrank[e]] : T(0);
        for (int e = tid; e < 3 * nc; e += nthr) {
            const int c = e / 3, t = e % 3;
            const int s = cslot[c];
            a.cache[k0 + nfix + nlc + e] = s >= 0 ? xn[nbil + 3 * s + t] : T(0);
        }
    }
    if (tid == 0) {
        kamino_residual rep;
        rep.iterations = it;
        rep.status = (converged ? 0 : KAMINO_WORLD_NOT_CONVERGED) | (world_bad ? KAMINO_WORLD_NONFINITE : 0) |
                     (stalled ? KAMINO_WORLD_STALLED : 0);
        rep.num_rows = m;
        rep.num_contacts = nact;
        rep.r_primal = (float)rp;
        rep.r_dual = (float)rd;
        rep.r_compl = (float)rc;
        rep.r_ncp = (float)lncp;
        a.res[w] = rep;
    }
}

// One world per CTA (256 threads), grid = number of worlds (or of entries in a.world_order); S = 1
// when every world has at most 256 PADMM units, else 2 (rows <= kMaxRowsPad = 288).
// Tensor-memory columns for the CTA (a.tmem: FP32, and the host guarantees one CTA per SM, so the
// allocation never waits); the address goes through the word misc[2] of the world layout.
template <typename T, int NB>
__device__ __forceinline__ uint32_t cta_tmem_alloc(const StepArgs<T> &a, unsigned char *smem) {
    uint32_t tbase = 0;
    if constexpr (sizeof(T) == 4) {
        const Layout L = make_layout<T>(a.nb_max, a.nj_max, a.nc_max, a.mp_max, NB, a.nl_max);
        int *slot = (int *)(smem + L.misc) + 2;
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(smem_addr(slot)), "r"(kTmemCols) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tmem_fence_before();
        __syncthreads();
        tmem_fence_after();
        tbase = (uint32_t)*slot;
        __syncthreads();                 // every thread has read the address before a world reuses the word
    }
    return tbase;
}
__device__ __forceinline__ void cta_tmem_free(uint32_t tbase) {
    tmem_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tmem_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(kTmemCols) : "memory");
    }
}

template <typename T, int NB, int S>
__global__ void __launch_bounds__(kThreads, 1) step_kernel(const StepArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = a.world_order ? a.world_order[blockIdx.x] : (int)blockIdx.x;
    const Group g{(int)threadIdx.x, kThreads, 0};
    const bool tm = sizeof(T) == 4 && a.tmem;
    const uint32_t tbase = tm ? cta_tmem_alloc<T, NB>(a, smem) : 0u;
    world_step<T, NB, S, false>(a, w, smem, g, tbase, tm);
    if (tm) cta_tmem_free(tbase);
}

// The sparse formulation, one world per CTA: no tensor memory, and a working set small enough for
// several CTAs per SM (hence the register bound of two resident CTAs, up to 2 units a thread; the
// largest worlds, up to 4 units a thread, keep their registers with one CTA per SM).
template <typename T, int S>
__global__ void __launch_bounds__(kThreads, S <= 2 ? 2 : 1) step_kernel_cr(const StepArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = a.world_order ? a.world_order[blockIdx.x] : (int)blockIdx.x;
    const Group g{(int)threadIdx.x, kThreads, 0};
    world_step<T, 16, S, true>(a, w, smem, g, 0u, false);
}

// Persistent launch over a list of worlds: the CTA is split into groups of `group` threads, each
// with its own slice of shared memory; every group pulls the next world from an atomic counter
// until the list is exhausted (dynamic load balance across worlds whose iteration counts differ).
template <typename T, int NB, bool CR>
__global__ void __launch_bounds__(kThreads, 1) step_persistent(const StepArgs<T> a, PersistentArgs p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int gi = threadIdx.x / p.group;
    const int ngroups = kThreads / p.group;
    const Group g{(int)threadIdx.x - gi * p.group, p.group, ngroups > 1 ? 1 + gi : 0};
    unsigned char *slice = smem + (size_t)gi * p.slice_bytes;
    int *slot = (int *)(smem + (size_t)ngroups * p.slice_bytes) + gi;
    // tensor memory only when one group fills the CTA (a.tmem is set by the host for such buckets)
    const bool tm = !CR && sizeof(T) == 4 && a.tmem && ngroups == 1;
    const uint32_t tbase = tm ? cta_tmem_alloc<T, NB>(a, smem) : 0u;
    for (int round = 0; round < p.count; ++round) {   // bounded: at most one world per round
        if (g.tid == 0) *slot = atomicAdd(p.counter, 1);
        g.sync();
        const int idx = *slot;
        g.sync();
        if (idx >= p.count) break;
        world_step<T, NB, kSlots, CR>(a, p.worlds[idx], slice, g, tbase, tm);
        g.sync();
    }
    if (tm) cta_tmem_free(tbase);
}

// ----------------------------------------------------------------------------- forward kinematics
// Gauss-Newton forward kinematics for resets (Sec. 6.3): poses consistent with the joint constraints
// and prescribed joint coordinates.  F(q) = [f(q); d_j(q) - target_j], f the errors of the joint
// rows (the dynamics' own rows, whose J is the rate of f), d_j the joint coordinate (hinge angle,
// wrapped into (-pi, pi], or slide).  Each iteration takes the minimum-norm least-squares step over
// the twists of the bodies that are not held, delta = -J^T P (P J J^T P + mu I)^-1 P F (P the row
// scaling to unit norm, mu = 1e-10: the loops make rows redundant and a partial selection leaves
// directions free), factorised as L D L^T in FP64, and moves the poses along it as the integrator
// does (r += delta_v, q = exp(delta_w) q).  One CTA per world; every quantity FP64 on chip.

__device__ __forceinline__ int joint_row_count(int type) {
    switch (type) {
        case KAMINO_JOINT_REVOLUTE: return 5;
        case KAMINO_JOINT_PRISMATIC: return 5;
        case KAMINO_JOINT_UNIVERSAL: return 4;
        case KAMINO_JOINT_SPHERICAL: return 3;
        case KAMINO_JOINT_FIXED: return 6;
        default: return 0;
    }
}

template <typename T>
__device__ void fk_world(const FkArgs<T> &a, int w, unsigned char *smem, const Group &g) {
    constexpr double kMu = 1e-10;
    const int tid = g.tid, lane = g.lane(), warp = g.warp(), nthr = g.size, nwarps = g.warps();
    const ModelView<T> &M = a.m;
    const int4 wa = M.world_a[w], wb = M.world_b[w];
    const int b0 = wa.x, j0 = wa.y, nb = wb.x, nj = wb.y;
    const FkLayout L = make_fk_layout(a.nb_max, a.m_max);
    double *bq = (double *)(smem + L.bq), *bq0 = (double *)(smem + L.bq0), *bRd = (double *)(smem + L.bRd);
    double *rJ = (double *)(smem + L.rJ);
    double *F = (double *)(smem + L.F), *y = (double *)(smem + L.y), *p = (double *)(smem + L.p);
    double *dinv = (double *)(smem + L.dinv), *dl = (double *)(smem + L.dl), *A = (double *)(smem + L.A);
    double *red = (double *)(smem + L.red);
    int *rbody = (int *)(smem + L.rbody), *bro = (int *)(smem + L.bro), *brow = (int *)(smem + L.brow);
    int *misc = (int *)(smem + L.misc);
    const int njr = nj > 0 ? M.joint_row[j0 + nj - 1] + joint_row_count(M.joint_meta[j0 + nj - 1].x) : 0;
    for (int i = tid; i < nb; i += nthr) {
        const T *gq = a.body_q + 7 * (size_t)(b0 + i);
        double q[7];
        for (int k = 0; k < 7; ++k) q[k] = (double)gq[k];
        const double qn = 1.0 / sqrt(q[3] * q[3] + q[4] * q[4] + q[5] * q[5] + q[6] * q[6]);
        for (int k = 0; k < 7; ++k) bq[7 * i + k] = k < 3 ? q[k] : q[k] * qn;
    }
    g.sync();
    int it = 0, m = njr;
    double res = INFINITY;
    for (it = 0;; ++it) {
        for (int i = tid; i < nb; i += nthr) quat_rot(bq + 7 * i + 3, bRd + 9 * i);
        g.sync();
        // joint rows (kbias 1: the row's value is f itself), then the selected coordinate rows
        for (int j = tid; j < nj; j += nthr) {
            const int4 meta = M.joint_meta[j0 + j];
            double wr[12];
            joint_rows<double>(meta.x, meta.y, meta.z, M.joint_frames + 14 * (size_t)(j0 + j), bq, bRd,
                               M.joint_row[j0 + j], 1.0, rbody, rJ, F, false, 0.0, wr);
        }
        if (warp == nwarps - 1) {
            int count = 0;
            for (int jb = 0; jb < nj; jb += 32) {
                const int j = jb + lane;
                bool sel = false;
                int4 meta = make_int4(0, 0, 0, -1);
                if (j < nj) {
                    meta = M.joint_meta[j0 + j];
                    const bool coord = meta.x == KAMINO_JOINT_REVOLUTE || meta.x == KAMINO_JOINT_PRISMATIC;
                    sel = coord && (a.select ? a.select[j0 + j] != 0 : meta.w >= 0);
                }
                const unsigned mask = __ballot_sync(0xffffffffu, sel);
                const int rank = count + __popc(mask & ((1u << lane) - 1u));
                if (sel) {
                    double d, Ja[6], Jb[6];
                    joint_coordinate(meta.x, meta.y, meta.z, M.joint_frames + 14 * (size_t)(j0 + j), bq, bRd, &d, Ja, Jb);
                    double diff = d - a.target[j0 + j];
                    if (meta.x == KAMINO_JOINT_REVOLUTE)
                        diff -= 2.0 * 3.141592653589793 * floor((diff + 3.141592653589793) / (2.0 * 3.141592653589793));
                    put_row(rbody, rJ, F, njr + rank, meta.y, meta.z, Ja, Jb, diff);
                }
                count += __popc(mask);
            }
            if (lane == 0) misc[0] = count;
        }
        g.sync();
        m = njr + misc[0];
        // held bodies are not unknowns: their blocks leave the rows
        for (int r = tid; r < m; r += nthr)
            for (int s = 0; s < 2; ++s) {
                const int b = rbody[2 * r + s];
                if (b >= 0 && a.fixed != nullptr && a.fixed[b0 + b] != 0) rbody[2 * r + s] = -1;
            }
        double lres = 0.0;
        for (int r = tid; r < m; r += nthr) lres = fmax(lres, fabs(F[r]));
        {
            double d0 = 0.0, d1 = 0.0, d2 = 0.0;
            group_reduce4(lres, d0, d1, d2, red, it & 1, g);
        }
        if (!isfinite(lres)) {
            // the last step diverged (a target out of reach near a singular configuration): keep
            // the poses it started from, whose residual is `res`
            for (int e = tid; e < 7 * nb; e += nthr) bq[e] = bq0[e];
            g.sync();
            break;
        }
        res = lres;
        if (res < a.tol || it >= a.iters) break;
        // row scaling to unit norm over the unknown blocks
        for (int r = tid; r < m; r += nthr) {
            double s = 0.0;
            for (int side = 0; side < 2; ++side)
                if (rbody[2 * r + side] >= 0)
                    for (int k = 0; k < 6; ++k) s += rJ[12 * r + 6 * side + k] * rJ[12 * r + 6 * side + k];
            p[r] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
        }
        g.sync();
        body_row_lists(g, nb, m, rbody, bro, brow);
        // P J J^T P + mu I, packed lower (warp per column, block-sparse over shared bodies)
        for (int j = warp; j < m; j += nwarps) {
            double *col = A + col_start(j, m) - j;
            const int ja = rbody[2 * j], jb = rbody[2 * j + 1];
            const double *Jj = rJ + 12 * j;
            for (int i = j + lane; i < m; i += 32) {
                const int ia = rbody[2 * i], ib = rbody[2 * i + 1];
                const double *Ji = rJ + 12 * i;
                double s = 0.0;
                if (ia >= 0 && ia == ja) for (int k = 0; k < 6; ++k) s += Ji[k] * Jj[k];
                if (ia >= 0 && ia == jb) for (int k = 0; k < 6; ++k) s += Ji[k] * Jj[6 + k];
                if (ib >= 0 && ib == ja) for (int k = 0; k < 6; ++k) s += Ji[6 + k] * Jj[k];
                if (ib >= 0 && ib == jb) for (int k = 0; k < 6; ++k) s += Ji[6 + k] * Jj[6 + k];
                col[i] = p[i] * p[j] * s + (i == j ? kMu : 0.0);
            }
        }
        g.sync();
        // L D L^T in place, right-looking (A(i, k) holds l_ik d_k): one barrier per column
        for (int k = 0; k < m; ++k) {
            const double dk = A[pidx(k, k, m)];
            const double idk = 1.0 / dk;
            for (int j = k + 1 + warp; j < m; j += nwarps) {
                const double ljk = A[pidx(j, k, m)] * idk;
                double *col = A + col_start(j, m) - j;
                const double *ck = A + col_start(k, m) - k;
                for (int i = j + lane; i < m; i += 32) col[i] -= ck[i] * ljk;
            }
            if (tid == 0) dinv[k] = idk;
            g.sync();
        }
        // y = -(L D L^T)^-1 P F: forward and backward substitution in one warp
        if (warp == 0) {
            for (int r = lane; r < m; r += 32) y[r] = -p[r] * F[r];
            __syncwarp();
            for (int k = 0; k < m; ++k) {
                const double zk = y[k], idk = dinv[k];
                const double *ck = A + col_start(k, m) - k;
                for (int i = k + 1 + lane; i < m; i += 32) y[i] -= ck[i] * idk * zk;
                __syncwarp();
            }
            for (int r = lane; r < m; r += 32) y[r] *= dinv[r];
            __syncwarp();
            for (int k = m - 1; k > 0; --k) {
                const double yk = y[k];
                for (int i = lane; i < k; i += 32) y[i] -= A[pidx(k, i, m)] * dinv[i] * yk;
                __syncwarp();
            }
        }
        g.sync();
        // delta = J^T P y per (body, component), then the poses move along it
        for (int t = tid; t < 6 * nb; t += nthr) {
            const int i = t / 6, k = t - 6 * (t / 6);
            double f = 0.0;
            for (int e = bro[i]; e < bro[i + 1]; ++e) {
                const int code = brow[e], r = code >> 1;
                f = fma(rJ[6 * code + k], p[r] * y[r], f);
            }
            dl[t] = f;
        }
        g.sync();
        for (int i = tid; i < nb; i += nthr) {
            double qn[7];
            pose_advance(bq + 7 * i, dl + 6 * i, dl + 6 * i + 3, 1.0, qn);
            for (int k = 0; k < 7; ++k) {
                bq0[7 * i + k] = bq[7 * i + k];
                bq[7 * i + k] = qn[k];
            }
        }
        g.sync();
    }
    const bool ok = res < a.tol;
    for (int i = tid; i < nb; i += nthr) {
        T *gq = a.body_q + 7 * (size_t)(b0 + i);
        for (int k = 0; k < 7; ++k) gq[k] = T(bq[7 * i + k]);
    }
    if (tid == 0) {
        kamino_residual rep{};
        rep.iterations = it;
        rep.status = ok ? 0 : KAMINO_WORLD_NOT_CONVERGED;
        rep.num_rows = m;
        rep.r_primal = (float)res;
        a.res[w] = rep;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) fk_kernel(const FkArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Group g{(int)threadIdx.x, kThreads, 0};
    fk_world<T>(a, (int)blockIdx.x, smem, g);
}

}  // namespace

template <typename T>
cudaError_t prepare_step(int nb_panel, size_t smem) {
    const int b = (int)smem;
    cudaError_t e = cudaFuncSetAttribute(step_kernel_cr<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel_cr<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel_cr<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e != cudaSuccess) return e;
    if (nb_panel == 16) {
        e = cudaFuncSetAttribute(step_kernel<T, 16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, 16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        return e;
    }
    e = cudaFuncSetAttribute(step_kernel<T, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(step_kernel<T, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

template <typename T>
cudaError_t launch_step(const StepArgs<T> &args, int num_worlds, int nb_panel, size_t smem, cudaStream_t stream) {
    if (num_worlds <= 0) return cudaSuccess;
    const bool one = args.mp_max <= kThreads;     // units <= rows <= mp_max
    if (args.cr_iters > 0) {     // units <= rows <= mp_max
        if (one) step_kernel_cr<T, 1><<<num_worlds, kThreads, smem, stream>>>(args);
        else if (args.mp_max <= 2 * kThreads) step_kernel_cr<T, 2><<<num_worlds, kThreads, smem, stream>>>(args);
        else step_kernel_cr<T, 4><<<num_worlds, kThreads, smem, stream>>>(args);
    } else if (nb_panel == 16) {
        if (one) step_kernel<T, 16, 1><<<num_worlds, kThreads, smem, stream>>>(args);
        else step_kernel<T, 16, 2><<<num_worlds, kThreads, smem, stream>>>(args);
    } else {
        if (one) step_kernel<T, 8, 1><<<num_worlds, kThreads, smem, stream>>>(args);
        else step_kernel<T, 8, 2><<<num_worlds, kThreads, smem, stream>>>(args);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t prepare_persistent(int nb_panel, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(step_persistent<T, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    if (nb_panel == 16)
        return cudaFuncSetAttribute(step_persistent<T, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaFuncSetAttribute(step_persistent<T, 8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
cudaError_t occupancy_persistent(int nb_panel, size_t smem, int cr, int *blocks_per_sm) {
    if (cr) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, step_persistent<T, 16, true>, kThreads, smem);
    if (nb_panel == 16)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, step_persistent<T, 16, false>, kThreads, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, step_persistent<T, 8, false>, kThreads, smem);
}

template <typename T>
cudaError_t launch_persistent(const StepArgs<T> &args, const PersistentArgs &p, int nb_panel, int grid, size_t smem,
                              cudaStream_t stream) {
    if (p.count <= 0 || grid <= 0) return cudaSuccess;
    if (args.cr_iters > 0)
        step_persistent<T, 16, true><<<grid, kThreads, smem, stream>>>(args, p);
    else if (nb_panel == 16)
        step_persistent<T, 16, false><<<grid, kThreads, smem, stream>>>(args, p);
    else
        step_persistent<T, 8, false><<<grid, kThreads, smem, stream>>>(args, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fk(const FkArgs<T> &args, int num_worlds, size_t smem, cudaStream_t stream) {
    if (num_worlds <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fk_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fk_kernel<T><<<num_worlds, kThreads, smem, stream>>>(args);
    return cudaGetLastError();
}

namespace {
// Counting sort of the worlds by the PADMM iterations of their previous step, most first (keys
// clamped to kKeys - 1): a histogram in shared memory, the start of every key (thread 0), then every
// world takes the next slot of its key.  The order within a key is arbitrary; it is a permutation.
constexpr int kOrderKeys = 1024;
__global__ void __launch_bounds__(1024, 1) order_kernel(const kamino_residual *res, int W, int *order) {
    __shared__ int start[kOrderKeys];
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int k = tid; k < kOrderKeys; k += nthr) start[k] = 0;
    __syncthreads();
    for (int w = tid; w < W; w += nthr) atomicAdd(&start[min(max(res[w].iterations, 0), kOrderKeys - 1)], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int k = kOrderKeys - 1; k >= 0; --k) {
            const int c = start[k];
            start[k] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int w = tid; w < W; w += nthr) {
        const int pos = atomicAdd(&start[min(max(res[w].iterations, 0), kOrderKeys - 1)], 1);
        order[pos] = w;
    }
}
}  // namespace

cudaError_t launch_order(const kamino_residual *res, int num_worlds, int *order, cudaStream_t stream) {
    if (num_worlds <= 0) return cudaSuccess;
    order_kernel<<<1, 1024, 0, stream>>>(res, num_worlds, order);
    return cudaGetLastError();
}

template cudaError_t launch_fk<float>(const FkArgs<float> &, int, size_t, cudaStream_t);
template cudaError_t launch_fk<double>(const FkArgs<double> &, int, size_t, cudaStream_t);
template cudaError_t prepare_step<float>(int, size_t);
template cudaError_t prepare_step<double>(int, size_t);
template cudaError_t launch_step<float>(const StepArgs<float> &, int, int, size_t, cudaStream_t);
template cudaError_t launch_step<double>(const StepArgs<double> &, int, int, size_t, cudaStream_t);
template cudaError_t prepare_persistent<float>(int, size_t);
template cudaError_t prepare_persistent<double>(int, size_t);
template cudaError_t occupancy_persistent<float>(int, size_t, int, int *);
template cudaError_t occupancy_persistent<double>(int, size_t, int, int *);
template cudaError_t launch_persistent<float>(const StepArgs<float> &, const PersistentArgs &, int, int, size_t,
                                              cudaStream_t);
template cudaError_t launch_persistent<double>(const StepArgs<double> &, const PersistentArgs &, int, int, size_t,
                                               cudaStream_t);

}  // namespace kamino
