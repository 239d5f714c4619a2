// Internal declarations shared by the host API (kamino_api.cu) and the step kernel
// (kamino_step.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "kamino.h"

namespace kamino {

constexpr int kThreads = 256;        // CTA size of the per-world step kernel (8 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRowsPad = 288;     // largest padded row count of the dense formulation (its matrix)
constexpr int kMaxRowsPadSparse = 1024;   // of the sparse formulation (units <= 4 per thread)
constexpr int kMaxChunks = kMaxRowsPad / 32;
constexpr int kMaxCandidates = 64;   // contact candidates per world
constexpr int kSlots = 4;            // PADMM units (joint rows / contacts) per thread: units <= kSlots * group

// Device-side view of a model (all pointers are device pointers; T = float or double).
template <typename T>
struct ModelView {
    int num_worlds;
    int n_act_max;
    const int4 *world_a;       // (body_offset, joint_offset, contact_offset, cache_offset)
    const int4 *world_b;       // (num_bodies, num_joints, num_candidates, fixed rows: joint + drive rows)
    const int4 *world_c;       // (limit candidates, 0, 0, 0); nullptr when no world has joint limits
    const T *world_mu;         // [W]
    const T *body_mass;        // [B]
    const T *body_inertia;     // [B*3]
    const int4 *joint_meta;    // (type, parent, child, actuator)
    const int *joint_row;      // first row of the joint inside its world
    // joint-space dynamics (Sec. 3, Eq. 2's R and v*); nullptr when the model has none
    const int *joint_drow;        // [J] row of the joint's drive row inside its world, or -1
    const int *joint_lslot;       // [J] first limit candidate of the joint inside its world, or -1
    const double *joint_dyn;      // [J*8] (mode, Kp, Kd, armature, damping, lower, upper, 0)
    // position-level data stays FP64 whatever T is: joint errors and contact distances are
    // multiplied by beta / dt in the bias, which would amplify FP32 rounding of anchors by 100-200
    const double *joint_frames;   // [J*14]: parent pos3 quat4, child pos3 quat4
    const int *contact_body;      // [C]
    const double *contact_point;  // [C*3]
    int terrain_kind, hf_nx, hf_ny;
    double hf_x0, hf_y0, hf_cell;
    const double *hf_heights;     // [ny*nx]
    T gx, gy, gz;
};

template <typename T>
struct StepArgs {
    ModelView<T> m;
    T *body_q;                 // [B*7]
    T *body_u;                 // [B*6]
    T *cache;                  // [cache_len]
    const T *warm;             // [cache_len] (external warm start) or nullptr
    kamino_residual *res;      // [W]
    const T *tau;              // [W*n_act_max] or nullptr
    const int *world_order;    // optional permutation of worlds (nullptr = identity)
    T dt, tol, eta, rho, beta, margin;
    int iters, nesterov, precond, warm_mode;
    int mixed;                 // 1: BF16 tiles of the inverse on tensor cores (KAMINO_MIXED)
    int midpoint;              // 1: Moreau-Jean midpoint scheme (KAMINO_INTEGRATOR_MIDPOINT)
    int refine64;              // 1: FP64 right-hand side and refinement residual near convergence
    int cr_iters;              // 0: dense formulation; k >= 1: sparse formulation, k CR iterations per x-step
    int ncp_stop;              // 1: converged also requires the natural-map NCP residual below tol
    int stall_window;          // > 0: the stall exit every stall_window iterations (dense formulation)
    int residual_every;        // >= 1: the refinement residual evaluated every residual_every iterations
    int tmem;                  // 1: keep the swept inverse in tensor memory (FP32, whole-CTA groups, mp <= 256)
    // shared-memory layout bounds (maxima over the launched worlds)
    int nb_max, nj_max, nc_max, mp_max, nl_max;
};

// Persistent launch over one bucket of worlds (see step_persistent).
struct PersistentArgs {
    const int *worlds;         // [count] world ids of the bucket
    int count;
    int *counter;              // device work counter, zero before the launch
    int group;                 // threads per world: 32, 64, 128 or 256
    size_t slice_bytes;        // shared memory per group (multiple of 16)
};

// Byte offsets of the per-world shared-memory working set.
struct Layout {
    size_t bq, bu, bRd, bI, bIinv, bminv, bufree, jwr, cid, cslot, rbody, rJ, rvs, rreg;
    size_t lgap, lJ, lrank, lcid;
    size_t vfd, p, x, xn, y, z, yh, zh, b, mut, mui, wv, fb, ust, bro, brow, X, A, red, misc, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Row stride of the transposed panels of the sweep: 8 words off a multiple of 32, so that rows
// k, k+1, k+2, k+3 of a panel start on banks 0, 8, 16, 24 (conflict-free tensor-core fragment loads);
// non-decreasing in mp, so a layout sized for the largest world fits every smaller one.
__host__ __device__ inline int panel_ld(int mp) { return mp + (mp % 32 == 0 ? 8 : 24); }

// nl: joint-limit candidates per world (0 when no world has limits).  dense: the dense formulation's
// working set (packed matrix, sweep panels, PADMM vectors in shared memory); otherwise the sparse
// formulation's, whose PADMM and Conjugate Residual vectors live in the owners' registers and whose
// scratch X holds, after assembly, the final y (FP64), the published vector w = P v and the per-body
// gather g (both sized for FP64).
template <typename T>
__host__ __device__ inline Layout make_layout(int nb, int nj, int nc, int mp, int nb_panel, int nl = 0,
                                              bool dense = true) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t &field, size_t bytes) { field = o; o = align_up(o + bytes, 16); };
    const size_t s = sizeof(T);
    take(L.bq, nb * 7 * sizeof(double));   // the pose the step is evaluated at, FP64
    take(L.bu, nb * 6 * s);
    take(L.bRd, nb * 9 * sizeof(double));
    take(L.bI, nb * 3 * s);
    take(L.bIinv, nb * 6 * s);
    take(L.bminv, nb * s);
    take(L.bufree, nb * 6 * s);
    take(L.jwr, nj * 12 * s);
    take(L.cid, nc * sizeof(int));
    take(L.cslot, nc * sizeof(int));
    take(L.rbody, mp * 2 * sizeof(int));
    take(L.rJ, mp * 12 * s);
    // the bias v* and the free velocity v_f are also kept in FP64: v_f has components outside the
    // range of J (redundant loop rows, contacts tied together by the joints) to which the dual
    // problem's solution is very sensitive, so its FP32 rounding alone moves u+ by up to ~2e-4
    take(L.rvs, mp * sizeof(double));
    take(L.rreg, mp * s);                  // R of Eq. 4 per row (drive rows; zero elsewhere)
    take(L.lgap, nl * sizeof(double));     // joint-limit candidates: gap, row blocks, rank, and the
    take(L.lJ, nl * 12 * s);               // candidate of every active limit row
    take(L.lrank, nl * sizeof(int));
    take(L.lcid, nl * sizeof(int));
    take(L.vfd, mp * sizeof(double));
    take(L.p, mp * s);
    take(L.x, mp * s);
    take(L.xn, mp * s);
    const int dv = dense ? mp : 0;         // vectors only the dense formulation keeps in shared memory
    take(L.y, dv * s);
    take(L.z, dv * s);
    take(L.yh, dv * s);
    take(L.zh, dv * s);
    take(L.b, dv * s);
    take(L.mut, (nc > 0 ? nc : 1) * s);
    take(L.mui, (nc > 0 ? nc : 1) * s);
    take(L.wv, dv * s);
    take(L.fb, (dense ? nb * 6 : 0) * s);
    take(L.ust, (dense ? nb * 6 : 0) * s);   // u+ at the last stall check
    take(L.bro, (nb + 1) * sizeof(int));
    take(L.brow, 2 * mp * sizeof(int));
    if (!dense) {
        size_t xb = (size_t)mp * 12 * s;                                     // M^-1 J^T blocks (assembly)
        const size_t cr = (2 * (size_t)mp + 6 * (size_t)nb) * sizeof(double);  // y64, w, g
        if (cr > xb) xb = cr;
        take(L.X, xb);
        take(L.A, 0);
        take(L.red, 2 * 4 * kWarps * sizeof(double));
        take(L.misc, 16 * sizeof(int));
        L.total = o;
        return L;
    }
    size_t xs = (size_t)mp * 12;
    size_t sweep = (size_t)2 * panel_ld(mp) * nb_panel + (size_t)nb_panel * nb_panel;
    if (sweep > xs) xs = sweep;
    if ((size_t)kWarps * mp > xs) xs = (size_t)kWarps * mp;
    // FP32 worlds: during PADMM the words past the mat-vec partials ([kWarps][mp]) hold the FP64
    // vectors of the refinement residual (b: mp; per-body velocities M^-1 J^T P x: 6 nb)
    if (s == 4 && (size_t)kWarps * mp + 2 * (size_t)mp + 12 * (size_t)nb > xs)
        xs = (size_t)kWarps * mp + 2 * (size_t)mp + 12 * (size_t)nb;
    take(L.X, xs * s);
    take(L.A, (size_t)mp * (mp + 1) / 2 * s);
    take(L.red, 2 * 4 * kWarps * s);
    take(L.misc, 16 * sizeof(int));
    L.total = o;
    return L;
}

// Forward kinematics for resets (fk_kernel): one world per CTA, everything in FP64 on chip.
template <typename T>
struct FkArgs {
    ModelView<T> m;
    T *body_q;                 // [B*7] poses, read and written
    kamino_residual *res;      // [W]
    const double *target;      // [J] joint-coordinate targets
    const int *select;         // [J] nonzero: prescribed coordinate; nullptr: the actuated joints
    const int *fixed;          // [B] nonzero: the body keeps its pose; nullptr: none
    int iters;
    double tol;
    int nb_max, m_max;         // bodies and rows of F (joint rows + coordinate rows) of the largest world
};

struct FkLayout {
    size_t bq, bq0, bRd, rbody, rJ, F, y, p, dinv, bro, brow, dl, A, red, misc, total;
};

// Shared memory of the FK kernel: the packed lower FP64 matrix of m_max rows dominates.
__host__ __device__ inline FkLayout make_fk_layout(int nb, int m) {
    FkLayout L{};
    size_t o = 0;
    auto take = [&](size_t &field, size_t bytes) { field = o; o = align_up(o + bytes, 16); };
    const int mm = m > 0 ? m : 1;
    take(L.bq, nb * 7 * sizeof(double));
    take(L.bq0, nb * 7 * sizeof(double));    // the poses before the last step
    take(L.bRd, nb * 9 * sizeof(double));
    take(L.rbody, mm * 2 * sizeof(int));
    take(L.rJ, mm * 12 * sizeof(double));
    take(L.F, mm * sizeof(double));
    take(L.y, mm * sizeof(double));
    take(L.p, mm * sizeof(double));
    take(L.dinv, mm * sizeof(double));
    take(L.bro, (nb + 1) * sizeof(int));
    take(L.brow, 2 * mm * sizeof(int));
    take(L.dl, nb * 6 * sizeof(double));
    take(L.A, (size_t)mm * (mm + 1) / 2 * sizeof(double));
    take(L.red, 2 * 4 * kWarps * sizeof(double));
    take(L.misc, 16 * sizeof(int));
    L.total = o;
    return L;
}

// Launchers (kamino_step.cu).  Return the launch error (cudaSuccess on success).
template <typename T>
cudaError_t launch_step(const StepArgs<T> &args, int num_worlds, int nb_panel, size_t smem,
                        cudaStream_t stream);
template <typename T>
cudaError_t prepare_step(int nb_panel, size_t smem);
template <typename T>
cudaError_t launch_persistent(const StepArgs<T> &args, const PersistentArgs &p, int nb_panel, int grid, size_t smem,
                              cudaStream_t stream);
template <typename T>
cudaError_t prepare_persistent(int nb_panel, size_t smem);
template <typename T>
cudaError_t occupancy_persistent(int nb_panel, size_t smem, int cr, int *blocks_per_sm);
template <typename T>
cudaError_t launch_fk(const FkArgs<T> &args, int num_worlds, size_t smem, cudaStream_t stream);
// Longest-first order of the worlds from the iterations of their previous step (one CTA).
cudaError_t launch_order(const kamino_residual *res, int num_worlds, int *order, cudaStream_t stream);

}  // namespace kamino
