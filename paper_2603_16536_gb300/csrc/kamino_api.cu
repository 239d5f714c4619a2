// Host implementation of the C ABI declared in include/kamino.h: validation of the world
// description, the device layout of a model (sum-allocated over worlds, Sec. 5.2 of the paper:
// arrays sized by the sum over worlds, launch bounds by the maximum), state memory and the launch
// of the fused step kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kamino.h"
#include "kamino_internal.h"
#include "kamino_mlp.h"

using namespace kamino;

namespace {

thread_local std::string g_error;

kamino_status fail(kamino_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
    return s;
}

kamino_status cuda_fail(cudaError_t e, const char *what) {
    return fail(KAMINO_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr size_t kMaxSmem = 232448;   // opt-in dynamic shared memory per CTA on sm_100 / sm_103

int rows_of(int type) {
    switch (type) {
        case KAMINO_JOINT_REVOLUTE: return 5;
        case KAMINO_JOINT_PRISMATIC: return 5;
        case KAMINO_JOINT_UNIVERSAL: return 4;
        case KAMINO_JOINT_SPHERICAL: return 3;
        case KAMINO_JOINT_FIXED: return 6;
        default: return -1;
    }
}

kamino_status check_params(const kamino_solver_params &p) {
    if (!(p.rho > 0.0) || !std::isfinite(p.rho)) return fail(KAMINO_E_INVALID_ARG, "params.rho must be > 0");
    if (!(p.eta >= 0.0) || !std::isfinite(p.eta)) return fail(KAMINO_E_INVALID_ARG, "params.eta must be >= 0");
    if (!(p.beta >= 0.0 && p.beta <= 1.0)) return fail(KAMINO_E_INVALID_ARG, "params.beta must be in [0, 1]");
    if (!(p.margin >= 0.0) || !std::isfinite(p.margin)) return fail(KAMINO_E_INVALID_ARG, "params.margin must be >= 0");
    if (p.warm_mode < KAMINO_WARM_COLD || p.warm_mode > KAMINO_WARM_EXTERNAL)
        return fail(KAMINO_E_INVALID_ARG, "params.warm_mode %d is not a KAMINO_WARM_* value", p.warm_mode);
    if (p.integrator != KAMINO_INTEGRATOR_EULER && p.integrator != KAMINO_INTEGRATOR_MIDPOINT)
        return fail(KAMINO_E_INVALID_ARG, "params.integrator %d is not a KAMINO_INTEGRATOR_* value", p.integrator);
    if (p.stall_window < 0) return fail(KAMINO_E_INVALID_ARG, "params.stall_window must be >= 0");
    if (p.residual_every < 0 || p.residual_every > 1024)
        return fail(KAMINO_E_INVALID_ARG, "params.residual_every must be in [0, 1024]");
    if (p.schedule != KAMINO_SCHEDULE_IN_ORDER && p.schedule != KAMINO_SCHEDULE_LONGEST_FIRST)
        return fail(KAMINO_E_INVALID_ARG, "params.schedule %d is not a KAMINO_SCHEDULE_* value", p.schedule);
    if (p.cr_iters < 0 || p.cr_iters > KAMINO_MAX_CR_ITERS)
        return fail(KAMINO_E_INVALID_ARG, "params.cr_iters must be in [0, %d] (got %d)", KAMINO_MAX_CR_ITERS, p.cr_iters);
    return KAMINO_OK;
}

}  // namespace

struct Bucket {
    int rows_pad = 0, count = 0;           // padded row bound, worlds
    int nb = 0, nj = 0, nc = 0, rows = 0;  // layout maxima over the bucket
    int units = 0;                         // max PADMM units (joint rows + contacts)
    int group = 256, panel = 16, grid = 0, per_cta = 1;
    size_t slice = 0, smem = 0;
    float tuned_ms = 0.0f;
    int *d_worlds = nullptr;
    std::vector<int> worlds;
};

struct kamino_model_s {
    int precision = KAMINO_FP32;
    int W = 0, B = 0, J = 0, C = 0;
    int nb_max = 0, nj_max = 0, nc_max = 0, mp_max = 0, max_rows = 0, n_act_max = 0, cache_len = 0;
    int fk_rows_max = 0;                   // joint rows + revolute / prismatic joints of a world (FK)
    int nb_panel = 16;
    size_t smem = 0;
    bool prepared = false;
    kamino_solver_params params{};
    // device arrays
    std::vector<void *> allocs;
    int4 *world_a = nullptr, *world_b = nullptr, *world_c = nullptr, *joint_meta = nullptr;
    int *joint_row = nullptr, *contact_body = nullptr, *joint_drow = nullptr, *joint_lslot = nullptr;
    double *joint_dyn = nullptr;
    int nl_max = 0;                        // joint-limit candidates of one world
    std::vector<int> world_cache;          // impulse-cache length of every world
    void *world_mu = nullptr, *body_mass = nullptr, *body_inertia = nullptr, *joint_frames = nullptr;
    void *contact_point = nullptr, *hf_heights = nullptr, *q0 = nullptr, *u0 = nullptr;
    int terrain_kind = 0, hf_nx = 0, hf_ny = 0;
    double hf_x0 = 0, hf_y0 = 0, hf_cell = 0, g[3] = {0, 0, 0};
    // heterogeneous plan
    std::vector<Bucket> buckets;
    int launch_mode = KAMINO_LAUNCH_SINGLE;
    bool plan_ready = false;
    int sm_count = 0;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;

    ~kamino_model_s() {
        for (void *p : allocs) cudaFree(p);
        for (cudaStream_t st : side) cudaStreamDestroy(st);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
    }
};

struct kamino_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct kamino_state_s {
    kamino_model_t model = nullptr;
    char *base = nullptr;
    bool owned = false;
    size_t off_q = 0, off_u = 0, off_cache = 0, off_warm = 0, off_res = 0, off_tau = 0, off_cnt = 0, off_order = 0;
    size_t bytes = 0;
    void *ptr(size_t off) const { return base + off; }
};

namespace {

template <typename T>
kamino_status upload(kamino_model_s *m, void **dst, const void *src, size_t bytes) {
    (void)sizeof(T);
    if (bytes == 0) { *dst = nullptr; return KAMINO_OK; }
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (model)");
    m->allocs.push_back(d);
    e = cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (model)");
    *dst = d;
    return KAMINO_OK;
}

template <typename T>
std::vector<T> convert(const double *src, size_t n) {
    std::vector<T> v(n);
    for (size_t i = 0; i < n; ++i) v[i] = (T)src[i];
    return v;
}

// Host arrays of the joint-space dynamics (empty when the model has none).
struct JointDyn {
    std::vector<int4> wc;       // per world (limit candidates, 0, 0, 0)
    std::vector<int> drow, lslot;
    std::vector<double> dyn;    // [J*8]
};

template <typename T>
kamino_status build_device(kamino_model_s *m, const kamino_model_desc *d, const std::vector<int4> &wa,
                           const std::vector<int4> &wb, const std::vector<int4> &jm, const std::vector<int> &jrow,
                           const std::vector<double> &frames, const std::vector<double> &q0, const JointDyn &jd) {
    kamino_status s;
    if ((s = upload<T>(m, (void **)&m->world_a, wa.data(), wa.size() * sizeof(int4)))) return s;
    if ((s = upload<T>(m, (void **)&m->world_b, wb.data(), wb.size() * sizeof(int4)))) return s;
    if (!jd.dyn.empty()) {
        if ((s = upload<T>(m, (void **)&m->world_c, jd.wc.data(), jd.wc.size() * sizeof(int4)))) return s;
        if ((s = upload<T>(m, (void **)&m->joint_drow, jd.drow.data(), jd.drow.size() * sizeof(int)))) return s;
        if ((s = upload<T>(m, (void **)&m->joint_lslot, jd.lslot.data(), jd.lslot.size() * sizeof(int)))) return s;
        if ((s = upload<T>(m, (void **)&m->joint_dyn, jd.dyn.data(), jd.dyn.size() * sizeof(double)))) return s;
    }
    auto mu = convert<T>(d->world_mu, m->W);
    if ((s = upload<T>(m, &m->world_mu, mu.data(), mu.size() * sizeof(T)))) return s;
    auto mass = convert<T>(d->body_mass, m->B);
    if ((s = upload<T>(m, &m->body_mass, mass.data(), mass.size() * sizeof(T)))) return s;
    auto inert = convert<T>(d->body_inertia, 3 * (size_t)m->B);
    if ((s = upload<T>(m, &m->body_inertia, inert.data(), inert.size() * sizeof(T)))) return s;
    if ((s = upload<T>(m, (void **)&m->joint_meta, jm.data(), jm.size() * sizeof(int4)))) return s;
    if ((s = upload<T>(m, (void **)&m->joint_row, jrow.data(), jrow.size() * sizeof(int)))) return s;
    if ((s = upload<T>(m, &m->joint_frames, frames.data(), frames.size() * sizeof(double)))) return s;
    if (m->C > 0) {
        if ((s = upload<T>(m, (void **)&m->contact_body, d->contact_body, (size_t)m->C * sizeof(int)))) return s;
        if ((s = upload<T>(m, &m->contact_point, d->contact_point, 3 * (size_t)m->C * sizeof(double)))) return s;
    }
    if (m->terrain_kind == KAMINO_TERRAIN_HEIGHTFIELD) {
        if ((s = upload<T>(m, &m->hf_heights, d->hf_heights, (size_t)m->hf_nx * m->hf_ny * sizeof(double)))) return s;
    }
    auto qq = convert<T>(q0.data(), q0.size());
    if ((s = upload<T>(m, &m->q0, qq.data(), qq.size() * sizeof(T)))) return s;
    std::vector<T> uu(6 * (size_t)m->B, T(0));
    if (d->body_u0)
        for (size_t i = 0; i < uu.size(); ++i) uu[i] = (T)d->body_u0[i];
    if ((s = upload<T>(m, &m->u0, uu.data(), uu.size() * sizeof(T)))) return s;
    return KAMINO_OK;
}

template <typename T>
ModelView<T> view(const kamino_model_s *m) {
    ModelView<T> v{};
    v.num_worlds = m->W;
    v.n_act_max = m->n_act_max;
    v.world_a = m->world_a;
    v.world_b = m->world_b;
    v.world_c = m->world_c;
    v.joint_drow = m->joint_drow;
    v.joint_lslot = m->joint_lslot;
    v.joint_dyn = m->joint_dyn;
    v.world_mu = (const T *)m->world_mu;
    v.body_mass = (const T *)m->body_mass;
    v.body_inertia = (const T *)m->body_inertia;
    v.joint_meta = m->joint_meta;
    v.joint_row = m->joint_row;
    v.joint_frames = (const double *)m->joint_frames;
    v.contact_body = m->contact_body;
    v.contact_point = (const double *)m->contact_point;
    v.terrain_kind = m->terrain_kind;
    v.hf_nx = m->hf_nx;
    v.hf_ny = m->hf_ny;
    v.hf_x0 = m->hf_x0;
    v.hf_y0 = m->hf_y0;
    v.hf_cell = m->hf_cell;
    v.hf_heights = (const double *)m->hf_heights;
    v.gx = (T)m->g[0];
    v.gy = (T)m->g[1];
    v.gz = (T)m->g[2];
    return v;
}

size_t esize(const kamino_model_s *m) { return m->precision == KAMINO_FP64 ? sizeof(double) : sizeof(float); }

// Shared memory of a persistent CTA for bucket b with `group` threads per world and panel `nbp`;
// 0 when the configuration does not fit.
size_t persistent_smem(const kamino_model_s *m, const Bucket &b, int group, int nbp, size_t *slice) {
    if (b.units > kSlots * group) return 0;
    const int mp = std::max(((b.rows + 15) / 16) * 16, 16);
    const bool dense = m->params.cr_iters == 0;
    if (mp > (dense ? kMaxRowsPad : kMaxRowsPadSparse)) return 0;
    const Layout L = esize(m) == sizeof(double) ? make_layout<double>(b.nb, b.nj, b.nc, mp, nbp, m->nl_max, dense)
                                                : make_layout<float>(b.nb, b.nj, b.nc, mp, nbp, m->nl_max, dense);
    const size_t sl = align_up(L.total, 16);
    const int per = kThreads / group;
    const size_t total = per * sl + align_up(per * sizeof(int), 16);
    if (total > kMaxSmem) return 0;
    if (slice) *slice = sl;
    return total;
}

bool set_config(const kamino_model_s *m, Bucket &b, int group, int nbp) {
    size_t slice = 0;
    const size_t smem = persistent_smem(m, b, group, nbp, &slice);
    if (!smem) return false;
    b.group = group;
    b.panel = nbp;
    b.slice = slice;
    b.smem = smem;
    b.per_cta = kThreads / group;
    return true;
}

// Size heuristic: one warp per world up to 32 rows, two warps up to 96, four up to 160, else the
// whole CTA; larger groups when the PADMM units or the shared memory demand it.
bool choose_default(const kamino_model_s *m, Bucket &b) {
    const int pref = b.rows_pad <= 32 ? 32 : b.rows_pad <= 96 ? 64 : b.rows_pad <= 160 ? 128 : 256;
    for (int g = pref; g <= kThreads; g *= 2)
        for (int nbp : {16, 8})
            if (set_config(m, b, g, nbp)) return true;
    return false;
}

template <typename T>
kamino_status ensure_plan_ready(kamino_model_s *m) {
    if (m->plan_ready) return KAMINO_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev);
    for (int nbp : {16, 8})
        if (e == cudaSuccess) e = prepare_persistent<T>(nbp, kMaxSmem);
    if (e != cudaSuccess) return cuda_fail(e, "persistent launch set-up");
    while (m->side.size() < m->buckets.size()) {
        cudaStream_t st;
        cudaEvent_t ev;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
        m->side.push_back(st);
        m->join.push_back(ev);
    }
    if (!m->fork && (e = cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "event");
    m->plan_ready = true;
    return KAMINO_OK;
}

template <typename T>
kamino_status grid_of(kamino_model_s *m, Bucket &b) {
    int per_sm = 0;
    cudaError_t e = occupancy_persistent<T>(b.panel, b.smem, m->params.cr_iters > 0 ? 1 : 0, &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    const int need = (b.count + b.per_cta - 1) / b.per_cta;
    b.grid = std::max(1, std::min(need, std::max(per_sm, 1) * m->sm_count));
    return KAMINO_OK;
}

template <typename T>
StepArgs<T> make_args(kamino_state_s *st, double dt, int iters, double tol, const void *tau) {
    kamino_model_s *m = st->model;
    StepArgs<T> a{};
    a.m = view<T>(m);
    a.body_q = (T *)st->ptr(st->off_q);
    a.body_u = (T *)st->ptr(st->off_u);
    a.cache = (T *)st->ptr(st->off_cache);
    a.warm = (const T *)st->ptr(st->off_warm);
    a.res = (kamino_residual *)st->ptr(st->off_res);
    a.tau = (const T *)tau;
    a.world_order = nullptr;
    a.dt = (T)dt;
    a.tol = (T)tol;
    a.eta = (T)m->params.eta;
    a.rho = (T)m->params.rho;
    a.beta = (T)m->params.beta;
    a.margin = (T)m->params.margin;
    a.iters = iters;
    a.nesterov = m->params.nesterov ? 1 : 0;
    a.precond = m->params.precond ? 1 : 0;
    a.mixed = m->precision == KAMINO_MIXED ? 1 : 0;
    a.midpoint = m->params.integrator == KAMINO_INTEGRATOR_MIDPOINT ? 1 : 0;
    a.refine64 = m->params.refine64 ? 1 : 0;
    a.cr_iters = m->params.cr_iters;
    a.ncp_stop = m->params.ncp_stop ? 1 : 0;
    a.stall_window = m->params.ncp_stop ? m->params.stall_window : 0;
    a.residual_every = m->params.residual_every > 1 ? m->params.residual_every : 1;
    // the inverse may live in tensor memory when a world's shared memory keeps a second CTA off the SM
    // (the 512-column allocation then never waits for another CTA); the sparse formulation has none
    a.tmem = (sizeof(T) == 4 && a.cr_iters == 0 && m->mp_max <= 256 && m->smem > kMaxSmem / 2) ? 1 : 0;
    a.warm_mode = m->params.warm_mode;
    a.nb_max = m->nb_max;
    a.nj_max = m->nj_max;
    a.nc_max = m->nc_max;
    a.mp_max = m->mp_max;
    a.nl_max = m->nl_max;
    return a;
}

// Persistent launch of one bucket on `stream` (its counter must be zero).
template <typename T>
kamino_status launch_bucket(kamino_state_s *st, const StepArgs<T> &base, int bi, cudaStream_t stream) {
    kamino_model_s *m = st->model;
    Bucket &b = m->buckets[bi];
    if (b.grid == 0) {
        kamino_status s = grid_of<T>(m, b);
        if (s) return s;
    }
    StepArgs<T> a = base;
    a.nb_max = b.nb;
    a.nj_max = b.nj;
    a.nc_max = b.nc;
    a.mp_max = std::max(((b.rows + 15) / 16) * 16, 16);
    // tensor memory when one 256-thread group fills the CTA and its shared memory keeps a second
    // CTA off the SM
    a.tmem = (sizeof(T) == 4 && a.cr_iters == 0 && b.group == kThreads && a.mp_max <= 256 && b.smem > kMaxSmem / 2)
                 ? 1 : 0;
    PersistentArgs p{};
    p.worlds = b.d_worlds;
    p.count = b.count;
    p.counter = (int *)st->ptr(st->off_cnt) + bi;
    p.group = b.group;
    p.slice_bytes = b.slice;
    cudaError_t e = launch_persistent<T>(a, p, b.panel, b.grid, b.smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "persistent step launch");
    return KAMINO_OK;
}

template <typename T>
kamino_status do_step(kamino_state_s *st, double dt, int iters, double tol, const void *tau, cudaStream_t stream) {
    kamino_model_s *m = st->model;
    const StepArgs<T> a = make_args<T>(st, dt, iters, tol, tau);
    if (m->launch_mode == KAMINO_LAUNCH_SINGLE) {
        if (!m->prepared) {
            cudaError_t e = prepare_step<T>(m->nb_panel, kMaxSmem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute (step kernel shared memory)");
            m->prepared = true;
        }
        StepArgs<T> b = a;
        if (m->params.schedule == KAMINO_SCHEDULE_LONGEST_FIRST && m->W > 1) {
            int *order = (int *)st->ptr(st->off_order);
            cudaError_t e = launch_order((const kamino_residual *)st->ptr(st->off_res), m->W, order, stream);
            if (e != cudaSuccess) return cuda_fail(e, "world order launch");
            b.world_order = order;
        }
        cudaError_t e = launch_step<T>(b, m->W, m->nb_panel, m->smem, stream);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel launch");
        return KAMINO_OK;
    }
    kamino_status s = ensure_plan_ready<T>(m);
    if (s) return s;
    const int nbk = (int)m->buckets.size();
    cudaError_t e = cudaMemsetAsync(st->ptr(st->off_cnt), 0, nbk * sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
    if (nbk > 1) {
        if ((e = cudaEventRecord(m->fork, stream)) != cudaSuccess) return cuda_fail(e, "fork");
        for (int b = 1; b < nbk; ++b)
            if ((e = cudaStreamWaitEvent(m->side[b], m->fork, 0)) != cudaSuccess) return cuda_fail(e, "fork wait");
    }
    for (int b = 0; b < nbk; ++b) {
        s = launch_bucket<T>(st, a, b, b == 0 ? stream : m->side[b]);
        if (s) return s;
    }
    for (int b = 1; b < nbk; ++b) {
        if ((e = cudaEventRecord(m->join[b], m->side[b])) != cudaSuccess) return cuda_fail(e, "join");
        if ((e = cudaStreamWaitEvent(stream, m->join[b], 0)) != cudaSuccess) return cuda_fail(e, "join wait");
    }
    return KAMINO_OK;
}

// Forward kinematics for resets over every world of the state (kamino_fk).
template <typename T>
kamino_status do_fk(kamino_state_s *st, const double *target, const int32_t *select, const int32_t *fixed,
                           int iters, double tol, cudaStream_t stream) {
    kamino_model_s *m = st->model;
    const FkLayout L = make_fk_layout(m->nb_max, m->fk_rows_max);
    if (L.total > kMaxSmem)
        return fail(KAMINO_E_UNSUPPORTED, "forward kinematics of a world with %d rows needs %zu bytes of shared memory "
                    "(at most %zu)", m->fk_rows_max, L.total, kMaxSmem);
    FkArgs<T> a{};
    a.m = view<T>(m);
    a.body_q = (T *)st->ptr(st->off_q);
    a.res = (kamino_residual *)st->ptr(st->off_res);
    a.target = target;
    a.select = select;
    a.fixed = fixed;
    a.iters = iters;
    a.tol = tol;
    a.nb_max = m->nb_max;
    a.m_max = m->fk_rows_max;
    cudaError_t e = launch_fk<T>(a, m->W, L.total, stream);
    if (e != cudaSuccess) return cuda_fail(e, "forward kinematics launch");
    return KAMINO_OK;
}

// Autotuner: time every feasible configuration of every bucket on the state's worlds.
template <typename T>
kamino_status autotune(kamino_state_s *st, double dt, int iters, double tol, const void *tau, cudaStream_t stream) {
    kamino_model_s *m = st->model;
    kamino_status s = ensure_plan_ready<T>(m);
    if (s) return s;
    const StepArgs<T> a = make_args<T>(st, dt, iters, tol, tau);
    char *snap = nullptr;
    cudaError_t e = cudaMalloc(&snap, st->bytes);
    if (e != cudaSuccess) return cuda_fail(e, "autotune snapshot");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    e = cudaMemcpyAsync(snap, st->base, st->bytes, cudaMemcpyDeviceToDevice, stream);
    for (size_t bi = 0; bi < m->buckets.size() && e == cudaSuccess && !s; ++bi) {
        Bucket &b = m->buckets[bi];
        const Bucket keep = b;
        float best = 1e30f;
        int best_g = b.group, best_nb = b.panel;
        for (int g : {32, 64, 128, 256}) {
            for (int nbp : {16, 8}) {
                if (!set_config(m, b, g, nbp)) continue;
                b.grid = 0;
                float t = 1e30f;
                for (int rep = 0; rep < 3 && !s; ++rep) {
                    cudaMemcpyAsync(st->base, snap, st->bytes, cudaMemcpyDeviceToDevice, stream);
                    cudaMemsetAsync(st->ptr(st->off_cnt), 0, m->buckets.size() * sizeof(int), stream);
                    cudaEventRecord(e0, stream);
                    s = launch_bucket<T>(st, a, (int)bi, stream);
                    cudaEventRecord(e1, stream);
                    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t = std::min(t, ms);
                }
                if (s || e != cudaSuccess) break;
                if (t < best) { best = t; best_g = g; best_nb = nbp; }
            }
            if (s || e != cudaSuccess) break;
        }
        if (s || e != cudaSuccess) { b = keep; break; }
        set_config(m, b, best_g, best_nb);
        b.grid = 0;
        b.tuned_ms = best;
    }
    // whole step: the tuned persistent plan against one CTA per world, keep the faster
    float t_mode[2] = {1e30f, 1e30f};
    const int modes[2] = {KAMINO_LAUNCH_PERSISTENT, KAMINO_LAUNCH_SINGLE};
    for (int mi = 0; mi < 2 && !s && e == cudaSuccess; ++mi) {
        m->launch_mode = modes[mi];
        for (int rep = 0; rep < 3 && !s; ++rep) {
            cudaMemcpyAsync(st->base, snap, st->bytes, cudaMemcpyDeviceToDevice, stream);
            cudaEventRecord(e0, stream);
            s = do_step<T>(st, dt, iters, tol, tau, stream);
            cudaEventRecord(e1, stream);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t_mode[mi] = std::min(t_mode[mi], ms);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(st->base, snap, st->bytes, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(snap);
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    m->launch_mode = t_mode[1] < t_mode[0] ? KAMINO_LAUNCH_SINGLE : KAMINO_LAUNCH_PERSISTENT;
    return KAMINO_OK;
}

}  // namespace

extern "C" {

const char *kamino_last_error(void) { return g_error.c_str(); }

// Shared-memory working set of the single-launch plan and the persistent configuration of every
// bucket, for the formulation the parameters select (dense, or sparse with params.cr_iters > 0).
static kamino_status configure(kamino_model_s *m) {
    const bool dense = m->params.cr_iters == 0;
    m->smem = 0;
    m->prepared = false;
    for (int nbp : {16, 8}) {
        const int mp = std::max(((m->max_rows + 15) / 16) * 16, 16);
        if (mp > (dense ? kMaxRowsPad : kMaxRowsPadSparse)) continue;
        const Layout L = m->precision == KAMINO_FP64
                             ? make_layout<double>(m->nb_max, m->nj_max, m->nc_max, mp, nbp, m->nl_max, dense)
                             : make_layout<float>(m->nb_max, m->nj_max, m->nc_max, mp, nbp, m->nl_max, dense);
        if (L.total <= kMaxSmem) {
            m->nb_panel = nbp;
            m->mp_max = mp;
            m->smem = L.total;
            break;
        }
    }
    if (m->smem == 0)
        return fail(KAMINO_E_UNSUPPORTED,
                    "a world needs %d constraint rows; the %s formulation's shared-memory working set exceeds %zu "
                    "bytes (max %d padded rows)", m->max_rows, dense ? "dense" : "sparse", kMaxSmem,
                    dense ? kMaxRowsPad : kMaxRowsPadSparse);
    for (auto &b : m->buckets) {
        b.grid = 0;
        if (!choose_default(m, b))
            return fail(KAMINO_E_UNSUPPORTED, "no persistent configuration fits the bucket of %d rows", b.rows_pad);
    }
    return KAMINO_OK;
}

kamino_status kamino_model_create(const kamino_model_desc *d, kamino_model_t *out) {
    if (!d || !out) return fail(KAMINO_E_INVALID_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (d->num_worlds < 1) return fail(KAMINO_E_INVALID_ARG, "num_worlds must be >= 1 (got %d)", d->num_worlds);
    if (d->precision != KAMINO_FP32 && d->precision != KAMINO_FP64 && d->precision != KAMINO_MIXED)
        return fail(KAMINO_E_INVALID_ARG, "precision must be KAMINO_FP32, KAMINO_MIXED or KAMINO_FP64");
    if (!d->world_body_offset || !d->world_joint_offset || !d->world_contact_offset || !d->world_num_actuators ||
        !d->world_mu)
        return fail(KAMINO_E_INVALID_ARG, "per-world arrays must not be NULL");
    kamino_status s = check_params(d->params);
    if (s) return s;
    const int W = d->num_worlds;
    if (d->world_body_offset[0] != 0 || d->world_joint_offset[0] != 0 || d->world_contact_offset[0] != 0)
        return fail(KAMINO_E_TOPOLOGY, "world offsets must start at 0");
    for (int w = 0; w < W; ++w) {
        if (d->world_body_offset[w + 1] <= d->world_body_offset[w])
            return fail(KAMINO_E_TOPOLOGY, "world %d has no bodies (offsets must increase)", w);
        if (d->world_joint_offset[w + 1] < d->world_joint_offset[w] ||
            d->world_contact_offset[w + 1] < d->world_contact_offset[w])
            return fail(KAMINO_E_TOPOLOGY, "world %d: joint/contact offsets decrease", w);
        if (d->world_num_actuators[w] < 0) return fail(KAMINO_E_TOPOLOGY, "world %d: negative actuator count", w);
        if (!(d->world_mu[w] >= 0.0) || !std::isfinite(d->world_mu[w]))
            return fail(KAMINO_E_TOPOLOGY, "world %d: friction must be finite and >= 0", w);
    }
    const int B = d->world_body_offset[W], J = d->world_joint_offset[W], C = d->world_contact_offset[W];
    if (!d->body_mass || !d->body_inertia) return fail(KAMINO_E_INVALID_ARG, "body arrays must not be NULL");
    if (J > 0 && (!d->joint_type || !d->joint_parent || !d->joint_child || !d->joint_actuator ||
                  !d->joint_frame_parent || !d->joint_frame_child))
        return fail(KAMINO_E_INVALID_ARG, "joint arrays must not be NULL");
    if (C > 0 && (!d->contact_body || !d->contact_point))
        return fail(KAMINO_E_INVALID_ARG, "contact arrays must not be NULL");
    for (int b = 0; b < B; ++b) {
        if (!(d->body_mass[b] > 0.0) || !std::isfinite(d->body_mass[b]))
            return fail(KAMINO_E_TOPOLOGY, "body %d: mass must be finite and > 0", b);
        for (int k = 0; k < 3; ++k)
            if (!(d->body_inertia[3 * b + k] > 0.0) || !std::isfinite(d->body_inertia[3 * b + k]))
                return fail(KAMINO_E_TOPOLOGY, "body %d: inertia must be finite and > 0", b);
    }
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(d->gravity[k])) return fail(KAMINO_E_INVALID_ARG, "gravity must be finite");
    for (int b = 0; b < B; ++b) {
        if (d->body_q0) {
            const double *q = d->body_q0 + 7 * (size_t)b;
            for (int k = 0; k < 7; ++k)
                if (!std::isfinite(q[k])) return fail(KAMINO_E_TOPOLOGY, "body %d: initial pose not finite", b);
            if (!(q[3] * q[3] + q[4] * q[4] + q[5] * q[5] + q[6] * q[6] > 1e-24))
                return fail(KAMINO_E_TOPOLOGY, "body %d: initial quaternion is not normalisable", b);
        }
        if (d->body_u0)
            for (int k = 0; k < 6; ++k)
                if (!std::isfinite(d->body_u0[6 * (size_t)b + k]))
                    return fail(KAMINO_E_TOPOLOGY, "body %d: initial twist not finite", b);
    }
    if (d->terrain_kind < KAMINO_TERRAIN_NONE || d->terrain_kind > KAMINO_TERRAIN_HEIGHTFIELD)
        return fail(KAMINO_E_INVALID_ARG, "terrain_kind %d is not a KAMINO_TERRAIN_* value", d->terrain_kind);
    if (d->terrain_kind == KAMINO_TERRAIN_HEIGHTFIELD) {
        if (d->hf_nx < 2 || d->hf_ny < 2 || !(d->hf_cell > 0.0) || !d->hf_heights)
            return fail(KAMINO_E_INVALID_ARG, "heightfield needs nx, ny >= 2, cell > 0 and heights");
        for (long i = 0; i < (long)d->hf_nx * d->hf_ny; ++i)
            if (!std::isfinite(d->hf_heights[i])) return fail(KAMINO_E_INVALID_ARG, "heightfield height %ld not finite", i);
    }

    auto *m = new kamino_model_s();
    m->precision = d->precision;
    m->W = W; m->B = B; m->J = J; m->C = C;
    m->params = d->params;
    m->terrain_kind = d->terrain_kind;
    m->hf_nx = d->hf_nx; m->hf_ny = d->hf_ny;
    m->hf_x0 = d->hf_origin[0]; m->hf_y0 = d->hf_origin[1]; m->hf_cell = d->hf_cell;
    for (int k = 0; k < 3; ++k) m->g[k] = d->gravity[k];

    std::vector<int4> wa(W), wb(W), jm(J);
    std::vector<int> jrow(J);
    std::vector<double> frames(14 * (size_t)J);
    const bool has_dyn = J > 0 && (d->joint_drive != nullptr || d->joint_limit != nullptr);
    JointDyn jd;
    if (has_dyn) {
        jd.wc.assign(W, make_int4(0, 0, 0, 0));
        jd.drow.assign(J, -1);
        jd.lslot.assign(J, -1);
        jd.dyn.assign(8 * (size_t)J, 0.0);
    }
    int cache = 0;
    for (int w = 0; w < W; ++w) {
        const int b0 = d->world_body_offset[w], nb = d->world_body_offset[w + 1] - b0;
        const int j0 = d->world_joint_offset[w], nj = d->world_joint_offset[w + 1] - j0;
        const int c0 = d->world_contact_offset[w], nc = d->world_contact_offset[w + 1] - c0;
        const int nact = d->world_num_actuators[w];
        int row = 0, ncoord = 0;
        for (int j = j0; j < j0 + nj; ++j) {
            const int t = d->joint_type[j], par = d->joint_parent[j], ch = d->joint_child[j], act = d->joint_actuator[j];
            if (rows_of(t) < 0) { delete m; return fail(KAMINO_E_TOPOLOGY, "joint %d: unknown type %d", j, t); }
            if (par < -1 || par >= nb || ch < 0 || ch >= nb || par == ch) {
                delete m;
                return fail(KAMINO_E_TOPOLOGY, "joint %d (world %d): parent %d / child %d out of range [0, %d) or equal",
                            j, w, par, ch, nb);
            }
            if (act < -1 || act >= nact) {
                delete m;
                return fail(KAMINO_E_TOPOLOGY, "joint %d: actuator slot %d out of range [-1, %d)", j, act, nact);
            }
            if (act >= 0 && t != KAMINO_JOINT_REVOLUTE && t != KAMINO_JOINT_PRISMATIC) {
                delete m;
                return fail(KAMINO_E_TOPOLOGY, "joint %d: only revolute and prismatic joints carry actuators", j);
            }
            for (int side = 0; side < 2; ++side) {
                const double *f = (side == 0 ? d->joint_frame_parent : d->joint_frame_child) + 7 * (size_t)j;
                const double n = std::sqrt(f[3] * f[3] + f[4] * f[4] + f[5] * f[5] + f[6] * f[6]);
                if (!(n > 1e-12) || !std::isfinite(n)) {
                    delete m;
                    return fail(KAMINO_E_TOPOLOGY, "joint %d: frame quaternion is not normalisable", j);
                }
                if (!std::isfinite(f[0]) || !std::isfinite(f[1]) || !std::isfinite(f[2])) {
                    delete m;
                    return fail(KAMINO_E_TOPOLOGY, "joint %d: frame position not finite", j);
                }
                double *o = frames.data() + 14 * (size_t)j + 7 * side;
                for (int k = 0; k < 3; ++k) o[k] = f[k];
                for (int k = 3; k < 7; ++k) o[k] = f[k] / n;
            }
            jm[j] = make_int4(t, par, ch, act);
            jrow[j] = row;
            row += rows_of(t);
            ncoord += (t == KAMINO_JOINT_REVOLUTE || t == KAMINO_JOINT_PRISMATIC) ? 1 : 0;
        }
        m->fk_rows_max = std::max(m->fk_rows_max, row + ncoord);
        // joint-space dynamics: a drive row per driven joint after the joint rows, then one limit
        // candidate per finite bound
        int nlc = 0;
        if (has_dyn) {
            for (int j = j0; j < j0 + nj; ++j) {
                const int t = d->joint_type[j];
                const bool coord = t == KAMINO_JOINT_REVOLUTE || t == KAMINO_JOINT_PRISMATIC;
                double *o = jd.dyn.data() + 8 * (size_t)j;
                o[5] = -INFINITY; o[6] = INFINITY;
                if (d->joint_drive) {
                    const double *dr = d->joint_drive + 5 * (size_t)j;
                    if (dr[0] != KAMINO_DRIVE_TORQUE && dr[0] != KAMINO_DRIVE_PD) {
                        delete m;
                        return fail(KAMINO_E_TOPOLOGY, "joint %d: drive mode %g is not a KAMINO_DRIVE_* value", j, dr[0]);
                    }
                    for (int k = 1; k < 5; ++k)
                        if (!(dr[k] >= 0.0) || !std::isfinite(dr[k])) {
                            delete m;
                            return fail(KAMINO_E_TOPOLOGY, "joint %d: drive gains must be finite and >= 0", j);
                        }
                    const bool pd = dr[0] == KAMINO_DRIVE_PD;
                    const bool any = dr[1] > 0.0 || dr[2] > 0.0 || dr[3] > 0.0 || dr[4] > 0.0;
                    if (any && !coord) {
                        delete m;
                        return fail(KAMINO_E_TOPOLOGY, "joint %d: only revolute and prismatic joints carry drives", j);
                    }
                    for (int k = 0; k < 5; ++k) o[k] = dr[k];
                    // torque mode applies the actuation as a force: its row holds armature and damping only
                    if (pd ? any : (dr[3] > 0.0 || dr[4] > 0.0)) jd.drow[j] = row++;
                }
            }
            for (int j = j0; j < j0 + nj; ++j) {
                if (!d->joint_limit) break;
                const double lo = d->joint_limit[2 * (size_t)j], hi = d->joint_limit[2 * (size_t)j + 1];
                if (std::isnan(lo) || std::isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY) {
                    delete m;
                    return fail(KAMINO_E_TOPOLOGY, "joint %d: limits (%g, %g) must satisfy lower <= upper", j, lo, hi);
                }
                const int nf = (std::isfinite(lo) ? 1 : 0) + (std::isfinite(hi) ? 1 : 0);
                if (nf == 0) continue;
                const int t = d->joint_type[j];
                if (t != KAMINO_JOINT_REVOLUTE && t != KAMINO_JOINT_PRISMATIC) {
                    delete m;
                    return fail(KAMINO_E_TOPOLOGY, "joint %d: only revolute and prismatic joints carry limits", j);
                }
                double *o = jd.dyn.data() + 8 * (size_t)j;
                o[5] = lo; o[6] = hi;
                jd.lslot[j] = nlc;
                nlc += nf;
            }
            jd.wc[w] = make_int4(nlc, 0, 0, 0);
            m->nl_max = std::max(m->nl_max, nlc);
        }
        for (int c = c0; c < c0 + nc; ++c) {
            if (d->contact_body[c] < 0 || d->contact_body[c] >= nb) {
                delete m;
                return fail(KAMINO_E_TOPOLOGY, "contact candidate %d: body %d out of range [0, %d)", c, d->contact_body[c], nb);
            }
            const double *pt = d->contact_point + 3 * (size_t)c;
            if (!std::isfinite(pt[0]) || !std::isfinite(pt[1]) || !std::isfinite(pt[2])) {
                delete m;
                return fail(KAMINO_E_TOPOLOGY, "contact candidate %d: point not finite", c);
            }
        }
        if (nc > kMaxCandidates) {
            delete m;
            return fail(KAMINO_E_UNSUPPORTED, "world %d has %d contact candidates (max %d)", w, nc, kMaxCandidates);
        }
        wa[w] = make_int4(b0, j0, c0, cache);
        wb[w] = make_int4(nb, nj, nc, row);
        {
            const int rows = row + nlc + 3 * nc;
            const int rp = std::max(32, ((rows + 31) / 32) * 32);
            Bucket *bk = nullptr;
            for (auto &b : m->buckets)
                if (b.rows_pad == rp) bk = &b;
            if (!bk) { m->buckets.emplace_back(); bk = &m->buckets.back(); bk->rows_pad = rp; }
            bk->worlds.push_back(w);
            bk->count++;
            bk->nb = std::max(bk->nb, nb);
            bk->nj = std::max(bk->nj, nj);
            bk->nc = std::max(bk->nc, nc);
            bk->rows = std::max(bk->rows, rows);
            bk->units = std::max(bk->units, row + nlc + nc);
        }
        cache += row + nlc + 3 * nc;
        m->world_cache.push_back(row + nlc + 3 * nc);
        m->nb_max = std::max(m->nb_max, nb);
        m->nj_max = std::max(m->nj_max, nj);
        m->nc_max = std::max(m->nc_max, nc);
        m->max_rows = std::max(m->max_rows, row + nlc + 3 * nc);
        m->n_act_max = std::max(m->n_act_max, nact);
    }
    m->cache_len = cache;
    std::sort(m->buckets.begin(), m->buckets.end(),
              [](const Bucket &a, const Bucket &b) { return a.rows_pad > b.rows_pad; });
    if (kamino_status st = configure(m)) {
        delete m;
        return st;
    }
    std::vector<double> q0(7 * (size_t)B, 0.0);
    for (int b = 0; b < B; ++b) {
        if (d->body_q0) {
            for (int k = 0; k < 7; ++k) q0[7 * b + k] = d->body_q0[7 * b + k];
        } else {
            q0[7 * b + 6] = 1.0;
        }
    }
    kamino_status st = d->precision == KAMINO_FP64 ? build_device<double>(m, d, wa, wb, jm, jrow, frames, q0, jd)
                                                   : build_device<float>(m, d, wa, wb, jm, jrow, frames, q0, jd);
    if (st) { delete m; return st; }
    for (auto &b : m->buckets) {
        if ((st = upload<float>(m, (void **)&b.d_worlds, b.worlds.data(), b.worlds.size() * sizeof(int)))) {
            delete m;
            return st;
        }
    }
    *out = m;
    return KAMINO_OK;
}

kamino_status kamino_model_destroy(kamino_model_t model) {
    delete model;
    return KAMINO_OK;
}

kamino_status kamino_model_get_info(kamino_model_t m, kamino_model_info *out) {
    if (!m || !out) return fail(KAMINO_E_INVALID_ARG, "model and out must not be NULL");
    out->num_worlds = m->W;
    out->num_bodies = m->B;
    out->max_bodies = m->nb_max;
    out->max_rows = m->max_rows;
    out->n_act_max = m->n_act_max;
    out->cache_len = m->cache_len;
    out->precision = m->precision;
    out->threads_per_world = kThreads;
    out->smem_bytes = (int64_t)m->smem;
    return KAMINO_OK;
}

kamino_status kamino_model_set_params(kamino_model_t m, const kamino_solver_params *p) {
    if (!m || !p) return fail(KAMINO_E_INVALID_ARG, "model and params must not be NULL");
    kamino_status s = check_params(*p);
    if (s) return s;
    const bool was_dense = m->params.cr_iters == 0;
    const kamino_solver_params keep = m->params;
    m->params = *p;
    if ((p->cr_iters == 0) != was_dense) {        // the other formulation: another working set
        if ((s = configure(m))) {
            m->params = keep;
            configure(m);
            return s;
        }
    }
    return KAMINO_OK;
}

static void state_layout(kamino_model_t m, kamino_state_s *s) {
    const size_t esz = m->precision == KAMINO_FP64 ? sizeof(double) : sizeof(float);
    size_t o = 0;
    auto take = [&](size_t &f, size_t bytes) { f = o; o = align_up(o + bytes, 256); };
    take(s->off_q, 7 * (size_t)m->B * esz);
    take(s->off_u, 6 * (size_t)m->B * esz);
    take(s->off_cache, (size_t)m->cache_len * esz);
    take(s->off_warm, (size_t)m->cache_len * esz);
    take(s->off_res, (size_t)m->W * sizeof(kamino_residual));
    take(s->off_tau, (size_t)m->W * std::max(m->n_act_max, 1) * esz);
    take(s->off_cnt, std::max<size_t>(m->buckets.size(), 1) * sizeof(int));
    take(s->off_order, (size_t)m->W * sizeof(int));
    s->bytes = o;
}

kamino_status kamino_state_bytes(kamino_model_t m, size_t *bytes) {
    if (!m || !bytes) return fail(KAMINO_E_INVALID_ARG, "model and bytes must not be NULL");
    kamino_state_s tmp;
    state_layout(m, &tmp);
    *bytes = tmp.bytes;
    return KAMINO_OK;
}

kamino_status kamino_state_alloc(kamino_model_t m, void *buffer, size_t bytes, kamino_state_t *out) {
    if (!m || !out) return fail(KAMINO_E_INVALID_ARG, "model and out must not be NULL");
    *out = nullptr;
    auto *s = new kamino_state_s();
    s->model = m;
    state_layout(m, s);
    if (buffer) {
        if (bytes < s->bytes) {
            const size_t need = s->bytes;
            delete s;
            return fail(KAMINO_E_NOMEM, "state buffer has %zu bytes, needs %zu", bytes, need);
        }
        if (((uintptr_t)buffer) % 256 != 0) {
            delete s;
            return fail(KAMINO_E_INVALID_ARG, "state buffer must be 256-byte aligned");
        }
        s->base = (char *)buffer;
    } else {
        cudaError_t e = cudaMalloc((void **)&s->base, s->bytes);
        if (e != cudaSuccess) { delete s; return cuda_fail(e, "cudaMalloc (state)"); }
        s->owned = true;
    }
    const size_t esz = m->precision == KAMINO_FP64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaMemset(s->base, 0, s->bytes);
    if (e == cudaSuccess) e = cudaMemcpy(s->ptr(s->off_q), m->q0, 7 * (size_t)m->B * esz, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->ptr(s->off_u), m->u0, 6 * (size_t)m->B * esz, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        if (s->owned) cudaFree(s->base);
        delete s;
        return cuda_fail(e, "state initialisation");
    }
    *out = s;
    return KAMINO_OK;
}

kamino_status kamino_state_free(kamino_state_t s) {
    if (!s) return KAMINO_OK;
    if (s->owned) cudaFree(s->base);
    delete s;
    return KAMINO_OK;
}

static kamino_status buffer_of(kamino_state_t s, kamino_buffer which, void **ptr, int64_t *count, size_t *esz) {
    const kamino_model_s *m = s->model;
    const size_t e = m->precision == KAMINO_FP64 ? sizeof(double) : sizeof(float);
    switch (which) {
        case KAMINO_BUF_BODY_Q: *ptr = s->ptr(s->off_q); *count = 7 * (int64_t)m->B; *esz = e; break;
        case KAMINO_BUF_BODY_U: *ptr = s->ptr(s->off_u); *count = 6 * (int64_t)m->B; *esz = e; break;
        case KAMINO_BUF_CACHE: *ptr = s->ptr(s->off_cache); *count = m->cache_len; *esz = e; break;
        case KAMINO_BUF_WARM: *ptr = s->ptr(s->off_warm); *count = m->cache_len; *esz = e; break;
        case KAMINO_BUF_RESIDUAL: *ptr = s->ptr(s->off_res); *count = m->W; *esz = sizeof(kamino_residual); break;
        case KAMINO_BUF_TAU: *ptr = s->ptr(s->off_tau); *count = (int64_t)m->W * m->n_act_max; *esz = e; break;
        default: return fail(KAMINO_E_INVALID_ARG, "unknown buffer %d", (int)which);
    }
    return KAMINO_OK;
}

kamino_status kamino_state_get(kamino_state_t s, kamino_buffer which, void **dev_ptr, int64_t *count) {
    if (!s || !dev_ptr || !count) return fail(KAMINO_E_INVALID_ARG, "state, dev_ptr and count must not be NULL");
    size_t esz;
    return buffer_of(s, which, dev_ptr, count, &esz);
}

static kamino_status copy(kamino_state_t s, kamino_buffer which, void *host, int64_t count, void *stream, bool up) {
    if (!s || !host) return fail(KAMINO_E_INVALID_ARG, "state and host pointer must not be NULL");
    void *dev;
    int64_t n;
    size_t esz;
    kamino_status st = buffer_of(s, which, &dev, &n, &esz);
    if (st) return st;
    if (count < 0 || count > n) return fail(KAMINO_E_INVALID_ARG, "count %lld outside [0, %lld]", (long long)count, (long long)n);
    cudaError_t e = up ? cudaMemcpyAsync(dev, host, (size_t)count * esz, cudaMemcpyHostToDevice, (cudaStream_t)stream)
                       : cudaMemcpyAsync(host, dev, (size_t)count * esz, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, up ? "state upload" : "state download");
    return KAMINO_OK;
}

kamino_status kamino_state_upload(kamino_state_t s, kamino_buffer which, const void *host, int64_t count, void *stream) {
    return copy(s, which, (void *)host, count, stream, true);
}

kamino_status kamino_state_download(kamino_state_t s, kamino_buffer which, void *host, int64_t count, void *stream) {
    return copy(s, which, host, count, stream, false);
}

kamino_status kamino_step(kamino_state_t s, double dt, int32_t iters, double tol, const void *tau_dev, void *stream) {
    if (!s) return fail(KAMINO_E_INVALID_ARG, "state must not be NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(KAMINO_E_INVALID_ARG, "dt must be finite and > 0");
    if (iters < 1) return fail(KAMINO_E_INVALID_ARG, "iters must be >= 1 (got %d)", iters);
    if (!(tol >= 0.0)) return fail(KAMINO_E_INVALID_ARG, "tol must be >= 0");
    return s->model->precision == KAMINO_FP64 ? do_step<double>(s, dt, iters, tol, tau_dev, (cudaStream_t)stream)
                                              : do_step<float>(s, dt, iters, tol, tau_dev, (cudaStream_t)stream);
}

kamino_status kamino_fk(kamino_state_t s, const double *joint_target_dev, const int32_t *joint_select_dev,
                        const int32_t *body_fixed_dev, int32_t max_iters, double tol, void *stream) {
    if (!s || !joint_target_dev) return fail(KAMINO_E_INVALID_ARG, "state and joint_target_dev must not be NULL");
    if (max_iters < 1) return fail(KAMINO_E_INVALID_ARG, "max_iters must be >= 1 (got %d)", max_iters);
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(KAMINO_E_INVALID_ARG, "tol must be finite and >= 0");
    return s->model->precision == KAMINO_FP64
               ? do_fk<double>(s, joint_target_dev, joint_select_dev, body_fixed_dev, max_iters, tol, (cudaStream_t)stream)
               : do_fk<float>(s, joint_target_dev, joint_select_dev, body_fixed_dev, max_iters, tol, (cudaStream_t)stream);
}

kamino_status kamino_residuals(kamino_state_t s, kamino_residual *out_dev, void *stream) {
    if (!s || !out_dev) return fail(KAMINO_E_INVALID_ARG, "state and out_dev must not be NULL");
    cudaError_t e = cudaMemcpyAsync(out_dev, s->ptr(s->off_res), (size_t)s->model->W * sizeof(kamino_residual),
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "residual copy");
    return KAMINO_OK;
}

kamino_status kamino_plan_get(kamino_model_t m, kamino_bucket_info *out, int32_t capacity, int32_t *count,
                              int32_t *mode) {
    if (!m || !count || !mode || (capacity > 0 && !out))
        return fail(KAMINO_E_INVALID_ARG, "model, count and mode must not be NULL");
    *count = (int32_t)m->buckets.size();
    *mode = m->launch_mode;
    for (int i = 0; i < capacity && i < (int)m->buckets.size(); ++i) {
        const Bucket &b = m->buckets[i];
        out[i].rows_pad = b.rows_pad;
        out[i].num_worlds = b.count;
        out[i].group_threads = b.group;
        out[i].panel = b.panel;
        out[i].grid = b.grid;
        out[i].worlds_per_cta = b.per_cta;
        out[i].tuned_ms = b.tuned_ms;
        out[i].reserved = 0.0f;
    }
    return KAMINO_OK;
}

kamino_status kamino_plan_set_mode(kamino_model_t m, int32_t mode) {
    if (!m) return fail(KAMINO_E_INVALID_ARG, "model must not be NULL");
    if (mode != KAMINO_LAUNCH_SINGLE && mode != KAMINO_LAUNCH_PERSISTENT)
        return fail(KAMINO_E_INVALID_ARG, "mode %d is not a KAMINO_LAUNCH_* value", mode);
    m->launch_mode = mode;
    return KAMINO_OK;
}

kamino_status kamino_autotune(kamino_state_t s, double dt, int32_t iters, double tol, const void *tau_dev,
                              void *stream) {
    if (!s) return fail(KAMINO_E_INVALID_ARG, "state must not be NULL");
    if (!(dt > 0.0) || iters < 1 || !(tol >= 0.0)) return fail(KAMINO_E_INVALID_ARG, "bad dt / iters / tol");
    return s->model->precision == KAMINO_FP64 ? autotune<double>(s, dt, iters, tol, tau_dev, (cudaStream_t)stream)
                                              : autotune<float>(s, dt, iters, tol, tau_dev, (cudaStream_t)stream);
}

kamino_status kamino_graph_create(kamino_state_t s, double dt, int32_t iters, double tol, const void *tau_dev,
                                  void *stream, kamino_graph_t *out) {
    if (!s || !out) return fail(KAMINO_E_INVALID_ARG, "state and out must not be NULL");
    *out = nullptr;
    if (!stream) return fail(KAMINO_E_INVALID_ARG, "graph capture needs a non-default stream");
    if (!(dt > 0.0) || iters < 1 || !(tol >= 0.0)) return fail(KAMINO_E_INVALID_ARG, "bad dt / iters / tol");
    kamino_model_s *m = s->model;
    kamino_status st;
    // everything that is not a stream operation happens before the capture
    if (m->precision == KAMINO_FP64) {
        if ((st = ensure_plan_ready<double>(m))) return st;
        for (auto &b : m->buckets)
            if (!b.grid && (st = grid_of<double>(m, b))) return st;
        if (!m->prepared) { prepare_step<double>(m->nb_panel, kMaxSmem); m->prepared = true; }
    } else {
        if ((st = ensure_plan_ready<float>(m))) return st;
        for (auto &b : m->buckets)
            if (!b.grid && (st = grid_of<float>(m, b))) return st;
        if (!m->prepared) { prepare_step<float>(m->nb_panel, kMaxSmem); m->prepared = true; }
    }
    auto *g = new kamino_graph_s();
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "begin capture"); }
    st = kamino_step(s, dt, iters, tol, tau_dev, stream);
    e = cudaStreamEndCapture(cs, &g->graph);
    if (st) { if (g->graph) cudaGraphDestroy(g->graph); delete g; return st; }
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "end capture"); }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g->graph); delete g; return cuda_fail(e, "graph instantiate"); }
    *out = g;
    return KAMINO_OK;
}

kamino_status kamino_graph_launch(kamino_graph_t g, void *stream) {
    if (!g) return fail(KAMINO_E_INVALID_ARG, "graph must not be NULL");
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return KAMINO_OK;
}

kamino_status kamino_graph_destroy(kamino_graph_t g) {
    if (!g) return KAMINO_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return KAMINO_OK;
}

}  // extern "C"

// ============================================================================ warm-start MLP

namespace {

constexpr int kHiddenLayers = 3;

struct MlpBufs {
    __nv_bfloat16 *Xb = nullptr, *dY = nullptr;
    float *Y = nullptr, *dYf = nullptr, *feat = nullptr;
    float *Z[kHiddenLayers] = {nullptr, nullptr, nullptr};
    __nv_bfloat16 *H[kHiddenLayers] = {nullptr, nullptr, nullptr};
    float *dZf[2] = {nullptr, nullptr};
    __nv_bfloat16 *dZb[2] = {nullptr, nullptr};
};

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double normal_draw(uint64_t &s) {   // Box-Muller on two uniform draws in (0, 1)
    const double u1 = ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((splitmix64(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

struct kamino_mlp_s {
    kamino_model_t model = nullptr;
    int device = 0;                        // the device that holds the network's arrays
    int count = 0, din = 0, dout = 0, hidden = 0, nact = 0, max_batch = 0, step = 0;
    int dims[kHiddenLayers + 2] = {0, 0, 0, 0, 0};
    long woff[kHiddenLayers + 1] = {0}, boff[kHiddenLayers + 1] = {0};
    long nparams = 0;
    int *d_worlds = nullptr;
    float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr, *norm = nullptr, *loss_tmp = nullptr;
    __nv_bfloat16 *PB = nullptr;
    unsigned char *isw = nullptr;
    MlpBufs b;
    std::vector<void *> allocs;
    ~kamino_mlp_s() {
        for (void *p : allocs) cudaFree(p);
    }
    float *xmean() const { return norm; }
    float *xinv() const { return norm + din; }
    float *ymean() const { return norm + 2 * din; }
    float *yinv() const { return norm + 2 * din + dout; }
};

namespace {

template <typename P>
cudaError_t mlp_alloc(kamino_mlp_s *n, P **ptr, size_t count) {
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, std::max<size_t>(count, 1) * sizeof(P));
    if (e == cudaSuccess) {
        n->allocs.push_back(d);
        *ptr = (P *)d;
    }
    return e;
}

// forward pass on n->b.Xb (batch rows), leaves Z, H and Y
cudaError_t mlp_forward(kamino_mlp_s *n, int batch, cudaStream_t s) {
    using namespace kamino::mlp;
    const __nv_bfloat16 *in = n->b.Xb;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l <= kHiddenLayers && e == cudaSuccess; ++l) {
        GemmArgs g{};
        g.M = batch;
        g.N = n->dims[l + 1];
        g.K = n->dims[l];
        g.A = in; g.sam = n->dims[l]; g.sak = 1;
        g.B = n->PB + n->woff[l]; g.sbk = 1; g.sbn = n->dims[l];
        g.bias = n->P + n->boff[l];
        if (l < kHiddenLayers) {
            g.epi = EPI_BIAS_GELU;
            g.Cf = n->b.Z[l]; g.ldcf = n->dims[l + 1];
            g.Cb = n->b.H[l]; g.ldcb = n->dims[l + 1];
            in = n->b.H[l];
        } else {
            g.epi = EPI_BIAS_F32;
            g.Cf = n->b.Y; g.ldcf = n->dout;
        }
        e = gemm(g, s);
    }
    return e;
}

// gradients into n->G for the batch whose forward pass and dY are in place
cudaError_t mlp_backward(kamino_mlp_s *n, int batch, cudaStream_t s) {
    using namespace kamino::mlp;
    const __nv_bfloat16 *dz = n->b.dY;
    const float *dzf = n->b.dYf;
    cudaError_t e = cudaSuccess;
    int cur = 0;
    for (int l = kHiddenLayers; l >= 0 && e == cudaSuccess; --l) {
        const int dout = n->dims[l + 1], din = n->dims[l];
        const __nv_bfloat16 *hin = l == 0 ? n->b.Xb : n->b.H[l - 1];
        GemmArgs gw{};   // dW_l = dZ_l^T H_{l-1}
        gw.M = dout; gw.N = din; gw.K = batch;
        gw.A = dz; gw.sam = 1; gw.sak = dout;
        gw.B = hin; gw.sbk = din; gw.sbn = 1;
        gw.epi = EPI_F32; gw.Cf = n->G + n->woff[l]; gw.ldcf = din;
        e = gemm(gw, s);
        if (e == cudaSuccess) e = colsum(dzf, batch, dout, dout, n->G + n->boff[l], s);
        if (l > 0 && e == cudaSuccess) {   // dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1})
            GemmArgs gh{};
            gh.M = batch; gh.N = din; gh.K = dout;
            gh.A = dz; gh.sam = dout; gh.sak = 1;
            gh.B = n->PB + n->woff[l]; gh.sbk = din; gh.sbn = 1;
            gh.epi = EPI_GELU_BWD;
            gh.Zin = n->b.Z[l - 1]; gh.ldz = din;
            gh.Cf = n->b.dZf[cur]; gh.ldcf = din;
            gh.Cb = n->b.dZb[cur]; gh.ldcb = din;
            e = gemm(gh, s);
            dz = n->b.dZb[cur];
            dzf = n->b.dZf[cur];
            cur ^= 1;
        }
    }
    return e;
}

kamino_status mlp_loss_and_grads(kamino_mlp_s *n, const float *x, const float *y, const int *rows, int batch,
                                 float *loss, cudaStream_t s) {
    using namespace kamino::mlp;
    if (batch < 1 || batch > n->max_batch) return fail(KAMINO_E_INVALID_ARG, "batch %d outside [1, %d]", batch, n->max_batch);
    if (!x || !y) return fail(KAMINO_E_INVALID_ARG, "x and y must not be NULL");
    cudaError_t e = normalize_rows(x, n->din, rows, batch, n->xmean(), n->xinv(), n->b.Xb, s);
    if (e == cudaSuccess) e = mlp_forward(n, batch, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->loss_tmp, 0, sizeof(float), s);
    if (e == cudaSuccess)
        e = loss_grad(n->b.Y, y, n->dout, rows, batch, n->ymean(), n->yinv(), n->b.dY, n->b.dYf, n->loss_tmp, s);
    if (e != cudaSuccess) return cuda_fail(e, "mlp forward");
    return KAMINO_OK;
}

}  // namespace

extern "C" {

kamino_status kamino_mlp_create(kamino_model_t m, const int32_t *worlds, int32_t count, int32_t hidden,
                                int32_t max_batch, uint64_t seed, kamino_mlp_t *out) {
    if (!m || !worlds || !out) return fail(KAMINO_E_INVALID_ARG, "model, worlds and out must not be NULL");
    *out = nullptr;
    if (count < 1 || hidden < 8 || hidden > 4096 || max_batch < 1)
        return fail(KAMINO_E_INVALID_ARG, "count >= 1, hidden in [8, 4096] and max_batch >= 1 required");
    // sizes of the first world define the type; all listed worlds must match
    std::vector<int4> wa(m->W), wb(m->W);
    cudaError_t e = cudaMemcpy(wa.data(), m->world_a, m->W * sizeof(int4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(wb.data(), m->world_b, m->W * sizeof(int4), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp create (read model)");
    for (int i = 0; i < count; ++i)
        if (worlds[i] < 0 || worlds[i] >= m->W) return fail(KAMINO_E_INVALID_ARG, "world %d out of range", worlds[i]);
    const int4 ref = wb[worlds[0]];
    for (int i = 1; i < count; ++i) {
        const int4 c = wb[worlds[i]];
        if (c.x != ref.x || c.y != ref.y || c.z != ref.z || c.w != ref.w ||
            m->world_cache[worlds[i]] != m->world_cache[worlds[0]])
            return fail(KAMINO_E_TOPOLOGY, "world %d does not match the sizes of world %d", worlds[i], worlds[0]);
    }
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "mlp create (device)");
    auto *n = new kamino_mlp_s();
    n->model = m;
    n->device = dev;
    n->count = count;
    n->hidden = hidden;
    n->nact = m->n_act_max;
    n->dout = m->world_cache[worlds[0]];   // the world's impulse-cache layout
    n->din = 13 * ref.x + 1 + n->nact + 4 * ref.z + n->dout;   // ... + the previous step's impulses
    n->max_batch = std::max(max_batch, count);
    n->dims[0] = n->din;
    for (int l = 1; l <= kHiddenLayers; ++l) n->dims[l] = hidden;
    n->dims[kHiddenLayers + 1] = n->dout;
    long off = 0;
    for (int l = 0; l <= kHiddenLayers; ++l) {
        n->woff[l] = off;
        off += (long)n->dims[l + 1] * n->dims[l];
        n->boff[l] = off;
        off += n->dims[l + 1];
    }
    n->nparams = off;
    const int B = n->max_batch;
    e = mlp_alloc(n, &n->d_worlds, count);
    if (e == cudaSuccess) e = cudaMemcpy(n->d_worlds, worlds, count * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->P, off);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->G, off);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->M1, off);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->M2, off);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->PB, off);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->isw, off);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->norm, 2 * (size_t)(n->din + n->dout));
    if (e == cudaSuccess) e = mlp_alloc(n, &n->loss_tmp, 1);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->b.Xb, (size_t)B * n->din);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->b.feat, (size_t)count * n->din);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->b.Y, (size_t)B * n->dout);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->b.dY, (size_t)B * n->dout);
    if (e == cudaSuccess) e = mlp_alloc(n, &n->b.dYf, (size_t)B * n->dout);
    for (int l = 0; l < kHiddenLayers && e == cudaSuccess; ++l) {
        e = mlp_alloc(n, &n->b.Z[l], (size_t)B * hidden);
        if (e == cudaSuccess) e = mlp_alloc(n, &n->b.H[l], (size_t)B * hidden);
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = mlp_alloc(n, &n->b.dZf[k], (size_t)B * hidden);
        if (e == cudaSuccess) e = mlp_alloc(n, &n->b.dZb[k], (size_t)B * hidden);
    }
    if (e != cudaSuccess) { delete n; return cuda_fail(e, "mlp allocation"); }
    // initial parameters and identity normalisation
    std::vector<float> p(off, 0.0f);
    std::vector<unsigned char> isw(off, 0);
    uint64_t st = seed;
    for (int l = 0; l <= kHiddenLayers; ++l) {
        const double sd = std::sqrt(2.0 / n->dims[l]) * (l == kHiddenLayers ? 0.5 : 1.0);
        for (long i = 0; i < (long)n->dims[l + 1] * n->dims[l]; ++i) {
            p[n->woff[l] + i] = (float)(sd * normal_draw(st));
            isw[n->woff[l] + i] = 1;
        }
    }
    std::vector<float> nm(2 * (size_t)(n->din + n->dout), 0.0f);
    for (int i = 0; i < n->din; ++i) nm[n->din + i] = 1.0f;
    for (int i = 0; i < n->dout; ++i) nm[2 * n->din + n->dout + i] = 1.0f;
    e = cudaMemcpy(n->P, p.data(), off * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n->isw, isw.data(), off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(n->norm, nm.data(), nm.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->M1, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->M2, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->PB, 0, off * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = kamino::mlp::to_bf16(n->P, n->PB, (int)off, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { delete n; return cuda_fail(e, "mlp initialisation"); }
    *out = n;
    return KAMINO_OK;
}

kamino_status kamino_mlp_destroy(kamino_mlp_t n) {
    delete n;
    return KAMINO_OK;
}

kamino_status kamino_mlp_get_info(kamino_mlp_t n, kamino_mlp_info *out) {
    if (!n || !out) return fail(KAMINO_E_INVALID_ARG, "mlp and out must not be NULL");
    out->num_worlds = n->count;
    out->d_in = n->din;
    out->d_hidden = n->hidden;
    out->hidden_layers = kHiddenLayers;
    out->d_out = n->dout;
    out->max_batch = n->max_batch;
    out->num_params = n->nparams;
    return KAMINO_OK;
}

kamino_status kamino_mlp_features(kamino_mlp_t n, kamino_state_t s, const void *tau, float *out, void *stream) {
    if (!n || !s || !out) return fail(KAMINO_E_INVALID_ARG, "mlp, state and out must not be NULL");
    if (s->model != n->model) return fail(KAMINO_E_INVALID_ARG, "state belongs to another model");
    cudaError_t e;
    if (n->model->precision == KAMINO_FP64) {
        kamino::mlp::FeatureArgs<double> a{};
        a.m = view<double>(n->model);
        a.q = (const double *)s->ptr(s->off_q); a.u = (const double *)s->ptr(s->off_u); a.tau = (const double *)tau;
        a.cache = (const double *)s->ptr(s->off_cache); a.dout = n->dout;
        a.worlds = n->d_worlds; a.count = n->count; a.din = n->din; a.nact = n->nact; a.out = out;
        e = kamino::mlp::features<double>(a, (cudaStream_t)stream);
    } else {
        kamino::mlp::FeatureArgs<float> a{};
        a.m = view<float>(n->model);
        a.q = (const float *)s->ptr(s->off_q); a.u = (const float *)s->ptr(s->off_u); a.tau = (const float *)tau;
        a.cache = (const float *)s->ptr(s->off_cache); a.dout = n->dout;
        a.worlds = n->d_worlds; a.count = n->count; a.din = n->din; a.nact = n->nact; a.out = out;
        e = kamino::mlp::features<float>(a, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mlp features");
    return KAMINO_OK;
}

kamino_status kamino_mlp_targets(kamino_mlp_t n, kamino_state_t s, float *out, void *stream) {
    if (!n || !s || !out) return fail(KAMINO_E_INVALID_ARG, "mlp, state and out must not be NULL");
    if (s->model != n->model) return fail(KAMINO_E_INVALID_ARG, "state belongs to another model");
    cudaError_t e = n->model->precision == KAMINO_FP64
        ? kamino::mlp::targets<double>(n->model->world_a, n->d_worlds, n->count, n->dout,
                                       (const double *)s->ptr(s->off_cache), out, (cudaStream_t)stream)
        : kamino::mlp::targets<float>(n->model->world_a, n->d_worlds, n->count, n->dout,
                                      (const float *)s->ptr(s->off_cache), out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp targets");
    return KAMINO_OK;
}

kamino_status kamino_mlp_fit_normalization(kamino_mlp_t n, const float *x, const float *y, int64_t rows, void *stream) {
    if (!n || !x || !y || rows < 1) return fail(KAMINO_E_INVALID_ARG, "mlp, x, y and rows >= 1 required");
    cudaError_t e = kamino::mlp::colstats(x, rows, n->din, n->xmean(), n->xinv(), (cudaStream_t)stream);
    if (e == cudaSuccess) e = kamino::mlp::colstats(y, rows, n->dout, n->ymean(), n->yinv(), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp normalisation");
    return KAMINO_OK;
}

kamino_status kamino_mlp_gradients(kamino_mlp_t n, const float *x, const float *y, const int32_t *rows, int32_t batch,
                                   float *grad, float *loss, void *stream) {
    if (!n) return fail(KAMINO_E_INVALID_ARG, "mlp must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    kamino_status st = mlp_loss_and_grads(n, x, y, rows, batch, loss, s);
    if (st) return st;
    cudaError_t e = mlp_backward(n, batch, s);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, n->G, n->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, n->loss_tmp, sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "mlp backward");
    return KAMINO_OK;
}

kamino_status kamino_mlp_train_step(kamino_mlp_t n, const float *x, const float *y, const int32_t *rows, int32_t batch,
                                    float lr, float *loss, void *stream) {
    if (!n) return fail(KAMINO_E_INVALID_ARG, "mlp must not be NULL");
    if (!(lr > 0.0f)) return fail(KAMINO_E_INVALID_ARG, "lr must be > 0");
    kamino_status st = kamino_mlp_gradients(n, x, y, rows, batch, nullptr, loss, stream);
    if (st) return st;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)n->step), c2 = 1.0f - std::pow(b2, (float)n->step);
    cudaError_t e = kamino::mlp::adam(n->P, n->G, n->M1, n->M2, (int)n->nparams, lr, b1, b2, 1e-8f, c1, c2, n->PB,
                                      n->isw, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mlp adam");
    return KAMINO_OK;
}

kamino_status kamino_mlp_predict(kamino_mlp_t n, const float *x, int32_t batch, float *y, void *stream) {
    if (!n || !x || !y) return fail(KAMINO_E_INVALID_ARG, "mlp, x and y must not be NULL");
    if (batch < 1 || batch > n->max_batch) return fail(KAMINO_E_INVALID_ARG, "batch %d outside [1, %d]", batch, n->max_batch);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = kamino::mlp::normalize_rows(x, n->din, nullptr, batch, n->xmean(), n->xinv(), n->b.Xb, s);
    if (e == cudaSuccess) e = mlp_forward(n, batch, s);
    if (e == cudaSuccess) e = kamino::mlp::denormalize(n->b.Y, batch, n->dout, n->ymean(), n->yinv(), y, s);
    if (e != cudaSuccess) return cuda_fail(e, "mlp predict");
    return KAMINO_OK;
}

kamino_status kamino_mlp_warm_start(kamino_mlp_t n, kamino_state_t s, const void *tau, void *stream) {
    if (!n || !s) return fail(KAMINO_E_INVALID_ARG, "mlp and state must not be NULL");
    kamino_status st = kamino_mlp_features(n, s, tau, n->b.feat, stream);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = kamino::mlp::normalize_rows(n->b.feat, n->din, nullptr, n->count, n->xmean(), n->xinv(), n->b.Xb, cs);
    if (e == cudaSuccess) e = mlp_forward(n, n->count, cs);
    if (e == cudaSuccess)
        e = n->model->precision == KAMINO_FP64
            ? kamino::mlp::warm_write<double>(n->model->world_a, n->d_worlds, n->count, n->dout, n->b.Y, n->ymean(),
                                              n->yinv(), (double *)s->ptr(s->off_warm), cs)
            : kamino::mlp::warm_write<float>(n->model->world_a, n->d_worlds, n->count, n->dout, n->b.Y, n->ymean(),
                                             n->yinv(), (float *)s->ptr(s->off_warm), cs);
    if (e != cudaSuccess) return cuda_fail(e, "mlp warm start");
    return KAMINO_OK;
}

kamino_status kamino_mlp_get_params(kamino_mlp_t n, float *host, int64_t count) {
    if (!n || !host || count != n->nparams) return fail(KAMINO_E_INVALID_ARG, "need num_params floats");
    cudaError_t e = cudaMemcpy(host, n->P, count * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp get params");
    return KAMINO_OK;
}

kamino_status kamino_mlp_set_params(kamino_mlp_t n, const float *host, int64_t count) {
    if (!n || !host || count != n->nparams) return fail(KAMINO_E_INVALID_ARG, "need num_params floats");
    cudaError_t e = cudaMemcpy(n->P, host, count * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = kamino::mlp::to_bf16(n->P, n->PB, (int)count, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "mlp set params");
    return KAMINO_OK;
}

kamino_status kamino_mlp_get_normalization(kamino_mlp_t n, float *host) {
    if (!n || !host) return fail(KAMINO_E_INVALID_ARG, "mlp and host must not be NULL");
    cudaError_t e = cudaMemcpy(host, n->norm, 2 * (size_t)(n->din + n->dout) * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp get normalisation");
    return KAMINO_OK;
}

kamino_status kamino_mlp_set_normalization(kamino_mlp_t n, const float *host) {
    if (!n || !host) return fail(KAMINO_E_INVALID_ARG, "mlp and host must not be NULL");
    cudaError_t e = cudaMemcpy(n->norm, host, 2 * (size_t)(n->din + n->dout) * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "mlp set normalisation");
    return KAMINO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------- internal accessors
kamino_status kamino::report_error(kamino_status s, const char *msg) { return fail(s, "%s", msg); }

bool kamino::mlp::net_view(const struct kamino_mlp_s *n, NetView *out) {
    if (!n || !out) return false;
    out->din = n->din;
    out->dout = n->dout;
    out->hidden = n->hidden;
    out->layers = kHiddenLayers;
    out->max_batch = n->max_batch;
    out->device = n->device;
    out->P = n->P;
    out->PB = n->PB;
    for (int l = 0; l <= kHiddenLayers; ++l) {
        out->woff[l] = n->woff[l];
        out->boff[l] = n->boff[l];
    }
    out->xmean = n->xmean();
    out->xinv = n->xinv();
    out->ymean = n->ymean();
    out->yinv = n->yinv();
    return true;
}
