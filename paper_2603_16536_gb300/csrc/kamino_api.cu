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
    int nb_panel = 16;
    size_t smem = 0;
    bool prepared = false;
    kamino_solver_params params{};
    // device arrays
    std::vector<void *> allocs;
    int4 *world_a = nullptr, *world_b = nullptr, *joint_meta = nullptr;
    int *joint_row = nullptr, *contact_body = nullptr;
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
    size_t off_q = 0, off_u = 0, off_cache = 0, off_warm = 0, off_res = 0, off_tau = 0, off_cnt = 0, bytes = 0;
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

template <typename T>
kamino_status build_device(kamino_model_s *m, const kamino_model_desc *d, const std::vector<int4> &wa,
                           const std::vector<int4> &wb, const std::vector<int4> &jm, const std::vector<int> &jrow,
                           const std::vector<double> &frames, const std::vector<double> &q0) {
    kamino_status s;
    if ((s = upload<T>(m, (void **)&m->world_a, wa.data(), wa.size() * sizeof(int4)))) return s;
    if ((s = upload<T>(m, (void **)&m->world_b, wb.data(), wb.size() * sizeof(int4)))) return s;
    auto mu = convert<T>(d->world_mu, m->W);
    if ((s = upload<T>(m, &m->world_mu, mu.data(), mu.size() * sizeof(T)))) return s;
    auto mass = convert<T>(d->body_mass, m->B);
    if ((s = upload<T>(m, &m->body_mass, mass.data(), mass.size() * sizeof(T)))) return s;
    auto inert = convert<T>(d->body_inertia, 3 * (size_t)m->B);
    if ((s = upload<T>(m, &m->body_inertia, inert.data(), inert.size() * sizeof(T)))) return s;
    if ((s = upload<T>(m, (void **)&m->joint_meta, jm.data(), jm.size() * sizeof(int4)))) return s;
    if ((s = upload<T>(m, (void **)&m->joint_row, jrow.data(), jrow.size() * sizeof(int)))) return s;
    auto fr = convert<T>(frames.data(), frames.size());
    if ((s = upload<T>(m, &m->joint_frames, fr.data(), fr.size() * sizeof(T)))) return s;
    if (m->C > 0) {
        if ((s = upload<T>(m, (void **)&m->contact_body, d->contact_body, (size_t)m->C * sizeof(int)))) return s;
        auto cp = convert<T>(d->contact_point, 3 * (size_t)m->C);
        if ((s = upload<T>(m, &m->contact_point, cp.data(), cp.size() * sizeof(T)))) return s;
    }
    if (m->terrain_kind == KAMINO_TERRAIN_HEIGHTFIELD) {
        auto hh = convert<T>(d->hf_heights, (size_t)m->hf_nx * m->hf_ny);
        if ((s = upload<T>(m, &m->hf_heights, hh.data(), hh.size() * sizeof(T)))) return s;
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
    v.world_mu = (const T *)m->world_mu;
    v.body_mass = (const T *)m->body_mass;
    v.body_inertia = (const T *)m->body_inertia;
    v.joint_meta = m->joint_meta;
    v.joint_row = m->joint_row;
    v.joint_frames = (const T *)m->joint_frames;
    v.contact_body = m->contact_body;
    v.contact_point = (const T *)m->contact_point;
    v.terrain_kind = m->terrain_kind;
    v.hf_nx = m->hf_nx;
    v.hf_ny = m->hf_ny;
    v.hf_x0 = (T)m->hf_x0;
    v.hf_y0 = (T)m->hf_y0;
    v.hf_cell = (T)m->hf_cell;
    v.hf_heights = (const T *)m->hf_heights;
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
    const int mp = std::max(((b.rows + nbp - 1) / nbp) * nbp, nbp);
    if (mp > kMaxRowsPad) return 0;
    const Layout L = esize(m) == sizeof(double) ? make_layout<double>(b.nb, b.nj, b.nc, mp, nbp)
                                                : make_layout<float>(b.nb, b.nj, b.nc, mp, nbp);
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
    cudaError_t e = occupancy_persistent<T>(b.panel, b.smem, &per_sm);
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
    a.warm_mode = m->params.warm_mode;
    a.nb_max = m->nb_max;
    a.nj_max = m->nj_max;
    a.nc_max = m->nc_max;
    a.mp_max = m->mp_max;
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
    a.mp_max = std::max(((b.rows + b.panel - 1) / b.panel) * b.panel, b.panel);
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
        cudaError_t e = launch_step<T>(a, m->W, m->nb_panel, m->smem, stream);
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
    if (e == cudaSuccess) e = cudaMemcpyAsync(st->base, snap, st->bytes, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(snap);
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    m->launch_mode = KAMINO_LAUNCH_PERSISTENT;
    return KAMINO_OK;
}

}  // namespace

extern "C" {

const char *kamino_last_error(void) { return g_error.c_str(); }

kamino_status kamino_model_create(const kamino_model_desc *d, kamino_model_t *out) {
    if (!d || !out) return fail(KAMINO_E_INVALID_ARG, "desc and out must not be NULL");
    *out = nullptr;
    if (d->num_worlds < 1) return fail(KAMINO_E_INVALID_ARG, "num_worlds must be >= 1 (got %d)", d->num_worlds);
    if (d->precision != KAMINO_FP32 && d->precision != KAMINO_FP64)
        return fail(KAMINO_E_INVALID_ARG, "precision must be KAMINO_FP32 or KAMINO_FP64");
    if (!d->world_body_offset || !d->world_joint_offset || !d->world_contact_offset || !d->world_num_actuators ||
        !d->world_mu)
        return fail(KAMINO_E_INVALID_ARG, "per-world arrays must not be NULL");
    kamino_status s = check_params(d->params);
    if (s) return s;
    const int W = d->num_worlds;
    for (int k = 0; k < 3; ++k)
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
    int cache = 0;
    for (int w = 0; w < W; ++w) {
        const int b0 = d->world_body_offset[w], nb = d->world_body_offset[w + 1] - b0;
        const int j0 = d->world_joint_offset[w], nj = d->world_joint_offset[w + 1] - j0;
        const int c0 = d->world_contact_offset[w], nc = d->world_contact_offset[w + 1] - c0;
        const int nact = d->world_num_actuators[w];
        int row = 0;
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
                double *o = frames.data() + 14 * (size_t)j + 7 * side;
                for (int k = 0; k < 3; ++k) o[k] = f[k];
                for (int k = 3; k < 7; ++k) o[k] = f[k] / n;
            }
            jm[j] = make_int4(t, par, ch, act);
            jrow[j] = row;
            row += rows_of(t);
        }
        for (int c = c0; c < c0 + nc; ++c)
            if (d->contact_body[c] < 0 || d->contact_body[c] >= nb) {
                delete m;
                return fail(KAMINO_E_TOPOLOGY, "contact candidate %d: body %d out of range [0, %d)", c, d->contact_body[c], nb);
            }
        if (nc > kMaxCandidates) {
            delete m;
            return fail(KAMINO_E_UNSUPPORTED, "world %d has %d contact candidates (max %d)", w, nc, kMaxCandidates);
        }
        wa[w] = make_int4(b0, j0, c0, cache);
        wb[w] = make_int4(nb, nj, nc, row);
        {
            const int rows = row + 3 * nc;
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
            bk->units = std::max(bk->units, row + nc);
        }
        cache += row + 3 * nc;
        m->nb_max = std::max(m->nb_max, nb);
        m->nj_max = std::max(m->nj_max, nj);
        m->nc_max = std::max(m->nc_max, nc);
        m->max_rows = std::max(m->max_rows, row + 3 * nc);
        m->n_act_max = std::max(m->n_act_max, nact);
    }
    m->cache_len = cache;
    const size_t esz = d->precision == KAMINO_FP64 ? sizeof(double) : sizeof(float);
    m->smem = 0;
    for (int nbp : {16, 8}) {
        const int mp = std::max(((m->max_rows + nbp - 1) / nbp) * nbp, nbp);
        if (mp > kMaxRowsPad) continue;
        const Layout L = esz == sizeof(double) ? make_layout<double>(m->nb_max, m->nj_max, m->nc_max, mp, nbp)
                                               : make_layout<float>(m->nb_max, m->nj_max, m->nc_max, mp, nbp);
        if (L.total <= kMaxSmem) {
            m->nb_panel = nbp;
            m->mp_max = mp;
            m->smem = L.total;
            break;
        }
    }
    if (m->smem == 0) {
        const int rows = m->max_rows;
        delete m;
        return fail(KAMINO_E_UNSUPPORTED,
                    "a world needs %d constraint rows; the shared-memory working set exceeds %zu bytes "
                    "(max %d padded rows)", rows, kMaxSmem, kMaxRowsPad);
    }
    std::sort(m->buckets.begin(), m->buckets.end(),
              [](const Bucket &a, const Bucket &b) { return a.rows_pad > b.rows_pad; });
    for (auto &b : m->buckets) {
        if (!choose_default(m, b)) {
            const int rp = b.rows_pad;
            delete m;
            return fail(KAMINO_E_UNSUPPORTED, "no persistent configuration fits the bucket of %d rows", rp);
        }
    }
    std::vector<double> q0(7 * (size_t)B, 0.0);
    for (int b = 0; b < B; ++b) {
        if (d->body_q0) {
            for (int k = 0; k < 7; ++k) q0[7 * b + k] = d->body_q0[7 * b + k];
        } else {
            q0[7 * b + 6] = 1.0;
        }
    }
    kamino_status st = d->precision == KAMINO_FP64 ? build_device<double>(m, d, wa, wb, jm, jrow, frames, q0)
                                                   : build_device<float>(m, d, wa, wb, jm, jrow, frames, q0);
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
    m->params = *p;
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
