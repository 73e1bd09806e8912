// pm_api.cu -- host side of the C ABI declared in include/pm.h: the context,
// argument validation, the heading tables, launch configuration and the
// host-buffer convenience call. No arithmetic of the method runs here; every
// numeric step is a kernel of this library.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "pm.h"
#include "pm_kernels.cuh"

struct pm_ctx {
    int device = 0;
    int sm_count = 0;
    int clock_khz = 0;
    int cc = 0;
    size_t smem_optin = 0;
    // device staging owned by the context (host-buffer call, probe sink)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // scratch of the belief update: per-chunk accumulators and a ticket word
    void *post_scratch = nullptr;
    size_t post_scratch_bytes = 0;
    unsigned *ticket = nullptr;
    // scratch of the log-likelihood adjoint: per-trajectory partials
    void *adj_scratch = nullptr;
    size_t adj_scratch_bytes = 0;
    // asynchronous host-buffer predictions: two staging slots, a copy stream,
    // and per slot the event after which its copy-out has read it
    void *slot[2] = {nullptr, nullptr};
    size_t slot_bytes[2] = {0, 0};
    cudaEvent_t slot_free[2] = {nullptr, nullptr};
    cudaEvent_t computed = nullptr;
    cudaStream_t copy_stream = nullptr;
    int next_slot = 0;
    // page-locked host staging of the host-buffer calls' inputs (one per slot,
    // and [2] for the synchronous call) and the event after which its upload
    // has read it
    char *hin[3] = {nullptr, nullptr, nullptr};
    size_t hin_bytes[3] = {0, 0, 0};
    cudaEvent_t hin_read[3] = {nullptr, nullptr, nullptr};
};

struct pm_batch {
    pm_ctx *ctx = nullptr;
    pm_model shared{};
    int max_humans = 0;
    std::vector<pm_human> humans;
    // device
    pm::BatchHuman *d_humans = nullptr;
    pm::PostHuman *d_post = nullptr;
    int2 *d_items = nullptr;
    size_t items_cap = 0;
    int *d_meta = nullptr; // [0] tiles, [1] humans
    unsigned *d_head = nullptr;
    float *d_post_part = nullptr;
    unsigned *d_post_ticket = nullptr;
    float2 *d_prev = nullptr;        // [max_humans] start of the last prediction per slot (NaN: none), then a ticket word
    bool zero_reach = false;         // zero only the reachable cells (pm_batch_set_zeroing)
    float step_max = 0.0f;           // longest Euler step of the shared control set (upper bound)
    int t_max = 1;                   // longest horizon of the batch (sizes the zeroing grid)
    pm::SmoothSrc *d_srcs = nullptr; // union source records, one per human
    uint8_t *d_flags = nullptr;      // block occupancy flags of every human's histogram
    size_t flags_cap = 0;
    bool block_flags = false;        // pm_batch_predict marks occupied blocks
    size_t post_stride = 0; // floats of posterior scratch per human
    // page-locked staging of the uploads
    char *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    cudaEvent_t staged = nullptr;
    // launch shape
    int threads = 128;
    bool warp_hist = true;  // warp-combined emplacement, persistent warps (else shared-memory window)
    int ctas_per_sm = 0;
    int window_kib = 48;
    int n_items = 0;
    int max_chunks = 0;
    int max_J = 1;
    int occ = 0; // resident CTAs per SM of the current shape (queried outside any capture)
};

// A named NVTX range over one C ABI call, so that a profiler attributes the
// call's device work to it; without an attached tool it costs one check.
struct CallRange {
    explicit CallRange(const char *name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange &) = delete;
    CallRange &operator=(const CallRange &) = delete;
};
#define PM_RANGE(name) CallRange pm_call_range_(name)

namespace {

thread_local std::string g_err;

pm_status fail(pm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

pm_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(PM_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Makes the context's device current for the duration of a call.
struct DeviceScope {
    int prev = -1, want;
    explicit DeviceScope(int d) : want(d)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
    }
    ~DeviceScope()
    {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

// Unit vector of theta_k = 2 pi k / K by reduction to a quarter turn and a
// first-octant angle (exact at multiples of a quarter turn).
void unit_heading(int K, int k, double *c, double *s)
{
    const long long k4 = 4LL * k;
    const long long q = k4 / K;
    const long long rem = k4 - q * K;
    double cb, sb;
    if (rem == 0) {
        cb = 1.0;
        sb = 0.0;
    } else if (2 * rem <= K) {
        const double phi = (M_PI / 2.0) * (double)rem / (double)K;
        cb = std::cos(phi);
        sb = std::sin(phi);
    } else {
        const double phi = (M_PI / 2.0) * (double)(K - rem) / (double)K;
        cb = std::sin(phi);
        sb = std::cos(phi);
    }
    switch (q & 3) {
    case 0: *c = cb; *s = sb; break;
    case 1: *c = -sb; *s = cb; break;
    case 2: *c = -cb; *s = -sb; break;
    default: *c = sb; *s = -cb; break;
    }
}

// The control set has several speeds, or one speed with a multiplier != 1.
bool multi_speed(const pm_model *m)
{
    return m->n_speeds >= 2 || (m->n_speeds == 1 && m->speed_mult[0] != 1.0f);
}

uint64_t enabled_mask(const pm_model *m)
{
    const uint64_t allK = (m->K >= 64) ? ~0ull : ((1ull << m->K) - 1ull);
    return allK & ~m->heading_off;
}

pm_status check_model(const pm_model *m, bool need_tables = true)
{
    if (!m) return fail(PM_EINVAL, "model is NULL");
    if (m->K < 1 || m->K > PM_MAX_HEADINGS) return fail(PM_EINVAL, "K=%d outside [1, %d]", m->K, PM_MAX_HEADINGS);
    if (m->G < 1 || m->G > PM_MAX_GOALS) return fail(PM_EINVAL, "G=%d outside [1, %d]", m->G, PM_MAX_GOALS);
    if (m->B < 1 || (long long)m->G * m->B > PM_MAX_COMPONENTS)
        return fail(PM_EINVAL, "G*B=%lld outside [1, %d]", (long long)m->G * m->B, PM_MAX_COMPONENTS);
    if (!finite_pos(m->speed)) return fail(PM_EINVAL, "speed must be finite and > 0");
    if (!finite_pos(m->dt)) return fail(PM_EINVAL, "dt must be finite and > 0");
    if (!std::isfinite(m->w1) || !std::isfinite(m->w2) || m->w2 < 0.0f)
        return fail(PM_EINVAL, "w1 must be finite and w2 finite and >= 0");
    if (need_tables && (!m->goals || !m->beta)) return fail(PM_EINVAL, "goals/beta device pointers are NULL");
    if (enabled_mask(m) == 0) return fail(PM_EINVAL, "every heading is disabled");
    const double s = (double)m->speed * (double)m->dt;
    if (!(s * s > 1e-30) || !std::isfinite(s)) return fail(PM_EINVAL, "step v*dt out of range");
    if (m->n_speeds < 0 || m->n_speeds > PM_MAX_SPEEDS)
        return fail(PM_EINVAL, "n_speeds=%d outside [0, %d]", m->n_speeds, PM_MAX_SPEEDS);
    for (int sp = 0; sp < m->n_speeds; ++sp)
        if (!finite_pos(m->speed_mult[sp]) || !(s * m->speed_mult[sp] * s * m->speed_mult[sp] > 1e-30))
            return fail(PM_EINVAL, "speed_mult[%d] must be finite and > 0", sp);
    if (m->n_speeds > 0 && (m->speed_off & ((1u << m->n_speeds) - 1u)) == ((1u << m->n_speeds) - 1u))
        return fail(PM_EINVAL, "every speed is disabled");
    if (multi_speed(m)) {
        if (m->K % 4 != 0 || enabled_mask(m) != ((m->K >= 64) ? ~0ull : ((1ull << m->K) - 1ull)))
            return fail(PM_EINVAL, "several speeds need K a multiple of 4 with every heading enabled");
        if (m->n_speeds * m->K > 256) return fail(PM_EINVAL, "n_speeds*K=%d above 256", m->n_speeds * m->K);
    }
    if (m->snap_heading != 0 && m->snap_heading != 1)
        return fail(PM_EINVAL, "snap_heading=%d must be 0 or 1", m->snap_heading);
    return PM_OK;
}

pm_status check_grid(const pm_grid *g)
{
    if (!g) return fail(PM_EINVAL, "grid is NULL");
    if (!finite_pos(g->res) || !std::isfinite(g->x0) || !std::isfinite(g->y0))
        return fail(PM_EINVAL, "grid origin must be finite and res > 0");
    if (g->W < 1 || g->H < 1 || g->W > (1 << 22) || g->H > (1 << 22) || (long long)g->W * g->H > (1LL << 31))
        return fail(PM_EINVAL, "grid W=%d H=%d out of range", g->W, g->H);
    return PM_OK;
}

void fill_rollout_tables(const pm_model *m, pm::RolloutArgs &a)
{
    const double s = (double)m->speed * (double)m->dt;
    std::memset(&a.tab, 0, sizeof a.tab);
    for (int k = 0; k < m->K; ++k) {
        double c, sn;
        unit_heading(m->K, k, &c, &sn);
        a.tab.ux[k] = (float)c;
        a.tab.uy[k] = (float)sn;
        a.tab.sx[k] = (float)(s * c);
        a.tab.sy[k] = (float)(s * sn);
        a.tab.tx[k] = (float)(2.0 * s * c);
        a.tab.ty[k] = (float)(2.0 * s * sn);
        a.tab.cdf[k][0] = (float)c;
        a.tab.cdf[k][1] = (float)(c - (double)a.tab.cdf[k][0]);
        a.tab.sdf[k][0] = (float)sn;
        a.tab.sdf[k][1] = (float)(sn - (double)a.tab.sdf[k][0]);
    }
    a.enabled = enabled_mask(m);
    a.tab.s = (float)s;
    a.tab.v = m->speed;
    a.tab.dt = m->dt;
    a.tab.w1 = m->w1;
    a.tab.w2 = m->w2;
    a.tab.K = m->K;
    a.tab.lb_gap = (float)(2.0 * s * std::sin(3.14159265358979323846 / (2.0 * m->K)));
    a.s2 = (float)(s * s);
    const double w2l = (double)m->w2 * 1.4426950408889634, w1l = (double)m->w1 * s * 1.4426950408889634;
    a.w2_log2e = (float)w2l;
    a.w1_vdt_log2e = (float)w1l;
    a.tab.w2l[0] = a.w2_log2e;
    a.tab.w2l[1] = (float)(w2l - (double)a.w2_log2e);
    a.tab.w1l[0] = a.w1_vdt_log2e;
    a.tab.w1l[1] = (float)(w1l - (double)a.w1_vdt_log2e);
    a.tab.S = 0; // one speed: the heading kernels
    if (multi_speed(m)) {
        a.tab.S = m->n_speeds;
        double smax = 0.0;
        for (int sp = 0; sp < m->n_speeds; ++sp) {
            const double sl = (double)m->speed * (double)m->speed_mult[sp] * (double)m->dt;
            a.tab.mult[sp] = m->speed_mult[sp];
            a.tab.inv_mult[sp] = 1.0f / m->speed_mult[sp];
            a.tab.sl[sp] = (float)sl;
            if (!((m->speed_off >> sp) & 1u)) {
                a.tab.speed_on |= 1u << sp;
                smax = std::max(smax, sl);
            }
            for (int k = 0; k < m->K; ++k) {
                double c, sn;
                unit_heading(m->K, k, &c, &sn);
                a.tab.msx[sp][k] = (float)(sl * c);
                a.tab.msy[sp][k] = (float)(sl * sn);
            }
        }
        a.tab.lb_gap = (float)(2.0 * smax * std::sin(3.14159265358979323846 / (2.0 * m->K)));
    }
    a.K = m->K;
    a.G = m->G;
    a.B = m->B;
    a.goals = m->goals;
    a.beta = m->beta;
}

// The speed set of the belief update and the adjoint (S = 0: one speed).
void fill_speed_set(const pm_model *m, pm::SpeedSet &sp)
{
    std::memset(&sp, 0, sizeof sp);
    sp.w1 = m->w1;
    if (!multi_speed(m)) return;
    sp.S = m->n_speeds;
    for (int q = 0; q < m->n_speeds; ++q) {
        sp.mult[q] = m->speed_mult[q];
        sp.sl[q] = (float)((double)m->speed * (double)m->speed_mult[q] * (double)m->dt);
        if (!((m->speed_off >> q) & 1u)) sp.speed_on |= 1u << q;
    }
}

// Heading tables and model constants of the belief update (per-human tables
// and observations are set by the caller).
void fill_posterior_args(const pm_model *m, pm::PosteriorArgs &a)
{
    std::memset(&a, 0, sizeof a);
    const double s = (double)m->speed * (double)m->dt;
    for (int k = 0; k < m->K; ++k) {
        double c, sn;
        unit_heading(m->K, k, &c, &sn);
        a.ux[k] = (float)c;
        a.uy[k] = (float)sn;
    }
    a.enabled = enabled_mask(m);
    a.s = (float)s;
    a.s2 = (float)(s * s);
    a.two_s = (float)(2.0 * s);
    a.w2 = m->w2;
    a.K = m->K;
    a.G = m->G;
    a.B = m->B;
    a.goals = m->goals;
    a.beta = m->beta;
    a.snap = m->snap_heading;
    fill_speed_set(m, a.sp);
}

pm_status ensure_stage(pm_ctx *ctx, size_t bytes)
{
    if (ctx->stage_bytes >= bytes) return PM_OK;
    if (ctx->stage) cudaFree(ctx->stage);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->stage, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PM_ENOMEM, "cudaMalloc(%zu) for context staging failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->stage_bytes = bytes;
    return PM_OK;
}

// Word 3 of the context's counter block is its device status word.
unsigned *status_word(pm_ctx *ctx) { return ctx->ticket ? ctx->ticket + 3 : nullptr; }

pm_status ensure_posterior_scratch(pm_ctx *ctx, size_t bytes)
{
    if (!ctx->ticket) {
        cudaError_t e = cudaMalloc((void **)&ctx->ticket, 256);
        if (e == cudaSuccess) e = cudaMemset(ctx->ticket, 0, 256);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->ticket = nullptr;
            return fail(PM_ENOMEM, "ticket allocation failed: %s", cudaGetErrorString(e));
        }
    }
    if (ctx->post_scratch_bytes >= bytes) return PM_OK;
    if (ctx->post_scratch) cudaFree(ctx->post_scratch);
    ctx->post_scratch = nullptr;
    ctx->post_scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->post_scratch, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PM_ENOMEM, "cudaMalloc(%zu) for belief-update scratch failed", bytes);
    }
    ctx->post_scratch_bytes = bytes;
    return PM_OK;
}

pm_status predict_impl(pm_ctx *ctx, const pm_model *model, const float *log_belief, float z0x,
                       float z0y, int32_t n_particles, int32_t horizon, const pm_grid *grid,
                       uint64_t seed, uint32_t human_id, uint32_t *counts, uint32_t *oob,
                       int32_t n_trace, float *states, uint8_t *headings, int32_t *components,
                       cudaStream_t stream, bool zero = true)
{
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    pm_status st = check_model(model);
    if (st != PM_OK) return st;
    if (!log_belief) return fail(PM_EINVAL, "log_belief is NULL");
    if (n_particles < 1) return fail(PM_EINVAL, "n_particles=%d must be >= 1", n_particles);
    if (horizon < 1 || horizon > PM_MAX_HORIZON)
        return fail(PM_EINVAL, "horizon=%d outside [1, %d]", horizon, PM_MAX_HORIZON);
    if (!std::isfinite(z0x) || !std::isfinite(z0y)) return fail(PM_EINVAL, "z0 must be finite");
    if ((counts == nullptr) != (oob == nullptr)) return fail(PM_EINVAL, "counts and oob must both be set or both NULL");
    const bool hist = counts != nullptr;
    if (hist) {
        st = check_grid(grid);
        if (st != PM_OK) return st;
    }
    if (n_trace < 0 || n_trace > n_particles) return fail(PM_EINVAL, "n_trace=%d outside [0, n_particles]", n_trace);
    // the kernel stores each traced state as one 8-byte pair
    if (n_trace > 0 && states && ((uintptr_t)states & 7u))
        return fail(PM_EINVAL, "states must be 8-byte aligned");
    if (!hist && n_trace == 0) return fail(PM_EINVAL, "nothing to compute: no histogram and no trace");
    DeviceScope dev(ctx->device);

    pm::RolloutArgs a;
    std::memset(&a, 0, sizeof a);
    fill_rollout_tables(model, a);
    a.log_b = log_belief;
    a.z0x = z0x;
    a.z0y = z0y;
    a.N = n_particles;
    a.T = horizon;
    a.seed = seed;
    a.human = human_id;
    a.n_trace = n_trace;
    a.tr_states = states;
    a.tr_head = headings;
    a.tr_comp = components;
    a.status = status_word(ctx);
    if (hist) {
        a.gx0 = grid->x0;
        a.gy0 = grid->y0;
        a.inv_res = 1.0f / grid->res;
        a.W = grid->W;
        a.H = grid->H;
        a.counts = counts;
        a.oob = oob;
    } else {
        a.W = a.H = 1;
        a.inv_res = 1.0f;
    }
    // persistent warps take 32-particle chunks from a context-owned counter
    // (word 2 of the counter block, word 4 counts the warps that are done);
    // the last warp leaves both at zero, and the zeroing launch resets the
    // counter too
    st = ensure_posterior_scratch(ctx, 0);
    if (st != PM_OK) return st;
    unsigned *head = ctx->ticket + 2;
    const size_t words = hist ? (size_t)grid->W * (size_t)grid->H * (size_t)horizon : 0;
    // (the rollout leaves its chunk counter at zero; without `zero` the
    // caller has zeroed the outputs)
    cudaError_t ez = zero ? pm::launch_zero_outputs(hist ? counts : nullptr, words, hist ? oob : nullptr, horizon,
                                                    head, ctx->sm_count, stream)
                          : cudaSuccess;
    if (ez != cudaSuccess) return cuda_fail(ez, "zeroing counts, oob and the chunk counter");
    cudaError_t e = pm::launch_rollout(a, head, ctx->sm_count, stream);
    if (e != cudaSuccess) return cuda_fail(e, "rollout launch");
    return PM_OK;
}

pm_status posterior_impl(pm_ctx *ctx, const pm_model *model, const float *obs_xy, int32_t n_obs,
                         const float *log_prior, float *log_belief, cudaStream_t stream)
{
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    pm_status st = check_model(model);
    if (st != PM_OK) return st;
    if (n_obs < 0) return fail(PM_EINVAL, "n_obs=%d must be >= 0", n_obs);
    if (!log_belief) return fail(PM_EINVAL, "log_belief is NULL");
    if (!log_prior) return fail(PM_EINVAL, "log_prior is NULL");
    const size_t J = (size_t)model->G * (size_t)model->B;
    if (log_prior != log_belief && log_prior < log_belief + J && log_belief < log_prior + J)
        return fail(PM_EINVAL, "log_prior and log_belief overlap without being the same buffer");
    if (n_obs == 0) {
        if (log_prior == log_belief) return PM_OK;
        DeviceScope dev(ctx->device);
        cudaError_t e = cudaMemcpyAsync(log_belief, log_prior, J * sizeof(float), cudaMemcpyDeviceToDevice, stream);
        return e == cudaSuccess ? PM_OK : cuda_fail(e, "copying the prior");
    }
    if (!obs_xy) return fail(PM_EINVAL, "obs_xy is NULL");
    DeviceScope dev(ctx->device);
    pm::PosteriorArgs a;
    fill_posterior_args(model, a);
    a.obs = obs_xy;
    a.n_obs = n_obs;
    a.log_prior = log_prior;
    a.log_b = log_belief;
    const int n_chunks = pm::posterior_chunks(n_obs, &a.steps_per_chunk);
    st = ensure_posterior_scratch(ctx, pm::posterior_scratch_bytes(n_chunks, model->G * model->B));
    if (st != PM_OK) return st;
    a.part = (float *)ctx->post_scratch;
    a.ticket = ctx->ticket;
    a.status = status_word(ctx);
    cudaError_t e = pm::launch_posterior(a, n_chunks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "posterior launch");
    return PM_OK;
}

pm_status loglik_impl(pm_ctx *ctx, const pm_model *model, int32_t M, const int32_t *offsets, int32_t n_points,
                      const float *traj_xy, const float *log_prior, bool want_grad, float grad_out, float *loglik,
                      float *d_goals, float *d_speed, float *d_w, cudaStream_t stream)
{
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    pm_status st = check_model(model);
    if (st != PM_OK) return st;
    if (M < 1) return fail(PM_EINVAL, "M=%d must be >= 1", M);
    if (n_points < 0) return fail(PM_EINVAL, "n_points must be >= 0");
    if (!offsets || !traj_xy || !log_prior || !loglik) return fail(PM_EINVAL, "a device pointer is NULL");
    if (want_grad && (!d_goals || !d_speed || !d_w)) return fail(PM_EINVAL, "gradient outputs are NULL");
    if (!std::isfinite(grad_out)) return fail(PM_EINVAL, "grad_out must be finite");
    DeviceScope dev(ctx->device);
    st = ensure_posterior_scratch(ctx, 0); // allocates the ticket word
    if (st != PM_OK) return st;
    const size_t bytes = pm::adjoint_scratch_bytes(M, model->G, model->G * model->B);
    if (ctx->adj_scratch_bytes < bytes) {
        if (ctx->adj_scratch) cudaFree(ctx->adj_scratch);
        ctx->adj_scratch = nullptr;
        ctx->adj_scratch_bytes = 0;
        cudaError_t e = cudaMalloc(&ctx->adj_scratch, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ENOMEM, "cudaMalloc(%zu) for adjoint scratch failed", bytes);
        }
        ctx->adj_scratch_bytes = bytes;
    }
    pm::AdjointArgs a;
    std::memset(&a, 0, sizeof a);
    const double s = (double)model->speed * (double)model->dt;
    for (int k = 0; k < model->K; ++k) {
        double c, sn;
        unit_heading(model->K, k, &c, &sn);
        a.ux[k] = (float)c;
        a.uy[k] = (float)sn;
    }
    a.snap = model->snap_heading;
    a.enabled = enabled_mask(model);
    a.s = (float)s;
    a.s2 = (float)(s * s);
    a.two_s = (float)(2.0 * s);
    a.w2 = model->w2;
    a.dt = model->dt;
    a.v = model->speed;
    a.K = model->K;
    fill_speed_set(model, a.sp);
    a.G = model->G;
    a.B = model->B;
    a.goals = model->goals;
    a.beta = model->beta;
    a.M = M;
    a.offsets = offsets;
    a.n_points = n_points;
    a.traj = traj_xy;
    a.log_prior = log_prior;
    a.want_grad = want_grad ? 1 : 0;
    a.grad_out = grad_out;
    pm::adjoint_scratch_layout(ctx->adj_scratch, M, model->G, model->G * model->B, a);
    a.ticket = ctx->ticket + 1; // its own word of the ticket block
    a.status = status_word(ctx);
    a.loglik = loglik;
    a.d_goals = d_goals;
    a.d_speed = d_speed;
    a.d_w = d_w;
    cudaError_t e = pm::launch_adjoint(a, stream);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    return PM_OK;
}


// ---------------------------------------------------------------------------
// batched prediction
// ---------------------------------------------------------------------------
pm_status check_human(const pm_human &h, int i, const pm_model &shared)
{
    if (!h.goals || !h.beta || !h.log_belief || !h.z0_xy || !h.counts || !h.oob)
        return fail(PM_EINVAL, "human %d: a device pointer is NULL", i);
    if (h.G < 1 || h.G > PM_MAX_GOALS || h.B < 1 || (long long)h.G * h.B > PM_MAX_COMPONENTS)
        return fail(PM_EINVAL, "human %d: G=%d B=%d out of range", i, h.G, h.B);
    if (h.n_particles < 1) return fail(PM_EINVAL, "human %d: n_particles must be >= 1", i);
    if (h.horizon < 1 || h.horizon > PM_MAX_HORIZON) return fail(PM_EINVAL, "human %d: horizon out of range", i);
    if (h.n_obs < 0 || (h.n_obs > 0 && !h.obs_xy)) return fail(PM_EINVAL, "human %d: observations", i);
    pm_status st = check_grid(&h.grid);
    if (st != PM_OK) return fail(st, "human %d: %s", i, g_err.c_str());
    if (h.center && (h.grid.W % 2 == 0 || h.grid.H % 2 == 0))
        return fail(PM_EINVAL, "human %d: a centred output window needs odd W and H", i);
    if (!h.center && (std::abs((long long)h.cx_off) + h.grid.W > (1LL << 22) ||
                      std::abs((long long)h.cy_off) + h.grid.H > (1LL << 22)))
        return fail(PM_EINVAL, "human %d: window offset more than 2^22 cells from the grid origin", i);
    if (h.speed_off != 0u) {
        if (!multi_speed(&shared)) return fail(PM_EINVAL, "human %d: speed_off needs a model with several speeds", i);
        const uint32_t all = (1u << shared.n_speeds) - 1u;
        if (((shared.speed_off | h.speed_off) & all) == all)
            return fail(PM_EINVAL, "human %d: every speed is disabled", i);
    }
    return PM_OK;
}

// Speeds enabled for one human of a batch (several speeds only).
uint32_t human_speed_on(const pm_model &shared, const pm_human &h)
{
    if (!multi_speed(&shared)) return 0u;
    return ((1u << shared.n_speeds) - 1u) & ~(shared.speed_off | h.speed_off);
}

// The longest step of the control set, v dt times the largest multiplier.
double max_step(const pm_model &m)
{
    double mult = 1.0;
    if (multi_speed(&m))
        for (int q = 0; q < m.n_speeds; ++q) mult = std::max(mult, (double)m.speed_mult[q]);
    return (double)m.speed * (double)m.dt * mult;
}

int batch_radius_cap(int window_kib, int threads)
{
    // two windows of 16-bit counts and two lists of `threads` entries
    const long long cells = (((long long)window_kib * 1024 - (long long)threads * 4) / 2 - 32) / 2;
    int r = 0;
    while ((2LL * (r + 1) + 1) * (2LL * (r + 1) + 1) <= cells && 2 * (r + 1) + 1 <= 255) ++r;
    return r;
}

pm::RolloutShape batch_shape_of(const pm_batch *b) { return pm::RolloutShape{b->threads, 1, b->warp_hist}; }

size_t batch_dyn_smem(const pm_batch *b)
{
    if (b->warp_hist) return pm::batch_warp_tables_bytes(b->threads, multi_speed(&b->shared));
    const int r = batch_radius_cap(b->window_kib, b->threads);
    const size_t cells = (size_t)(2 * r + 1) * (2 * r + 1);
    const size_t stride_words = (((cells + 1) / 2) + 3) & ~(size_t)3;
    return 2 * stride_words * 4 + 2 * (size_t)b->threads * 2;
}

unsigned *zero_ticket(pm_batch *b)
{
    return reinterpret_cast<unsigned *>(b->d_prev + b->max_humans);
}

// Forget the starts of the last predictions: the next prediction zeroes every
// cell of every human (stream-ordered).
cudaError_t forget_starts(pm_batch *b, cudaStream_t stream)
{
    return cudaMemsetAsync(b->d_prev, 0xFF, (size_t)b->max_humans * sizeof(float2), stream);
}

pm_status batch_upload(pm_batch *b, cudaStream_t stream)
{
    const int n = (int)b->humans.size();
    const double s = max_step(b->shared); // reach of the fastest control
    // an upper bound on every FP32 step of the table (each rounded once from s cos, s sin)
    b->step_max = (float)(s * (1.0 + 0x1p-16));
    // the slots may now hold other humans or other buffers
    if (b->zero_reach) {
        cudaError_t ef = forget_starts(b, stream);
        if (ef != cudaSuccess) return cuda_fail(ef, "batch start records");
    }
    std::vector<int2> items;
    for (int h = 0; h < n; ++h)
        for (int p0 = 0; p0 < b->humans[h].n_particles; p0 += (b->warp_hist ? 32 : b->threads))
            items.push_back(make_int2(h, p0));
    std::stable_sort(items.begin(), items.end(), [&](const int2 &x, const int2 &y) {
        return b->humans[x.x].horizon > b->humans[y.x].horizon;
    });
    std::vector<pm::BatchHuman> hd(n);
    std::vector<pm::PostHuman> ph(n);
    int max_chunks = 0, max_J = 1;
    // block occupancy flags (written by the warp-combined emplacement only)
    std::vector<size_t> foff(n + 1, 0);
    for (int h = 0; h < n; ++h) {
        const pm_human &u = b->humans[h];
        const size_t fbx = ((size_t)u.grid.W + pm::kFlagBlock - 1) >> pm::kFlagShift;
        const size_t fby = ((size_t)u.grid.H + pm::kFlagBlock - 1) >> pm::kFlagShift;
        foff[h + 1] = foff[h] + (((size_t)u.horizon * fbx * fby + 15) & ~(size_t)15);
    }
    const bool marks = b->block_flags && b->warp_hist;
    if (marks && foff[n] > b->flags_cap) {
        if (b->d_flags) cudaFree(b->d_flags);
        b->d_flags = nullptr;
        b->flags_cap = 0;
        cudaError_t ef = cudaMalloc(&b->d_flags, foff[n]);
        if (ef == cudaSuccess) ef = cudaMemset(b->d_flags, 0, foff[n]);
        if (ef != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ENOMEM, "cudaMalloc(%zu) for block flags failed", foff[n]);
        }
        b->flags_cap = foff[n];
    }
    for (int h = 0; h < n; ++h) {
        const pm_human &u = b->humans[h];
        pm::BatchHuman &d = hd[h];
        d.goals = u.goals;
        d.beta = u.beta;
        d.G = u.G;
        d.B = u.B;
        d.log_b = u.log_belief;
        d.z0 = u.z0_xy;
        d.N = u.n_particles;
        d.T = u.horizon;
        d.gx0 = u.grid.x0;
        d.gy0 = u.grid.y0;
        d.inv_res = 1.0f / u.grid.res;
        d.W = u.grid.W;
        d.H = u.grid.H;
        d.center = u.center ? 1 : 0;
        d.cx_off = u.cx_off;
        d.cy_off = u.cy_off;
        d.reach_cells = (int)std::fmin(std::ceil((double)u.horizon * s / (double)u.grid.res) + 1.0, 1 << 20);
        d.seed = u.seed;
        d.human = u.human_id;
        d.counts = u.counts;
        d.oob = u.oob;
        d.speed_on = human_speed_on(b->shared, u);
        d.fbx = (u.grid.W + pm::kFlagBlock - 1) >> pm::kFlagShift;
        d.fby = (u.grid.H + pm::kFlagBlock - 1) >> pm::kFlagShift;
        d.flags = (marks && b->d_flags) ? b->d_flags + foff[h] : nullptr;
        pm::PostHuman &q = ph[h];
        q.goals = u.goals;
        q.beta = u.beta;
        q.G = u.G;
        q.B = u.B;
        q.obs = u.obs_xy;
        q.n_obs = u.n_obs;
        int spc = 1;
        const int nch = u.n_obs > 0 ? pm::posterior_chunks(u.n_obs, &spc) : 0;
        q.steps_per_chunk = spc;
        q.log_prior = u.log_belief;
        q.log_b = u.log_belief;
        q.part = b->d_post_part + (size_t)h * b->post_stride;
        q.ticket = b->d_post_ticket + h;
        q.speed_on = d.speed_on;
        max_chunks = std::max(max_chunks, nch);
        max_J = std::max(max_J, u.G * u.B);
    }
    if (items.size() > b->items_cap) {
        cudaStreamSynchronize(stream);
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        b->items_cap = 0;
        cudaError_t e = cudaMalloc(&b->d_items, items.size() * sizeof(int2));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ENOMEM, "cudaMalloc for %zu work items failed", items.size());
        }
        b->items_cap = items.size();
    }
    const size_t bh = (size_t)n * sizeof(pm::BatchHuman), bp = (size_t)n * sizeof(pm::PostHuman);
    const size_t bi = items.size() * sizeof(int2);
    const size_t need = bh + bp + 16 + bi + 64;
    cudaError_t e = cudaEventSynchronize(b->staged); // the previous upload has left the staging buffer
    if (e != cudaSuccess) return cuda_fail(e, "staging event");
    if (need > b->h_stage_bytes) {
        if (b->h_stage) cudaFreeHost(b->h_stage);
        b->h_stage = nullptr;
        b->h_stage_bytes = 0;
        e = cudaMallocHost((void **)&b->h_stage, need * 2);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ENOMEM, "page-locked staging of %zu bytes failed", need * 2);
        }
        b->h_stage_bytes = need * 2;
    }
    char *p = b->h_stage;
    std::memcpy(p, hd.data(), bh);
    std::memcpy(p + bh, ph.data(), bp);
    int t_max = 1;
    for (const pm_human &u : b->humans) t_max = std::max(t_max, (int)u.horizon);
    b->t_max = t_max;
    int meta[3] = {(int)items.size(), n, t_max};
    std::memcpy(p + bh + bp, meta, sizeof meta);
    if (bi) std::memcpy(p + bh + bp + 16, items.data(), bi);
    if (bh) e = cudaMemcpyAsync(b->d_humans, p, bh, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && bp) e = cudaMemcpyAsync(b->d_post, p + bh, bp, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_meta, p + bh + bp, sizeof meta, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && bi) e = cudaMemcpyAsync(b->d_items, p + bh + bp + 16, bi, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->staged, stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch upload");
    b->n_items = (int)items.size();
    b->max_chunks = std::max(b->max_chunks, max_chunks);
    b->max_J = std::max(b->max_J, max_J);
    pm::RolloutArgs t;
    std::memset(&t, 0, sizeof t);
    fill_rollout_tables(&b->shared, t);
    b->occ = pm::batch_rollout_occupancy(b->shared.K, t.enabled, t.tab.S, b->block_flags && b->warp_hist,
                                         batch_shape_of(b), batch_dyn_smem(b));
    cudaGetLastError();
    return PM_OK;
}

pm_status batch_zero_impl(pm_batch *b, cudaStream_t stream)
{
    cudaError_t e = pm::launch_batch_zero(b->d_humans, b->d_meta + 1, b->max_humans, b->ctx->sm_count, b->t_max,
                                          b->zero_reach ? b->d_prev : nullptr, zero_ticket(b), b->step_max, stream);
    if (e != cudaSuccess) return cuda_fail(e, "zero launch");
    return PM_OK;
}

pm_status batch_rollout_impl(pm_batch *b, cudaStream_t stream)
{
    pm_ctx *ctx = b->ctx;
    cudaError_t e = cudaMemsetAsync(b->d_head, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    pm::RolloutArgs t;
    std::memset(&t, 0, sizeof t);
    fill_rollout_tables(&b->shared, t);
    pm::BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.tab = t.tab;
    a.enabled = t.enabled;
    a.s2 = t.s2;
    a.w2_log2e = t.w2_log2e;
    a.w1_vdt_log2e = t.w1_vdt_log2e;
    a.K = b->shared.K;
    a.humans = b->d_humans;
    a.items = b->d_items;
    a.n_items = b->d_meta;
    a.head = b->d_head;
    a.win_radius_cap = batch_radius_cap(b->window_kib, b->threads);
    a.status = status_word(ctx);
    a.marks = (b->block_flags && b->warp_hist && b->d_flags) ? 1 : 0;
    const size_t dyn = batch_dyn_smem(b);
    int occ = b->occ;
    if (occ < 1)
        return fail(PM_EINVAL, "launch shape (%d threads, %s) does not fit an SM", b->threads,
                    b->warp_hist ? "warp emplacement" : "shared window");
    if (b->ctas_per_sm > 0) occ = std::min(occ, b->ctas_per_sm);
    e = pm::launch_batch_rollout(a, batch_shape_of(b), ctx->sm_count * occ, dyn, stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch rollout launch");
    return PM_OK;
}

pm_status batch_predict_impl(pm_batch *b, cudaStream_t stream)
{
    pm_status st = batch_zero_impl(b, stream);
    return st != PM_OK ? st : batch_rollout_impl(b, stream);
}

} // namespace

// Belief update on caller-supplied scratch (used by the entry point that
// allocates nothing): `part` holds the per-chunk accumulators and the [J]
// doubles, `ticket` one zero word; at most `max_chunks` CTAs are used.
pm_status pm_internal_error(pm_status st, const char *msg) { return fail(st, "%s", msg); }

pm_status pm_internal_posterior_on_scratch(const pm_model *model, const float *obs_xy, int32_t n_obs,
                                           float *log_belief, float *part, unsigned *ticket, size_t part_bytes,
                                           int max_chunks, void *stream)
{
    PM_RANGE("pm_internal_posterior_on_scratch");
    pm_status st = check_model(model);
    if (st != PM_OK) return st;
    if (n_obs < 0) return fail(PM_EINVAL, "n_obs=%d must be >= 0", n_obs);
    if (!log_belief) return fail(PM_EINVAL, "log_belief is NULL");
    if (n_obs == 0) return PM_OK;
    if (!obs_xy) return fail(PM_EINVAL, "obs_xy is NULL");
    pm::PosteriorArgs a;
    fill_posterior_args(model, a);
    a.obs = obs_xy;
    a.n_obs = n_obs;
    a.log_prior = log_belief;
    a.log_b = log_belief;
    a.steps_per_chunk = (n_obs + max_chunks - 1) / max_chunks;
    const int n_chunks = (n_obs + a.steps_per_chunk - 1) / a.steps_per_chunk;
    if (pm::posterior_scratch_bytes(n_chunks, model->G * model->B) > part_bytes)
        return fail(PM_EINVAL, "scratch of %zu bytes is too small for G*B=%d", part_bytes, model->G * model->B);
    a.part = part;
    a.ticket = ticket;
    // the ticket must start at zero; a call that did not finish could have left it set
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the ticket");
    e = pm::launch_posterior(a, n_chunks, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "posterior launch");
    return PM_OK;
}

extern "C" {

pm_status pm_create(pm_ctx **out, int device)
{
    PM_RANGE("pm_create");
    if (!out) return fail(PM_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(PM_EINVAL, "device %d outside [0, %d)", device, n);
    cudaDeviceProp p;
    e = cudaGetDeviceProperties(&p, device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    pm_ctx *c = new pm_ctx();
    c->device = device;
    c->sm_count = p.multiProcessorCount;
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
    c->clock_khz = clk;
    c->cc = p.major * 10 + p.minor;
    c->smem_optin = p.sharedMemPerBlockOptin;
    {
        DeviceScope dev(device);
        pm_status st = ensure_posterior_scratch(c, 0); // the counter words and the status word
        if (st != PM_OK) {
            delete c;
            return st;
        }
    }
    *out = c;
    return PM_OK;
}

void pm_destroy(pm_ctx *ctx)
{
    PM_RANGE("pm_destroy");
    if (!ctx) return;
    {
        DeviceScope dev(ctx->device);
        if (ctx->stage) cudaFree(ctx->stage);
        if (ctx->post_scratch) cudaFree(ctx->post_scratch);
        if (ctx->ticket) cudaFree(ctx->ticket);
        if (ctx->adj_scratch) cudaFree(ctx->adj_scratch);
        if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
        for (int i = 0; i < 2; ++i) {
            if (ctx->slot[i]) cudaFree(ctx->slot[i]);
            if (ctx->slot_free[i]) cudaEventDestroy(ctx->slot_free[i]);
        }
        if (ctx->computed) cudaEventDestroy(ctx->computed);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        for (int i = 0; i < 3; ++i) {
            if (ctx->hin_read[i]) cudaEventSynchronize(ctx->hin_read[i]);
            if (ctx->hin[i]) cudaFreeHost(ctx->hin[i]);
            if (ctx->hin_read[i]) cudaEventDestroy(ctx->hin_read[i]);
        }
    }
    delete ctx;
}

const char *pm_last_error(void) { return g_err.c_str(); }

const char *pm_version(void) { return "pm 0.1.0 (sm_103a)"; }

pm_status pm_sync_status(pm_ctx *ctx, void *stream)
{
    PM_RANGE("pm_sync_status");
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    DeviceScope dev(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    unsigned word = 0u;
    e = cudaMemcpy(&word, status_word(ctx), sizeof word, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && word) e = cudaMemset(status_word(ctx), 0, sizeof word);
    if (e != cudaSuccess) return cuda_fail(e, "reading the status word");
    if (!word) return PM_OK;
    std::string what;
    if (word & pm::kStatusModel) what += " non-finite goal or beta;";
    if (word & pm::kStatusBelief) what += " log-belief NaN, +inf or all -inf;";
    if (word & pm::kStatusObs) what += " non-finite observed state (its steps were skipped);";
    if (word & pm::kStatusTraj) what += " non-finite trajectory point (its steps were skipped);";
    return fail(PM_EDEVICE, "kernels reported (status 0x%x):%s", word, what.c_str());
}

pm_status pm_graph_launch(void *graph_exec, void *stream, void *done, int32_t wait)
{
    PM_RANGE("pm_graph_launch");
    if (!graph_exec) return fail(PM_EINVAL, "graph_exec is NULL");
    cudaError_t e = cudaGraphLaunch((cudaGraphExec_t)graph_exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    if (done) {
        e = cudaEventRecord((cudaEvent_t)done, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "event record");
    }
    if (wait) {
        e = done ? cudaEventSynchronize((cudaEvent_t)done) : cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "graph wait");
    }
    return PM_OK;
}

pm_status pm_update_posterior(pm_ctx *ctx, const pm_model *model, const float *obs_xy, int32_t n_obs,
                              float *log_belief, void *stream)
{
    PM_RANGE("pm_update_posterior");
    return posterior_impl(ctx, model, obs_xy, n_obs, log_belief, log_belief, (cudaStream_t)stream);
}

pm_status pm_update_posterior_into(pm_ctx *ctx, const pm_model *model, const float *obs_xy, int32_t n_obs,
                                   const float *log_prior, float *log_belief, void *stream)
{
    PM_RANGE("pm_update_posterior_into");
    return posterior_impl(ctx, model, obs_xy, n_obs, log_prior, log_belief, (cudaStream_t)stream);
}

pm_status pm_predict_occupancy(pm_ctx *ctx, const pm_model *model, const float *log_belief, float z0x,
                               float z0y, int32_t n_particles, int32_t horizon, const pm_grid *grid,
                               uint64_t seed, uint32_t human_id, uint32_t *counts, uint32_t *oob,
                               void *stream)
{
    PM_RANGE("pm_predict_occupancy");
    if (!counts || !oob) return fail(PM_EINVAL, "counts and oob are required");
    return predict_impl(ctx, model, log_belief, z0x, z0y, n_particles, horizon, grid, seed, human_id,
                        counts, oob, 0, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}


pm_status pm_zero_occupancy(pm_ctx *ctx, int32_t horizon, const pm_grid *grid, uint32_t *counts, uint32_t *oob,
                            void *stream)
{
    PM_RANGE("pm_zero_occupancy");
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    if (!counts || !oob) return fail(PM_EINVAL, "counts and oob are required");
    if (horizon < 1 || horizon > PM_MAX_HORIZON)
        return fail(PM_EINVAL, "horizon=%d outside [1, %d]", horizon, PM_MAX_HORIZON);
    pm_status st = check_grid(grid);
    if (st != PM_OK) return st;
    DeviceScope dev(ctx->device);
    const size_t words = (size_t)grid->W * (size_t)grid->H * (size_t)horizon;
    cudaError_t e = pm::launch_zero_outputs(counts, words, oob, horizon, nullptr, ctx->sm_count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "zeroing counts and oob");
    return PM_OK;
}

pm_status pm_rollout_occupancy(pm_ctx *ctx, const pm_model *model, const float *log_belief, float z0x,
                               float z0y, int32_t n_particles, int32_t horizon, const pm_grid *grid,
                               uint64_t seed, uint32_t human_id, uint32_t *counts, uint32_t *oob,
                               void *stream)
{
    PM_RANGE("pm_rollout_occupancy");
    if (!counts || !oob) return fail(PM_EINVAL, "counts and oob are required");
    return predict_impl(ctx, model, log_belief, z0x, z0y, n_particles, horizon, grid, seed, human_id,
                        counts, oob, 0, nullptr, nullptr, nullptr, (cudaStream_t)stream, false);
}

pm_status pm_predict_occupancy_traced(pm_ctx *ctx, const pm_model *model, const float *log_belief,
                                      float z0x, float z0y, int32_t n_particles, int32_t horizon,
                                      const pm_grid *grid, uint64_t seed, uint32_t human_id,
                                      uint32_t *counts, uint32_t *oob, int32_t n_trace, float *states,
                                      uint8_t *headings, int32_t *components, void *stream)
{
    PM_RANGE("pm_predict_occupancy_traced");
    return predict_impl(ctx, model, log_belief, z0x, z0y, n_particles, horizon, grid, seed, human_id,
                        counts, oob, n_trace, states, headings, components, (cudaStream_t)stream);
}

namespace {

// Host-buffer prediction on a device staging area `base` of `cap` bytes (or
// the context's synchronous stage when base is NULL): inputs in, belief
// update and rollout on `s`, outputs out on `out_stream` after `s` has
// computed them (same stream: in order).
pm_status predict_host_impl(pm_ctx *ctx, const pm_model *model, const float *goals, const float *beta,
                            const float *obs_xy, int32_t n_obs, const float *log_prior, int32_t n_particles,
                            int32_t horizon, const pm_grid *grid, uint64_t seed, uint32_t human_id,
                            float *posterior_out, uint32_t *counts_out, uint32_t *oob_out, cudaStream_t s,
                            int slot)
{
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    pm_status st = check_model(model, false);
    if (st != PM_OK) return st;
    st = check_grid(grid);
    if (st != PM_OK) return st;
    if (!goals || !beta || !obs_xy || !log_prior || !posterior_out || !counts_out || !oob_out)
        return fail(PM_EINVAL, "a host pointer is NULL");
    if (n_obs < 0) return fail(PM_EINVAL, "n_obs must be >= 0");
    if (horizon < 1 || horizon > PM_MAX_HORIZON) return fail(PM_EINVAL, "horizon out of range");
    if (n_particles < 1) return fail(PM_EINVAL, "n_particles must be >= 1");
    DeviceScope dev(ctx->device);
    const int J = model->G * model->B;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t plane = (size_t)grid->W * (size_t)grid->H;
    const size_t b_goals = al((size_t)model->G * 2 * 4), b_beta = al((size_t)model->B * 4);
    const size_t b_obs = al((size_t)(n_obs + 1) * 2 * 4), b_lb = al((size_t)J * 4);
    const size_t b_counts = al(plane * (size_t)horizon * 4), b_oob = al((size_t)horizon * 4);
    const size_t need = b_goals + b_beta + b_obs + b_lb + b_counts + b_oob;
    char *p;
    cudaStream_t out_stream = s;
    if (slot < 0) {
        st = ensure_stage(ctx, need);
        if (st != PM_OK) return st;
        p = (char *)ctx->stage;
    } else {
        cudaError_t e = cudaSuccess;
        if (!ctx->copy_stream) e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i)
            if (!ctx->slot_free[i]) e = cudaEventCreateWithFlags(&ctx->slot_free[i], cudaEventDisableTiming);
        if (e == cudaSuccess && !ctx->computed) e = cudaEventCreateWithFlags(&ctx->computed, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "copy stream or events");
        // the slot's previous copy-out must have read it before it is refilled
        e = cudaStreamWaitEvent(s, ctx->slot_free[slot], 0);
        if (e != cudaSuccess) return cuda_fail(e, "waiting for the staging slot");
        if (ctx->slot_bytes[slot] < need) {
            cudaStreamSynchronize(s); // the slot may still be read by an earlier copy-out
            if (ctx->slot[slot]) cudaFree(ctx->slot[slot]);
            ctx->slot[slot] = nullptr;
            ctx->slot_bytes[slot] = 0;
            e = cudaMalloc(&ctx->slot[slot], need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(PM_ENOMEM, "cudaMalloc(%zu) for a staging slot failed", need);
            }
            ctx->slot_bytes[slot] = need;
        }
        p = (char *)ctx->slot[slot];
        out_stream = ctx->copy_stream;
    }
    char *const d_in = p;
    float *d_goals = (float *)p; p += b_goals;
    float *d_beta = (float *)p; p += b_beta;
    float *d_obs = (float *)p; p += b_obs;
    float *d_lb = (float *)p; p += b_lb;
    uint32_t *d_counts = (uint32_t *)p; p += b_counts;
    uint32_t *d_oob = (uint32_t *)p;
    // the four inputs go through page-locked staging with the device layout,
    // so one upload carries them and the caller's buffers are free on return
    const size_t in_bytes = b_goals + b_beta + b_obs + b_lb;
    const int hs = slot < 0 ? 2 : slot;
    cudaError_t e = cudaSuccess;
    if (!ctx->hin_read[hs]) e = cudaEventCreateWithFlags(&ctx->hin_read[hs], cudaEventDisableTiming);
    // the staging's previous upload must have read it before it is refilled
    if (e == cudaSuccess) e = cudaEventSynchronize(ctx->hin_read[hs]);
    if (e != cudaSuccess) return cuda_fail(e, "input staging event");
    if (ctx->hin_bytes[hs] < in_bytes) {
        if (ctx->hin[hs]) cudaFreeHost(ctx->hin[hs]);
        ctx->hin[hs] = nullptr;
        ctx->hin_bytes[hs] = 0;
        const size_t cap = std::max(in_bytes, (size_t)4096);
        e = cudaHostAlloc((void **)&ctx->hin[hs], cap, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PM_ENOMEM, "cudaHostAlloc(%zu) for the input staging failed", cap);
        }
        ctx->hin_bytes[hs] = cap;
    }
    char *h = ctx->hin[hs];
    std::memcpy(h, goals, (size_t)model->G * 8);
    std::memcpy(h + b_goals, beta, (size_t)model->B * 4);
    std::memcpy(h + b_goals + b_beta, obs_xy, (size_t)(n_obs + 1) * 8);
    std::memcpy(h + b_goals + b_beta + b_obs, log_prior, (size_t)J * 4);
    e = cudaMemcpyAsync(d_in, h, in_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->hin_read[hs], s);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    pm_model m = *model;
    m.goals = d_goals;
    m.beta = d_beta;
    st = posterior_impl(ctx, &m, d_obs, n_obs, d_lb, d_lb, s);
    if (st != PM_OK) return st;
    const float z0x = obs_xy[2 * n_obs], z0y = obs_xy[2 * n_obs + 1];
    st = predict_impl(ctx, &m, d_lb, z0x, z0y, n_particles, horizon, grid, seed, human_id, d_counts, d_oob, 0,
                      nullptr, nullptr, nullptr, s);
    if (st != PM_OK) return st;
    if (out_stream != s) {
        e = cudaEventRecord(ctx->computed, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(out_stream, ctx->computed, 0);
        if (e != cudaSuccess) return cuda_fail(e, "ordering the copy-out");
    }
    e = cudaMemcpyAsync(posterior_out, d_lb, (size_t)J * 4, cudaMemcpyDeviceToHost, out_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts_out, d_counts, plane * (size_t)horizon * 4, cudaMemcpyDeviceToHost, out_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(oob_out, d_oob, (size_t)horizon * 4, cudaMemcpyDeviceToHost, out_stream);
    if (e == cudaSuccess && slot >= 0) e = cudaEventRecord(ctx->slot_free[slot], out_stream);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    return PM_OK;
}

} // namespace

pm_status pm_predict_host(pm_ctx *ctx, const pm_model *model, const float *goals, const float *beta,
                          const float *obs_xy, int32_t n_obs, const float *log_prior, int32_t n_particles,
                          int32_t horizon, const pm_grid *grid, uint64_t seed, uint32_t human_id,
                          float *posterior_out, uint32_t *counts_out, uint32_t *oob_out, void *stream)
{
    PM_RANGE("pm_predict_host");
    cudaStream_t s = (cudaStream_t)stream;
    pm_status st = predict_host_impl(ctx, model, goals, beta, obs_xy, n_obs, log_prior, n_particles, horizon, grid,
                                     seed, human_id, posterior_out, counts_out, oob_out, s, -1);
    if (st != PM_OK) return st;
    DeviceScope dev(ctx->device);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    return PM_OK;
}

pm_status pm_predict_host_async(pm_ctx *ctx, const pm_model *model, const float *goals, const float *beta,
                                const float *obs_xy, int32_t n_obs, const float *log_prior, int32_t n_particles,
                                int32_t horizon, const pm_grid *grid, uint64_t seed, uint32_t human_id,
                                float *posterior_out, uint32_t *counts_out, uint32_t *oob_out, void *stream)
{
    PM_RANGE("pm_predict_host_async");
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    const int slot = ctx->next_slot;
    pm_status st = predict_host_impl(ctx, model, goals, beta, obs_xy, n_obs, log_prior, n_particles, horizon, grid,
                                     seed, human_id, posterior_out, counts_out, oob_out, (cudaStream_t)stream, slot);
    if (st == PM_OK) ctx->next_slot = slot ^ 1;
    return st;
}

pm_status pm_host_fence(pm_ctx *ctx, void *stream)
{
    PM_RANGE("pm_host_fence");
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    DeviceScope dev(ctx->device);
    for (int i = 0; i < 2; ++i) {
        if (!ctx->slot_free[i]) continue;
        cudaError_t e = cudaStreamWaitEvent((cudaStream_t)stream, ctx->slot_free[i], 0);
        if (e != cudaSuccess) return cuda_fail(e, "fence");
    }
    return PM_OK;
}


pm_status pm_batch_create(pm_ctx *ctx, const pm_model *shared, int32_t max_humans, pm_batch **out)
{
    PM_RANGE("pm_batch_create");
    if (!ctx || !out) return fail(PM_EINVAL, "ctx/out is NULL");
    *out = nullptr;
    pm_status st = check_model(shared, false);
    if (st != PM_OK) return st;
    if (max_humans < 1 || max_humans > 65535) return fail(PM_EINVAL, "max_humans=%d out of range", max_humans);
    DeviceScope dev(ctx->device);
    pm_batch *b = new pm_batch();
    b->ctx = ctx;
    b->shared = *shared;
    b->shared.goals = nullptr;
    b->shared.beta = nullptr;
    b->max_humans = max_humans;
    b->post_stride = pm::posterior_scratch_bytes(64, PM_MAX_COMPONENTS) / sizeof(float);
    b->items_cap = (size_t)max_humans * 2048;
    cudaError_t e = cudaMalloc(&b->d_humans, (size_t)max_humans * sizeof(pm::BatchHuman));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_post, (size_t)max_humans * sizeof(pm::PostHuman));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, b->items_cap * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_meta, 256);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_srcs, (size_t)max_humans * sizeof(pm::SmoothSrc));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_head, 256);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_post_part, (size_t)max_humans * b->post_stride * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_post_ticket, (size_t)max_humans * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_post_ticket, 0, (size_t)max_humans * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_prev, (size_t)max_humans * sizeof(float2) + 16);
    if (e == cudaSuccess) e = cudaMemset(b->d_prev, 0xFF, (size_t)max_humans * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(reinterpret_cast<char *>(b->d_prev) + (size_t)max_humans * sizeof(float2), 0, 16);
    if (e == cudaSuccess) e = cudaMemset(b->d_meta, 0, 256);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        pm_batch_destroy(b);
        return fail(PM_ENOMEM, "batch allocation failed: %s", cudaGetErrorString(e));
    }
    *out = b;
    return PM_OK;
}

void pm_batch_destroy(pm_batch *b)
{
    PM_RANGE("pm_batch_destroy");
    if (!b) return;
    DeviceScope dev(b->ctx->device);
    if (b->staged) {
        cudaEventSynchronize(b->staged);
        cudaEventDestroy(b->staged);
    }
    cudaFree(b->d_humans);
    cudaFree(b->d_post);
    cudaFree(b->d_items);
    cudaFree(b->d_meta);
    cudaFree(b->d_srcs);
    cudaFree(b->d_flags);
    cudaFree(b->d_head);
    cudaFree(b->d_post_part);
    cudaFree(b->d_post_ticket);
    cudaFree(b->d_prev);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    delete b;
}

pm_status pm_batch_set(pm_batch *b, const pm_human *humans, int32_t n_humans, void *stream)
{
    PM_RANGE("pm_batch_set");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    if (n_humans < 0 || n_humans > b->max_humans) return fail(PM_EINVAL, "n_humans=%d outside [0, %d]", n_humans, b->max_humans);
    if (n_humans > 0 && !humans) return fail(PM_EINVAL, "humans is NULL");
    for (int i = 0; i < n_humans; ++i) {
        pm_status st = check_human(humans[i], i, b->shared);
        if (st != PM_OK) return st;
    }
    DeviceScope dev(b->ctx->device);
    b->humans.assign(humans, humans + n_humans);
    return batch_upload(b, (cudaStream_t)stream);
}

pm_status pm_batch_update_posterior(pm_batch *b, void *stream)
{
    PM_RANGE("pm_batch_update_posterior");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    DeviceScope dev(b->ctx->device);
    pm::PosteriorArgs a;
    fill_posterior_args(&b->shared, a); // goals/beta per human
    a.status = status_word(b->ctx);
    cudaError_t e = pm::launch_posterior_batch(a, b->d_post, b->d_meta + 1, b->max_humans, b->max_chunks, b->max_J,
                                               (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "batched posterior launch");
    return PM_OK;
}

pm_status pm_batch_set_zeroing(pm_batch *b, int32_t reach, void *stream)
{
    PM_RANGE("pm_batch_set_zeroing");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    if (reach != 0 && reach != 1) return fail(PM_EINVAL, "reach=%d: 0 or 1", reach);
    DeviceScope dev(b->ctx->device);
    b->zero_reach = reach != 0;
    cudaError_t e = forget_starts(b, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch start records");
    return PM_OK;
}

pm_status pm_batch_zero(pm_batch *b, void *stream)
{
    PM_RANGE("pm_batch_zero");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    DeviceScope dev(b->ctx->device);
    return batch_zero_impl(b, (cudaStream_t)stream);
}

pm_status pm_batch_rollout(pm_batch *b, void *stream)
{
    PM_RANGE("pm_batch_rollout");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    DeviceScope dev(b->ctx->device);
    return batch_rollout_impl(b, (cudaStream_t)stream);
}

pm_status pm_batch_predict(pm_batch *b, void *stream)
{
    PM_RANGE("pm_batch_predict");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    DeviceScope dev(b->ctx->device);
    return batch_predict_impl(b, (cudaStream_t)stream);
}

namespace {

// Blur taps w_{-R..R} of the truncated, normalised Gaussian (computed in double).
pm_status smooth_taps(float sigma, pm::SmoothArgs &a)
{
    if (!(sigma >= 0.0f) || !(3.0 * (double)sigma <= (double)pm::kMaxSmoothR))
        return fail(PM_EINVAL, "sigma_cells=%g: need 0 <= ceil(3 sigma) <= %d", (double)sigma, pm::kMaxSmoothR);
    if (sigma == 0.0f) {
        a.R = 0;
        a.w[0] = 1.0f;
        return PM_OK;
    }
    const int R = (int)std::ceil(3.0 * (double)sigma); // <= kMaxSmoothR by the check above
    double w[2 * pm::kMaxSmoothR + 1], sum = 0.0;
    for (int i = -R; i <= R; ++i) sum += (w[i + R] = std::exp(-(double)i * i / (2.0 * (double)sigma * sigma)));
    for (int i = 0; i <= 2 * R; ++i) a.w[i] = (float)(w[i] / sum);
    a.R = R;
    return PM_OK;
}

} // namespace

pm_status pm_smooth_occupancy(pm_ctx *ctx, const uint32_t *counts, int32_t n_particles, int32_t horizon,
                              const pm_grid *grid, float sigma_cells, float *prob, void *stream)
{
    PM_RANGE("pm_smooth_occupancy");
    if (!ctx || !counts || !prob) return fail(PM_EINVAL, "ctx/counts/prob is NULL");
    if (n_particles < 1) return fail(PM_EINVAL, "n_particles=%d must be >= 1", n_particles);
    if (horizon < 1 || horizon > PM_MAX_HORIZON) return fail(PM_EINVAL, "horizon=%d out of range", horizon);
    pm_status st = check_grid(grid);
    if (st != PM_OK) return st;
    pm::SmoothArgs a;
    std::memset(&a, 0, sizeof a);
    st = smooth_taps(sigma_cells, a);
    if (st != PM_OK) return st;
    a.single.counts = counts;
    a.single.inv_n = 1.0f / (float)n_particles;
    a.single.small = n_particles < (1 << 23);
    a.single.T = horizon;
    a.single.W = grid->W;
    a.single.H = grid->H;
    a.out = prob;
    a.T = horizon;
    a.W = grid->W;
    a.H = grid->H;
    DeviceScope dev(ctx->device);
    cudaGetLastError();
    cudaError_t e = pm::launch_smooth_union(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "smoothing launch");
    return PM_OK;
}

pm_status pm_batch_union(pm_batch *b, float sigma_cells, int32_t horizon, const pm_grid *grid, float *prob,
                         void *stream)
{
    PM_RANGE("pm_batch_union");
    if (!b || !prob) return fail(PM_EINVAL, "batch/prob is NULL");
    if (horizon < 1 || horizon > PM_MAX_HORIZON) return fail(PM_EINVAL, "horizon=%d out of range", horizon);
    pm_status st = check_grid(grid);
    if (st != PM_OK) return st;
    for (size_t i = 0; i < b->humans.size(); ++i) {
        const pm_grid &g = b->humans[i].grid;
        if (g.x0 != grid->x0 || g.y0 != grid->y0 || g.res != grid->res)
            return fail(PM_EINVAL, "human %zu: grid origin/resolution differ from the shared grid", i);
    }
    pm::SmoothArgs a;
    std::memset(&a, 0, sizeof a);
    st = smooth_taps(sigma_cells, a);
    if (st != PM_OK) return st;
    a.srcs = b->d_srcs;
    a.n_srcs = b->d_meta + 1;
    a.out = prob;
    a.T = horizon;
    a.W = grid->W;
    a.H = grid->H;
    DeviceScope dev(b->ctx->device);
    cudaGetLastError();
    cudaError_t e = pm::launch_union_sources(b->d_humans, b->d_meta + 1, b->max_humans, b->d_srcs,
                                             (cudaStream_t)stream);
    if (e == cudaSuccess) e = pm::launch_smooth_union(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "union launch");
    return PM_OK;
}

pm_status pm_batch_get_config(const pm_batch *b, int32_t *threads, int32_t *shared_window, int32_t *ctas_per_sm,
                              int32_t *window_kib)
{
    PM_RANGE("pm_batch_get_config");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    if (threads) *threads = b->threads;
    if (shared_window) *shared_window = b->warp_hist ? 0 : 1;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (window_kib) *window_kib = b->window_kib;
    return PM_OK;
}

pm_status pm_batch_set_config(pm_batch *b, int32_t threads, int32_t shared_window, int32_t ctas_per_sm,
                              int32_t window_kib)
{
    PM_RANGE("pm_batch_set_config");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    if (shared_window != 0 && shared_window != 1) return fail(PM_EINVAL, "shared_window must be 0 or 1");
    if (threads < 32 || threads > 256 || threads % 32) return fail(PM_EINVAL, "threads=%d must be 32..256, multiple of 32", threads);
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(PM_EINVAL, "ctas_per_sm=%d out of range", ctas_per_sm);
    if (window_kib < 1 || window_kib > 200) return fail(PM_EINVAL, "window_kib=%d out of range", window_kib);
    if (shared_window && multi_speed(&b->shared))
        return fail(PM_EINVAL, "several speeds run only the warp-combined emplacement (shared_window=0)");
    DeviceScope dev(b->ctx->device);
    const bool retile = threads != b->threads || (shared_window == 0) != b->warp_hist;
    b->threads = threads;
    b->warp_hist = shared_window == 0;
    b->ctas_per_sm = ctas_per_sm;
    b->window_kib = window_kib;
    if (retile && !b->humans.empty()) return batch_upload(b, nullptr);
    pm::RolloutArgs t;
    std::memset(&t, 0, sizeof t);
    fill_rollout_tables(&b->shared, t);
    b->occ = pm::batch_rollout_occupancy(b->shared.K, t.enabled, t.tab.S, b->block_flags && b->warp_hist,
                                         batch_shape_of(b), batch_dyn_smem(b));
    cudaGetLastError();
    return PM_OK;
}

pm_status pm_batch_set_block_flags(pm_batch *b, int32_t enable, void *stream)
{
    PM_RANGE("pm_batch_set_block_flags");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    if (enable != 0 && enable != 1) return fail(PM_EINVAL, "enable must be 0 or 1");
    DeviceScope dev(b->ctx->device);
    b->block_flags = enable != 0;
    return b->humans.empty() ? PM_OK : batch_upload(b, (cudaStream_t)stream);
}

pm_status pm_batch_autotune(pm_batch *b, void *stream)
{
    PM_RANGE("pm_batch_autotune");
    if (!b) return fail(PM_EINVAL, "batch is NULL");
    if (b->humans.empty()) return PM_OK;
    DeviceScope dev(b->ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    struct Cand {
        int threads;
        bool warp;
        int window;
    };
    static const Cand cands[] = {{256, true, 48}, {128, true, 48}, {224, false, 48}, {256, false, 48},
                                 {256, false, 96}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Cand bc{b->threads, b->warp_hist, b->window_kib};
    for (const Cand &cd : cands) {
        if (!cd.warp && multi_speed(&b->shared)) continue; // several speeds: warp emplacement only
        b->threads = cd.threads;
        b->warp_hist = cd.warp;
        b->window_kib = cd.window;
        b->ctas_per_sm = 0;
        if (batch_upload(b, s) != PM_OK) continue;
        if (batch_predict_impl(b, s) != PM_OK) { // warm-up; a shape that does not fit is skipped
            cudaGetLastError();
            continue;
        }
        float total = 0.0f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            cudaEventRecord(e0, s);
            ok = batch_predict_impl(b, s) == PM_OK;
            cudaEventRecord(e1, s);
            float ms = 0.0f;
            if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                total += ms;
            else
                ok = false;
        }
        if (ok && total < best) {
            best = total;
            bc = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->threads = bc.threads;
    b->warp_hist = bc.warp;
    b->window_kib = bc.window;
    b->ctas_per_sm = 0;
    pm_status st = batch_upload(b, s);
    if (st != PM_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    return PM_OK;
}

pm_status pm_loglik_forward(pm_ctx *ctx, const pm_model *model, int32_t M, const int32_t *offsets,
                            int32_t n_points, const float *traj_xy, const float *log_prior, float *loglik,
                            void *stream)
{
    PM_RANGE("pm_loglik_forward");
    return loglik_impl(ctx, model, M, offsets, n_points, traj_xy, log_prior, false, 1.0f, loglik, nullptr,
                       nullptr, nullptr, (cudaStream_t)stream);
}

pm_status pm_loglik_backward(pm_ctx *ctx, const pm_model *model, int32_t M, const int32_t *offsets,
                             int32_t n_points, const float *traj_xy, const float *log_prior, float grad_out,
                             float *loglik, float *d_goals, float *d_speed, float *d_w, void *stream)
{
    PM_RANGE("pm_loglik_backward");
    return loglik_impl(ctx, model, M, offsets, n_points, traj_xy, log_prior, true, grad_out, loglik, d_goals,
                       d_speed, d_w, (cudaStream_t)stream);
}

pm_status pm_philox_blocks(pm_ctx *ctx, uint64_t seed, uint32_t human_id, uint32_t purpose, uint64_t particle0,
                           uint64_t block, int32_t n, uint64_t *out, void *stream)
{
    PM_RANGE("pm_philox_blocks");
    if (!ctx || !out) return fail(PM_EINVAL, "ctx/out is NULL");
    if (n < 0) return fail(PM_EINVAL, "n must be >= 0");
    if (n == 0) return PM_OK;
    DeviceScope dev(ctx->device);
    cudaError_t e = pm::launch_philox_blocks(seed, human_id, purpose, particle0, block, n, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "philox launch");
    return PM_OK;
}

pm_status pm_mppi_solve(pm_ctx *ctx, const pm_mppi *p, const float *z0, const float *u_ref, const float *delta,
                        const float *prob, int32_t prob_T, const pm_grid *grid, float *cost_to_go, float *u_opt,
                        void *stream)
{
    PM_RANGE("pm_mppi_solve");
    if (!ctx || !p || !z0 || !u_ref || !delta || !cost_to_go || !u_opt)
        return fail(PM_EINVAL, "ctx/params/z0/u_ref/delta/cost_to_go/u_opt is NULL");
    if ((uintptr_t)delta & 7u) return fail(PM_EINVAL, "delta must be 8-byte aligned (read as pairs)");
    if (p->n_samples < 1 || p->horizon < 1 || p->pred_stride < 1)
        return fail(PM_EINVAL, "n_samples=%d horizon=%d pred_stride=%d must be >= 1", p->n_samples, p->horizon,
                    p->pred_stride);
    if ((long long)p->n_samples * p->horizon > (1LL << 31)) return fail(PM_EINVAL, "n_samples x horizon too large");
    if (!finite_pos(p->dt) || !finite_pos(p->temperature)) return fail(PM_EINVAL, "dt and temperature must be > 0");
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(p->q[k]) || !std::isfinite(p->q_final[k]) || !std::isfinite(p->goal[k]) ||
            !std::isfinite(z0[k]))
            return fail(PM_EINVAL, "weights, goal and z0 must be finite");
    if (!std::isfinite(p->r[0]) || !std::isfinite(p->r[1]) || !std::isfinite(p->coll_threshold) ||
        !std::isfinite(p->coll_cost) || !std::isfinite(p->step_cost))
        return fail(PM_EINVAL, "costs must be finite");
    pm::MppiArgs a;
    std::memset(&a, 0, sizeof a);
    if (prob) {
        pm_status st = check_grid(grid);
        if (st != PM_OK) return st;
        if (prob_T < 1) return fail(PM_EINVAL, "prob_T=%d must be >= 1", prob_T);
        a.prob = prob;
        a.prob_T = prob_T;
        a.W = grid->W;
        a.H = grid->H;
        a.gx0 = grid->x0;
        a.gy0 = grid->y0;
        a.inv_res = 1.0f / grid->res;
    }
    a.N = p->n_samples;
    a.T = p->horizon;
    a.pred_stride = p->pred_stride;
    a.dt = p->dt;
    for (int k = 0; k < 4; ++k) {
        a.z0[k] = z0[k];
        a.q[k] = p->q[k];
        a.q_final[k] = p->q_final[k];
        a.goal[k] = p->goal[k];
    }
    a.r[0] = p->r[0];
    a.r[1] = p->r[1];
    a.coll_threshold = p->coll_threshold;
    a.coll_cost = p->coll_cost;
    a.step_cost = p->step_cost;
    a.temperature = p->temperature;
    a.u_ref = u_ref;
    a.delta = delta;
    a.ctg = cost_to_go;
    a.u_opt = u_opt;
    DeviceScope dev(ctx->device);
    cudaGetLastError();
    cudaError_t e = pm::launch_mppi(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mppi launch");
    return PM_OK;
}

pm_status pm_probe_sfu(pm_ctx *ctx, int op, double *results_per_s)
{
    PM_RANGE("pm_probe_sfu");
    if (!ctx || !results_per_s) return fail(PM_EINVAL, "ctx/results is NULL");
    if (op < 0 || op > 5) return fail(PM_EINVAL, "op %d outside [0, 5]", op);
    DeviceScope dev(ctx->device);
    const int threads = 256, blocks = ctx->sm_count * 8, iters = 4096;
    pm_status st = ensure_stage(ctx, (size_t)blocks * threads * sizeof(float));
    if (st != PM_OK) return st;
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "stream");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        e = pm::launch_sfu_probe(op, blocks, threads, iters, (float *)ctx->stage, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms > 0.0f && ms < best_ms) best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_fail(e, "sfu probe");
    const double per_instr = (op == 4) ? 2.0 : 1.0; // the packed FMA yields two results
    *results_per_s = (double)blocks * threads * iters * 8.0 * per_instr / (best_ms * 1e-3);
    return PM_OK;
}

pm_status pm_device_info(pm_ctx *ctx, int *sm_count, int *clock_khz, int *cc)
{
    PM_RANGE("pm_device_info");
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    if (sm_count) *sm_count = ctx->sm_count;
    if (clock_khz) *clock_khz = ctx->clock_khz;
    if (cc) *cc = ctx->cc;
    return PM_OK;
}

} // extern "C"
