// pm_api.cu -- host side of the C ABI declared in include/pm.h: the context,
// argument validation, the heading tables, launch configuration and the
// host-buffer convenience call. No arithmetic of the method runs here; every
// numeric step is a kernel of this library.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include <cuda_runtime.h>

#include "pm.h"
#include "pm_internal.cuh"

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
};

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
    return PM_OK;
}

pm_status check_grid(const pm_grid *g)
{
    if (!g) return fail(PM_EINVAL, "grid is NULL");
    if (!finite_pos(g->res) || !std::isfinite(g->x0) || !std::isfinite(g->y0))
        return fail(PM_EINVAL, "grid origin must be finite and res > 0");
    if (g->W < 1 || g->H < 1 || (long long)g->W * g->H > (1LL << 31))
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
    }
    a.enabled = enabled_mask(m);
    a.s2 = (float)(s * s);
    a.w2_log2e = (float)((double)m->w2 * 1.4426950408889634);
    a.K = m->K;
    a.G = m->G;
    a.B = m->B;
    a.goals = m->goals;
    a.beta = m->beta;
}

// Window of the shared-memory histogram: the cells within reach of z0 in T
// steps (|z_t - z0| <= T v dt), clipped to the grid and to 255 x 255 cells and
// to the shared-memory budget; particles outside it are counted directly.
void choose_window(const pm_model *m, const pm_grid *g, float z0x, float z0y, int T, int threads,
                   size_t smem_budget, pm::RolloutArgs &a, size_t *dyn_smem)
{
    const float inv_res = 1.0f / g->res;
    const double cx0 = std::floor((double)((z0x - g->x0) * inv_res));
    const double cy0 = std::floor((double)((z0y - g->y0) * inv_res));
    const double reach = std::ceil((double)T * (double)m->speed * (double)m->dt / (double)g->res) + 1.0;
    const size_t list_bytes = (size_t)threads * sizeof(uint16_t);
    long long r = (long long)std::fmin(reach, 127.0);
    for (;;) {
        long long x_lo = (long long)std::fmax(cx0 - r, 0.0), x_hi = (long long)std::fmin(cx0 + r, (double)g->W - 1);
        long long y_lo = (long long)std::fmax(cy0 - r, 0.0), y_hi = (long long)std::fmin(cy0 + r, (double)g->H - 1);
        long long w = x_hi - x_lo + 1, h = y_hi - y_lo + 1;
        if (w <= 0 || h <= 0) { // z0 is far outside the grid: no window
            a.win_x0 = a.win_y0 = 0;
            a.win_side = 0;
            *dyn_smem = list_bytes;
            return;
        }
        const size_t words = (size_t)((w * h + 1) / 2);
        const size_t bytes = ((words * 4 + 15) & ~(size_t)15) + list_bytes;
        if (bytes <= smem_budget || r <= 4) {
            a.win_x0 = (int)x_lo;
            a.win_y0 = (int)y_lo;
            a.win_side = (int)(w | (h << 16));
            *dyn_smem = bytes;
            return;
        }
        r = (r * 7) / 8;
    }
}

// Block size of the rollout: one particle per thread, all CTAs resident in
// one wave where possible, and the CTAs spread evenly over the SMs (the
// kernel time follows the most loaded SM: ceil(blocks / SMs) CTAs of
// `threads` particles each).
int choose_rollout_threads(pm_ctx *ctx, const pm_model *model, const pm_grid *grid, pm::RolloutArgs &a,
                           bool hist, size_t *dyn_out)
{
    static const int cand[] = {256, 224, 192, 160, 128};
    double best_eff = -1.0;
    int best_t = 256;
    size_t best_dyn = 0;
    pm::RolloutArgs trial = a;
    for (int t : cand) {
        size_t dyn = 0;
        if (hist) choose_window(model, grid, a.z0x, a.z0y, a.T, t, 64 * 1024, trial, &dyn);
        const int occ = pm::rollout_occupancy(trial, t, dyn);
        if (occ < 1) continue;
        const long long blocks = ((long long)a.N + t - 1) / t;
        const long long per_sm = (blocks + ctx->sm_count - 1) / ctx->sm_count;
        const double eff = (double)a.N / ((double)per_sm * t * ctx->sm_count) * (occ >= 2 ? 1.0 : 0.8);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best_t = t;
            best_dyn = dyn;
        }
    }
    if (hist) choose_window(model, grid, a.z0x, a.z0y, a.T, best_t, 64 * 1024, a, &best_dyn);
    *dyn_out = best_dyn;
    return best_t;
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
                       cudaStream_t stream)
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
    size_t dyn = 0;
    int threads = 256;
    if (hist) {
        a.gx0 = grid->x0;
        a.gy0 = grid->y0;
        a.inv_res = 1.0f / grid->res;
        a.W = grid->W;
        a.H = grid->H;
        a.counts = counts;
        a.oob = oob;
        const size_t plane = (size_t)grid->W * (size_t)grid->H;
        cudaError_t e = cudaMemsetAsync(counts, 0, plane * (size_t)horizon * sizeof(uint32_t), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(oob, 0, (size_t)horizon * sizeof(uint32_t), stream);
        if (e != cudaSuccess) return cuda_fail(e, "zeroing counts/oob");
    } else {
        a.W = a.H = 1;
        a.inv_res = 1.0f;
    }
    threads = choose_rollout_threads(ctx, model, grid, a, hist, &dyn);
    cudaError_t e = pm::launch_rollout(a, threads, dyn, stream);
    if (e != cudaSuccess) return cuda_fail(e, "rollout launch");
    return PM_OK;
}

pm_status posterior_impl(pm_ctx *ctx, const pm_model *model, const float *obs_xy, int32_t n_obs,
                         float *log_belief, cudaStream_t stream)
{
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    pm_status st = check_model(model);
    if (st != PM_OK) return st;
    if (n_obs < 0) return fail(PM_EINVAL, "n_obs=%d must be >= 0", n_obs);
    if (!log_belief) return fail(PM_EINVAL, "log_belief is NULL");
    if (n_obs == 0) return PM_OK;
    if (!obs_xy) return fail(PM_EINVAL, "obs_xy is NULL");
    DeviceScope dev(ctx->device);
    pm::PosteriorArgs a;
    std::memset(&a, 0, sizeof a);
    const double s = (double)model->speed * (double)model->dt;
    for (int k = 0; k < model->K; ++k) {
        double c, sn;
        unit_heading(model->K, k, &c, &sn);
        a.ux[k] = (float)c;
        a.uy[k] = (float)sn;
    }
    a.enabled = enabled_mask(model);
    a.s = (float)s;
    a.s2 = (float)(s * s);
    a.two_s = (float)(2.0 * s);
    a.w2 = model->w2;
    a.K = model->K;
    a.G = model->G;
    a.B = model->B;
    a.goals = model->goals;
    a.beta = model->beta;
    a.obs = obs_xy;
    a.n_obs = n_obs;
    a.log_b = log_belief;
    const int n_chunks = pm::posterior_chunks(n_obs, &a.steps_per_chunk);
    st = ensure_posterior_scratch(ctx, pm::posterior_scratch_bytes(n_chunks, model->G * model->B));
    if (st != PM_OK) return st;
    a.part = (float *)ctx->post_scratch;
    a.ticket = ctx->ticket;
    cudaError_t e = pm::launch_posterior(a, n_chunks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "posterior launch");
    return PM_OK;
}

} // namespace

extern "C" {

pm_status pm_create(pm_ctx **out, int device)
{
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
    *out = c;
    return PM_OK;
}

void pm_destroy(pm_ctx *ctx)
{
    if (!ctx) return;
    {
        DeviceScope dev(ctx->device);
        if (ctx->stage) cudaFree(ctx->stage);
        if (ctx->post_scratch) cudaFree(ctx->post_scratch);
        if (ctx->ticket) cudaFree(ctx->ticket);
    }
    delete ctx;
}

const char *pm_last_error(void) { return g_err.c_str(); }

const char *pm_version(void) { return "pm 0.1.0 (sm_103a)"; }

pm_status pm_update_posterior(pm_ctx *ctx, const pm_model *model, const float *obs_xy, int32_t n_obs,
                              float *log_belief, void *stream)
{
    return posterior_impl(ctx, model, obs_xy, n_obs, log_belief, (cudaStream_t)stream);
}

pm_status pm_predict_occupancy(pm_ctx *ctx, const pm_model *model, const float *log_belief, float z0x,
                               float z0y, int32_t n_particles, int32_t horizon, const pm_grid *grid,
                               uint64_t seed, uint32_t human_id, uint32_t *counts, uint32_t *oob,
                               void *stream)
{
    if (!counts || !oob) return fail(PM_EINVAL, "counts and oob are required");
    return predict_impl(ctx, model, log_belief, z0x, z0y, n_particles, horizon, grid, seed, human_id,
                        counts, oob, 0, nullptr, nullptr, nullptr, (cudaStream_t)stream);
}

pm_status pm_predict_occupancy_traced(pm_ctx *ctx, const pm_model *model, const float *log_belief,
                                      float z0x, float z0y, int32_t n_particles, int32_t horizon,
                                      const pm_grid *grid, uint64_t seed, uint32_t human_id,
                                      uint32_t *counts, uint32_t *oob, int32_t n_trace, float *states,
                                      uint8_t *headings, int32_t *components, void *stream)
{
    return predict_impl(ctx, model, log_belief, z0x, z0y, n_particles, horizon, grid, seed, human_id,
                        counts, oob, n_trace, states, headings, components, (cudaStream_t)stream);
}

pm_status pm_predict_host(pm_ctx *ctx, const pm_model *model, const float *goals, const float *beta,
                          const float *obs_xy, int32_t n_obs, const float *log_prior, int32_t n_particles,
                          int32_t horizon, const pm_grid *grid, uint64_t seed, uint32_t human_id,
                          float *posterior_out, uint32_t *counts_out, uint32_t *oob_out, void *stream)
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
    cudaStream_t s = (cudaStream_t)stream;
    const int J = model->G * model->B;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t plane = (size_t)grid->W * (size_t)grid->H;
    const size_t b_goals = al((size_t)model->G * 2 * 4), b_beta = al((size_t)model->B * 4);
    const size_t b_obs = al((size_t)(n_obs + 1) * 2 * 4), b_lb = al((size_t)J * 4);
    const size_t b_counts = al(plane * (size_t)horizon * 4), b_oob = al((size_t)horizon * 4);
    st = ensure_stage(ctx, b_goals + b_beta + b_obs + b_lb + b_counts + b_oob);
    if (st != PM_OK) return st;
    char *p = (char *)ctx->stage;
    float *d_goals = (float *)p; p += b_goals;
    float *d_beta = (float *)p; p += b_beta;
    float *d_obs = (float *)p; p += b_obs;
    float *d_lb = (float *)p; p += b_lb;
    uint32_t *d_counts = (uint32_t *)p; p += b_counts;
    uint32_t *d_oob = (uint32_t *)p;
    cudaError_t e = cudaMemcpyAsync(d_goals, goals, (size_t)model->G * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_beta, beta, (size_t)model->B * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_obs, obs_xy, (size_t)(n_obs + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_lb, log_prior, (size_t)J * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    pm_model m = *model;
    m.goals = d_goals;
    m.beta = d_beta;
    st = posterior_impl(ctx, &m, d_obs, n_obs, d_lb, s);
    if (st != PM_OK) return st;
    const float z0x = obs_xy[2 * n_obs], z0y = obs_xy[2 * n_obs + 1];
    st = predict_impl(ctx, &m, d_lb, z0x, z0y, n_particles, horizon, grid, seed, human_id, d_counts, d_oob, 0,
                      nullptr, nullptr, nullptr, s);
    if (st != PM_OK) return st;
    e = cudaMemcpyAsync(posterior_out, d_lb, (size_t)J * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts_out, d_counts, plane * (size_t)horizon * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(oob_out, d_oob, (size_t)horizon * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    return PM_OK;
}

pm_status pm_philox_blocks(pm_ctx *ctx, uint64_t seed, uint32_t human_id, uint32_t purpose, uint64_t particle0,
                           uint64_t block, int32_t n, uint64_t *out, void *stream)
{
    if (!ctx || !out) return fail(PM_EINVAL, "ctx/out is NULL");
    if (n < 0) return fail(PM_EINVAL, "n must be >= 0");
    if (n == 0) return PM_OK;
    DeviceScope dev(ctx->device);
    cudaError_t e = pm::launch_philox_blocks(seed, human_id, purpose, particle0, block, n, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "philox launch");
    return PM_OK;
}

pm_status pm_probe_sfu(pm_ctx *ctx, int op, double *results_per_s)
{
    if (!ctx || !results_per_s) return fail(PM_EINVAL, "ctx/results is NULL");
    if (op < 0 || op > 2) return fail(PM_EINVAL, "op %d outside [0, 2]", op);
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
    *results_per_s = (double)blocks * threads * iters * 8.0 / (best_ms * 1e-3);
    return PM_OK;
}

pm_status pm_device_info(pm_ctx *ctx, int *sm_count, int *clock_khz, int *cc)
{
    if (!ctx) return fail(PM_EINVAL, "ctx is NULL");
    if (sm_count) *sm_count = ctx->sm_count;
    if (clock_khz) *clock_khz = ctx->clock_khz;
    if (cc) *cc = ctx->cc;
    return PM_OK;
}

} // extern "C"
