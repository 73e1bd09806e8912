/*
 * pm_oracle.c -- plain, slow FP64 CPU oracle for confidence-aware human
 * prediction (Lu, Bui, Lyu, Chen, "Fast Confidence-Aware Human Prediction via
 * Hardware-accelerated Bayesian Inference for Safe Robot Navigation").
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. It shares
 * no code, header, table or constant generator with the CUDA library; each
 * side is written from the paper's equations and from the published Philox
 * definition on its own.
 *
 * Every routine is single-threaded and follows the paper's order of steps:
 *   orc_philox4x64      Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
 *   orc_log_policy      Eq. 2 (Boltzmann policy), running example Q of Sec. III-A
 *   orc_update_posterior Eq. 3 evaluated in log space as Eq. 7, per observed step
 *   orc_rollout         Algorithm 1 with the bootstrapped belief (Sec. III-B)
 *   orc_bin             the "emplace onto a grid" step of Algorithm 1
 *   orc_exact_occupancy Eq. 4 / Eq. 5: exact Markov propagation (small K, T)
 *   orc_loglik_grad     marginal log-likelihood of observed trajectories and its
 *                       analytic gradient (built on Eq. 2 / Eq. 3)
 *
 * Readings of points the paper leaves open:
 *   - Q(z, theta; g) = -w1*v*dt - w2*|| z + v*dt*(cos theta, sin theta) - g ||,
 *     evaluated at the next state (the running example's Q is heading-free).
 *   - K headings theta_k = 2*pi*k/K, counter-clockwise from +x; the controls
 *     are those headings at speeds v*mult[s] (one speed, mult = {1}, unless
 *     given), index u = s*K + k; a disabled heading or speed has Q = -inf.
 *   - the observed control is the continuous heading atan2(dy, dx) of the
 *     displacement at the enabled speed whose multiplier is nearest to its
 *     length / (v*dt) (ties: the lower index); Q is evaluated there and
 *     normalised over the controls; a displacement shorter than 1e-6 m leaves
 *     the belief unchanged. With `snap` set, the heading is read as the
 *     enabled heading theta_k nearest to atan2(dy, dx) instead (largest
 *     cos(theta - theta_k); ties: the lower index), so the observed control
 *     is one of the discrete controls.
 *   - belief index j = g*B + b (goal-major).
 *   - inverse-CDF sampling: smallest k with u*S < C_k, C_k the running sum in
 *     index order, S the total; u = (32-bit word >> 8) * 2^-24.
 *   - binning from the FP32 state: c = floor((x -f x0) *f inv_res) with
 *     inv_res the FP32 value 1/res; cells are half open; a particle outside
 *     the grid counts in oob[t] and stays alive.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * FP32 shadow state and binning follow IEEE single-precision operations).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PURPOSE_SELECT 1u
#define ORC_PURPOSE_STEP 2u

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, from the round function published by Salmon et al. (SC'11) */
/* ------------------------------------------------------------------------ */
static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *lo = (uint64_t)p;
    *hi = (uint64_t)(p >> 64);
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        orc_mulhilo64(M0, c0, &hi0, &lo0);
        orc_mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The 32-bit word w (0..7) of the block (particle, block, purpose) of stream
 * (seed, human). Word w is bits [32*(w&1), 32*(w&1)+32) of 64-bit output w>>1. */
static uint32_t orc_word(uint64_t seed, uint32_t human, uint64_t particle,
                         uint64_t block, uint32_t purpose, unsigned w)
{
    uint64_t ctr[4] = {particle, block, (uint64_t)purpose, 0};
    uint64_t key[2] = {seed, (uint64_t)human};
    uint64_t out[4];
    orc_philox4x64(ctr, key, out);
    return (uint32_t)(out[w >> 1] >> (32u * (w & 1u)));
}

/* Uniform in [0, 1 - 2^-24], exactly representable in FP32 and FP64. */
static double orc_uniform(uint32_t word) { return (double)(word >> 8) * (1.0 / 16777216.0); }

/* Uniform for the (beta, g) draw of particle i. */
double orc_uniform_select(uint64_t seed, uint32_t human, uint64_t i)
{
    return orc_uniform(orc_word(seed, human, i, 0, ORC_PURPOSE_SELECT, 0));
}

/* Uniform for the heading draw of particle i at prediction step t (t >= 1). */
double orc_uniform_step(uint64_t seed, uint32_t human, uint64_t i, int t)
{
    uint64_t q = (uint64_t)(t - 1);
    return orc_uniform(orc_word(seed, human, i, q >> 3, ORC_PURPOSE_STEP, (unsigned)(q & 7u)));
}

/* ------------------------------------------------------------------------ */
/* Model: Eq. 1 (kinematics), Eq. 2 (Boltzmann policy), Q of Sec. III-A      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int K;
    double v, dt, w1, w2;
    int G, B;
    const double *goals; /* [G][2] */
    const double *beta;  /* [B] */
    uint64_t mask_off;   /* bit k set: heading k disabled, Q = -inf */
    int S;               /* speeds: control u = s*K + k moves v*mult[s]*dt along theta_k */
    const double *mult;  /* [S] speed multipliers (> 0) */
    uint32_t speed_off;  /* bit s set: speed s disabled, Q = -inf (stationary masking) */
    int snap;            /* 1: the observed heading is read as the nearest enabled heading */
} orc_model;

/* Unit vector of heading k, theta_k = 2*pi*k/K. Quarter turns are exact. */
static void orc_heading(int K, int k, double *c, double *s)
{
    int q4 = 4 * k;
    if (q4 % K == 0) {
        int quarter = (q4 / K) & 3;
        static const double cq[4] = {1.0, 0.0, -1.0, 0.0};
        static const double sq[4] = {0.0, 1.0, 0.0, -1.0};
        *c = cq[quarter];
        *s = sq[quarter];
        return;
    }
    double th = 2.0 * M_PI * (double)k / (double)K;
    *c = cos(th);
    *s = sin(th);
}

static int orc_disabled(const orc_model *m, int u)
{
    int k = u % m->K, sp = u / m->K;
    return ((k < 64) && ((m->mask_off >> k) & 1u)) || ((m->speed_off >> sp) & 1u);
}

/* Q(z, u; g) = -w1*v*m_s*dt - w2*||z + v*m_s*dt*(cos, sin) - g|| for the
 * control of speed multiplier ms and heading (c, s). */
static double orc_Q(const orc_model *m, double zx, double zy, double c, double s, double ms,
                    double gx, double gy)
{
    double st = m->v * ms * m->dt;
    double dx = zx + st * c - gx, dy = zy + st * s - gy;
    return -m->w1 * m->v * ms * m->dt - m->w2 * sqrt(dx * dx + dy * dy);
}

/* The enabled speed whose multiplier is nearest to len / (v*dt) (lower index
 * on a tie): the speed of an observed displacement of length len. */
static int orc_snap_speed(const orc_model *m, double len)
{
    double r = len / (m->v * m->dt), best = INFINITY;
    int sb = 0;
    for (int sp = 0; sp < m->S; ++sp) {
        if ((m->speed_off >> sp) & 1u) continue;
        double d = fabs(m->mult[sp] - r);
        if (d < best) { best = d; sb = sp; }
    }
    return sb;
}

/* log pi(k | z; beta, g) for every heading k (Eq. 2); disabled headings get
 * -inf. Returns the LogSumExp of beta*Q over the enabled headings. */
double orc_log_policy_raw(const orc_model *m, double zx, double zy, double beta,
                          double gx, double gy, double *logpi)
{
    int U = m->S * m->K;
    double mx = -INFINITY;
    for (int u = 0; u < U; ++u) {
        double c, s;
        orc_heading(m->K, u % m->K, &c, &s);
        logpi[u] = orc_disabled(m, u) ? -INFINITY : beta * orc_Q(m, zx, zy, c, s, m->mult[u / m->K], gx, gy);
        if (logpi[u] > mx) mx = logpi[u];
    }
    double sum = 0.0;
    for (int u = 0; u < U; ++u)
        if (logpi[u] > -INFINITY) sum += exp(logpi[u] - mx);
    double lse = mx + log(sum);
    for (int u = 0; u < U; ++u) logpi[u] = logpi[u] - lse;
    return lse;
}

#define ORC_MODEL_ARGS int K, double v, double dt, double w1, double w2, uint64_t mask_off, \
                       int S, const double *mult, uint32_t speed_off, int snap
#define ORC_MODEL(G_, goals_, B_, beta_) {K, v, dt, w1, w2, G_, B_, goals_, beta_, mask_off, S, mult, speed_off, snap}

/* Flat-argument form of orc_log_policy_raw for the Python wrapper
 * (logpi [S*K], control u = s*K + k). */
void orc_log_policy(ORC_MODEL_ARGS, double zx, double zy, double beta, double gx, double gy, double *logpi)
{
    orc_model m = ORC_MODEL(1, NULL, 1, NULL);
    orc_log_policy_raw(&m, zx, zy, beta, gx, gy, logpi);
}

/* Direction (c, s) of the observed heading th: th itself, or with m->snap
 * the enabled heading nearest to it (largest cos(th - theta_k), the lower
 * index on a tie). */
static void orc_obs_heading(const orc_model *m, double th, double *c, double *s)
{
    if (!m->snap) {
        *c = cos(th);
        *s = sin(th);
        return;
    }
    double best = -INFINITY;
    int kb = 0;
    for (int k = 0; k < m->K; ++k) {
        if ((m->mask_off >> k) & 1u) continue;
        double d = cos(th - 2.0 * M_PI * (double)k / (double)m->K);
        if (d > best) { best = d; kb = k; }
    }
    orc_heading(m->K, kb, c, s);
}

/* log pi(u_obs | z; beta, g) for the observed control recovered from two
 * states (differential flatness): the heading th (continuous, or snapped)
 * and the enabled speed nearest to the displacement length len. */
static double orc_log_policy_obs(const orc_model *m, double zx, double zy, double th, double len,
                                 double beta, double gx, double gy, double *scratch)
{
    double lse = orc_log_policy_raw(m, zx, zy, beta, gx, gy, scratch);
    double ms = m->mult[orc_snap_speed(m, len)];
    double c, s;
    orc_obs_heading(m, th, &c, &s);
    return beta * orc_Q(m, zx, zy, c, s, ms, gx, gy) - lse;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3 / Eq. 7: sequential Bayesian update of the joint belief in log space */
/* ------------------------------------------------------------------------ */
static double orc_lse(const double *x, int n)
{
    double mx = -INFINITY;
    for (int i = 0; i < n; ++i)
        if (x[i] > mx) mx = x[i];
    if (mx == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(x[i] - mx);
    return mx + log(s);
}

/* obs: [n_obs+1][2]; log_b: [G*B] in/out, index j = g*B + b.
 * Returns the number of steps skipped as stationary. */
int orc_update_posterior(ORC_MODEL_ARGS, int G, const double *goals, int B, const double *beta,
                         const double *obs, int n_obs, double *log_b)
{
    orc_model m = ORC_MODEL(G, goals, B, beta);
    int J = G * B, skipped = 0;
    double *scratch = (double *)malloc(sizeof(double) * (size_t)(S * K > 0 ? S * K : 1));
    double *l = (double *)malloc(sizeof(double) * (size_t)J);
    for (int t = 0; t < n_obs; ++t) {
        double zx = obs[2 * t], zy = obs[2 * t + 1];
        double dx = obs[2 * t + 2] - zx, dy = obs[2 * t + 3] - zy;
        double len = sqrt(dx * dx + dy * dy);
        if (len < 1e-6) { ++skipped; continue; }
        double th = atan2(dy, dx);
        for (int j = 0; j < J; ++j) {
            int g = j / B, b = j % B;
            double lp = orc_log_policy_obs(&m, zx, zy, th, len, beta[b], goals[2 * g], goals[2 * g + 1], scratch);
            l[j] = lp + log_b[j];          /* log pi + log b^t              */
        }
        double lse = orc_lse(l, J);          /* log sum_{b',g'} pi * b^t      */
        for (int j = 0; j < J; ++j) log_b[j] = l[j] - lse;
    }
    free(scratch);
    free(l);
    return skipped;
}

/* ------------------------------------------------------------------------ */
/* Inverse CDF: smallest k with u*S < C_k; fallback: last k with e_k > 0.    */
/* ------------------------------------------------------------------------ */
static int orc_inverse_cdf(const double *e, int n, double u)
{
    double S = 0.0;
    for (int k = 0; k < n; ++k) S += e[k];
    double target = u * S, C = 0.0;
    for (int k = 0; k < n; ++k) {
        C += e[k];
        if (target < C) return k;
    }
    for (int k = n - 1; k >= 0; --k)
        if (e[k] > 0.0) return k;
    return 0;
}

/* The sampling rule on its own: weights e[n] (not normalised), uniform u. */
int orc_sample_index(const double *e, int n, double u) { return orc_inverse_cdf(e, n, u); }

/* Draw the (beta, g) index j of particle i from the belief exp(log_b). */
int orc_draw_component(int J, const double *log_b, uint64_t seed, uint32_t human, uint64_t i)
{
    double *e = (double *)malloc(sizeof(double) * (size_t)J);
    for (int j = 0; j < J; ++j) e[j] = exp(log_b[j]);
    int r = orc_inverse_cdf(e, J, orc_uniform_select(seed, human, i));
    free(e);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Binning of an FP32 state (the emplacement step of Algorithm 1).           */
/* Returns 1 and the cell if inside the grid, 0 if outside.                  */
/* ------------------------------------------------------------------------ */
int orc_bin(float x, float y, float x0, float y0, float inv_res, int W, int H, int *cx, int *cy)
{
    volatile float rx = x - x0;      /* FP32 subtraction, rounded */
    volatile float ry = y - y0;
    volatile float vx = rx * inv_res; /* FP32 multiplication, rounded */
    volatile float vy = ry * inv_res;
    float fx = floorf(vx), fy = floorf(vy);
    if (!(fx >= 0.0f && fx < (float)W && fy >= 0.0f && fy < (float)H)) return 0;
    *cx = (int)fx;
    *cy = (int)fy;
    return 1;
}

/* FP32 value 1/res, the binning scale. */
float orc_inv_res(float res)
{
    volatile float one = 1.0f;
    return one / res;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 with the bootstrapped belief, particles [i0, i1).             */
/*   counts [T][H][W] (+=), oob [T] (+=)       may be NULL                    */
/*   headings [i1-i0][T] (uint8 heading index)  may be NULL                   */
/*   states32 [i1-i0][T][2] (FP32 shadow state) may be NULL                   */
/*   states64 [i1-i0][T][2] (FP64 state)        may be NULL                   */
/*   comp [i1-i0] (drawn j)                     may be NULL                   */
/* A shadow FP32 state takes the same FP32 steps (float)(v*dt*cos theta_k)  */
/* and is what is binned. With decide_f32 = 0 the policy (Eq. 2) is          */
/* evaluated at the FP64 particle state; with decide_f32 = 1 at the FP32     */
/* state (the particle state of Algorithm 1 held in the paper's FP32, the    */
/* policy still computed in FP64), so that a draw differs from an FP32       */
/* implementation's only through the arithmetic of that draw.                */
/* ------------------------------------------------------------------------ */
void orc_rollout(ORC_MODEL_ARGS, int G, const double *goals, int B, const double *beta,
                 const double *log_b, float z0x, float z0y, int T,
                 uint64_t seed, uint32_t human, int64_t i0, int64_t i1,
                 float gx0, float gy0, float res, int W, int H,
                 uint32_t *counts, uint32_t *oob, uint8_t *headings,
                 float *states32, double *states64, int32_t *comp, int decide_f32)
{
    orc_model m = ORC_MODEL(G, goals, B, beta);
    int J = G * B, U = S * K;
    /* control u = s*K + k moves (v*mult[s]*dt) * (cos, sin)(theta_k); the FP32
     * shadow state moves by that product rounded once to FP32 */
    double *hc = (double *)malloc(sizeof(double) * (size_t)U);
    double *hs = (double *)malloc(sizeof(double) * (size_t)U);
    float *fx = (float *)malloc(sizeof(float) * (size_t)U);
    float *fy = (float *)malloc(sizeof(float) * (size_t)U);
    double *logpi = (double *)malloc(sizeof(double) * (size_t)U);
    double *e = (double *)malloc(sizeof(double) * (size_t)U);
    for (int u = 0; u < U; ++u) {
        double c, sn, st = v * mult[u / K] * dt;
        orc_heading(K, u % K, &c, &sn);
        hc[u] = st * c;
        hs[u] = st * sn;
        fx[u] = (float)(st * c);
        fy[u] = (float)(st * sn);
    }
    float inv_res = orc_inv_res(res);
    for (int64_t i = i0; i < i1; ++i) {
        int64_t li = i - i0;
        int j = orc_draw_component(J, log_b, seed, human, (uint64_t)i);
        if (comp) comp[li] = j;
        int g = j / B, b = j % B;
        double bt = beta[b], gx = goals[2 * g], gy = goals[2 * g + 1];
        double zx = (double)z0x, zy = (double)z0y;
        float sx = z0x, sy = z0y;
        for (int t = 1; t <= T; ++t) {
            if (decide_f32) orc_log_policy_raw(&m, (double)sx, (double)sy, bt, gx, gy, logpi);
            else orc_log_policy_raw(&m, zx, zy, bt, gx, gy, logpi);
            for (int u = 0; u < U; ++u) e[u] = exp(logpi[u]);
            int k = orc_inverse_cdf(e, U, orc_uniform_step(seed, human, (uint64_t)i, t));
            zx += hc[k];
            zy += hs[k];
            volatile float nx = sx + fx[k];
            volatile float ny = sy + fy[k];
            sx = nx;
            sy = ny;
            if (headings) headings[li * T + (t - 1)] = (uint8_t)k;
            if (states32) { states32[(li * T + (t - 1)) * 2] = sx; states32[(li * T + (t - 1)) * 2 + 1] = sy; }
            if (states64) { states64[(li * T + (t - 1)) * 2] = zx; states64[(li * T + (t - 1)) * 2 + 1] = zy; }
            if (counts || oob) {
                int cx, cy;
                if (orc_bin(sx, sy, gx0, gy0, inv_res, W, H, &cx, &cy)) {
                    if (counts) counts[((size_t)(t - 1) * (size_t)H + (size_t)cy) * (size_t)W + (size_t)cx] += 1u;
                } else if (oob) {
                    oob[t - 1] += 1u;
                }
            }
        }
    }
    free(hc); free(hs); free(fx); free(fy); free(logpi); free(e);
}

/* Histogram of given FP32 states [n][T][2] with the FP32 binning rule. */
void orc_bin_states(const float *states, int64_t n, int T, float x0, float y0, float res,
                    int W, int H, uint32_t *counts, uint32_t *oob)
{
    float inv_res = orc_inv_res(res);
    for (int64_t i = 0; i < n; ++i)
        for (int t = 0; t < T; ++t) {
            int cx, cy;
            const float *p = states + (i * T + t) * 2;
            if (orc_bin(p[0], p[1], x0, y0, inv_res, W, H, &cx, &cy))
                counts[((size_t)t * (size_t)H + (size_t)cy) * (size_t)W + (size_t)cx] += 1u;
            else
                oob[t] += 1u;
        }
}

/* ------------------------------------------------------------------------ */
/* Eq. 4 / Eq. 5: exact propagation of the occupancy distribution.           */
/* For even K (K/2 <= 4) a reachable position is the integer vector          */
/* m_i = n_i - n_{i+K/2} (i < K/2) of net moves along the first K/2 headings; */
/* position z0 + v*dt * sum_i m_i e_i. Each (beta, g) component is propagated */
/* separately with pi evaluated at the exact position, then mixed with b.     */
/* Output p[T][H][W] and p_oob[T] (FP64, binned from the FP64 position);      */
/* edge_mass[T]: mass of states within edge_tol of a cell edge.               */
/* Returns 0 on success, -1 if K is unsupported or memory is short.          */
/* ------------------------------------------------------------------------ */
int orc_exact_occupancy(ORC_MODEL_ARGS, int G, const double *goals, int B, const double *beta,
                        const double *log_b, double z0x, double z0y, int T,
                        double x0, double y0, double res, int W, int H, double edge_tol,
                        double *p, double *p_oob, double *edge_mass)
{
    if (K % 2 != 0 || K < 2 || K > 8 || S != 1 || mult[0] != 1.0) return -1; /* one speed: a lattice */
    orc_model m = ORC_MODEL(G, goals, B, beta);
    int D = K / 2, side = 2 * T + 1;
    size_t nstate = 1;
    for (int d = 0; d < D; ++d) nstate *= (size_t)side;
    double *cur = (double *)calloc(nstate, sizeof(double));
    double *nxt = (double *)calloc(nstate, sizeof(double));
    int64_t *act = (int64_t *)malloc(sizeof(int64_t) * nstate);
    int64_t *act2 = (int64_t *)malloc(sizeof(int64_t) * nstate);
    double *logpi = (double *)malloc(sizeof(double) * (size_t)K);
    double *hc = (double *)malloc(sizeof(double) * (size_t)K);
    double *hs = (double *)malloc(sizeof(double) * (size_t)K);
    if (!cur || !nxt || !act || !act2 || !logpi || !hc || !hs) {
        free(cur); free(nxt); free(act); free(act2); free(logpi); free(hc); free(hs);
        return -1;
    }
    for (int k = 0; k < K; ++k) orc_heading(K, k, &hc[k], &hs[k]);
    double st = v * dt;
    size_t plane = (size_t)H * (size_t)W;
    memset(p, 0, sizeof(double) * plane * (size_t)T);
    memset(p_oob, 0, sizeof(double) * (size_t)T);
    memset(edge_mass, 0, sizeof(double) * (size_t)T);
    int64_t stride[4] = {1, 1, 1, 1};
    for (int d = 1; d < D; ++d) stride[d] = stride[d - 1] * side;
    int64_t origin = 0;
    for (int d = 0; d < D; ++d) origin += (int64_t)T * stride[d];
    int J = G * B;
    for (int j = 0; j < J; ++j) {
        double wj = exp(log_b[j]);
        if (wj == 0.0) continue;
        int g = j / B, b = j % B;
        double bt = beta[b], gx = goals[2 * g], gy = goals[2 * g + 1];
        memset(cur, 0, sizeof(double) * nstate);
        cur[origin] = 1.0;
        int64_t nact = 1;
        act[0] = origin;
        for (int t = 1; t <= T; ++t) {
            int64_t nact2 = 0;
            for (int64_t a = 0; a < nact; ++a) {
                int64_t idx = act[a];
                double pr = cur[idx];
                if (pr == 0.0) continue;
                /* decode the integer move vector and the exact position */
                int64_t rem = idx;
                double zx = z0x, zy = z0y;
                int mv[4] = {0, 0, 0, 0};
                for (int d = 0; d < D; ++d) {
                    mv[d] = (int)(rem % side) - T;
                    rem /= side;
                }
                for (int d = 0; d < D; ++d) {
                    zx += st * (double)mv[d] * hc[d];
                    zy += st * (double)mv[d] * hs[d];
                }
                orc_log_policy_raw(&m, zx, zy, bt, gx, gy, logpi);
                for (int k = 0; k < K; ++k) {
                    if (logpi[k] == -INFINITY) continue;
                    double q = pr * exp(logpi[k]);
                    if (q == 0.0) continue;
                    int64_t to = (k < D) ? idx + stride[k] : idx - stride[k - D];
                    if (nxt[to] == 0.0) act2[nact2++] = to;
                    nxt[to] += q;
                }
                cur[idx] = 0.0;
            }
            /* bin the FP64 positions of step t */
            for (int64_t a = 0; a < nact2; ++a) {
                int64_t idx = act2[a];
                double pr = nxt[idx] * wj;
                int64_t rem = idx;
                double zx = z0x, zy = z0y;
                for (int d = 0; d < D; ++d) {
                    int mvd = (int)(rem % side) - T;
                    rem /= side;
                    zx += st * (double)mvd * hc[d];
                    zy += st * (double)mvd * hs[d];
                }
                double ux = (zx - x0) / res, uy = (zy - y0) / res;
                double fx = floor(ux), fy = floor(uy);
                double ex = fmin(ux - fx, fx + 1.0 - ux) * res;
                double ey = fmin(uy - fy, fy + 1.0 - uy) * res;
                if (ex < edge_tol || ey < edge_tol) edge_mass[t - 1] += pr;
                if (fx >= 0.0 && fx < (double)W && fy >= 0.0 && fy < (double)H)
                    p[(size_t)(t - 1) * plane + (size_t)fy * (size_t)W + (size_t)fx] += pr;
                else
                    p_oob[t - 1] += pr;
            }
            double *tmp = cur; cur = nxt; nxt = tmp;
            int64_t *ta = act; act = act2; act2 = ta;
            nact = nact2;
        }
    }
    free(cur); free(nxt); free(act); free(act2); free(logpi); free(hc); free(hs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Marginal log-likelihood of M observed trajectories and its gradient.      */
/*   L = sum_m log sum_j exp(log_prior_j + sum_t log pi_j(theta_{m,t}|z_{m,t}))*/
/*   dL/dp = sum_m sum_j w_{m,j} sum_t d log pi_j / dp,                        */
/*   d log pi / dp = beta * (dQ(theta_obs)/dp - sum_k pi_k dQ(theta_k)/dp),    */
/*   w_{m,j} the posterior of j given trajectory m.                            */
/* offsets [M+1] index points of traj [*][2]; trajectory m has points          */
/* offsets[m] .. offsets[m+1]-1 (steps = points - 1).                          */
/* Outputs: *L, d_goals [G][2], d_v, d_w [2]. Any output pointer may be NULL. */
/* A distance below 1e-9 gives the subgradient 0 for the distance term.       */
/* ------------------------------------------------------------------------ */
typedef struct { double q, dgx, dgy, dv, dw1, dw2; } orc_qgrad;

static orc_qgrad orc_Q_and_grad(const orc_model *m, double zx, double zy, double c, double s, double ms,
                                double gx, double gy)
{
    orc_qgrad r;
    double st = m->v * ms * m->dt;
    double dx = zx + st * c - gx, dy = zy + st * s - gy;
    double dist = sqrt(dx * dx + dy * dy);
    double ux = 0.0, uy = 0.0;
    if (dist >= 1e-9) { ux = dx / dist; uy = dy / dist; }
    r.q = -m->w1 * m->v * ms * m->dt - m->w2 * dist;
    r.dgx = m->w2 * ux;                 /* dQ/dg = w2 (z' - g)/||z' - g|| */
    r.dgy = m->w2 * uy;
    r.dv = -m->w1 * ms * m->dt - m->w2 * ms * m->dt * (c * ux + s * uy);
    r.dw1 = -m->v * ms * m->dt;
    r.dw2 = -dist;
    return r;
}

int orc_loglik_grad(ORC_MODEL_ARGS, int G, const double *goals, int B, const double *beta,
                    int M, const int32_t *offsets, const double *traj, const double *log_prior,
                    double *L_out, double *d_goals, double *d_v, double *d_w)
{
    if (G > 64 || K < 1 || S < 1) return -1;
    orc_model m = ORC_MODEL(G, goals, B, beta);
    int J = G * B, U = S * K;
    double *A = (double *)malloc(sizeof(double) * (size_t)J);
    double *gr = (double *)malloc(sizeof(double) * (size_t)J * 5); /* dgx dgy dv dw1 dw2 */
    orc_qgrad *qk = (orc_qgrad *)malloc(sizeof(orc_qgrad) * (size_t)U);
    double *hc = (double *)malloc(sizeof(double) * (size_t)K);
    double *hs = (double *)malloc(sizeof(double) * (size_t)K);
    double *pk = (double *)malloc(sizeof(double) * (size_t)U);
    for (int k = 0; k < K; ++k) orc_heading(K, k, &hc[k], &hs[k]);
    double Lsum = 0.0;
    double acc_g[2 * 64 + 8];
    double acc_v = 0.0, acc_w1 = 0.0, acc_w2 = 0.0;
    memset(acc_g, 0, sizeof(acc_g));
    for (int mm = 0; mm < M; ++mm) {
        for (int j = 0; j < J; ++j) {
            A[j] = log_prior[j];
            for (int q = 0; q < 5; ++q) gr[j * 5 + q] = 0.0;
        }
        for (int pt = offsets[mm]; pt + 1 < offsets[mm + 1]; ++pt) {
            double zx = traj[2 * pt], zy = traj[2 * pt + 1];
            double dx = traj[2 * pt + 2] - zx, dy = traj[2 * pt + 3] - zy;
            double len = sqrt(dx * dx + dy * dy);
            if (len < 1e-6) continue;
            double co, so;
            orc_obs_heading(&m, atan2(dy, dx), &co, &so);
            double mo = mult[orc_snap_speed(&m, len)]; /* the observed control's speed */
            for (int j = 0; j < J; ++j) {
                int g = j / B, b = j % B;
                double bt = beta[b], gx = goals[2 * g], gy = goals[2 * g + 1];
                double mx = -INFINITY;
                for (int k = 0; k < U; ++k) {
                    qk[k] = orc_Q_and_grad(&m, zx, zy, hc[k % K], hs[k % K], mult[k / K], gx, gy);
                    pk[k] = orc_disabled(&m, k) ? -INFINITY : bt * qk[k].q;
                    if (pk[k] > mx) mx = pk[k];
                }
                double Ssum = 0.0;
                for (int k = 0; k < U; ++k) { pk[k] = (pk[k] == -INFINITY) ? 0.0 : exp(pk[k] - mx); Ssum += pk[k]; }
                double lse = mx + log(Ssum);
                orc_qgrad qo = orc_Q_and_grad(&m, zx, zy, co, so, mo, gx, gy);
                A[j] += bt * qo.q - lse;
                double e_gx = 0, e_gy = 0, e_v = 0, e_w1 = 0, e_w2 = 0;
                for (int k = 0; k < U; ++k) {
                    double pi = pk[k] / Ssum;
                    e_gx += pi * qk[k].dgx; e_gy += pi * qk[k].dgy; e_v += pi * qk[k].dv;
                    e_w1 += pi * qk[k].dw1; e_w2 += pi * qk[k].dw2;
                }
                gr[j * 5 + 0] += bt * (qo.dgx - e_gx);
                gr[j * 5 + 1] += bt * (qo.dgy - e_gy);
                gr[j * 5 + 2] += bt * (qo.dv - e_v);
                gr[j * 5 + 3] += bt * (qo.dw1 - e_w1);
                gr[j * 5 + 4] += bt * (qo.dw2 - e_w2);
            }
        }
        double lse = orc_lse(A, J);
        Lsum += lse;
        for (int j = 0; j < J; ++j) {
            double w = exp(A[j] - lse);
            int g = j / B;
            acc_g[2 * g] += w * gr[j * 5 + 0];
            acc_g[2 * g + 1] += w * gr[j * 5 + 1];
            acc_v += w * gr[j * 5 + 2];
            acc_w1 += w * gr[j * 5 + 3];
            acc_w2 += w * gr[j * 5 + 4];
        }
    }
    if (L_out) *L_out = Lsum;
    if (d_goals) for (int g = 0; g < G; ++g) { d_goals[2 * g] = acc_g[2 * g]; d_goals[2 * g + 1] = acc_g[2 * g + 1]; }
    if (d_v) *d_v = acc_v;
    if (d_w) { d_w[0] = acc_w1; d_w[1] = acc_w2; }
    free(A); free(gr); free(qk); free(hc); free(hs); free(pk);
    return 0;
}
