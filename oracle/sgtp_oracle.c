/*
 * sgtp_oracle.c -- plain, slow, FP64 CPU oracle of the SGTP best-response
 * hot path.  TEST INFRASTRUCTURE ONLY: the product library never links,
 * loads or calls this file; only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark do.
 *
 * It shares no code, header, table or constant generator with the CUDA path.
 * Every function states the passage of the SGTP paper (Li et al.,
 * "SGTP: Sampling-based Game-Theoretic Planning for Real-Time Multi-Vehicle
 * Autonomous Racing") that it follows.  Where the paper is silent the reading
 * taken is written next to the code.
 *
 * Everything is computed in double precision.  Inputs arrive as double arrays
 * holding exactly the float32 values the GPU receives.  The per-sample loop
 * over k may run on several POSIX threads; each k is computed by one thread
 * from start to end, so threading never changes a result.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Parameters (Sec. IV-B lists the paper's values; names follow it).   */
/* ------------------------------------------------------------------ */
typedef struct {
    double dt, wheelbase;
    double a_min, a_max, delta_max, v_min, v_max;
    double sigma_a, sigma_delta;
    double Q[4], R[2], S[2];
    double w_game, w_contest, w_long, w_block, w_safety;
    double s_contest, s_role, mu_tail, g_safe, eps_alpha, m_bd, d_col;
} orc_params;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11).  Written from the published round        */
/* function: two 32x32->64 multiplies per round, a Weyl key schedule.    */
/* ------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n[4];
    n[0] = hi1 ^ c[1] ^ k[0];
    n[1] = lo1;
    n[2] = hi0 ^ c[3] ^ k[1];
    n[3] = lo0;
    memcpy(c, n, sizeof n);
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* Counter layout of the noise of sample k at step tau (part of the ABI so
 * that any sample can be reproduced): one Philox call serves the two steps
 * 2m and 2m+1; words (0,1) feed the even step, (2,3) the odd one.
 *   key = (seed low 32 bits, seed high 32 bits)
 *   ctr = (k, (tau >> 1) | stream << 31, agent | round << 16, race)       */
static void noise_words(uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                        uint32_t stream, uint32_t k, int tau, uint32_t *w0, uint32_t *w1)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {k, ((uint32_t)tau >> 1) | (stream << 31), agent | (round << 16), race};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    if ((tau & 1) == 0) { *w0 = o[0]; *w1 = o[1]; }
    else                { *w0 = o[2]; *w1 = o[3]; }
}

/* Uniform in (0,1): the top 23 bits of a word plus one half, times 2^-23.
 * Every value is exact in float32 and float64, so both sides see the same u. */
static double uniform_open(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box-Muller transform: two independent N(0,1) draws (Sec. II: the
 * perturbation eps ~ N(0, diag(sigma_a^2, sigma_delta^2)) of each k, tau). */
void orc_std_normals(uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                     uint32_t stream, uint32_t k, int tau, double *z_a, double *z_d)
{
    uint32_t w0, w1;
    noise_words(seed, race, agent, round, stream, k, tau, &w0, &w1);
    const double u1 = uniform_open(w0), u2 = uniform_open(w1);
    const double r = sqrt(-2.0 * log(u1));
    *z_a = r * cos(2.0 * M_PI * u2);
    *z_d = r * sin(2.0 * M_PI * u2);
}

/* ------------------------------------------------------------------ */
/* Raceline G (Sec. II, Preliminaries): waypoints (x, y, psi, v^r) with  */
/* left/right widths, arc-length parameterised, closed loop.             */
/* ------------------------------------------------------------------ */
typedef struct {
    int N;
    const double *xr;   /* N x 4: x, y, psi, v^r */
    const double *wl, *wr;
    double *s;          /* N+1 cumulative arc length, s[N] = L */
    double L;
} orc_track;

static int track_init(orc_track *t, const double *xr, const double *wl, const double *wr, int N)
{
    t->N = N; t->xr = xr; t->wl = wl; t->wr = wr;
    t->s = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    if (!t->s) return -1;
    t->s[0] = 0.0;
    for (int j = 0; j < N; ++j) {
        const int jn = (j + 1) % N;
        const double dx = xr[4 * jn] - xr[4 * j], dy = xr[4 * jn + 1] - xr[4 * j + 1];
        t->s[j + 1] = t->s[j] + sqrt(dx * dx + dy * dy);
    }
    t->L = t->s[N];
    return 0;
}
static void track_free(orc_track *t) { free(t->s); t->s = NULL; }

/* Wrap a progress difference into (-L/2, L/2] (closed-track reading). */
static double wrap_len(double x, double L) { return x - L * ceil(x / L - 0.5); }
/* Wrap an angle into (-pi, pi]. */
static double wrap_pi(double a) { return a - 2.0 * M_PI * ceil(a / (2.0 * M_PI) - 0.5); }

/* Frenet projection s(x; G), d(x; G) (Sec. II): the globally nearest point of
 * the closed polyline, by brute force over every segment; equidistant
 * segments resolve to the lowest index.  d > 0 left of the travel direction. */
void orc_frenet_raw(const orc_track *t, double px, double py, double *s_out, double *d_out, int *seg_out)
{
    double best = INFINITY, bs = 0.0, bd = 0.0;
    int bj = 0;
    for (int j = 0; j < t->N; ++j) {
        const int jn = (j + 1) % t->N;
        const double ax = t->xr[4 * j], ay = t->xr[4 * j + 1];
        const double ex = t->xr[4 * jn] - ax, ey = t->xr[4 * jn + 1] - ay;
        const double len2 = ex * ex + ey * ey;
        double u = ((px - ax) * ex + (py - ay) * ey) / len2;
        if (u < 0.0) u = 0.0;
        if (u > 1.0) u = 1.0;
        const double cx = ax + u * ex, cy = ay + u * ey;
        const double dist = sqrt((px - cx) * (px - cx) + (py - cy) * (py - cy));
        if (dist < best) {
            best = dist;
            bj = j;
            bs = t->s[j] + u * (t->s[j + 1] - t->s[j]);
            const double cr = ex * (py - ay) - ey * (px - ax);
            bd = (cr >= 0.0) ? dist : -dist;
        }
    }
    *s_out = bs; *d_out = bd;
    if (seg_out) *seg_out = bj;
}

/* Continuous reference maps x^r(s), w^L(s), w^R(s) (Sec. II): linear in s
 * between waypoints; heading along the shorter arc.  s is taken modulo L. */
static void track_at(const orc_track *t, double s, double xr_out[4], double *wl, double *wr)
{
    double sm = fmod(s, t->L);
    if (sm < 0.0) sm += t->L;
    int j = 0;
    while (j + 1 < t->N && t->s[j + 1] <= sm) ++j;     /* segment with s_j <= sm < s_{j+1} */
    const int jn = (j + 1) % t->N;
    const double u = (sm - t->s[j]) / (t->s[j + 1] - t->s[j]);
    const double *a = t->xr + 4 * j, *b = t->xr + 4 * jn;
    if (xr_out) {
        xr_out[0] = a[0] + u * (b[0] - a[0]);
        xr_out[1] = a[1] + u * (b[1] - a[1]);
        xr_out[2] = a[2] + u * wrap_pi(b[2] - a[2]);
        xr_out[3] = a[3] + u * (b[3] - a[3]);
    }
    if (wl) *wl = t->wl[j] + u * (t->wl[jn] - t->wl[j]);
    if (wr) *wr = t->wr[j] + u * (t->wr[jn] - t->wr[j]);
}

/* Kinematic bicycle model f (Sec. II, the model of the cited reference,
 * read as: rear-axle reference point, steering angle as input, explicit
 * forward Euler with step dt, speed clamped to [v_min, v_max]). */
static void bicycle_step(const orc_params *p, const double x[4], double a, double delta, double xn[4])
{
    xn[0] = x[0] + p->dt * x[3] * cos(x[2]);
    xn[1] = x[1] + p->dt * x[3] * sin(x[2]);
    xn[2] = x[2] + p->dt * x[3] * tan(delta) / p->wheelbase;
    double v = x[3] + p->dt * a;
    if (v < p->v_min) v = p->v_min;
    if (v > p->v_max) v = p->v_max;
    xn[3] = v;
}

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Size of the tail index set T_tail (Sec. III-A, blocking term): the final
 * mu_tail share of the horizon, at least one step.  mu*H is rounded up after
 * subtracting 1e-4 so that the float32 rounding of mu (0.3f > 0.3) does not
 * add a step. */
int orc_tail_count(double mu_tail, int H)
{
    int n = (int)ceil(mu_tail * (double)H - 1e-4);
    if (n < 1) n = 1;
    if (n > H) n = H;
    return n;
}

/* Trajectory summary of a fixed opponent prediction xi_hat_j (Sec. III-A):
 * unwrapped progress at t and t+H and the tail-mean lateral offset. */
typedef struct { double s0, sH, dbar; } orc_opp_summary;

/* Unwrapped Frenet progress/offset along a state trajectory (T+1 states). */
static void frenet_traj(const orc_track *t, const double *states, int T, double *s_unw, double *d)
{
    double s_prev = 0.0;
    for (int tau = 0; tau <= T; ++tau) {
        double sr, dr;
        orc_frenet_raw(t, states[4 * tau], states[4 * tau + 1], &sr, &dr, NULL);
        if (tau == 0) s_prev = sr;
        else s_prev = s_prev + wrap_len(sr - s_prev, t->L);
        s_unw[tau] = s_prev;
        d[tau] = dr;
    }
}

static void opp_summaries(const orc_track *t, const double *opp, int n_opp, int T, int n_tail,
                          orc_opp_summary *out)
{
    double *s = (double *)malloc(sizeof(double) * (size_t)(T + 1));
    double *d = (double *)malloc(sizeof(double) * (size_t)(T + 1));
    for (int j = 0; j < n_opp; ++j) {
        frenet_traj(t, opp + (size_t)j * (T + 1) * 4, T, s, d);
        double acc = 0.0;
        for (int tau = T - n_tail + 1; tau <= T; ++tau) acc += d[tau];
        out[j].s0 = s[0];
        out[j].sH = s[T];
        out[j].dbar = acc / (double)n_tail;
    }
    free(s); free(d);
}

/* ------------------------------------------------------------------ */
/* One best-response problem (Alg. 1, the body of the vehicle loop).    */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_params *p;
    orc_track trk;
    const double *x0;        /* 4 */
    const double *u_nom;     /* T x 2 */
    double vref_scale;
    const double *opp;       /* n_opp x (T+1) x 4 */
    const double *opp_pos;   /* states whose positions enter the distance terms (NULL: opp) */
    int n_opp, T;
    uint64_t seed;
    uint32_t race, agent, round, stream;
    int game_on, zero_noise;
    /* optional per-step proposal (T x 4: mean a, mean delta, sigma a,
       sigma delta) for the first K_prop samples */
    const double *prop;
    int K_prop;
    /* per-problem data */
    double *xref;            /* (T+1) x 4 reference states, index 0 unused */
    orc_opp_summary *opp_sum;
    double s_t, d_t;         /* Frenet of x0 */
    int n_tail;
} orc_problem;

typedef struct {
    double cost, viol;
    int feasible;
    double c_track, c_game;
    /* distances of the indicator arguments to their thresholds (used by the
       parity tests to recognise near-threshold candidates) */
    double m_bd, m_obs, m_game;
} orc_sample_result;

static int problem_init(orc_problem *P)
{
    const int T = P->T;
    P->xref = (double *)calloc((size_t)(T + 1) * 4, sizeof(double));
    P->opp_sum = (orc_opp_summary *)calloc((size_t)(P->n_opp > 0 ? P->n_opp : 1), sizeof(orc_opp_summary));
    if (!P->xref || !P->opp_sum) return -1;
    P->n_tail = orc_tail_count(P->p->mu_tail, T);
    orc_frenet_raw(&P->trk, P->x0[0], P->x0[1], &P->s_t, &P->d_t, NULL);
    /* Reference progress recursion (Sec. III-A, overall ranking):
     * s^r_0 = s_{i,t}, s^r_{tau+1} = s^r_tau + dt * v^r(s^r_tau); the agent's
     * reference speed profile is v^r scaled by vref_scale (Sec. IV-B scales
     * the opponents' by 0.9). */
    double sr = P->s_t;
    for (int tau = 0; tau < T; ++tau) {
        double xr[4];
        track_at(&P->trk, sr, xr, NULL, NULL);
        sr = sr + P->p->dt * (P->vref_scale * xr[3]);
        track_at(&P->trk, sr, P->xref + 4 * (tau + 1), NULL, NULL);
        P->xref[4 * (tau + 1) + 3] *= P->vref_scale;
    }
    if (P->n_opp > 0) opp_summaries(&P->trk, P->opp, P->n_opp, T, P->n_tail, P->opp_sum);
    return 0;
}
static void problem_free(orc_problem *P) { free(P->xref); free(P->opp_sum); }

/* Sampled controls of candidate k (Sec. II, Algorithm Formulation):
 * u = Pi_U(u_nom + eps), Pi_U clipping a to [a_min,a_max], delta to
 * [-delta_max, delta_max].  With a proposal (not in the paper), candidates
 * k < K_prop draw u = Pi_U(mean_tau + sigma_tau z) instead, their noise
 * taken from counter stream 1 so that it never repeats a plain sample's. */
static void sample_controls(const orc_problem *P, uint32_t k, double *u)
{
    const orc_params *p = P->p;
    const int from_prop = P->prop != NULL && k < (uint32_t)P->K_prop;
    for (int tau = 0; tau < P->T; ++tau) {
        double za = 0.0, zd = 0.0;
        if (!P->zero_noise)
            orc_std_normals(P->seed, P->race, P->agent, P->round, from_prop ? 1u : P->stream, k, tau, &za, &zd);
        double ma = P->u_nom[2 * tau], md = P->u_nom[2 * tau + 1], sa = p->sigma_a, sd = p->sigma_delta;
        if (from_prop) {
            const double *q = P->prop + 4 * tau;
            ma = q[0]; md = q[1]; sa = q[2]; sd = q[3];
        }
        u[2 * tau] = clampd(ma + sa * za, p->a_min, p->a_max);
        u[2 * tau + 1] = clampd(md + sd * zd, -p->delta_max, p->delta_max);
    }
}

/* Roll out, score and check one candidate whose controls u (T x 2) are given.
 * states (T+1)x4 and frenet (T+1)x2 are written when non-NULL. */
static orc_sample_result eval_candidate(const orc_problem *P, const double *u, double *states, double *frenet)
{
    const orc_params *p = P->p;
    const int T = P->T;
    double x[4] = {P->x0[0], P->x0[1], P->x0[2], P->x0[3]};
    if (states) memcpy(states, x, sizeof x);
    if (frenet) { frenet[0] = P->s_t; frenet[1] = P->d_t; }

    double c_state = 0.0, c_ctrl = 0.0, c_smooth = 0.0;
    double rho_bd = INFINITY;
    double s_prev = P->s_t, d_tail = 0.0;
    double gmin2[16];
    for (int j = 0; j < P->n_opp; ++j) gmin2[j] = INFINITY;

    for (int tau = 0; tau < T; ++tau) {
        const double a = u[2 * tau], dl = u[2 * tau + 1];
        /* control cost ||u_tau||_R^2, tau = 0..H-1 (Eq. ctrack) */
        c_ctrl += p->R[0] * a * a + p->R[1] * dl * dl;
        /* smoothness ||u_tau - u_{tau-1}||_S^2, tau = 1..H-1 (Eq. ctrack) */
        if (tau >= 1) {
            const double da = a - u[2 * (tau - 1)], dd = dl - u[2 * (tau - 1) + 1];
            c_smooth += p->S[0] * da * da + p->S[1] * dd * dd;
        }
        double xn[4];
        bicycle_step(p, x, a, dl, xn);
        memcpy(x, xn, sizeof x);
        const int st = tau + 1;
        if (states) memcpy(states + 4 * st, x, sizeof x);

        /* Frenet of the new state, unwrapped along the rollout */
        double sr, dr;
        orc_frenet_raw(&P->trk, x[0], x[1], &sr, &dr, NULL);
        s_prev = s_prev + wrap_len(sr - s_prev, P->trk.L);
        if (frenet) { frenet[2 * st] = s_prev; frenet[2 * st + 1] = dr; }

        /* tracking term ||x - x^r||_Q^2, tau = 1..H (Eq. ctrack) */
        const double *xr = P->xref + 4 * st;
        const double ex = x[0] - xr[0], ey = x[1] - xr[1];
        const double ep = wrap_pi(x[2] - xr[2]), ev = x[3] - xr[3];
        c_state += p->Q[0] * ex * ex + p->Q[1] * ey * ey + p->Q[2] * ep * ep + p->Q[3] * ev * ev;

        /* track-boundary clearance (Sec. III-B, Eq. selection-boundary) */
        double wl, wr;
        track_at(&P->trk, sr, NULL, &wl, &wr);
        const double rb = fmin(wr + dr, wl - dr);
        if (rb < rho_bd) rho_bd = rb;

        /* tail lateral offsets for the blocking term */
        if (st >= T - P->n_tail + 1) d_tail += dr;

        /* time-aligned distances to each opponent (Eq. Dmin) */
        for (int j = 0; j < P->n_opp; ++j) {
            const double *q = (P->opp_pos ? P->opp_pos : P->opp) + ((size_t)j * (T + 1) + st) * 4;
            const double dx = x[0] - q[0], dy = x[1] - q[1];
            const double g2 = dx * dx + dy * dy;
            if (g2 < gmin2[j]) gmin2[j] = g2;
        }
    }

    orc_sample_result r;
    r.c_track = c_state + c_ctrl + c_smooth;

    /* game-aware cost, summed over opponents (Eq. game_cost) */
    double c_game = 0.0, rho_obs = INFINITY, m_game = INFINITY;
    const double dbar_i = d_tail / (double)P->n_tail;
    for (int j = 0; j < P->n_opp; ++j) {
        const orc_opp_summary *o = &P->opp_sum[j];
        const double ds_t = wrap_len(P->s_t - o->s0, P->trk.L);
        const double ds_H = ds_t + (s_prev - P->s_t) - (o->sH - o->s0);
        /* contest-state term (Eq. c_contest) */
        const double c_contest = -p->w_contest * ((fabs(ds_H) < p->s_contest) ? 1.0 : 0.0);
        m_game = fmin(m_game, fabs(fabs(ds_H) - p->s_contest));
        m_game = fmin(m_game, fmin(fabs(ds_t - p->s_role), fabs(ds_t - p->s_contest)));
        /* longitudinal advantage (Eq. c_long) with adaptive alpha */
        const double alpha = 1.0 / (1.0 + fabs(ds_t) / (p->s_contest + p->eps_alpha));
        const double c_long = -p->w_long * alpha * ds_H;
        /* blocking alignment (Eq. c_block), gate gamma on the current gap */
        const double gamma = p->w_block * ((ds_t > p->s_role) ? 1.0 : 0.0) * ((ds_t < p->s_contest) ? 1.0 : 0.0);
        const double c_block = -gamma / (1.0 + fabs(dbar_i - o->dbar));
        /* safety separation (Eqs. Dmin, c_safety) */
        const double gmin = sqrt(gmin2[j]);
        const double sh = fmax(0.0, p->g_safe - gmin);
        const double c_safety = p->w_safety * sh * sh;
        c_game += c_contest + c_long + c_block + c_safety;
        if (gmin < rho_obs) rho_obs = gmin;
    }
    r.c_game = c_game;
    /* total cost (Eq. allc); the initial round runs without the game term */
    r.cost = r.c_track + (P->game_on ? p->w_game * c_game : 0.0);
    if (isnan(r.cost)) r.cost = INFINITY;
    /* feasibility h = b * o (Eqs. selection-boundary, selection-vehicle) */
    const int b = rho_bd >= p->m_bd;
    const int ob = rho_obs >= p->d_col;     /* no opponents: rho_obs = +inf */
    r.feasible = b && ob;
    /* least-violation measure (Sec. III-B, fallback) */
    r.viol = fmax(0.0, p->m_bd - rho_bd) + fmax(0.0, p->d_col - rho_obs);
    if (isnan(r.viol)) r.viol = INFINITY;
    r.m_bd = fabs(rho_bd - p->m_bd);
    r.m_obs = P->n_opp > 0 ? fabs(rho_obs - p->d_col) : INFINITY;
    r.m_game = m_game;
    return r;
}

/* ------------------------------------------------------------------ */
/* Threaded loop over candidates                                        */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_problem *P;
    const int32_t *k_list;
    int n, begin, end;
    double *cost, *viol, *states, *frenet, *controls, *c_track, *c_game, *margins;
    unsigned char *feas;
} orc_job;

static void *job_run(void *arg)
{
    orc_job *J = (orc_job *)arg;
    const int T = J->P->T;
    double *u = (double *)malloc(sizeof(double) * (size_t)T * 2);
    for (int i = J->begin; i < J->end; ++i) {
        const uint32_t k = J->k_list ? (uint32_t)J->k_list[i] : (uint32_t)i;
        sample_controls(J->P, k, u);
        orc_sample_result r = eval_candidate(J->P, u,
                                             J->states ? J->states + (size_t)i * (T + 1) * 4 : NULL,
                                             J->frenet ? J->frenet + (size_t)i * (T + 1) * 2 : NULL);
        J->cost[i] = r.cost;
        J->viol[i] = r.viol;
        J->feas[i] = (unsigned char)r.feasible;
        if (J->c_track) J->c_track[i] = r.c_track;
        if (J->c_game) J->c_game[i] = r.c_game;
        if (J->margins) { J->margins[3 * i] = r.m_bd; J->margins[3 * i + 1] = r.m_obs; J->margins[3 * i + 2] = r.m_game; }
        if (J->controls) memcpy(J->controls + (size_t)i * T * 2, u, sizeof(double) * (size_t)T * 2);
    }
    free(u);
    return NULL;
}

static void run_jobs(const orc_problem *P, const int32_t *k_list, int n, int nthreads, double *cost, unsigned char *feas,
                     double *viol, double *states, double *frenet, double *controls, double *c_track, double *c_game,
                     double *margins)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    orc_job *jobs = (orc_job *)calloc((size_t)nthreads, sizeof(orc_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        orc_job *J = &jobs[t];
        J->P = P; J->k_list = k_list; J->n = n;
        J->begin = (int)((int64_t)n * t / nthreads);
        J->end = (int)((int64_t)n * (t + 1) / nthreads);
        J->cost = cost; J->viol = viol; J->feas = feas; J->states = states; J->frenet = frenet;
        J->controls = controls; J->c_track = c_track; J->c_game = c_game; J->margins = margins;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, job_run, &jobs[t]);
    job_run(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th);
}

/* Selection (Eq. selection and the least-violation fallback, Sec. III-B):
 * lowest cost among feasible candidates; if none is feasible, lowest total
 * violation.  Ties go to the lowest index; NaN ranks as +inf. */
int orc_select(const double *cost, const unsigned char *feas, const double *viol, int n, int *any_feasible)
{
    int best = -1, anyf = 0;
    for (int i = 0; i < n; ++i) if (feas[i]) { anyf = 1; break; }
    double bv = INFINITY;
    for (int i = 0; i < n; ++i) {
        double v;
        if (anyf) { if (!feas[i]) continue; v = cost[i]; }
        else v = viol[i];
        if (isnan(v)) v = INFINITY;
        if (best < 0 || v < bv) { best = i; bv = v; }
    }
    if (any_feasible) *any_feasible = anyf;
    return best;
}

static int setup_problem(orc_problem *P, const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                         const double *x0, const double *u_nom, double vref_scale, const double *opp, int n_opp,
                         int T, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round, uint32_t stream,
                         int game_on, int zero_noise)
{
    memset(P, 0, sizeof *P);
    if (N < 3 || T < 1 || n_opp < 0 || n_opp > 16) return -1;
    P->p = p; P->x0 = x0; P->u_nom = u_nom; P->vref_scale = vref_scale; P->opp = opp; P->n_opp = n_opp; P->T = T;
    P->seed = seed; P->race = race; P->agent = agent; P->round = round; P->stream = stream;
    P->game_on = game_on; P->zero_noise = zero_noise;
    if (track_init(&P->trk, xr, wl, wr, N)) return -1;
    if (problem_init(P)) { track_free(&P->trk); return -1; }
    return 0;
}
static void teardown_problem(orc_problem *P) { problem_free(P); track_free(&P->trk); }

/* Per-candidate costs, flags and violations (Alg. 1, sampling, cost and
 * feasibility steps).  k_list (n entries) selects which k to evaluate; when it
 * is NULL, k = 0..n-1.  Optional per-candidate outputs may be NULL; prop
 * (T x 4, may be NULL) and K_prop add the proposal of sample_controls. */
/* The same with perturbed opponent data (orc_perturb_prediction): opp_pos
 * (n_opp x (T+1) x 4) gives the positions of the distance terms and
 * sum_delta (n_opp x 2) the shifts of each prediction's progress gain and
 * tail-mean offset; the summaries themselves come from opp. */
int orc_rollout_costs_perturbed(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                                const double *x0, const double *u_nom, double vref_scale, const double *opp,
                                const double *opp_pos, const double *sum_delta, int n_opp, int T,
                                const int32_t *k_list, int n, uint64_t seed, uint32_t race, uint32_t agent,
                                uint32_t round, int game_on, double *cost, unsigned char *feas, double *viol,
                                double *states, double *controls, double *margins, int nthreads)
{
    orc_problem P;
    if (setup_problem(&P, p, xr, wl, wr, N, x0, u_nom, vref_scale, opp, n_opp, T, seed, race, agent, round, 0,
                      game_on, 0))
        return -1;
    P.opp_pos = opp_pos;
    for (int j = 0; j < n_opp; ++j) {
        P.opp_sum[j].sH += sum_delta[2 * j];
        P.opp_sum[j].dbar += sum_delta[2 * j + 1];
    }
    run_jobs(&P, k_list, n, nthreads, cost, feas, viol, states, NULL, controls, NULL, NULL, margins);
    teardown_problem(&P);
    return 0;
}

int orc_rollout_costs(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                      const double *x0, const double *u_nom, double vref_scale, const double *opp, int n_opp,
                      int T, const int32_t *k_list, int n, uint64_t seed, uint32_t race, uint32_t agent,
                      uint32_t round, uint32_t stream, int game_on, int zero_noise,
                      double *cost, unsigned char *feas, double *viol, double *states, double *frenet,
                      double *controls, double *c_track, double *c_game, double *margins, const double *prop,
                      int K_prop, int nthreads)
{
    orc_problem P;
    if (setup_problem(&P, p, xr, wl, wr, N, x0, u_nom, vref_scale, opp, n_opp, T, seed, race, agent, round,
                      stream, game_on, zero_noise))
        return -1;
    P.prop = prop;
    P.K_prop = prop ? K_prop : 0;
    run_jobs(&P, k_list, n, nthreads, cost, feas, viol, states, frenet, controls, c_track, c_game, margins);
    teardown_problem(&P);
    return 0;
}

/* Evaluate explicitly given control sequences (n x T x 2, already inside the
 * admissible set) through the same rollout, cost and checks. */
int orc_eval_controls(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                      const double *x0, const double *u, int n, double vref_scale, const double *opp, int n_opp,
                      int T, int game_on, double *cost, unsigned char *feas, double *viol, double *states,
                      double *frenet)
{
    orc_problem P;
    if (setup_problem(&P, p, xr, wl, wr, N, x0, u, vref_scale, opp, n_opp, T, 0, 0, 0, 0, 0, game_on, 1))
        return -1;
    for (int i = 0; i < n; ++i) {
        orc_sample_result r = eval_candidate(&P, u + (size_t)i * T * 2,
                                             states ? states + (size_t)i * (T + 1) * 4 : NULL,
                                             frenet ? frenet + (size_t)i * (T + 1) * 2 : NULL);
        cost[i] = r.cost; feas[i] = (unsigned char)r.feasible; viol[i] = r.viol;
    }
    teardown_problem(&P);
    return 0;
}

/* One best response (Alg. 1, one pass of the vehicle loop): all K samples,
 * selection, and the selected trajectory xi* ((T+1)x4) and controls U* (Tx2).
 * prop (T x 4, may be NULL) and K_prop add the proposal of sample_controls;
 * cost_out (K, may be NULL) receives every candidate's cost and viol_out (K,
 * may be NULL) every violation. */
static int br_core(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                   const double *x0, const double *u_nom, double vref_scale, const double *opp, int n_opp, int T,
                   int K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round, uint32_t stream,
                   int game_on, const double *prop, int K_prop, const double *opp_pos, const double *sum_delta,
                   int *k_star, double *u_star, double *xi_star, int *any_feasible, double *cost_out,
                   double *viol_out, int nthreads)
{
    orc_problem P;
    if (K < 1 || K_prop < 0 || K_prop > K) return -1;
    if (setup_problem(&P, p, xr, wl, wr, N, x0, u_nom, vref_scale, opp, n_opp, T, seed, race, agent, round,
                      stream, game_on, 0))
        return -1;
    P.opp_pos = opp_pos;
    if (sum_delta)
        for (int j = 0; j < n_opp; ++j) {
            P.opp_sum[j].sH += sum_delta[2 * j];
            P.opp_sum[j].dbar += sum_delta[2 * j + 1];
        }
    P.prop = prop;
    P.K_prop = prop ? K_prop : 0;
    double *cost = (double *)malloc(sizeof(double) * (size_t)K);
    double *viol = (double *)malloc(sizeof(double) * (size_t)K);
    unsigned char *feas = (unsigned char *)malloc((size_t)K);
    run_jobs(&P, NULL, K, nthreads, cost, feas, viol, NULL, NULL, NULL, NULL, NULL, NULL);
    const int ks = orc_select(cost, feas, viol, K, any_feasible);
    *k_star = ks;
    double *u = (double *)malloc(sizeof(double) * (size_t)T * 2);
    sample_controls(&P, (uint32_t)ks, u);
    eval_candidate(&P, u, xi_star, NULL);
    if (u_star) memcpy(u_star, u, sizeof(double) * (size_t)T * 2);
    if (cost_out) memcpy(cost_out, cost, sizeof(double) * (size_t)K);
    if (viol_out) memcpy(viol_out, viol, sizeof(double) * (size_t)K);
    free(u); free(cost); free(viol); free(feas);
    teardown_problem(&P);
    return 0;
}

int orc_best_response_mixed(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                            const double *x0, const double *u_nom, double vref_scale, const double *opp, int n_opp,
                            int T, int K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                            uint32_t stream, int game_on, const double *prop, int K_prop, int *k_star,
                            double *u_star, double *xi_star, int *any_feasible, double *cost_out,
                            double *viol_out, int nthreads)
{
    return br_core(p, xr, wl, wr, N, x0, u_nom, vref_scale, opp, n_opp, T, K, seed, race, agent, round, stream,
                   game_on, prop, K_prop, NULL, NULL, k_star, u_star, xi_star, any_feasible, cost_out, viol_out,
                   nthreads);
}

/* Perturbed prediction of opponent jv as seen by vehicle `observer` in
 * round `round` (robustness study of Sec. IV-F, Table II; the paper's
 * perturbation model is a cited one that is not available, so this is plain
 * Gaussian noise in Frenet coordinates, first order): every predicted
 * position p_tau, tau = 1..T, moves by sigma_lon z_1 along the unit direction
 * of its nearest raceline segment and by sigma_lat z_2 along that segment's
 * left normal, (z_1, z_2) the Box-Muller pair of counter
 * (2^30 | jv, (tau-1) >> 1, observer | round << 16, race), a counter no
 * sample uses (samples have k < 2^30).  The prediction's progress gain moves
 * by sigma_lon z_1 at tau = T and its tail-mean offset by the mean of
 * sigma_lat z_2 over the tail steps: delta_out = (d gain, d tail mean).
 * The current state (tau = 0), headings and speeds are unchanged. */
int orc_perturb_prediction(const double *xr, const double *wl, const double *wr, int N, const double *states, int T,
                           uint64_t seed, uint32_t race, uint32_t observer, uint32_t round, uint32_t jv,
                           double sigma_lon, double sigma_lat, int n_tail, double *out_states, double *delta_out)
{
    orc_track trk;
    if (track_init(&trk, xr, wl, wr, N)) return -1;
    memcpy(out_states, states, sizeof(double) * (size_t)(T + 1) * 4);
    double dgain = 0.0, dsum = 0.0;
    for (int tau = 1; tau <= T; ++tau) {
        double z1, z2, s, d;
        int j;
        orc_std_normals(seed, race, observer, round, 0, (1u << 30) | jv, tau - 1, &z1, &z2);
        const double *q = states + 4 * tau;
        orc_frenet_raw(&trk, q[0], q[1], &s, &d, &j);
        const int jn = (j + 1) % N;
        const double ex = xr[4 * jn] - xr[4 * j], ey = xr[4 * jn + 1] - xr[4 * j + 1];
        const double len = sqrt(ex * ex + ey * ey);
        const double tx = ex / len, ty = ey / len;
        out_states[4 * tau] = q[0] + sigma_lon * z1 * tx - sigma_lat * z2 * ty;
        out_states[4 * tau + 1] = q[1] + sigma_lon * z1 * ty + sigma_lat * z2 * tx;
        if (tau == T) dgain = sigma_lon * z1;
        if (tau > T - n_tail) dsum += sigma_lat * z2;
    }
    delta_out[0] = dgain;
    delta_out[1] = dsum / (double)n_tail;
    track_free(&trk);
    return 0;
}

int orc_best_response(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                      const double *x0, const double *u_nom, double vref_scale, const double *opp, int n_opp,
                      int T, int K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round, uint32_t stream,
                      int game_on, int *k_star, double *u_star, double *xi_star, int *any_feasible,
                      double *cost_out, int nthreads)
{
    return orc_best_response_mixed(p, xr, wl, wr, N, x0, u_nom, vref_scale, opp, n_opp, T, K, seed, race, agent,
                                   round, stream, game_on, NULL, 0, k_star, u_star, xi_star, any_feasible, cost_out,
                                   NULL, nthreads);
}

/* Zero-noise (nominal) rollout of a control sequence, controls clipped to
 * the admissible set: the opponents' predictions before the first round. */
static void nominal_rollout(const orc_params *p, const double *x0, const double *u_nom, int T, double *states)
{
    double x[4] = {x0[0], x0[1], x0[2], x0[3]};
    memcpy(states, x, sizeof x);
    for (int tau = 0; tau < T; ++tau) {
        const double a = clampd(u_nom[2 * tau], p->a_min, p->a_max);
        const double dl = clampd(u_nom[2 * tau + 1], -p->delta_max, p->delta_max);
        double xn[4];
        bicycle_step(p, x, a, dl, xn);
        memcpy(x, xn, sizeof x);
        memcpy(states + 4 * (tau + 1), x, sizeof x);
    }
}

/* GA-IBR-MPPI best response (Sec. IV-A, the second ablation): the same K
 * samples, rollouts, tracking cost and game-aware cost as the SGTP best
 * response, but no feasibility selection.  The nominal sequence becomes the
 * path-integral (importance-weighted) mean of the sampled controls, the
 * update of standard MPPI that the paper cites:
 *     w_k = exp(-(c_k - c_min) / lambda),   U_new = sum_k w_k U^(k) / sum_k w_k.
 * The paper gives no temperature; lambda is an input.  Readings: U^(k) are
 * the clipped controls sample k was rolled out with, so U_new is admissible;
 * a sample whose cost is not finite weighs nothing, and when no sample has a
 * finite cost the clipped nominal is kept; the new trajectory xi_new
 * ((T+1)x4) is the rollout of U_new; k_min is the lowest-cost sample (lowest
 * index on ties), reported for inspection only.  cost_out (K, may be NULL)
 * receives every sample's cost. */
int orc_best_response_mppi(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                           const double *x0, const double *u_nom, double vref_scale, const double *opp, int n_opp,
                           int T, int K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round, int game_on,
                           double lambda, int *k_min, double *u_new, double *xi_new, double *cost_out, int nthreads)
{
    orc_problem P;
    if (K < 1 || !(lambda > 0.0)) return -1;
    if (setup_problem(&P, p, xr, wl, wr, N, x0, u_nom, vref_scale, opp, n_opp, T, seed, race, agent, round, 0,
                      game_on, 0))
        return -1;
    double *cost = (double *)malloc(sizeof(double) * (size_t)K);
    double *viol = (double *)malloc(sizeof(double) * (size_t)K);
    unsigned char *feas = (unsigned char *)malloc((size_t)K);
    double *u = (double *)malloc(sizeof(double) * (size_t)T * 2);
    run_jobs(&P, NULL, K, nthreads, cost, feas, viol, NULL, NULL, NULL, NULL, NULL, NULL);
    int kb = -1;
    double c_min = INFINITY;
    for (int k = 0; k < K; ++k)
        if (isfinite(cost[k]) && cost[k] < c_min) { c_min = cost[k]; kb = k; }
    *k_min = kb;
    if (kb < 0) {
        for (int tau = 0; tau < T; ++tau) {
            u_new[2 * tau] = clampd(u_nom[2 * tau], p->a_min, p->a_max);
            u_new[2 * tau + 1] = clampd(u_nom[2 * tau + 1], -p->delta_max, p->delta_max);
        }
    } else {
        double w_sum = 0.0;
        for (int q = 0; q < 2 * T; ++q) u_new[q] = 0.0;
        for (int k = 0; k < K; ++k) {
            if (!isfinite(cost[k])) continue;
            const double w = exp(-(cost[k] - c_min) / lambda);
            sample_controls(&P, (uint32_t)k, u);
            for (int q = 0; q < 2 * T; ++q) u_new[q] += w * u[q];
            w_sum += w;
        }
        for (int q = 0; q < 2 * T; ++q) u_new[q] /= w_sum;
    }
    eval_candidate(&P, u_new, xi_new, NULL);
    if (cost_out) memcpy(cost_out, cost, sizeof(double) * (size_t)K);
    free(u); free(cost); free(viol); free(feas);
    teardown_problem(&P);
    return 0;
}

/* The planning loop of Alg. 1, shared by both update rules.
 *   round 0: every vehicle best-responds, without the game term, to the
 *            others' nominal rollouts (Alg. 1 initialisation, read as the
 *            feasibility-selected tracking response);
 *   rounds 1..L: Jacobi iterative best response against the previous round;
 *   finally one extra ego response (round tag L+1) against round L.
 * After each best response the vehicle's nominal controls become the
 * response's controls (warm start): the selected sample's (SGTP, lambda <= 0)
 * or the path-integral mean (GA-IBR-MPPI, lambda > 0).  xi_out holds
 * round-L trajectories, except the ego's, which is its extra response.
 * k_star_out has (L+1)*n_v+1 entries: round-major, then the extra ego
 * response (the selected sample; for GA-IBR-MPPI the lowest-cost one).
 * xi_hist (optional) has (L+2) x n_v x (T+1) x 4 entries: slot r holds the
 * round-r trajectory of every vehicle; slot L+1 holds round L again except
 * the ego's extra response.  u_hist likewise with (L+2) x n_v x T x 2
 * nominal controls after each round. */
static int plan_loop(const orc_params *p, const double *xr, const double *wl, const double *wr, int N, int n_v,
                     const double *X0, double *U_io, const double *vref_scale, int T, int K, int L, int ego,
                     uint64_t seed, uint32_t race, double lambda, double sigma_lon, double sigma_lat,
                     double *xi_out, int *k_star_out, double *xi_hist, double *u_hist, int nthreads)
{
    if (n_v < 1 || n_v > 17 || ego < 0 || ego >= n_v || L < 0) return -1;
    const int perturb = sigma_lon != 0.0 || sigma_lat != 0.0;
    if (perturb && lambda > 0.0) return -1;
    const int n_tail = orc_tail_count(p->mu_tail, T);
    const size_t traj = (size_t)(T + 1) * 4;
    double *xi = (double *)malloc(sizeof(double) * traj * (size_t)n_v);
    double *xi_new = (double *)malloc(sizeof(double) * traj * (size_t)n_v);
    double *opp = (double *)malloc(sizeof(double) * traj * (size_t)(n_v > 1 ? n_v - 1 : 1));
    double *u_new = (double *)malloc(sizeof(double) * (size_t)T * 2 * (size_t)n_v);
    double *opp_pos = (double *)malloc(sizeof(double) * traj * (size_t)(n_v > 1 ? n_v - 1 : 1));
    double *delta = (double *)malloc(sizeof(double) * 2 * (size_t)(n_v > 1 ? n_v - 1 : 1));
    for (int i = 0; i < n_v; ++i) nominal_rollout(p, X0 + 4 * i, U_io + (size_t)i * T * 2, T, xi + traj * i);
    int nk = 0, rc = 0;
    for (int round = 0; round <= L + 1 && rc == 0; ++round) {
        const int extra = (round == L + 1);
        for (int i = 0; i < n_v && rc == 0; ++i) {
            if (extra && i != ego) continue;
            int m = 0;
            for (int j = 0; j < n_v; ++j) {
                if (j == i) continue;
                memcpy(opp + traj * m, xi + traj * j, sizeof(double) * traj);
                if (perturb)
                    orc_perturb_prediction(xr, wl, wr, N, xi + traj * j, T, seed, race, (uint32_t)i, (uint32_t)round,
                                           (uint32_t)j, sigma_lon, sigma_lat, n_tail, opp_pos + traj * m,
                                           delta + 2 * m);
                ++m;
            }
            int ks, anyf;
            if (lambda > 0.0)
                rc = orc_best_response_mppi(p, xr, wl, wr, N, X0 + 4 * i, U_io + (size_t)i * T * 2, vref_scale[i],
                                            opp, n_v - 1, T, K, seed, race, (uint32_t)i, (uint32_t)round, round > 0,
                                            lambda, &ks, u_new + (size_t)i * T * 2, xi_new + traj * i, NULL,
                                            nthreads);
            else
                rc = br_core(p, xr, wl, wr, N, X0 + 4 * i, U_io + (size_t)i * T * 2, vref_scale[i], opp, n_v - 1, T,
                             K, seed, race, (uint32_t)i, (uint32_t)round, 0, round > 0, NULL, 0,
                             perturb ? opp_pos : NULL, perturb ? delta : NULL, &ks, u_new + (size_t)i * T * 2,
                             xi_new + traj * i, &anyf, NULL, NULL, nthreads);
            k_star_out[nk++] = ks;
        }
        /* Jacobi: all vehicles of the round updated together */
        for (int i = 0; i < n_v; ++i) {
            if (extra && i != ego) continue;
            memcpy(xi + traj * i, xi_new + traj * i, sizeof(double) * traj);
            memcpy(U_io + (size_t)i * T * 2, u_new + (size_t)i * T * 2, sizeof(double) * (size_t)T * 2);
        }
        if (xi_hist) memcpy(xi_hist + traj * (size_t)n_v * round, xi, sizeof(double) * traj * (size_t)n_v);
        if (u_hist) memcpy(u_hist + (size_t)T * 2 * n_v * round, U_io, sizeof(double) * (size_t)T * 2 * n_v);
    }
    memcpy(xi_out, xi, sizeof(double) * traj * (size_t)n_v);
    free(xi); free(xi_new); free(opp); free(u_new); free(opp_pos); free(delta);
    return rc;
}

/* The SGTP planning call (Alg. 1): plan_loop with feasibility selection. */
int orc_ibr_plan(const orc_params *p, const double *xr, const double *wl, const double *wr, int N, int n_v,
                 const double *X0, double *U_io, const double *vref_scale, int T, int K, int L, int ego,
                 uint64_t seed, uint32_t race, double *xi_out, int *k_star_out, double *xi_hist,
                 double *u_hist, int nthreads)
{
    return plan_loop(p, xr, wl, wr, N, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, 0.0, 0.0, 0.0, xi_out,
                     k_star_out, xi_hist, u_hist, nthreads);
}

/* The SGTP planning call with every opponent prediction perturbed before
 * each best response (orc_perturb_prediction, per observer and round). */
int orc_ibr_plan_perturbed(const orc_params *p, const double *xr, const double *wl, const double *wr, int N, int n_v,
                           const double *X0, double *U_io, const double *vref_scale, int T, int K, int L, int ego,
                           uint64_t seed, uint32_t race, double sigma_lon, double sigma_lat, double *xi_out,
                           int *k_star_out, double *xi_hist, double *u_hist, int nthreads)
{
    return plan_loop(p, xr, wl, wr, N, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, 0.0, sigma_lon, sigma_lat,
                     xi_out, k_star_out, xi_hist, u_hist, nthreads);
}

/* The GA-IBR-MPPI planning call (Sec. IV-A ablation): the same loop with the
 * path-integral update of orc_best_response_mppi at temperature lambda > 0. */
int orc_ibr_plan_mppi(const orc_params *p, const double *xr, const double *wl, const double *wr, int N, int n_v,
                      const double *X0, double *U_io, const double *vref_scale, int T, int K, int L, int ego,
                      uint64_t seed, uint32_t race, double lambda, double *xi_out, int *k_star_out,
                      double *xi_hist, double *u_hist, int nthreads)
{
    if (!(lambda > 0.0)) return -1;
    return plan_loop(p, xr, wl, wr, N, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, lambda, 0.0, 0.0,
                     xi_out, k_star_out, xi_hist, u_hist, nthreads);
}

/* Exposed pieces used by the oracle's own checks. */
int orc_frenet(const double *xr, const double *wl, const double *wr, int N, const double *pts, int n,
               double *s, double *d, int32_t *seg)
{
    orc_track t;
    if (track_init(&t, xr, wl, wr, N)) return -1;
    for (int i = 0; i < n; ++i) {
        int j;
        orc_frenet_raw(&t, pts[2 * i], pts[2 * i + 1], &s[i], &d[i], &j);
        if (seg) seg[i] = j;
    }
    track_free(&t);
    return 0;
}

double orc_track_length(const double *xr, int N)
{
    orc_track t;
    if (track_init(&t, xr, NULL, NULL, N)) return -1.0;
    const double L = t.L;
    track_free(&t);
    return L;
}

int orc_reference(const orc_params *p, const double *xr, const double *wl, const double *wr, int N,
                  const double *x0, double vref_scale, int T, double *xref /* (T+1) x 4, row 0 = 0 */)
{
    orc_problem P;
    double dummy_u[2] = {0, 0};
    (void)dummy_u;
    double *u = (double *)calloc((size_t)T * 2, sizeof(double));
    if (setup_problem(&P, p, xr, wl, wr, N, x0, u, vref_scale, NULL, 0, T, 0, 0, 0, 0, 0, 0, 1)) { free(u); return -1; }
    memcpy(xref, P.xref, sizeof(double) * (size_t)(T + 1) * 4);
    teardown_problem(&P);
    free(u);
    return 0;
}

void orc_rollout(const orc_params *p, const double *x0, const double *u, int T, double *states)
{
    nominal_rollout(p, x0, u, T, states);
}

/* Batch of standard normals for samples k0..k0+nk-1, steps 0..T-1:
 * out[(k - k0) * T * 2 + tau * 2 + {0,1}] (used by the oracle's own checks). */
void orc_std_normals_batch(uint64_t seed, uint32_t race, uint32_t agent, uint32_t round, uint32_t stream,
                           uint32_t k0, int nk, int T, double *out)
{
    for (int i = 0; i < nk; ++i)
        for (int tau = 0; tau < T; ++tau)
            orc_std_normals(seed, race, agent, round, stream, k0 + (uint32_t)i, tau,
                            &out[((size_t)i * T + tau) * 2], &out[((size_t)i * T + tau) * 2 + 1]);
}

/* Raw Philox4x32-10 blocks of counters (k0 + i, c1, c2, c3), i = 0..n-1,
 * under key (key lo, key hi): out[4 i .. 4 i + 3] (used by the parity tests
 * of the device generator; the same function as orc_philox4x32_10). */
void orc_philox_batch(uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, int n, uint32_t key_lo, uint32_t key_hi,
                      uint32_t *out)
{
    const uint32_t key[2] = {key_lo, key_hi};
    for (int i = 0; i < n; ++i) {
        const uint32_t ctr[4] = {k0 + (uint32_t)i, c1, c2, c3};
        orc_philox4x32_10(ctr, key, out + 4 * (size_t)i);
    }
}
