// sgtp_rollout.cuh -- one sampled candidate of a best response, in registers.
//
// A candidate k of vehicle i (Alg. 1, sampling/cost/feasibility steps):
//   u_tau = Pi_U(u_nom_tau + eps_tau)                       (Sec. II)
//   x_{tau+1} = f(x_tau, u_tau), kinematic bicycle, Euler   (Sec. II)
//   c = c_track (Eq. ctrack) + w_game * sum_j c_game,ij     (Eqs. game_cost, allc)
//   h = b * o (Eqs. selection-boundary, selection-vehicle), nu (fallback)
// The horizon loop keeps the state, one running cost sum, the running
// boundary clearance and one running minimum distance per opponent in
// registers; nothing of the trajectory is stored unless asked for.
#pragma once

#include "sgtp_device.cuh"

namespace sgtp {

// Read-only view of one best-response problem, staged in shared memory.
struct BRView {
    TrackView tv;
    SegWindow win;
    const float2 *ubar;   // [T]          nominal controls
    const float4 *ref;    // [T+1]        reference states, row 0 unused
    const float2 *opp;    // [T][n_opp]   opponent positions at tau = 1..T (row tau-1)
    const float4 *osum;   // [n_opp]      (ds_t, alpha, gamma, prog)
    const float *odbar;   // [n_opp]      tail-mean lateral offset of each opponent
    float4 x0;
    float s_t, d_t;
    int r0;               // window-local segment of x0
    int T, n_opp, n_tail;
    float invL;
    // noise counter words
    uint2 key;
    unsigned ctr_agent_round, ctr_race, stream_bit;
};

template <int MAXO>
struct SampleState {
    float x, y, psi, v;
    float a_prev, d_prev;
    float s;          // unwrapped progress
    int r, dr;        // window-local nearest segment, last shift
    float c;          // running c_track
    float rho_bd, d_tail;
    float g2[MAXO];
};

// Clipped control from a nominal control and a normal pair z (Pi_U).
__device__ __forceinline__ float2 sample_control(const sgtp_params &p, float2 ubar, float2 z)
{
    const float a = fminf(fmaxf(__fmaf_rn(p.sigma_a, z.x, ubar.x), p.a_min), p.a_max);
    const float d = fminf(fmaxf(__fmaf_rn(p.sigma_delta, z.y, ubar.y), -p.delta_max), p.delta_max);
    return make_float2(a, d);
}

// One forward-Euler step of the kinematic bicycle (rear-axle reference,
// steering input, speed clamp), every right-hand side at the old state.
__device__ __forceinline__ void bicycle_step(const sgtp_params &p, float &x, float &y, float &psi, float &v, float a,
                                             float delta)
{
    float sn, cs;
    __sincosf(wrap_angle(psi), &sn, &cs);
    float sd, cd;
    __sincosf(delta, &sd, &cd);
    const float dv = __fmul_rn(p.dt, v);
    const float x1 = __fmaf_rn(dv, cs, x);
    const float y1 = __fmaf_rn(dv, sn, y);
    const float psi1 = psi + __fdividef(__fmul_rn(dv, sd), __fmul_rn(cd, p.wheelbase));
    const float v1 = fminf(fmaxf(__fmaf_rn(p.dt, a, v), p.v_min), p.v_max);
    x = x1; y = y1; psi = psi1; v = v1;
}

// Noise words of candidate k at steps 2m, 2m+1.
__device__ __forceinline__ uint4 noise_block(const BRView &bv, unsigned k, int m)
{
    return philox4x32_10(make_uint4(k, (unsigned)m | bv.stream_bit, bv.ctr_agent_round, bv.ctr_race), bv.key);
}

template <int MAXO>
__device__ __forceinline__ void sample_init(SampleState<MAXO> &S, const BRView &bv)
{
    S.x = bv.x0.x; S.y = bv.x0.y; S.psi = bv.x0.z; S.v = bv.x0.w;
    S.a_prev = 0.f; S.d_prev = 0.f;
    S.s = bv.s_t;
    S.r = bv.r0; S.dr = 0;
    S.c = 0.f;
    S.rho_bd = __int_as_float(0x7f800000);
    S.d_tail = 0.f;
#pragma unroll
    for (int o = 0; o < MAXO; ++o) S.g2[o] = __int_as_float(0x7f800000);
}

// Advance a candidate by one step tau with control u; optional outputs.
template <int MAXO, bool OUT>
__device__ __forceinline__ void sample_step(SampleState<MAXO> &S, const BRView &bv, const sgtp_params &p, int tau,
                                            float2 u, int &flag, float *st_out, float *fr_out)
{
    // control cost, tau = 0..H-1, and smoothness, tau = 1..H-1 (Eq. ctrack)
    float cc = __fmaf_rn(p.R[0], __fmul_rn(u.x, u.x), __fmul_rn(p.R[1], __fmul_rn(u.y, u.y)));
    if (tau > 0) {
        const float da = u.x - S.a_prev, dd = u.y - S.d_prev;
        cc = __fmaf_rn(p.S[0], __fmul_rn(da, da), cc);
        cc = __fmaf_rn(p.S[1], __fmul_rn(dd, dd), cc);
    }
    S.a_prev = u.x; S.d_prev = u.y;

    bicycle_step(p, S.x, S.y, S.psi, S.v, u.x, u.y);
    const int st = tau + 1;

    // Frenet of the new state, progress unwrapped along the rollout
    const FrenetPt f = frenet_walk(bv.tv, bv.win, S.r, S.dr, S.x, S.y, flag);
    S.s = S.s + wrap_len(f.s - S.s, bv.tv.L, bv.invL);

    // tracking term, tau = 1..H (Eq. ctrack), heading error wrapped
    const float4 r = bv.ref[st];
    const float ex = S.x - r.x, ey = S.y - r.y, ep = wrap_angle(S.psi - r.z), ev = S.v - r.w;
    cc = __fmaf_rn(p.Q[0], __fmul_rn(ex, ex), cc);
    cc = __fmaf_rn(p.Q[1], __fmul_rn(ey, ey), cc);
    cc = __fmaf_rn(p.Q[2], __fmul_rn(ep, ep), cc);
    cc = __fmaf_rn(p.Q[3], __fmul_rn(ev, ev), cc);
    S.c = S.c + cc;

    // boundary clearance (Sec. III-B) with widths at the foot point
    S.rho_bd = fminf(S.rho_bd, fminf(f.wr + f.d, f.wl - f.d));

    // tail lateral offsets (blocking term)
    if (st > bv.T - bv.n_tail) S.d_tail = S.d_tail + f.d;

    // time-aligned distances to every opponent (Eq. Dmin)
    const float2 *op = bv.opp + (size_t)tau * bv.n_opp;
#pragma unroll
    for (int o = 0; o < MAXO; ++o) {
        if (o < bv.n_opp) {
            const float2 q = op[o];
            const float dx = S.x - q.x, dy = S.y - q.y;
            S.g2[o] = fminf(S.g2[o], __fmaf_rn(dx, dx, __fmul_rn(dy, dy)));
        }
    }
    if (OUT) {
        if (st_out) {
            st_out[4 * st + 0] = S.x; st_out[4 * st + 1] = S.y; st_out[4 * st + 2] = S.psi; st_out[4 * st + 3] = S.v;
        }
        if (fr_out) { fr_out[2 * st] = S.s; fr_out[2 * st + 1] = f.d; }
    }
}

struct SampleResult {
    float cost, viol;
    bool feasible;
};

// Terminal game cost per opponent (Eqs. c_contest, c_long, c_block,
// c_safety), total cost (Eq. allc), feasibility and violation (Sec. III-B).
template <int MAXO>
__device__ __forceinline__ SampleResult sample_finish(const SampleState<MAXO> &S, const BRView &bv,
                                                      const sgtp_params &p, bool game_on)
{
    const float dbar_i = S.d_tail / (float)bv.n_tail;
    const float prog_i = S.s - bv.s_t;
    float c_game = 0.f;
    float rho_obs = __int_as_float(0x7f800000);
#pragma unroll
    for (int o = 0; o < MAXO; ++o) {
        if (o < bv.n_opp) {
            const float4 os = bv.osum[o];            // ds_t, alpha, gamma, prog_j
            const float ds_H = os.x + (prog_i - os.w);
            const float c_contest = fabsf(ds_H) < p.s_contest ? -p.w_contest : 0.f;
            const float c_long = -p.w_long * os.y * ds_H;
            const float c_block = os.z != 0.f ? -os.z / (1.f + fabsf(dbar_i - bv.odbar[o])) : 0.f;
            const float g = sqrtf(S.g2[o]);
            const float sh = fmaxf(0.f, p.g_safe - g);
            const float c_safety = p.w_safety * sh * sh;
            c_game = c_game + (c_contest + c_long + c_block + c_safety);
            rho_obs = fminf(rho_obs, g);
        }
    }
    SampleResult r;
    r.cost = game_on ? __fmaf_rn(p.w_game, c_game, S.c) : S.c;
    const bool b = S.rho_bd >= p.m_bd;
    const bool ob = rho_obs >= p.d_col;
    r.feasible = b && ob;
    r.viol = fmaxf(0.f, p.m_bd - S.rho_bd) + fmaxf(0.f, p.d_col - rho_obs);
    return r;
}

// Full candidate: noise, controls, rollout, finish.  Optional outputs are
// written when OUT (states (T+1)x4, frenet (T+1)x2, controls Tx2).
template <int MAXO, bool OUT>
__device__ __forceinline__ SampleResult run_candidate(const BRView &bv, const sgtp_params &p, unsigned k, bool game_on,
                                                      bool zero_noise, int &flag, float *st_out, float *fr_out,
                                                      float *u_out)
{
    SampleState<MAXO> S;
    sample_init(S, bv);
    if (OUT) {
        if (st_out) { st_out[0] = S.x; st_out[1] = S.y; st_out[2] = S.psi; st_out[3] = S.v; }
        if (fr_out) { fr_out[0] = bv.s_t; fr_out[1] = bv.d_t; }
    }
    for (int m = 0; 2 * m < bv.T; ++m) {
        float2 z0 = make_float2(0.f, 0.f), z1 = z0;
        if (!zero_noise) {
            const uint4 w = noise_block(bv, k, m);
            z0 = box_muller(w.x, w.y);
            z1 = box_muller(w.z, w.w);
        }
        const int t0 = 2 * m;
        const float2 u0 = sample_control(p, bv.ubar[t0], z0);
        if (OUT && u_out) { u_out[2 * t0] = u0.x; u_out[2 * t0 + 1] = u0.y; }
        sample_step<MAXO, OUT>(S, bv, p, t0, u0, flag, st_out, fr_out);
        if (t0 + 1 < bv.T) {
            const float2 u1 = sample_control(p, bv.ubar[t0 + 1], z1);
            if (OUT && u_out) { u_out[2 * t0 + 2] = u1.x; u_out[2 * t0 + 3] = u1.y; }
            sample_step<MAXO, OUT>(S, bv, p, t0 + 1, u1, flag, st_out, fr_out);
        }
    }
    return sample_finish(S, bv, p, game_on);
}

}  // namespace sgtp
