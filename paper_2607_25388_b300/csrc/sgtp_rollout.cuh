// sgtp_rollout.cuh -- one sampled candidate of a best response, in registers.
//
// A candidate k of vehicle i (Alg. 1, sampling/cost/feasibility steps):
//   u_tau = Pi_U(u_nom_tau + eps_tau)                       (Sec. II)
//   x_{tau+1} = f(x_tau, u_tau), kinematic bicycle, Euler   (Sec. II)
//   c = c_track (Eq. ctrack) + w_game * sum_j c_game,ij     (Eqs. game_cost, allc)
//   h = b * o (Eqs. selection-boundary, selection-vehicle), nu (fallback)
// The horizon loop keeps the state, a running cost pair, the running
// boundary clearance and one running minimum distance per opponent in
// registers; nothing of the trajectory is stored unless asked for.  Paired
// quantities (x/y errors, a/delta controls, two opponents) use the packed
// f32x2 arithmetic of sm_100-class GPUs.
//
// Every per-problem array lives in shared memory at a compile-time offset
// (BRTile below), so the sample loop holds no pointers in registers.
#pragma once

#include "sgtp_device.cuh"

namespace sgtp {

constexpr int kWinTile = 512;          // track window of a best-response tile (segments)
constexpr int kTileSingle = 256;       // samples of a work item of the plan kernel
constexpr float kFarAway = 1.0e15f;    // position of an absent opponent slot

// Scalars of one best-response problem (shared memory).
struct BRScalars {
    TrackView tv;         // global track (out-of-window segments)
    float4 x0;
    float s_t, d_t;
    float psi0, psi_off;  // x0's heading wrapped into (-pi, pi], and x0.z - psi0 (rollouts run from
                          // psi0 and add psi_off back to every heading they output)
    float pos0;           // continuous segment position of x0 (window-local segment + parameter)
    float ppred0;         // first predicted position: pos0 + advance at v0 - 1/2
    int r0;               // window-local segment of x0
    int w0, Wn;           // window: segments w0 .. w0 + Wn - 1 of the ring-extended arrays
    int lap0;             // 1 when x0's segment sits past the ring's end (w0 + r0 >= N)
    int T, n_opp, n_tail;
    float invL;
    uint2 key;            // noise counter words
    unsigned ctr_agent_round, ctr_race, stream_bit;
    int K_prop;           // samples k < K_prop come from the proposal distribution
    int pad[1];
};

// A heading wrapped into (-pi, pi] and the offset that restores it: the
// rollouts start from the wrapped heading, so that the sine and cosine
// approximations of the dynamics stay in their accurate range without a
// wrap at every step, and add the offset to every heading they output.
__device__ __forceinline__ float2 heading_split(float psi)
{
    const float w = wrap_angle(psi);
    return make_float2(w, psi - w);
}

// Shared-memory tile of one best response: fixed offsets for a given MAXO.
// The track window holds the sample-loop projection records G0..G3 of
// kWinTile segments; the scratch area serves the proposal network and the
// GA-IBR-MPPI sums.
template <int MAXO>
struct BRTile {
    static constexpr int NP = (MAXO + 1) / 2;           // opponent pairs per step
    static constexpr unsigned kBar = 0;                 // TMA mbarrier (8 B)
    static constexpr unsigned kScal = 16;
    static constexpr unsigned kF0 = (kScal + sizeof(BRScalars) + 15) & ~15u;
    static constexpr unsigned kF1 = kF0 + 16u * kWinTile;
    static constexpr unsigned kF2 = kF1 + 16u * kWinTile;
    static constexpr unsigned kF3 = kF2 + 16u * kWinTile;
    static constexpr unsigned kRef = kF3 + 8u * kWinTile;
    static constexpr unsigned kUbar = kRef + 16u * (SGTP_MAX_T + 1);   // float4 [2][T]: plain, proposal
    static constexpr unsigned kOpp = kUbar + 32u * SGTP_MAX_T;
    static constexpr unsigned kOsum = kOpp + 16u * SGTP_MAX_T * NP;
    static constexpr unsigned kOdbar = kOsum + 16u * SGTP_MAX_AGENTS;
    static constexpr unsigned kCtl = kOdbar + 4u * SGTP_MAX_AGENTS;
    static constexpr unsigned kSt = kCtl + 8u * SGTP_MAX_T;          // states of one rollout (T+1)
    static constexpr unsigned kFr = kSt + 16u * (SGTP_MAX_T + 1);     // their (s, d)
    static constexpr unsigned kScr = kFr + 8u * SGTP_MAX_T;           // scratch
    static constexpr unsigned kScrBytes = 8192u;
    static constexpr unsigned kBytes = kScr + kScrBytes;
};

extern __shared__ __align__(16) unsigned char g_smem[];

template <int MAXO>
struct Tile {
    using L = BRTile<MAXO>;
    static __device__ __forceinline__ unsigned long long *bar() { return (unsigned long long *)(g_smem + L::kBar); }
    static __device__ __forceinline__ BRScalars &sc() { return *(BRScalars *)(g_smem + L::kScal); }
    static __device__ __forceinline__ float4 *F0() { return (float4 *)(g_smem + L::kF0); }
    static __device__ __forceinline__ float4 *F1() { return (float4 *)(g_smem + L::kF1); }
    static __device__ __forceinline__ float4 *F2() { return (float4 *)(g_smem + L::kF2); }
    static __device__ __forceinline__ float2 *F3() { return (float2 *)(g_smem + L::kF3); }
    static __device__ __forceinline__ float4 *ref() { return (float4 *)(g_smem + L::kRef); }
    // per-step sampling distribution (mean a, mean delta, sigma a, sigma delta):
    // dist()[tau] for the plain sampler, dist()[SGTP_MAX_T + tau] for the proposal
    static __device__ __forceinline__ float4 *dist() { return (float4 *)(g_smem + L::kUbar); }
    static __device__ __forceinline__ float4 *opp() { return (float4 *)(g_smem + L::kOpp); }
    static __device__ __forceinline__ float4 *osum() { return (float4 *)(g_smem + L::kOsum); }
    static __device__ __forceinline__ float *odbar() { return (float *)(g_smem + L::kOdbar); }
    static __device__ __forceinline__ float2 *ctl() { return (float2 *)(g_smem + L::kCtl); }
    static __device__ __forceinline__ float4 *st() { return (float4 *)(g_smem + L::kSt); }
    static __device__ __forceinline__ float2 *fr() { return (float2 *)(g_smem + L::kFr); }
    static __device__ __forceinline__ unsigned char *scratch() { return g_smem + L::kScr; }
    // Issue the window's bulk copies (one thread; completes on bar()).
    static __device__ __forceinline__ void stage_window(const TrackView &tv, int w0, int Wn)
    {
        mbar_expect_tx(bar(), (unsigned)Wn * 56u);
        bulk_g2s(F0(), tv.G0 + w0, (unsigned)Wn * 16u, bar());
        bulk_g2s(F1(), tv.G1 + w0, (unsigned)Wn * 16u, bar());
        bulk_g2s(F2(), tv.G2 + w0, (unsigned)Wn * 16u, bar());
        bulk_g2s(F3(), tv.G3 + w0, (unsigned)Wn * 8u, bar());
    }
    // Once the copies have landed (all threads; the caller synchronises
    // after): the arc lengths of window segments on another lap of the ring
    // than x0's segment move by that lap's multiple of L, so that progress
    // read from the window is unwrapped relative to s_t.
    static __device__ __forceinline__ void fix_laps(const BRScalars &S)
    {
        const int N = S.tv.N;
        for (int r = threadIdx.x; r < S.Wn; r += blockDim.x) {
            const int dl = (S.w0 + r >= N ? 1 : 0) - S.lap0;
            if (dl != 0) F3()[r].y = F3()[r].y + (float)dl * S.tv.L;
        }
    }
};

// True when a window fill needs fix_laps: it reaches past the ring's end.
__device__ __forceinline__ bool window_wraps(const BRScalars &S) { return S.w0 + S.Wn > S.tv.N; }

// ---------------------------------------------------------------- Frenet of rollout states
// Frenet projection s(x; G), d(x; G) (Sec. II) of a state p on segment j of
// the polyline, from the records G0..G3 (see TrackView):
//   along = u_j . (p - P_j), perp = u_j x (p - P_j) (> 0 left of travel),
//   t = clamp(along / |e_j|, 0, 1), foot P_j + t e_j,
//   |p - foot|^2 = (along - t |e_j|)^2 + perp^2, d = sign(perp) |p - foot|,
//   s = s_j + t |e_j|, widths at the foot by linear interpolation in t,
//   boundary clearance min(wR + d, wL - d) = h - |d - c|.
struct GeoPt {
    float s, d, tc, rho;
};

__device__ __forceinline__ GeoPt frenet_eval(float4 g1, float4 g2, float2 g3, float len, float px, float py)
{
    GeoPt f;
    const float along = __fmaf_rn(px, g1.x, __fmaf_rn(py, g1.y, -g1.z));
    const float perp = __fmaf_rn(py, g1.x, __fmaf_rn(-px, g1.y, -g1.w));
    const float tc = __saturatef(__fmul_rn(along, g2.x));
    const float ex = __fmaf_rn(-tc, len, along);
    const float q2 = __fmaf_rn(ex, ex, __fmul_rn(perp, perp));
    f.d = copysignf(sqrt_ftz(q2), perp);
    f.s = __fmaf_rn(tc, len, g3.y);
    f.tc = tc;
    const float h = __fmaf_rn(tc, g2.z, g2.y), c = __fmaf_rn(tc, g3.x, g2.w);
    f.rho = h - fabsf(f.d - c);
    return f;
}

// p lies strictly past the bisector of waypoint j (record q = G0[j]): then
// segment j is nearer than segment j-1 (ties go to the lower index).
__device__ __forceinline__ bool past_bisector(float4 q, float px, float py)
{
    return __fmaf_rn(px, q.x, __fmaf_rn(py, q.y, -q.z)) > 0.f;
}

// Global segment of window-local index r (any r) and its lap relative to
// the window's first lap.
__device__ __forceinline__ int lap_of(int g, int N) { return g >= 0 ? g / N : -((N - 1 - g) / N); }

template <int MAXO>
__device__ __forceinline__ float4 bisector_at(const BRScalars &S, int r)
{
    if ((unsigned)r < (unsigned)S.Wn) return Tile<MAXO>::F0()[r];
    const int g = S.w0 + r;
    const int j = g - lap_of(g, S.tv.N) * S.tv.N;
    return __ldg(S.tv.G0 + j);
}

// Records of window-local segment r: from the window, or from global
// memory with the same lap correction of the arc length as fix_laps.
template <int MAXO>
__device__ __forceinline__ void segment_at(const BRScalars &S, int r, float4 &g1, float4 &g2, float2 &g3, float &len)
{
    using T = Tile<MAXO>;
    if ((unsigned)r < (unsigned)S.Wn) {
        g1 = T::F1()[r]; g2 = T::F2()[r]; g3 = T::F3()[r]; len = T::F0()[r].w;
    } else {
        const int g = S.w0 + r, N = S.tv.N;
        const int lap = lap_of(g, N);
        const int j = g - lap * N;
        g1 = __ldg(S.tv.G1 + j); g2 = __ldg(S.tv.G2 + j); g3 = __ldg(S.tv.G3 + j); len = __ldg(S.tv.G0 + j).w;
        const int dl = lap - S.lap0;
        if (dl != 0) g3.y = g3.y + (float)dl * S.tv.L;
    }
}

// Segment of p by a walk over the bisectors from window-local segment r:
// forward while p is past the next bisector, else backward while it is not
// past the current one.  The result m has p past bisector m and not past
// bisector m+1, i.e. segment m is nearer than both neighbours: a local
// minimum of the distance over the segment index, which for points within
// the track's reach is the global nearest segment of the projection (ties
// to the lower index).  A walk longer than kMaxMoves stops and sets flag.
template <int MAXO>
__device__ __noinline__ int bisector_walk(const BRScalars &S, int r, float px, float py, int &flag)
{
    bool moved = false;
    for (int it = 0; it < kMaxMoves; ++it) {
        if (!past_bisector(bisector_at<MAXO>(S, r + 1), px, py)) break;
        r += 1;
        moved = true;
        if (it == kMaxMoves - 1) flag = 1;
    }
    if (!moved) {
        for (int it = 0; it < kMaxMoves; ++it) {
            if (past_bisector(bisector_at<MAXO>(S, r), px, py)) break;
            r -= 1;
            if (it == kMaxMoves - 1) flag = 1;
        }
    }
    return r;
}

// Segment of the next rollout state.  The sample carries a continuous
// segment position pos (window-local segment + parameter) and the predicted
// position of its next state, ppred = pos + last advance - 1/2.  With
// c = floor(ppred) clamped into the window (wlim = S.Wn - 2), the bisectors of
// c, c+1, c+2 certify segment c or c+1 when p is past the first and not past
// the third (three plane tests against shared memory); the segment's records
// are read unconditionally, and `ok` is false when the certificate fails or
// c had to be clamped, in which case frenet_relocate must run.
struct SegPick {
    float4 g1, g2;
    float2 g3;
    float len;
    int m;
    bool ok;
};

template <int MAXO>
__device__ __forceinline__ SegPick frenet_locate(int wlim, float px, float py, float ppred)
{
    using T = Tile<MAXO>;
    SegPick q;
    const int craw = __float2int_rd(ppred);
    const int c = min(max(craw, 0), wlim - 1);
    const float4 q0 = T::F0()[c], q1 = T::F0()[c + 1], q2 = T::F0()[c + 2];
    const bool b0 = past_bisector(q0, px, py), b1 = past_bisector(q1, px, py), b2 = past_bisector(q2, px, py);
    q.m = b1 ? c + 1 : c;
    q.len = b1 ? q1.w : q0.w;
    q.g1 = T::F1()[q.m]; q.g2 = T::F2()[q.m]; q.g3 = T::F3()[q.m];
    q.ok = b0 && !b2 && c == craw;
    return q;
}

// The rare case: the bisector walk from the predicted segment (or from the
// last one when the prediction is far off), records from the window or
// global memory.
template <int MAXO>
__device__ __noinline__ SegPick frenet_relocate(const BRScalars &S, float px, float py, float pos, float ppred, int &flag)
{
    SegPick q;
    const int c = __float2int_rd(ppred), r = __float2int_rd(pos);
    const int start = (c < r - kMaxMoves || c > r + kMaxMoves) ? r : c;
    q.m = bisector_walk<MAXO>(S, start, px, py, flag);
    segment_at<MAXO>(S, q.m, q.g1, q.g2, q.g3, q.len);
    q.ok = true;
    return q;
}

// Frenet of the state from its segment, and its continuous segment
// position np = m + t (the next prediction follows from it, frenet_advance).
__device__ __forceinline__ GeoPt frenet_point(const SegPick &q, float px, float py, float &np)
{
    const GeoPt f = frenet_eval(q.g1, q.g2, q.g3, q.len, px, py);
    np = (float)q.m + f.tc;
    return f;
}

// The next step's predicted position from the new position np.
__device__ __forceinline__ void frenet_advance(float np, float &pos, float &ppred)
{
    ppred = __fmaf_rn(2.f, np, -(pos + 0.5f));
    pos = np;
}


// Clipped control from a nominal control and a normal pair z (Pi_U).
__device__ __forceinline__ float2 sample_control(const sgtp_params &p, float2 ubar, float2 z)
{
    const float a = fminf(fmaxf(__fmaf_rn(p.sigma_a, z.x, ubar.x), p.a_min), p.a_max);
    const float d = fminf(fmaxf(__fmaf_rn(p.sigma_delta, z.y, ubar.y), -p.delta_max), p.delta_max);
    return make_float2(a, d);
}

// Clipped control from a per-step distribution d = (mean a, mean delta,
// sigma a, sigma delta); for the plain sampler d = (U-bar, sigma_a,
// sigma_delta) and the result equals sample_control's.
__device__ __forceinline__ float2 sample_control_d(const sgtp_params &p, float4 d, float2 z)
{
    const float a = fminf(fmaxf(__fmaf_rn(d.z, z.x, d.x), p.a_min), p.a_max);
    const float e = fminf(fmaxf(__fmaf_rn(d.w, z.y, d.y), -p.delta_max), p.delta_max);
    return make_float2(a, e);
}

// Stream bit of the noise counter: 1 for proposal samples.
__device__ __forceinline__ unsigned stream_bit_of(unsigned k, int K_prop) { return k < (unsigned)K_prop ? 0x80000000u : 0u; }

// One forward-Euler step of the kinematic bicycle (rear-axle reference,
// steering input, speed clamp), every right-hand side at the old state.  The
// heading is used as given (a rollout keeps it near (-pi, pi], see
// heading_split); bicycle_step_wrap wraps it first.
__device__ __forceinline__ void bicycle_step(const sgtp_params &p, float &x, float &y, float &psi, float &v, float a,
                                             float delta)
{
    const float sn = sin_ftz(psi), cs = cos_ftz(psi);
    const float sd = sin_ftz(delta), cd = cos_ftz(delta);
    const float dv = __fmul_rn(p.dt, v);
    const float x1 = __fmaf_rn(dv, cs, x);
    const float y1 = __fmaf_rn(dv, sn, y);
    const float psi1 = psi + __fmul_rn(__fmul_rn(dv, sd), rcp_ftz(__fmul_rn(cd, p.wheelbase)));
    const float v1 = fminf(fmaxf(__fmaf_rn(p.dt, a, v), p.v_min), p.v_max);
    x = x1; y = y1; psi = psi1; v = v1;
}

// bicycle_step for a heading of any size (the closed-loop plant).
__device__ __forceinline__ void bicycle_step_wrap(const sgtp_params &p, float &x, float &y, float &psi, float &v,
                                                  float a, float delta)
{
    const float pw = wrap_angle(psi);
    const float sn = sin_ftz(pw), cs = cos_ftz(pw);
    const float sd = sin_ftz(delta), cd = cos_ftz(delta);
    const float dv = __fmul_rn(p.dt, v);
    const float x1 = __fmaf_rn(dv, cs, x);
    const float y1 = __fmaf_rn(dv, sn, y);
    const float psi1 = psi + __fmul_rn(__fmul_rn(dv, sd), rcp_ftz(__fmul_rn(cd, p.wheelbase)));
    const float v1 = fminf(fmaxf(__fmaf_rn(p.dt, a, v), p.v_min), p.v_max);
    x = x1; y = y1; psi = psi1; v = v1;
}

// bicycle_step with the steering terms sin(delta) and 1/(cos(delta) L)
// computed beforehand (same instructions, so the same bits): the
// sequential rollout of a fixed control sequence then carries only the
// state recursion.
__device__ __forceinline__ void bicycle_step_pre(const sgtp_params &p, float &x, float &y, float &psi, float &v, float a,
                                                 float2 steer)
{
    const float sn = sin_ftz(psi), cs = cos_ftz(psi);
    const float dv = __fmul_rn(p.dt, v);
    const float x1 = __fmaf_rn(dv, cs, x);
    const float y1 = __fmaf_rn(dv, sn, y);
    const float psi1 = psi + __fmul_rn(__fmul_rn(dv, steer.x), steer.y);
    const float v1 = fminf(fmaxf(__fmaf_rn(p.dt, a, v), p.v_min), p.v_max);
    x = x1; y = y1; psi = psi1; v = v1;
}

__device__ __forceinline__ float2 steer_terms(const sgtp_params &p, float delta)
{
    return make_float2(sin_ftz(delta), rcp_ftz(__fmul_rn(cos_ftz(delta), p.wheelbase)));
}

// Normal pairs of candidate k at steps 2m and 2m+1 (one Philox block).
// The round keys are a kernel parameter (constant-bank operands).
__device__ __forceinline__ void noise_pair(const BRScalars &S, const RoundKeys &rk, unsigned k, unsigned sbit, int m,
                                           float2 &z0, float2 &z1)
{
    const uint4 w = philox4x32_10_rk(make_uint4(k, (unsigned)m | sbit, S.ctr_agent_round, S.ctr_race), rk);
    z0 = box_muller(w.x, w.y);
    z1 = box_muller(w.z, w.w);
}

// Running sums of the tracking cost (Eq. ctrack) per component: squared
// state errors (x, y, psi, v) over tau = 1..H, squared controls over
// tau = 0..H-1 and squared control differences over tau = 1..H-1; the
// weights Q, R, S multiply them once per candidate.
struct TrackSums {
    float ex, ey, epsi, ev, ua, ud, da, dd;
};

template <int MAXO>
struct SampleState {
    float x, y, psi, v;
    float a_prev, d_prev;
    float s;          // progress, unwrapped relative to s_t
    float pos, ppred; // continuous segment position and the next step's prediction
    TrackSums c;
    float rho_bd, d_tail;
    float g2[MAXO];
};

template <int MAXO>
__device__ __forceinline__ void sample_init(SampleState<MAXO> &St, const BRScalars &S)
{
    St.x = S.x0.x; St.y = S.x0.y; St.psi = S.psi0; St.v = S.x0.w;
    St.a_prev = 0.f; St.d_prev = 0.f;
    St.s = S.s_t;
    St.pos = S.pos0; St.ppred = S.ppred0;
    St.c = TrackSums{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    St.rho_bd = __int_as_float(0x7f800000);
    St.d_tail = 0.f;
#pragma unroll
    for (int o = 0; o < MAXO; ++o) St.g2[o] = __int_as_float(0x7f800000);
}

// Pieces of one rollout step.

// control cost terms, tau = 0..H-1, and smoothness terms, tau = 1..H-1 (Eq. ctrack)
__device__ __forceinline__ void step_control_cost(TrackSums &c, float &a_prev, float &d_prev, float2 u, int tau)
{
    c.ua = __fmaf_rn(u.x, u.x, c.ua);
    c.ud = __fmaf_rn(u.y, u.y, c.ud);
    if (tau > 0) {
        const float da = u.x - a_prev, dd = u.y - d_prev;
        c.da = __fmaf_rn(da, da, c.da);
        c.dd = __fmaf_rn(dd, dd, c.dd);
    }
    a_prev = u.x; d_prev = u.y;
}

// tracking terms at the new state, tau = 1..H (Eq. ctrack), heading error wrapped
__device__ __forceinline__ void step_tracking_cost(TrackSums &c, float x, float y, float psi, float v, float4 r)
{
    const float ex = x - r.x, ey = y - r.y, ep = wrap_angle(psi - r.z), ev = v - r.w;
    c.ex = __fmaf_rn(ex, ex, c.ex);
    c.ey = __fmaf_rn(ey, ey, c.ey);
    c.epsi = __fmaf_rn(ep, ep, c.epsi);
    c.ev = __fmaf_rn(ev, ev, c.ev);
}

// c_track from the running sums
__device__ __forceinline__ float track_cost(const sgtp_params &p, const TrackSums &c)
{
    float t = __fmul_rn(p.Q[0], c.ex);
    t = __fmaf_rn(p.Q[1], c.ey, t);
    t = __fmaf_rn(p.Q[2], c.epsi, t);
    t = __fmaf_rn(p.Q[3], c.ev, t);
    t = __fmaf_rn(p.R[0], c.ua, t);
    t = __fmaf_rn(p.R[1], c.ud, t);
    t = __fmaf_rn(p.S[0], c.da, t);
    return __fmaf_rn(p.S[1], c.dd, t);
}

// time-aligned distances to opponents [2 Q0, 2 Q1) of one step (Eq. Dmin),
// two at a time, and to the odd last one when ODD
template <int Q0, int Q1, bool ODD, int MAXO>
__device__ __forceinline__ void step_opponents(float *g2, float x, float y, const float4 *row)
{
    const f2p X = pk(x, x), Y = pk(y, y);
#pragma unroll
    for (int q = Q0; q < Q1; ++q) {
        const float4 o = row[q];
        const f2p dx = sub2(X, pk(o.x, o.y));
        const f2p dy = sub2(Y, pk(o.z, o.w));
        const float2 d2 = upk(fma2(dx, dx, mul2(dy, dy)));
        g2[2 * q] = fminf(g2[2 * q], d2.x);
        g2[2 * q + 1] = fminf(g2[2 * q + 1], d2.y);
    }
    if (ODD && (MAXO & 1)) {
        // the odd last opponent alone: the same operations on one lane
        const float4 o = row[MAXO / 2];
        const float dx = __fsub_rn(x, o.x), dy = __fsub_rn(y, o.z);
        const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        g2[MAXO - 1] = fminf(g2[MAXO - 1], d2);
    }
}

// Advance NI candidates (one thread's) by one step tau with controls u:
// control costs, the bicycle step, Frenet of the new states with their
// boundary clearance (Sec. III-B, widths at the foot point) and tail
// offsets, tracking costs, opponent distances; optional outputs (NI = 1).
// The candidates' chains are independent, so their instructions interleave.
template <int MAXO, int NI, bool OUT>
__device__ __forceinline__ void sample_steps(SampleState<MAXO> (&St)[NI], const BRScalars &S, const sgtp_params &p,
                                             int tau, int tail0, int wlim, const float2 (&u)[NI], int &flag,
                                             float *st_out, float *fr_out)
{
    using T = Tile<MAXO>;
    // each state's Frenet point from its predicted segment right away; only
    // the point (not the segment's records) waits for the rare relocation
    GeoPt f[NI];
    float np[NI];
    bool ok[NI];
    bool miss = false;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        step_control_cost(St[i].c, St[i].a_prev, St[i].d_prev, u[i], tau);
        bicycle_step(p, St[i].x, St[i].y, St[i].psi, St[i].v, u[i].x, u[i].y);
        const SegPick q = frenet_locate<MAXO>(wlim, St[i].x, St[i].y, St[i].ppred);
        f[i] = frenet_point(q, St[i].x, St[i].y, np[i]);
        ok[i] = q.ok;
        miss = miss || !q.ok;
    }
    if (__any_sync(__activemask(), miss)) {
#pragma unroll
        for (int i = 0; i < NI; ++i)
            if (!ok[i]) {
                const SegPick q = frenet_relocate<MAXO>(S, St[i].x, St[i].y, St[i].pos, St[i].ppred, flag);
                f[i] = frenet_point(q, St[i].x, St[i].y, np[i]);
            }
    }
    const int st = tau + 1;
    const float4 r = T::ref()[st];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        frenet_advance(np[i], St[i].pos, St[i].ppred);
        St[i].s = f[i].s;
        St[i].rho_bd = fminf(St[i].rho_bd, f[i].rho);
        if (st > tail0) St[i].d_tail = St[i].d_tail + f[i].d;
        step_tracking_cost(St[i].c, St[i].x, St[i].y, St[i].psi, St[i].v, r);
        step_opponents<0, MAXO / 2, true, MAXO>(St[i].g2, St[i].x, St[i].y, T::opp() + tau * BRTile<MAXO>::NP);
        if (OUT) {
            if (st_out) {
                st_out[4 * st + 0] = St[i].x; st_out[4 * st + 1] = St[i].y;
                st_out[4 * st + 2] = St[i].psi + S.psi_off; st_out[4 * st + 3] = St[i].v;
            }
            if (fr_out) { fr_out[2 * st] = St[i].s; fr_out[2 * st + 1] = f[i].d; }
        }
    }
}

struct SampleResult {
    float cost, viol;
    bool feasible;
};

// Terminal game cost per opponent (Eqs. c_contest, c_long, c_block,
// c_safety), total cost (Eq. allc), feasibility and violation (Sec. III-B).
template <int MAXO>
__device__ __forceinline__ SampleResult finish_terms(float c_track, float s, float rho_bd, float d_tail, const float *g2,
                                                     const BRScalars &S, const sgtp_params &p, bool game_on)
{
    using T = Tile<MAXO>;
    const float dbar_i = __fdiv_rn(d_tail, (float)S.n_tail);
    const float prog_i = __fsub_rn(s, S.s_t);
    float c_game = 0.f;
    float rho_obs = __int_as_float(0x7f800000);
#pragma unroll
    for (int o = 0; o < MAXO; ++o) {
        if (o < S.n_opp) {
            // every operation explicitly rounded (no fused contraction left
            // to the compiler), so that all builds give the same bits
            const float4 os = T::osum()[o];          // ds_t, alpha, gamma, prog_j
            const float ds_H = __fadd_rn(os.x, __fsub_rn(prog_i, os.w));
            const float c_contest = fabsf(ds_H) < p.s_contest ? -p.w_contest : 0.f;
            const float c_long = __fmul_rn(__fmul_rn(-p.w_long, os.y), ds_H);
            const float c_block =
                os.z != 0.f ? __fdiv_rn(-os.z, __fadd_rn(1.f, fabsf(__fsub_rn(dbar_i, T::odbar()[o])))) : 0.f;
            const float g = sqrtf(g2[o]);
            const float sh = fmaxf(0.f, __fsub_rn(p.g_safe, g));
            const float c_safety = __fmul_rn(__fmul_rn(p.w_safety, sh), sh);
            c_game = __fadd_rn(c_game, __fadd_rn(__fadd_rn(__fadd_rn(c_contest, c_long), c_block), c_safety));
            rho_obs = fminf(rho_obs, g);
        }
    }
    SampleResult r;
    r.cost = game_on ? __fmaf_rn(p.w_game, c_game, c_track) : c_track;
    const bool b = rho_bd >= p.m_bd;
    const bool ob = rho_obs >= p.d_col;
    r.feasible = b && ob;
    r.viol = __fadd_rn(fmaxf(0.f, __fsub_rn(p.m_bd, rho_bd)), fmaxf(0.f, __fsub_rn(p.d_col, rho_obs)));
    return r;
}

template <int MAXO>
__device__ __forceinline__ SampleResult sample_finish(const SampleState<MAXO> &St, const BRScalars &S,
                                                      const sgtp_params &p, bool game_on)
{
    return finish_terms<MAXO>(track_cost(p, St.c), St.s, St.rho_bd, St.d_tail, St.g2, S, p, game_on);
}

// NI full candidates k[0..NI) in one thread: noise, controls, rollout,
// finish.  Optional outputs are written when OUT (NI = 1; states (T+1)x4,
// frenet (T+1)x2, controls Tx2).
template <int MAXO, int NI, bool OUT>
__device__ __forceinline__ void run_candidates(const BRScalars &S, const sgtp_params &p, const RoundKeys &rk,
                                               const unsigned (&k)[NI], bool game_on, int &flag,
                                               SampleResult (&res)[NI], float *st_out, float *fr_out, float *u_out)
{
    using T = Tile<MAXO>;
    static_assert(!OUT || NI == 1, "per-candidate outputs take one candidate per thread");
    SampleState<MAXO> St[NI];
    unsigned sbit[NI];
    const float4 *dist[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        sample_init(St[i], S);
        const bool prop = k[i] < (unsigned)S.K_prop;
        sbit[i] = prop ? 0x80000000u : S.stream_bit;
        dist[i] = T::dist() + (prop ? SGTP_MAX_T : 0);
    }
    if (OUT) {
        if (st_out) { st_out[0] = S.x0.x; st_out[1] = S.x0.y; st_out[2] = S.x0.z; st_out[3] = S.x0.w; }
        if (fr_out) { fr_out[0] = S.s_t; fr_out[1] = S.d_t; }
    }
    const int Tn = S.T, tail0 = S.T - S.n_tail, wlim = S.Wn - 2;
    for (int m = 0; 2 * m < Tn; ++m) {
        float2 z0[NI], z1[NI], u[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) noise_pair(S, rk, k[i], sbit[i], m, z0[i], z1[i]);
        const int t0 = 2 * m;
#pragma unroll
        for (int i = 0; i < NI; ++i) u[i] = sample_control_d(p, dist[i][t0], z0[i]);
        if (OUT && u_out) { u_out[2 * t0] = u[0].x; u_out[2 * t0 + 1] = u[0].y; }
        sample_steps<MAXO, NI, OUT>(St, S, p, t0, tail0, wlim, u, flag, st_out, fr_out);
        if (t0 + 1 < Tn) {
#pragma unroll
            for (int i = 0; i < NI; ++i) u[i] = sample_control_d(p, dist[i][t0 + 1], z1[i]);
            if (OUT && u_out) { u_out[2 * t0 + 2] = u[0].x; u_out[2 * t0 + 3] = u[0].y; }
            sample_steps<MAXO, NI, OUT>(St, S, p, t0 + 1, tail0, wlim, u, flag, st_out, fr_out);
        }
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) res[i] = sample_finish(St[i], S, p, game_on);
}

// One full candidate per thread.
template <int MAXO, bool OUT>
__device__ __forceinline__ SampleResult run_candidate(const BRScalars &S, const sgtp_params &p,
                                                      const RoundKeys &rk, unsigned k, bool game_on, int &flag,
                                                      float *st_out, float *fr_out, float *u_out)
{
    const unsigned kk[1] = {k};
    SampleResult r[1];
    run_candidates<MAXO, 1, OUT>(S, p, rk, kk, game_on, flag, r, st_out, fr_out, u_out);
    return r[0];
}

// Stage one best response's opponent positions into the pair layout:
// src(tau, o) gives opponent o's position at step tau = 1..T.  Absent slots
// hold a far-away point.  Cooperative over the CTA's threads.
template <int MAXO, typename F>
__device__ __forceinline__ void stage_opponents(int T, int n_opp, F src)
{
    constexpr int NP = BRTile<MAXO>::NP;
    float4 *dst = Tile<MAXO>::opp();
    for (int q = threadIdx.x; q < T * NP; q += blockDim.x) {
        const int tau = q / NP, pr = q - tau * NP;
        const int o0 = 2 * pr, o1 = 2 * pr + 1;
        const float2 p0 = o0 < n_opp ? src(tau + 1, o0) : make_float2(kFarAway, kFarAway);
        const float2 p1 = o1 < n_opp ? src(tau + 1, o1) : make_float2(kFarAway, kFarAway);
        dst[q] = make_float4(p0.x, p1.x, p0.y, p1.y);
    }
}

// Roll out the controls ctl()[0..T) from x0 cooperatively: warp 0 prepares
// the steering terms of every step (in the opponent area, which only the
// sample phase uses), then its thread 0 runs the bicycle recurrence (the
// same arithmetic as the sample loop, so the states are bit-identical to the
// evaluated candidate's) into st(); then every thread projects one state
// onto the track by the bisector walk from a guess (the signed chord from
// x0 in segment lengths), which reaches the sample loop's segment; progress
// comes out unwrapped relative to s_t.  Outputs (any may be NULL):
// positions (T+1), states twice (T+1)x4, and the prediction summary
// (progress gain s_H - s_t, tail-mean offset); tan_out (T+1, entry 0
// unused) receives the unit direction of each state's segment, the
// longitudinal axis of a perturbed prediction.  Uses the tile's window,
// which must be staged for x0's segment j0.  All threads of the CTA must
// call it.
template <int MAXO>
__device__ void roll_cooperative(const sgtp_params &p, float4 x0, float s_t, int j0, int T, int n_tail,
                                 float2 *pos_out, float *xi_a, float *xi_b, float2 *summ_out, int &flag,
                                 float2 *tan_out = nullptr)
{
    using Tl = Tile<MAXO>;
    const BRScalars &S = Tl::sc();
    float4 *st = Tl::st();
    float2 *fr = Tl::fr();
    float2 *steer = (float2 *)Tl::opp();
    if (threadIdx.x < 32) {
        for (int q = threadIdx.x; q < T; q += 32) steer[q] = steer_terms(p, Tl::ctl()[q].y);
        __syncwarp();
        if (threadIdx.x == 0) {
            const float2 h = heading_split(x0.z);
            float x = x0.x, y = x0.y, psi = h.x, v = x0.w;
            st[0] = x0;
#pragma unroll 4
            for (int tau = 0; tau < T; ++tau) {
                bicycle_step_pre(p, x, y, psi, v, Tl::ctl()[tau].x, steer[tau]);
                st[tau + 1] = make_float4(x, y, psi + h.y, v);
            }
        }
    }
    __syncthreads();
    const int r0 = wrap_index(j0 - S.w0, S.tv.N);
    const float4 b0 = __ldg(S.tv.B + j0);
    for (int q = threadIdx.x; q < T; q += blockDim.x) {
        const float4 v = st[q + 1];
        const int guess = r0 + chord_guess(v.x - x0.x, v.y - x0.y, b0, 4 * kWinTile);
        const int m = bisector_walk<MAXO>(S, guess, v.x, v.y, flag);
        float4 g1, g2;
        float2 g3;
        float len;
        segment_at<MAXO>(S, m, g1, g2, g3, len);
        const GeoPt f = frenet_eval(g1, g2, g3, len, v.x, v.y);
        if (tan_out) tan_out[q + 1] = make_float2(g1.x, g1.y);
        fr[q] = make_float2(f.s, f.d);
    }
    __syncthreads();
    if (threadIdx.x == 0 && summ_out) {
        float dsum = 0.f;
        for (int tau = T - n_tail; tau < T; ++tau) dsum = dsum + fr[tau].y;
        *summ_out = make_float2(fr[T - 1].x - s_t, dsum / (float)n_tail);
    }
    for (int q = threadIdx.x; q <= T; q += blockDim.x) {
        const float4 v = st[q];
        if (pos_out) pos_out[q] = make_float2(v.x, v.y);
        if (xi_a) ((float4 *)xi_a)[q] = v;
        if (xi_b) ((float4 *)xi_b)[q] = v;
    }
}

}  // namespace sgtp
