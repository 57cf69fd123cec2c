// sgtp_sim.cu -- closed-loop race simulation on the batch layout: every race
// of an sgtp_batch is one trial that re-plans every control period.  After a
// planning call, sgtp_sim_step applies the first n_apply control steps of
// each vehicle's plan (its controls, or pure pursuit on its trajectory),
// steps every vehicle with the planner's kinematic bicycle, projects each one
// on the globally nearest raceline segment (Sec. II), checks the ego's
// contacts and keeps the sums behind the trial metrics of Sec. IV-C
// (progress gains for Wins and FPR, duration, close-interaction segments for
// CSD, ego speed, control smoothness for MCS).
//
// One CTA of 256 threads per trial: thread i < n_v steps vehicle i, warp w
// projects vehicles w, w + 8 (brute force over the track, lowest index on
// ties), thread 0 updates the trial record.
#include <cmath>

#include "sgtp_batch.hpp"
#include "sgtp_host.hpp"
#include "sgtp_rollout.cuh"

using namespace sgtp;

namespace {

struct SimArgs {
    const RaceDev *races;
    const TrackDesc *tdesc;
    const float4 *A, *B, *W, *C;
    const float *S;
    sgtp_params p;
    sgtp_sim_params sp;
    float *X;
    float *U;
    const float *xi;
    sgtp_sim_race *st;
};

__device__ __forceinline__ TrackView sim_track(const SimArgs &a, int id)
{
    const TrackDesc d = a.tdesc[id];
    TrackView v;
    v.A = a.A + d.offset; v.B = a.B + d.offset; v.W = a.W + d.offset; v.S = a.S + d.offset;
    v.C = a.C + d.offset;
    v.N = d.N; v.L = d.L;
    return v;
}

// Projection on the globally nearest segment by one warp (every lane gets it).
__device__ __forceinline__ FrenetPt project_warp(const TrackView &tv, float px, float py)
{
    const int j = nearest_segment_warp(tv, px, py);
    return frenet_at(tv, j, px, py);
}

// Pure pursuit toward the planned position `preview` steps after substep m
// of vehicle i's plan; the acceleration tracks the planned speed of the
// next step.  Clipped to the admissible controls.
__device__ __forceinline__ float2 pure_pursuit(const SimArgs &a, const RaceDev &R, int i, int m, float4 x)
{
    const float4 *plan = (const float4 *)(a.xi + R.xi_off + (size_t)i * (R.T + 1) * 4);
    const float4 tgt = plan[min(m + a.sp.pp_preview, R.T)];
    const float dx = tgt.x - x.x, dy = tgt.y - x.y;
    const float ld = sqrtf(dx * dx + dy * dy);
    float delta = 0.f;
    if (ld > 1e-6f) {
        const float alpha = atan2f(dy, dx) - x.z;
        delta = atanf(2.f * a.p.wheelbase * sinf(alpha) / ld);
    }
    delta = fminf(fmaxf(delta, -a.p.delta_max), a.p.delta_max);
    const float vp = plan[min(m + 1, R.T)].w;
    const float acc = fminf(fmaxf((vp - x.w) / a.p.dt, a.p.a_min), a.p.a_max);
    return make_float2(acc, delta);
}

__global__ void __launch_bounds__(256) sim_reset_kernel(SimArgs a)
{
    const RaceDev R = a.races[blockIdx.x];
    sgtp_sim_race *S = a.st + blockIdx.x;
    const TrackView tv = sim_track(a, R.track_id);
    __shared__ float s_sh[SGTP_MAX_AGENTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int i = warp; i < R.n_v; i += nwarps) {
        const float *x = a.X + 4 * (size_t)(R.agent_off + i);
        const FrenetPt f = project_warp(tv, x[0], x[1]);
        if (lane == 0) { s_sh[i] = f.s; S->s_raw[i] = f.s; S->d[i] = f.d; }
    }
    __syncthreads();
    const int i = threadIdx.x;
    if (i < SGTP_MAX_AGENTS) {
        S->progress[i] = 0.f;
        S->close_run[i] = 0;
        S->rel0[i] = i < R.n_v ? wrap_len(s_sh[i] - s_sh[R.ego], tv.L, 1.0f / tv.L) : 0.f;
        if (i >= R.n_v) { S->s_raw[i] = 0.f; S->d[i] = 0.f; }
    }
    if (i == 0) {
        S->alive = 1; S->steps = 0; S->ego_collision = 0;
        S->close_segments = 0; S->close_steps = 0;
        S->ego_speed_sum = 0.f; S->ego_du2_sum = 0.f;
        S->u_prev[0] = 0.f; S->u_prev[1] = 0.f;
        S->pad0 = 0; S->pad1[0] = 0; S->pad1[1] = 0;
    }
}

__global__ void __launch_bounds__(256) sim_step_kernel(SimArgs a)
{
    const RaceDev R = a.races[blockIdx.x];
    sgtp_sim_race *S = a.st + blockIdx.x;
    if (!S->alive) return;
    const TrackView tv = sim_track(a, R.track_id);
    const float invL = 1.0f / tv.L;
    const int n_v = R.n_v, T = R.T, ego = R.ego;
    __shared__ float4 xs[SGTP_MAX_AGENTS];
    __shared__ float2 fs[SGTP_MAX_AGENTS];     // (s, d) after the substep
    __shared__ float2 fw[SGTP_MAX_AGENTS];     // (w^L, w^R) there
    __shared__ int alive_sh, applied_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    if (tid < n_v) {
        const float *x = a.X + 4 * (size_t)(R.agent_off + tid);
        xs[tid] = make_float4(x[0], x[1], x[2], x[3]);
    }
    if (tid == 0) { alive_sh = 1; applied_sh = 0; }
    __syncthreads();
    for (int m = 0; m < a.sp.n_apply; ++m) {
        if (!alive_sh) break;
        if (tid < n_v) {
            float4 x = xs[tid];
            float2 u;
            if (a.sp.tracker == SGTP_TRACK_PURE_PURSUIT) {
                u = pure_pursuit(a, R, tid, m, x);
            } else {
                const float *Ui = a.U + R.u_off + (size_t)tid * T * 2;
                u = make_float2(Ui[2 * m], Ui[2 * m + 1]);
            }
            if (tid == ego) {
                if (S->steps > 0) {
                    const float da = u.x - S->u_prev[0], dd = u.y - S->u_prev[1];
                    S->ego_du2_sum += da * da + dd * dd;
                }
                S->u_prev[0] = u.x;
                S->u_prev[1] = u.y;
            }
            bicycle_step_wrap(a.p, x.x, x.y, x.z, x.w, u.x, u.y);
            xs[tid] = x;
            if (tid == ego) S->ego_speed_sum += x.w;
        }
        __syncthreads();
        for (int i = warp; i < n_v; i += nwarps) {
            const float4 x = xs[i];
            const FrenetPt f = project_warp(tv, x.x, x.y);
            if (lane == 0) { fs[i] = make_float2(f.s, f.d); fw[i] = make_float2(f.wl, f.wr); }
        }
        __syncthreads();
        if (tid == 0) {
            for (int i = 0; i < n_v; ++i) {
                S->progress[i] += wrap_len(fs[i].x - S->s_raw[i], tv.L, invL);
                S->s_raw[i] = fs[i].x;
                S->d[i] = fs[i].y;
            }
            const int steps = S->steps + 1;
            S->steps = steps;
            int coll = 0;
            const float4 xe = xs[ego];
            for (int j = 0; j < n_v; ++j) {
                if (j == ego) continue;
                const float dx = xs[j].x - xe.x, dy = xs[j].y - xe.y;
                if (dx * dx + dy * dy < a.sp.contact_dist * a.sp.contact_dist) coll = 1;
            }
            if (!coll) {
                const float clear = fminf(fw[ego].y + fs[ego].y, fw[ego].x - fs[ego].y);
                if (clear < a.sp.wall_margin) coll = 2;
            }
            for (int j = 0; j < n_v; ++j) {
                if (j == ego) continue;
                const float ds = wrap_len(fs[ego].x - fs[j].x, tv.L, invL);
                const float dd = fs[ego].y - fs[j].y;
                if (fabsf(ds) < a.sp.close_ds && fabsf(dd) < a.sp.close_dd) {
                    S->close_run[j] += 1;
                } else if (S->close_run[j] > 0) {
                    S->close_segments += 1;
                    S->close_steps += S->close_run[j];
                    S->close_run[j] = 0;
                }
            }
            if (coll || steps >= a.sp.max_steps) {
                if (coll) S->ego_collision = coll;
                S->alive = 0;
                for (int j = 0; j < n_v; ++j) {
                    if (S->close_run[j] > 0) {
                        S->close_segments += 1;
                        S->close_steps += S->close_run[j];
                        S->close_run[j] = 0;
                    }
                }
                alive_sh = 0;
            }
            applied_sh = m + 1;
        }
        __syncthreads();
    }
    if (tid < n_v) {
        float *x = a.X + 4 * (size_t)(R.agent_off + tid);
        const float4 v = xs[tid];
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    // warm start shifted by the steps applied, the last control repeated; a
    // warp per vehicle moves chunks of 32 steps forward (reads of a chunk
    // lie past every earlier write)
    const int n = applied_sh;
    for (int i = warp; i < n_v; i += nwarps) {
        float2 *Ui = (float2 *)(a.U + R.u_off + (size_t)i * T * 2);
        const float2 last = Ui[T - 1];
        __syncwarp();
        for (int base = 0; base < T; base += 32) {
            const int tau = base + lane;
            float2 v = last;
            if (tau + n < T) v = Ui[tau + n];
            __syncwarp();
            if (tau < T) Ui[tau] = v;
            __syncwarp();
        }
    }
}

sgtp_status fill_args(SimArgs &a, const sgtp_batch *b)
{
    SGTP_CHECK(b != nullptr && b->trk != nullptr, "batch is NULL");
    const sgtp_track *t = b->trk;
    a.races = b->races_dev;
    a.tdesc = t->desc_dev;
    a.A = t->A; a.B = t->B; a.W = t->W; a.C = t->C; a.S = t->S;
    return SGTP_OK;
}

}  // namespace

extern "C" sgtp_status sgtp_sim_reset(const sgtp_batch *b, const float *X, sgtp_sim_race *state, void *stream)
{
    SimArgs a{};
    sgtp_status st = fill_args(a, b);
    if (st) return st;
    SGTP_CHECK(X != nullptr && state != nullptr, "NULL array");
    SGTP_CHECK(aligned16(state), "state must be 16-byte aligned");
    a.X = const_cast<float *>(X);
    a.st = state;
    sim_reset_kernel<<<b->n_races, 256, 0, (cudaStream_t)stream>>>(a);
    SGTP_CUDA(cudaGetLastError());
    count_launch();
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_sim_step(const sgtp_batch *b, const sgtp_params *p, const sgtp_sim_params *sp,
                                     float *X_io, float *U_io, const float *xi, sgtp_sim_race *state, void *stream)
{
    SimArgs a{};
    sgtp_status st = fill_args(a, b);
    if (st) return st;
    st = check_params(p);
    if (st) return st;
    SGTP_CHECK(sp != nullptr, "sim params are NULL");
    SGTP_CHECK(X_io != nullptr && U_io != nullptr && state != nullptr, "NULL array");
    SGTP_CHECK(aligned16(state), "state must be 16-byte aligned");
    SGTP_CHECK(sp->n_apply >= 1 && sp->n_apply <= b->minT, "n_apply=%d out of range [1, %d]", sp->n_apply,
               b->minT);
    SGTP_CHECK(sp->max_steps >= 1, "max_steps must be >= 1");
    SGTP_CHECK(sp->tracker == SGTP_TRACK_CONTROLS || sp->tracker == SGTP_TRACK_PURE_PURSUIT, "unknown tracker %d",
               sp->tracker);
    SGTP_CHECK(sp->tracker != SGTP_TRACK_PURE_PURSUIT || (xi != nullptr && sp->pp_preview >= 1),
               "pure pursuit needs xi and pp_preview >= 1");
    SGTP_CHECK(std::isfinite(sp->contact_dist) && sp->contact_dist >= 0.f && std::isfinite(sp->wall_margin) &&
                   std::isfinite(sp->close_ds) && sp->close_ds >= 0.f && std::isfinite(sp->close_dd) &&
                   sp->close_dd >= 0.f,
               "sim distances must be finite (and >= 0 except wall_margin)");
    a.p = *p;
    a.sp = *sp;
    a.X = X_io;
    a.U = U_io;
    a.xi = xi;
    a.st = state;
    sim_step_kernel<<<b->n_races, 256, 0, (cudaStream_t)stream>>>(a);
    SGTP_CUDA(cudaGetLastError());
    count_launch();
    return SGTP_OK;
}
