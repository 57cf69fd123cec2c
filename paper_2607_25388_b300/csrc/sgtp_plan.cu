// sgtp_plan.cu -- the SGTP planning call (Alg. 1) as one persistent
// cooperative kernel, for one race or a batch of independent races.
//
// Phases of the kernel:
//   setup   : per vehicle, Frenet of x_{i,t} (global search), reference
//             trajectory (Sec. III-A), nominal rollout of the current U-bar
//             = the opponents' predictions for round 0 (then a grid
//             barrier);
//   proposal: with the learned proposal, per vehicle, features, network and
//             the per-step Gaussian of its next best response;
//   round r : every (race, vehicle, sample tile) item evaluates its samples
//             and folds their selection keys into the best response's key;
//   winner r: per vehicle, re-roll of the selected sample k*, warm start
//             U-bar <- U^(k*) (Alg. 1, update step), and the new prediction
//             (positions, progress gain, tail offset) for the next round.
// Rounds 0..L are Jacobi rounds over all vehicles (round 0 without the game
// term); round L+1 is the extra ego response.  Under the lock-step schedule
// a grid barrier separates the phases; under the queue schedule the items
// are claimed from one device counter and wait only for their own race's
// (or vehicle's) earlier items (see wait_count / signal_done).
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

#include "sgtp_batch.hpp"
#include "sgtp_host.hpp"
#include "sgtp_mlp.h"
#include "sgtp_rollout.cuh"

using namespace sgtp;

namespace {

struct AgentDev {
    float4 x0;
    float s_t, d_t;
    int j0, race;
    float t0;                 // segment parameter of x_{i,t}
    float pad[3];
};

struct PlanArgs {
    const TrackDesc *tdesc;
    const float4 *A, *B, *W, *C;
    const float *S;
    const float4 *G0, *G1, *G2;
    const float2 *G3;
    sgtp_params p;
    const RaceDev *races;     // NULL: single race `one`
    RaceDev one;
    int n_races, n_agents;
    int K, L;
    // per round kind ([0] Jacobi rounds, [1] the extra ego round): samples
    // each thread rolls out at once, samples per tile, tiles per best
    // response, work items (vehicles x tiles), and the items' total work
    // (batches: items weighted by their race's T; see RaceDev)
    int ni[2], tile[2], tiles[2], items[2];
    long long w[2];
    long long w_units_all, w_units_ego;   // total work per sample tile
    int maxT;
    const float *X0;
    float *U_io;
    const float *vref;
    uint2 key;
    RoundKeys rk;             // the key's Weyl schedule
    float *xi_out;
    int *k_star_out;
    float *xi_hist, *u_hist;
    long long xi_total, u_total;
    int *status;
    // workspace
    unsigned *bar;            // [0] count, [1] generation
    unsigned long long *keys; // per race: (L+1)*n_v + 1
    AgentDev *agents;
    float4 *ref;              // per vehicle: T+1
    float2 *pos[2];           // per vehicle: T+1 predicted positions
    float2 *summ[2];          // per vehicle: (progress gain, tail-mean d)
    int Wn, back;
    long long timeout_ns;
    int debug_flags;
    long long *trace;          // optional phase stamps (CTA 0)
    // learned proposal
    const __nv_bfloat16 *mlp_wb;   // BF16 parameters (NULL: plain sampler only)
    const float *mlp_wf;           // FP32 master parameters (biases)
    int K_prop;                    // proposal samples per best response
    float4 *prop;                  // per vehicle: maxT steps (mean a, mean delta, sigma a, sigma delta)
    float *feat_out;               // optional: (L+2) x n_agents x 64 features of each best response
    float4 *prop_out;              // optional: (L+2) x n_agents x maxT proposals of each best response
    // GA-IBR-MPPI (mppi_il > 0): path-integral update instead of selection
    float mppi_il;                 // 1 / lambda
    float *mppi_part;              // per vehicle x tile: m_t, sum w u (2T), sum w; stride 2 maxT + 2
    // perturbed opponent predictions (sig_lon or sig_lat > 0)
    float sig_lon, sig_lat;
    float2 *ptan[2];               // per vehicle: T+1 unit directions of the predictions' nearest segments
    // per-race round progression (queue != 0): after the setup, work items
    // are claimed from one queue in the order samples of round 0, winners of
    // round 0, samples of round 1, ...; a race moves to its next round as
    // soon as its own winners are in, never waiting for another race
    int queue;
    unsigned long long *qhead;     // next queue position to claim
    unsigned *wdone;               // per race: winner items completed
    unsigned *tdone;               // per vehicle: sample tiles completed (all rounds)
    unsigned *pdone;               // per vehicle: proposal items completed (learned proposal)
};

__device__ __forceinline__ void stamp(const PlanArgs &a, int i)
{
    if (a.trace && blockIdx.x == 0 && threadIdx.x == 0) a.trace[i] = (long long)global_ns();
}

__device__ __forceinline__ RaceDev get_race(const PlanArgs &a, int r) { return a.races ? a.races[r] : a.one; }

// Workspace written inside the launch by other CTAs is read through L2.
__device__ __forceinline__ AgentDev load_agent(const AgentDev *p)
{
    const float4 *q = (const float4 *)p;
    const float4 u = __ldcg(q), w = __ldcg(q + 1), z = __ldcg(q + 2);
    AgentDev A;
    A.x0 = u;
    A.s_t = w.x; A.d_t = w.y; A.j0 = __float_as_int(w.z); A.race = __float_as_int(w.w);
    A.t0 = z.x;
    return A;
}

__device__ __forceinline__ TrackView get_track(const PlanArgs &a, int id)
{
    const TrackDesc d = a.tdesc[id];
    TrackView v;
    v.A = a.A + d.offset; v.B = a.B + d.offset; v.W = a.W + d.offset; v.S = a.S + d.offset;
    v.C = a.C + d.offset;
    v.G0 = a.G0 + d.offset; v.G1 = a.G1 + d.offset; v.G2 = a.G2 + d.offset; v.G3 = a.G3 + d.offset;
    v.N = d.N; v.L = d.L;
    return v;
}

// last race r with field(r) <= x (races sorted by every prefix field)
template <typename F>
__device__ __forceinline__ int find_race(const PlanArgs &a, int x, F field)
{
    if (!a.races) return 0;
    int lo = 0, hi = a.n_races - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (field(a.races[mid]) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// First item of a round whose work starts at or after x (batches): the race
// holding x by its work prefix, then ceil((x - prefix) / T) items into it.
// Every item of a race weighs its horizon T, so that the CTAs' shares of a
// round, cut at equal work, take about equal time across races of
// different horizons.
__device__ __forceinline__ int first_item_at(const PlanArgs &a, long long x, bool extra)
{
    int lo = 0, hi = a.n_races - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long w = (extra ? a.races[mid].wcum_ego : a.races[mid].wcum_all) * a.tiles[extra];
        if (w <= x) lo = mid; else hi = mid - 1;
    }
    const RaceDev R = a.races[lo];
    const long long w0 = (extra ? R.wcum_ego : R.wcum_all) * a.tiles[extra];
    const long long n = (long long)(extra ? 1 : R.n_v) * a.tiles[extra];
    const long long k = (x - w0 + R.T - 1) / R.T;
    const long long first = (long long)(extra ? lo : R.agent_off) * a.tiles[extra];
    return (int)(first + (k < n ? k : n));
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_status(const int *p) { return *(const volatile int *)p; }

// Grid-wide barrier of a cooperative launch: one arrival counter that only
// grows (zeroed at launch).  Barrier e of the launch is passed once it reaches
// e x gridDim.x; arrival is an acquire-release add by each CTA's thread 0
// after the CTA's bar.sync, so the CTA's writes are visible to every CTA that
// passes.  Every wait has a limit: a CTA whose wait runs out records
// SGTP_E_TIMEOUT and returns false, and every other waiter stops as soon as
// it sees a fatal status.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits (thread 0, bounded by the launch's timeout) until the counter *p has
// reached `target`; every thread returns false when the wait ran out
// (SGTP_E_TIMEOUT recorded) or another CTA recorded a fatal status.  What the
// counter's producers wrote before their release is visible to the whole CTA
// afterwards (thread 0's acquire, then the CTA barrier).
__device__ bool wait_count(const PlanArgs &a, const unsigned *p, unsigned target)
{
    __shared__ int wc_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if ((int)(ld_acquire(p) - target) < 0) {
            const unsigned long long t0 = global_ns();
            while ((int)(ld_acquire(p) - target) < 0) {
                if (ld_status(a.status) & 0xff) { ok = 0; break; }
                if (global_ns() - t0 > (unsigned long long)a.timeout_ns) {
                    atomicOr(a.status, SGTP_E_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        wc_sh = ok;
    }
    __syncthreads();
    return wc_sh != 0;
}

// Marks one item done: the CTA's writes for it, then a release increment.
__device__ __forceinline__ void signal_done(unsigned *p)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_add_release(p, 1u);
    }
}

// Claims the next queue position for this CTA into q_sh (all threads; the
// position is CTA-uniform, so it lives in shared memory, not in registers
// across the sample loop).
__device__ __forceinline__ void claim_item(const PlanArgs &a, unsigned long long &q_sh)
{
    __syncthreads();
    if (threadIdx.x == 0) q_sh = atomicAdd(a.qhead, 1ull);
    __syncthreads();
}

__shared__ unsigned g_bar_epoch;      // barriers this CTA has entered (thread 0's count)

__device__ bool grid_barrier(const PlanArgs &a, bool skip_arrival)
{
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned *count = a.bar;
        const unsigned target = (g_bar_epoch += 1u) * gridDim.x;
        bool passed = false;
        if (!skip_arrival) passed = atom_add_acq_rel(count, 1u) + 1u == target;
        if (!passed) {
            const unsigned long long t0 = global_ns();
            while ((int)(ld_acquire(count) - target) < 0) {
                if (ld_status(a.status) & 0xff) break;
                if (global_ns() - t0 > (unsigned long long)a.timeout_ns) {
                    atomicOr(a.status, SGTP_E_TIMEOUT);
                    break;
                }
            }
        }
        ok_sh = (ld_status(a.status) & 0xff) == 0;
    }
    __syncthreads();
    return ok_sh != 0;
}

// The window in shared memory: its track (A array), first segment and the
// lap of the vehicle it was corrected for; g_win_fix asks the threads to run
// the lap correction once the copies have landed.
__shared__ const float4 *g_win_track;
__shared__ int g_win_w0, g_win_lap0, g_win_fix;

// The reference recursion's stretch of track in the tile's scratch area.
template <int MAXO>
__device__ __forceinline__ SegWindow stage_ref_window(const TrackView &tv, int j0, const float4 *&Cw)
{
    static_assert(kRefStretchBytes <= BRTile<MAXO>::kScrBytes, "reference stretch exceeds the scratch area");
    return stage_ref_stretch(tv, j0, Tile<MAXO>::scratch(), Cw);
}

// Stage the sample window of a vehicle whose state lies on segment j0
// (thread 0 issues the bulk copies and returns true; every thread then
// calls window_ready) and fill the tile scalars' window fields.  The window
// starts `back` segments behind j0 (rounded down to a multiple of 4), a
// function of j0 alone, so every CTA and every launch shape sees the same
// window for a vehicle; a window already in shared memory for the same
// track, start and lap is reused without a copy.
template <int MAXO>
__device__ __forceinline__ bool stage_vehicle_window(const PlanArgs &a, const TrackView &tv, int j0)
{
    using T = Tile<MAXO>;
    bool issued = false;
    if (threadIdx.x == 0) {
        BRScalars &S = T::sc();
        const int Wn = min(a.Wn, (tv.N + 3) & ~3);
        const int back = min(a.back, Wn / 4);
        S.tv = tv;
        S.Wn = Wn;
        S.invL = 1.0f / tv.L;
        S.w0 = window_start(j0, back, tv.N);
        S.r0 = wrap_index(j0 - S.w0, tv.N);
        S.lap0 = S.w0 + S.r0 >= tv.N ? 1 : 0;
        if (!(g_win_track == tv.A && g_win_w0 == S.w0 && g_win_lap0 == S.lap0)) {
            T::stage_window(tv, S.w0, Wn);
            g_win_track = tv.A;
            g_win_w0 = S.w0;
            g_win_lap0 = S.lap0;
            g_win_fix = window_wraps(S) ? 1 : 0;
            issued = true;
        }
    }
    return issued;
}

// Completes a staging: thread 0 waits (bounded) for the copies it issued,
// then every thread takes part in the lap correction when one is due.
// Returns false (on every thread) when the wait ran out.
template <int MAXO>
__device__ __forceinline__ bool window_ready(const PlanArgs &a, bool issued, unsigned &phase)
{
    using T = Tile<MAXO>;
    __shared__ int wok_sh;
    if (threadIdx.x == 0) {
        wok_sh = 1;
        if (issued) {
            if (!mbar_wait_bounded(T::bar(), phase, (unsigned long long)a.timeout_ns)) {
                atomicOr(a.status, SGTP_E_TIMEOUT);
                wok_sh = 0;
            }
            phase ^= 1u;
        }
    }
    __syncthreads();
    const bool ok = wok_sh != 0;
    if (g_win_fix) {
        if (ok) T::fix_laps(T::sc());
        __syncthreads();
        if (threadIdx.x == 0) g_win_fix = 0;
    }
    return ok;
}

// ---------------------------------------------------------------- learned proposal
// Features of vehicle i before a best response (layout in sgtp_mlp.h):
// Frenet-relative ego state, raceline curvature ahead, and the nine nearest
// opponents by |Delta s| (ties by index after rounding |Delta s| to mm).
// All threads of the CTA (at least 64); thread 0 writes the ego terms,
// threads 1..4 one curvature each, threads 32.. one opponent each (rank by
// counting), and the slots of absent opponents are zeroed.
// key_sh: SGTP_MAX_AGENTS floats of shared scratch.
__device__ void compute_features(const PlanArgs &a, const RaceDev &R, int i, int bin, bool game_on, float *f,
                                 float *key_sh)
{
    const TrackView tv = get_track(a, R.track_id);
    const int tid = threadIdx.x;
    const int n_opp = R.n_v - 1;
    const float invL = 1.0f / tv.L;
    const int jo = tid - 32;                 // opponent handled by this thread (vehicle index)
    const bool opp_thread = jo >= 0 && jo < R.n_v && jo != i;
    AgentDev A = load_agent(a.agents + R.agent_off + i);
    AgentDev B;
    float ds = 0.f;
    if (opp_thread) {
        B = load_agent(a.agents + R.agent_off + jo);
        ds = wrap_len(B.s_t - A.s_t, tv.L, invL);
        key_sh[jo] = floorf(fabsf(ds) * 1000.f);
    }
    if (tid == 0) {
        const float4 c0 = __ldg(tv.C + A.j0);
        const float e = wrap_angle(__fsub_rn(A.x0.z, __fmaf_rn(A.t0, c0.y, c0.x)));
        float sn, cs;
        sincosf(e, &sn, &cs);
        f[0] = A.d_t / 5.f;
        f[1] = sn;
        f[2] = cs;
        f[3] = A.x0.w / 60.f;
        f[62] = (float)n_opp / 9.f;
        f[63] = game_on ? 1.f : 0.f;
    } else if (tid <= 4) {
        // segment holding arc position s_i + ahead: jump by the local segment
        // length, then step to the segment whose [S_j, S_j+1) holds it
        const float ahead = tid == 1 ? 0.f : tid == 2 ? 20.f : tid == 3 ? 40.f : 80.f;
        const float tgt = A.s_t + ahead;
        const int N = tv.N;
        auto sj = [&](int j) {
            const int lap = j >= 0 ? j / N : -((-j + N - 1) / N);
            return __fmaf_rn((float)lap, tv.L, __ldg(tv.S + (j - lap * N)));
        };
        int j = A.j0 + (int)(ahead / __ldg(tv.B + A.j0).w);
        for (int it = 0; it < 4 * N && sj(j) > tgt; ++it) --j;
        for (int it = 0; it < 4 * N && sj(j + 1) <= tgt; ++it) ++j;
        const int jm = ((j % N) + N) % N;
        f[4 + tid - 1] = 100.f * __ldg(tv.C + jm).y / __ldg(tv.B + jm).w;
    }
    __syncthreads();
    if (opp_thread) {
        const float k = key_sh[jo];
        int rank = 0;
        for (int m = 0; m < R.n_v; ++m) {
            if (m == i || m == jo) continue;
            const float km = key_sh[m];
            rank += (km < k || (km == k && m < jo)) ? 1 : 0;
        }
        if (rank < 9) {
            const float prog = __ldcg(a.summ[bin] + R.agent_off + jo).x;
            const float horizon_gain = __fmul_rn(__fmul_rn(A.x0.w, (float)R.T), a.p.dt);
            float *o = f + 8 + 6 * rank;
            o[0] = 1.f;
            o[1] = ds / 40.f;
            o[2] = B.d_t / 5.f;
            o[3] = (B.x0.w - A.x0.w) / 10.f;
            o[4] = wrap_angle(B.x0.z - A.x0.z);
            o[5] = __fdiv_rn(__fsub_rn(prog, horizon_gain), 40.f);
        }
    }
    for (int q = tid; q < 9 * 6; q += blockDim.x)
        if (q / 6 >= n_opp) f[8 + q] = 0.f;
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const unsigned a[4], const unsigned b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One layer of the network for one input row on the tensor cores.  The row
// (BF16, K values) sits in shared memory and is row 0 of the mma's A tile;
// lanes of rows 1..15 feed zeros.  Weights come in the fragment order of
// sgtp_mlp.cu (per 8-column tile and 16-deep k-step, 32 lanes x {b0, b1}),
// so each warp's load is one coalesced 256-byte piece.  Each warp owns up
// to four tiles at once so that their loads are in flight together.  Output
// row 0 = act(acc + b): BF16 ReLU into `next`, or FP32 into `yout`.
__device__ void mlp_layer(const __nv_bfloat16 *act, const uint2 *frag, const float *bias, int N, int K,
                          __nv_bfloat16 *next, float *yout)
{
    constexpr int NT = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int ksteps = K >> 4, n_tiles = (N + 7) >> 3;
    const unsigned *act32 = (const unsigned *)act;
    for (int base = warp; base < n_tiles; base += nwarps * NT) {
        float acc[NT][4];
        const uint2 *fp[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int tile = min(base + j * nwarps, n_tiles - 1);
            fp[j] = frag + (size_t)tile * ksteps * 32 + lane;
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
        }
#pragma unroll 4
        for (int ks = 0; ks < ksteps; ++ks) {
            uint2 bv[NT];
#pragma unroll
            for (int j = 0; j < NT; ++j) bv[j] = __ldg(fp[j] + ks * 32);
            unsigned af[4] = {0u, 0u, 0u, 0u};
            if (g == 0) {
                af[0] = act32[ks * 8 + t];
                af[2] = act32[ks * 8 + 4 + t];
            }
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const unsigned bf[2] = {bv[j].x, bv[j].y};
                mma_bf16_16816(acc[j], af, bf);
            }
        }
        if (g == 0) {
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int tile = base + j * nwarps;
                if (tile >= n_tiles) continue;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = tile * 8 + 2 * t + q;
                    if (c >= N) continue;
                    const float v = acc[j][q] + bias[c];
                    if (next) next[c] = __float2bfloat16(fmaxf(v, 0.f));
                    else yout[c] = v;
                }
            }
        }
    }
}

// Proposal of vehicle i for its next best response: features, network, and
// the per-step Gaussian (mean = U-bar + sigma_plain * mu, a residual around
// the plain sampler's centre, sigma = sigma_plain * exp(clamp(logsig, -5,
// 2))).  All threads of the CTA; shared scratch at buf.
__device__ void proposal_for(const PlanArgs &a, const RaceDev &R, int i, int bin, bool game_on, int round,
                             unsigned char *buf)
{
    float *x = (float *)buf;                                    // 64 features
    float *y = x + 64;                                          // 4T outputs
    float *key_sh = y + 4 * SGTP_MAX_T;                         // SGTP_MAX_AGENTS keys
    __nv_bfloat16 *act0 = (__nv_bfloat16 *)(key_sh + SGTP_MAX_AGENTS);
    __nv_bfloat16 *act1 = act0 + SGTP_MLP_HIDDEN;
    const int ag = R.agent_off + i;
    compute_features(a, R, i, bin, game_on, x, key_sh);
    __syncthreads();
    if (a.feat_out && threadIdx.x < 64)
        a.feat_out[((size_t)round * a.n_agents + ag) * 64 + threadIdx.x] = x[threadIdx.x];
    if (!a.mlp_wb) return;
    if (threadIdx.x < 64) act0[threadIdx.x] = __float2bfloat16(x[threadIdx.x]);
    __syncthreads();
    const int T = R.T, OUT = 4 * T, H = SGTP_MLP_HIDDEN;
    long long off = 0, foff = 0;
    const __nv_bfloat16 *cur = act0;
    __nv_bfloat16 *nxt = act1;
    for (int l = 0; l < 4; ++l) {
        const int K = l == 0 ? SGTP_MLP_IN : H;
        const int N = l == 3 ? OUT : H;
        mlp_layer(cur, (const uint2 *)(a.mlp_wb + foff), a.mlp_wf + off + (long long)N * K, N, K,
                  l == 3 ? nullptr : nxt, y);
        off += (long long)N * K + N;
        foff += (long long)((N + 7) & ~7) * K;
        __syncthreads();
        const __nv_bfloat16 *t = cur; cur = nxt; nxt = (__nv_bfloat16 *)t;
    }
    float4 *dst = a.prop + (size_t)ag * a.maxT;
    const float *U = a.U_io + R.u_off + (size_t)i * T * 2;
    for (int q = threadIdx.x; q < T; q += blockDim.x) {
        const float la = fminf(fmaxf(y[2 * T + q], -5.f), 2.f);
        const float ld = fminf(fmaxf(y[3 * T + q], -5.f), 2.f);
        const float4 d = make_float4(__fmaf_rn(a.p.sigma_a, y[q], __ldcg(U + 2 * q)),
                                     __fmaf_rn(a.p.sigma_delta, y[T + q], __ldcg(U + 2 * q + 1)),
                                     a.p.sigma_a * expf(la), a.p.sigma_delta * expf(ld));
        dst[q] = d;
        if (a.prop_out) a.prop_out[((size_t)round * a.n_agents + ag) * a.maxT + q] = d;
    }
}

// ---------------------------------------------------------------- perturbed predictions
// Gaussian pair of step tau (1..T) of opponent jv's prediction as seen by
// the best response with counter word ar = observer | round << 16: counter
// (2^30 | jv, (tau-1) >> 1, ar, race), a word no sample uses (k < 2^30).
__device__ __forceinline__ float2 pred_noise(uint2 key, unsigned jv, int tau, unsigned ar, unsigned race)
{
    const uint4 w = philox4x32_10(make_uint4((1u << 30) | jv, (unsigned)((tau - 1) >> 1), ar, race), key);
    return ((tau - 1) & 1) ? box_muller(w.z, w.w) : box_muller(w.x, w.y);
}

// Predicted position p of step tau moved by sig_lon z_1 along the unit
// direction t of its nearest segment and sig_lat z_2 along t's left normal.
__device__ __forceinline__ float2 perturb_point(const PlanArgs &a, float2 p, float2 t, unsigned jv, int tau,
                                                unsigned ar, unsigned race)
{
    const float2 z = pred_noise(a.key, jv, tau, ar, race);
    // explicitly rounded operations: every build gives the same bits
    const float ds = __fmul_rn(a.sig_lon, z.x), dd = __fmul_rn(a.sig_lat, z.y);
    return make_float2(__fsub_rn(__fmaf_rn(ds, t.x, p.x), __fmul_rn(dd, t.y)),
                       __fmaf_rn(dd, t.x, __fmaf_rn(ds, t.y, p.y)));
}

// ---------------------------------------------------------------- GA-IBR-MPPI
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Path-integral partial sums of one tile of kTileSingle samples (all threads
// of the CTA; the tile's costs are in Tl::st() as floats, +inf for a
// non-finite cost or k >= K).  With m_t the tile's minimum cost, every sample
// weighs w = exp((m_t - c) / lambda) and its clipped controls are drawn again
// from the same counter; w u is summed over each 32-sample group by a
// shuffle butterfly over lanes (lane = k mod 32), then over the groups in
// order, so the sums depend on k alone, not on the launch shape.  Output
// row of mppi_part: [0] m_t, [1 + 2 tau + c] sum w u_tau,c, [1 + 2T] sum w.
// Group sums are kept in the tile's scratch area.
template <int MAXO>
__device__ void mppi_tile(const PlanArgs &a, int t, int ag, int T)
{
    using Tl = Tile<MAXO>;
    constexpr int kGroups = kTileSingle / 32;
    const BRScalars &S = Tl::sc();
    float *mc = (float *)Tl::st();
    float *gw = mc + kTileSingle;
    float *grp = (float *)Tl::scratch();
    __shared__ float m_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (warp == 0) {
        float m = __int_as_float(0x7f800000);
        for (int q = lane; q < kTileSingle; q += 32) m = fminf(m, mc[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) m_sh = m;
    }
    __syncthreads();
    const float m = m_sh;
    const float4 *dist = Tl::dist();
    for (unsigned j = threadIdx.x; j < (unsigned)kTileSingle; j += blockDim.x) {
        const unsigned k = (unsigned)t * kTileSingle + j;
        const float c = mc[j];
        const float w = c <= 3.402823466e38f ? expf(__fmul_rn(m - c, a.mppi_il)) : 0.f;
        float *gs = grp + (j >> 5) * (2 * T);
        for (int mm = 0; 2 * mm < T; ++mm) {
            float2 z0, z1;
            noise_pair(S, a.rk, k, S.stream_bit, mm, z0, z1);
            const int t0 = 2 * mm;
            const float2 u0 = sample_control_d(a.p, dist[t0], z0);
            float v0 = __fmul_rn(w, u0.x), v1 = __fmul_rn(w, u0.y), v2 = 0.f, v3 = 0.f;
            if (t0 + 1 < T) {
                const float2 u1 = sample_control_d(a.p, dist[t0 + 1], z1);
                v2 = __fmul_rn(w, u1.x);
                v3 = __fmul_rn(w, u1.y);
            }
            v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2); v3 = warp_sum(v3);
            if (lane == 0) {
                gs[2 * t0] = v0;
                gs[2 * t0 + 1] = v1;
                if (t0 + 1 < T) { gs[2 * t0 + 2] = v2; gs[2 * t0 + 3] = v3; }
            }
        }
        const float ws = warp_sum(w);
        if (lane == 0) gw[j >> 5] = ws;
    }
    __syncthreads();
    float *out = a.mppi_part + ((size_t)ag * a.tiles[0] + t) * (size_t)(2 * a.maxT + 2);
    for (int v = threadIdx.x; v <= 2 * T; v += blockDim.x) {
        float acc = 0.f;
#pragma unroll
        for (int g = 0; g < kGroups; ++g) acc += v < 2 * T ? grp[g * 2 * T + v] : gw[g];
        out[1 + v] = acc;
    }
    if (threadIdx.x == 0) out[0] = m;
    __syncthreads();
}

// The GA-IBR-MPPI update of vehicle ag (all threads of the CTA): c_min =
// min_t m_t, then sum_t exp((c_min - m_t) / lambda) x row_t over the tiles in
// index order (factors staged in the scratch area in chunks), and U-bar <-
// sum w u / sum w, clipped (rounding may leave the box by an ulp).  With no
// finite cost the clipped nominal is kept.  Writes Tl::ctl(), U_io, u_hist.
template <int MAXO>
__device__ void mppi_update(const PlanArgs &a, int ag, int T, size_t uo, int round)
{
    using Tl = Tile<MAXO>;
    constexpr int kChunk = BRTile<MAXO>::kScrBytes / 4;
    const size_t stride = (size_t)(2 * a.maxT + 2);
    const float *part = a.mppi_part + (size_t)ag * a.tiles[0] * stride;
    float *acc = (float *)Tl::st();
    float *e = (float *)Tl::scratch();
    __shared__ float red_sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float ml = __int_as_float(0x7f800000);
    for (int q = threadIdx.x; q < a.tiles[0]; q += blockDim.x) ml = fminf(ml, __ldcg(part + (size_t)q * stride));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ml = fminf(ml, __shfl_xor_sync(0xffffffffu, ml, o));
    if (lane == 0) red_sh[warp] = ml;
    for (int v = threadIdx.x; v <= 2 * T; v += blockDim.x) acc[v] = 0.f;
    __syncthreads();
    float cmin = red_sh[0];
    for (int w = 1; w < nwarps; ++w) cmin = fminf(cmin, red_sh[w]);
    for (int base = 0; base < a.tiles[0]; base += kChunk) {
        const int n = min(kChunk, a.tiles[0] - base);
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const float mt = __ldcg(part + (size_t)(base + q) * stride);
            e[q] = mt <= 3.402823466e38f ? expf(__fmul_rn(cmin - mt, a.mppi_il)) : 0.f;
        }
        __syncthreads();
        for (int v = threadIdx.x; v <= 2 * T; v += blockDim.x) {
            const float *pv = part + (size_t)base * stride + 1 + v;
            float sum = acc[v];
#pragma unroll 8
            for (int q = 0; q < n; ++q) sum = __fmaf_rn(e[q], __ldcg(pv + (size_t)q * stride), sum);
            acc[v] = sum;
        }
    }
    __syncthreads();
    const float W = acc[2 * T];
    const bool ok = cmin <= 3.402823466e38f && W > 0.f;
    for (int q = threadIdx.x; q < T; q += blockDim.x) {
        const float2 ubar = ok ? make_float2(__fdiv_rn(acc[2 * q], W), __fdiv_rn(acc[2 * q + 1], W))
                               : make_float2(__ldcg(a.U_io + uo + 2 * q), __ldcg(a.U_io + uo + 2 * q + 1));
        const float2 u = sample_control(a.p, ubar, make_float2(0.f, 0.f));
        Tl::ctl()[q] = u;
        a.U_io[uo + 2 * q] = u.x;
        a.U_io[uo + 2 * q + 1] = u.y;
        if (a.u_hist) {
            a.u_hist[(size_t)round * a.u_total + uo + 2 * q] = u.x;
            a.u_hist[(size_t)round * a.u_total + uo + 2 * q + 1] = u.y;
        }
    }
}

// Register budgets of the persistent kernel (MODE):
//   kWide3: 256 threads x 3 CTAs per SM, 80 registers, one sample per thread;
//   kWide2: 256 x 2 CTAs, 128 registers, one sample per thread;
//   kIlp:   128 x 3 CTAs, 168 registers, one to three samples per thread at
//           once (chosen per round, so that a round fits in one wave where
//           it can): independent rollouts interleaved in one thread hide
//           each other's latency, and 168 registers hold three of them.
// In every SGTP build a round that fits the grid twice over at one sample
// per thread takes half tiles (the CTA's first half of threads), so that
// its lone-sample chains spread over twice the CTAs.
// Every mode computes every sample with the same code.  MPPI selects the
// GA-IBR-MPPI update (a build of its own, so that the SGTP builds carry none
// of its code); its kIlp build rolls two samples per thread, so that a tile
// is the 256 samples of its path-integral partial sums in every build.
constexpr int kWide3 = 0, kWide2 = 1, kIlp = 2;

template <int MAXO, int MODE, bool MPPI>
__device__ __forceinline__ void plan_body(const PlanArgs &a);

template <int MAXO, int MINB, bool MPPI>
__global__ void __launch_bounds__(256, MINB) plan_kernel(PlanArgs a)
{
    plan_body<MAXO, MINB == 3 ? kWide3 : kWide2, MPPI>(a);
}

template <int MAXO, bool MPPI>
__global__ void __launch_bounds__(128, 3) plan_kernel_ilp(PlanArgs a)
{
    plan_body<MAXO, kIlp, MPPI>(a);
}

// Selection key of the NI candidates k0 + i blockDim of this thread (all
// threads of the tile call it; candidates k >= K key as ~0).  GA-IBR-MPPI
// keys every sample as feasible and keeps each sample's cost (+inf when not
// finite or k >= K) at its place in the tile for the partial sums.
template <int MAXO, int NI, bool MPPI = false>
__device__ __forceinline__ unsigned long long tile_keys(const BRScalars &S, const PlanArgs &a, unsigned k0, int round,
                                                        int &flag)
{
    unsigned kk[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) kk[i] = k0 + (unsigned)i * blockDim.x;
    SampleResult r[NI];
    run_candidates<MAXO, NI, false>(S, a.p, a.rk, kk, round > 0, flag, r, nullptr, nullptr, nullptr);
    unsigned long long best = ~0ull;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
        const unsigned long long key = make_key(r[i].feasible || MPPI, r[i].cost, r[i].viol, kk[i]);
        if (kk[i] < (unsigned)a.K && key < best) best = key;
        if constexpr (MPPI) {
            const bool fin = kk[i] < (unsigned)a.K && fabsf(r[i].cost) <= 3.402823466e38f;
            ((float *)Tile<MAXO>::st())[threadIdx.x + i * blockDim.x] = fin ? r[i].cost : __int_as_float(0x7f800000);
        }
    }
    return best;
}

template <int MAXO, int MODE, bool MPPI>
__device__ __forceinline__ void plan_body(const PlanArgs &a)
{
    using Tl = Tile<MAXO>;
    __shared__ unsigned long long cta_key;
    __shared__ int abort_sh, j0_sh;
    __shared__ unsigned ks_sh;
    BRScalars &S = Tl::sc();

    const int lane = threadIdx.x & 31;
    const bool skip = (a.debug_flags & SGTP_DEBUG_SKIP_BARRIER_ARRIVAL) && blockIdx.x == 0;
    int flag = 0;
    unsigned phase = 0;
    bool ok = true;
    if (threadIdx.x == 0) {
        mbar_init(Tl::bar(), 1);
        g_bar_epoch = 0u;
        g_win_track = nullptr;
        g_win_fix = 0;
    }
    stamp(a, 0);

    // ------------------------------------------------------------ setup (one CTA per vehicle)
    for (int ag = blockIdx.x; ag < a.n_agents; ag += gridDim.x) {
        const int ri = find_race(a, ag, [](const RaceDev &r) { return r.agent_off; });
        const RaceDev R = get_race(a, ri);
        const int i = ag - R.agent_off;
        const TrackView tv = get_track(a, R.track_id);
        const float4 x0 = make_float4(a.X0[4 * ag], a.X0[4 * ag + 1], a.X0[4 * ag + 2], a.X0[4 * ag + 3]);
        __syncthreads();
        for (int q = threadIdx.x; q < R.T; q += blockDim.x) {
            // nominal controls, clipped: the zero-noise sample
            const float *U = a.U_io + R.u_off + (size_t)i * R.T * 2;
            Tl::ctl()[q] = sample_control(a.p, make_float2(U[2 * q], U[2 * q + 1]), make_float2(0.f, 0.f));
        }
        {
            const int j = nearest_segment_cta(tv, x0.x, x0.y, &cta_key);
            if (threadIdx.x == 0) j0_sh = j;
        }
        __syncthreads();
        const int j0 = j0_sh;
        // the window copy, the reference stretch and x0's projection are
        // all in flight before the CTA waits for the copy
        const bool issued = stage_vehicle_window<MAXO>(a, tv, j0);
        const float4 *ref_c;
        const SegWindow ref_w = stage_ref_window<MAXO>(tv, j0, ref_c);
        const FrenetPt f = frenet_at(tv, j0, x0.x, x0.y);
        window_ready<MAXO>(a, issued, phase);
        AgentDev A;
        A.x0 = x0; A.s_t = f.s; A.d_t = f.d; A.j0 = j0; A.race = ri; A.t0 = f.t;
        if ((threadIdx.x >> 5) == 1) {
            // reference recursion (warp 1, the staged stretch of track)
            // alongside the nominal rollout's dynamics (warp 0)
            if (threadIdx.x == 32) a.agents[ag] = A;
            reference_traj(tv, ref_w, ref_c, j0, f.s, a.p.dt, a.vref[ag], R.T,
                           a.ref + (size_t)R.pos_off + (size_t)i * (R.T + 1));
        }
        roll_cooperative<MAXO>(a.p, x0, f.s, j0, R.T, R.n_tail, a.pos[0] + R.pos_off + (size_t)i * (R.T + 1), nullptr,
                               nullptr, a.summ[0] + ag, flag,
                               a.ptan[0] ? a.ptan[0] + R.pos_off + (size_t)i * (R.T + 1) : nullptr);
    }
    {
        // fresh selection keys for every best response of the plan
        const RaceDev last = get_race(a, a.n_races - 1);
        const int n_keys = last.ks_off + (a.L + 1) * last.n_v + 1;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_keys; q += gridDim.x * blockDim.x)
            a.keys[q] = ~0ull;
        if (a.queue) {
            const int n_cnt = a.n_races + 2 * a.n_agents;
            for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_cnt; q += gridDim.x * blockDim.x)
                a.wdone[q] = 0u;      // wdone, tdone and pdone are contiguous
            if (blockIdx.x == 0 && threadIdx.x == 0) *a.qhead = 0ull;
        }
    }
    ok = grid_barrier(a, skip);
    stamp(a, 1);
    // queue schedule: q_sh is this CTA's claimed position; a round holds
    // (with the learned proposal) one proposal item per vehicle, then
    // items[kind] sample items, then one winner item per vehicle
    const bool queue = a.queue != 0;
    const bool learned = a.mlp_wb || a.feat_out;
    const unsigned long long round_items =
        (unsigned long long)((learned ? a.n_agents : 0) + a.items[0] + a.n_agents);
    __shared__ unsigned long long q_sh;
    if (ok && queue) claim_item(a, q_sh);

    for (int round = 0; ok && round <= a.L + 1; ++round) {
        const bool extra = round == a.L + 1;
        const int bin = round & 1, bout = bin ^ 1;
        unsigned long long base = (unsigned long long)round * round_items;
        if (learned) {
            // -------------------------------------------------- proposals (one CTA per vehicle)
            // queue: a proposal needs the race's previous round complete
            for (int ag = blockIdx.x;; ag += gridDim.x) {
                if (queue) {
                    if (q_sh >= base + (unsigned long long)a.n_agents) break;
                    ag = (int)(q_sh - base);
                } else if (ag >= a.n_agents) {
                    break;
                }
                const int ri = find_race(a, ag, [](const RaceDev &r) { return r.agent_off; });
                const RaceDev R = get_race(a, ri);
                const int i = ag - R.agent_off;
                const bool active = !extra || i == R.ego;
                if (queue && active && round > 0 && !wait_count(a, a.wdone + ri, (unsigned)(round * R.n_v))) {
                    ok = false;
                    break;
                }
                if (active) {
                    __syncthreads();
                    proposal_for(a, R, i, bin, round > 0, round, Tl::scratch());
                }
                if (queue) {
                    // only a proposal that ran counts: the extra round's
                    // idle items (claimed as early as any) must not stand
                    // in for a vehicle's proposal of an earlier round
                    if (active) signal_done(a.pdone + ag);
                    claim_item(a, q_sh);
                }
            }
            if (!ok) break;
            if (!queue && !grid_barrier(a, skip)) break;
            base += (unsigned long long)a.n_agents;
        }
        stamp(a, 2 + 3 * round);
        // lock step: this CTA's share of the round, equal item counts for one
        // race, equal work (items weighted by their race's horizon) for a
        // batch; queue: the positions base .. base + items - 1 as claimed
        int i0 = 0, i1 = 0;
        if (queue) {
        } else if (!a.races) {
            const int n_items = a.items[extra];
            i0 = (int)((long long)n_items * blockIdx.x / gridDim.x);
            i1 = (int)((long long)n_items * (blockIdx.x + 1) / gridDim.x);
        } else {
            const long long W = a.w[extra];
            i0 = first_item_at(a, W * blockIdx.x / gridDim.x, extra);
            i1 = first_item_at(a, W * (blockIdx.x + 1) / gridDim.x, extra);
        }
        int cur = -1;                 // vehicle (global index) staged
        unsigned long long *cur_slot = nullptr;
        for (int item = i0;; ++item) {
            if (queue) {
                if (q_sh >= base + (unsigned long long)a.items[extra]) break;
                item = (int)(q_sh - base);
            } else if (item >= i1) {
                break;
            }
            // item = vehicle (all vehicles of all races in a Jacobi round, the
            // races' egos in the extra round) x tile of that vehicle's samples
            int ri, i;
            const int unit = item / a.tiles[extra], t = item - unit * a.tiles[extra];
            if (!extra) {
                ri = find_race(a, unit, [](const RaceDev &r) { return r.agent_off; });
                i = unit - get_race(a, ri).agent_off;
            } else {
                ri = unit;
                i = get_race(a, ri).ego;
            }
            const RaceDev R = get_race(a, ri);
            const int ag = R.agent_off + i;
            // queue: the race's previous round must be complete (its n_v
            // winners per round); with the learned proposal, the vehicle's
            // proposal of this round, which waited for that itself
            if (queue && (learned || round > 0) &&
                !(learned ? wait_count(a, a.pdone + ag, (unsigned)(round + 1))
                          : wait_count(a, a.wdone + ri, (unsigned)(round * R.n_v)))) {
                ok = false;
                break;
            }
            if (ag != cur) {
                // flush the previous vehicle's key (lock step; the queue
                // flushes after every item), then stage this one
                __syncthreads();
                if (threadIdx.x == 0 && cur_slot && !queue) atomicMin(cur_slot, cta_key);
                const TrackView tv = get_track(a, R.track_id);
                const AgentDev A = load_agent(a.agents + ag);
                const int T = R.T, n_opp = R.n_v - 1;
                const bool issued = stage_vehicle_window<MAXO>(a, tv, A.j0);
                if (threadIdx.x == 0) {
                    cta_key = ~0ull;
                    S.x0 = A.x0; S.s_t = A.s_t; S.d_t = A.d_t;
                    const float2 hs = heading_split(A.x0.z);
                    S.psi0 = hs.x; S.psi_off = hs.y;
                    S.pos0 = (float)S.r0 + A.t0;
                    S.ppred0 = S.pos0 + __fdiv_rn(__fmul_rn(a.p.dt, A.x0.w), __ldg(tv.B + A.j0).w) - 0.5f;
                    S.T = T; S.n_opp = n_opp; S.n_tail = R.n_tail;
                    S.key = a.key;
                    S.ctr_agent_round = (unsigned)i | ((unsigned)round << 16);
                    S.ctr_race = R.race_tag;
                    S.stream_bit = 0u;
                    S.K_prop = a.mlp_wb ? a.K_prop : 0;
                }
                const float *U = a.U_io + R.u_off + (size_t)i * T * 2;
                const float4 *P = a.prop + (size_t)ag * a.maxT;
                for (int q = threadIdx.x; q < T; q += blockDim.x) {
                    Tl::dist()[q] = make_float4(__ldcg(U + 2 * q), __ldcg(U + 2 * q + 1), a.p.sigma_a, a.p.sigma_delta);
                    if (a.mlp_wb) Tl::dist()[SGTP_MAX_T + q] = __ldcg(P + q);
                }
                const float4 *gref = a.ref + (size_t)R.pos_off + (size_t)i * (T + 1);
                for (int q = threadIdx.x; q <= T; q += blockDim.x) Tl::ref()[q] = __ldcg(gref + q);
                const float2 *pin = a.pos[bin] + R.pos_off;
                const float2 *tin = a.ptan[bin] ? a.ptan[bin] + R.pos_off : nullptr;
                const unsigned ar = (unsigned)i | ((unsigned)round << 16);
                stage_opponents<MAXO>(T, n_opp, [&](int tau, int o) {
                    const int jv = o < i ? o : o + 1;
                    const float2 q = __ldcg(pin + (size_t)jv * (T + 1) + tau);
                    if (!tin) return q;
                    return perturb_point(a, q, __ldcg(tin + (size_t)jv * (T + 1) + tau), (unsigned)jv, tau, ar,
                                         R.race_tag);
                });
                if (threadIdx.x < n_opp) {
                    const int o = threadIdx.x;
                    const int jv = o < i ? o : o + 1;
                    const AgentDev B = load_agent(a.agents + R.agent_off + jv);
                    float2 sm = __ldcg(a.summ[bin] + R.agent_off + jv);
                    if (tin) {
                        // the perturbed prediction's progress gain and tail-mean offset
                        sm.x = __fmaf_rn(a.sig_lon, pred_noise(a.key, (unsigned)jv, T, ar, R.race_tag).x, sm.x);
                        float dsum = 0.f;
                        for (int tau = T - R.n_tail + 1; tau <= T; ++tau)
                            dsum = __fmaf_rn(a.sig_lat, pred_noise(a.key, (unsigned)jv, tau, ar, R.race_tag).y, dsum);
                        sm.y = __fadd_rn(sm.y, __fdiv_rn(dsum, (float)R.n_tail));
                    }
                    const float ds_t = wrap_len(A.s_t - B.s_t, tv.L, 1.0f / tv.L);
                    const float alpha = 1.0f / (1.0f + fabsf(ds_t) / (a.p.s_contest + a.p.eps_alpha));
                    const float gamma = (ds_t > a.p.s_role && ds_t < a.p.s_contest) ? a.p.w_block : 0.f;
                    Tl::osum()[o] = make_float4(ds_t, alpha, gamma, sm.x);
                    Tl::odbar()[o] = sm.y;
                }
                cur = ag;
                cur_slot = a.keys + R.ks_off + (extra ? (a.L + 1) * R.n_v : round * R.n_v + i);
                __syncthreads();
                window_ready<MAXO>(a, issued, phase);
                if (threadIdx.x == 0) abort_sh = (ld_status(a.status) & 0xff) != 0;
                __syncthreads();
                if (abort_sh) { ok = false; break; }
            }
            // a tile of a.tile[extra] samples: in the kIlp build one to three
            // per thread at once (a.ni[extra], candidates k, k + blockDim,
            // k + 2 blockDim), otherwise a.tile / blockDim.x in turn;
            // GA-IBR-MPPI keys every sample as feasible (its k* is the lowest
            // cost) and keeps the tile's costs for its partial sums
            constexpr bool mppi = MPPI;
            unsigned long long best = ~0ull;
            if constexpr (MODE == kIlp && MPPI) {
                best = tile_keys<MAXO, 2, true>(S, a, (unsigned)t * a.tile[extra] + threadIdx.x, round, flag);
            } else if constexpr (MODE == kIlp) {
                const unsigned k0 = (unsigned)t * a.tile[extra] + threadIdx.x;
                const int ni = a.ni[extra];
                if (ni == 3) best = tile_keys<MAXO, 3>(S, a, k0, round, flag);
                else if (ni == 2) best = tile_keys<MAXO, 2>(S, a, k0, round, flag);
                else if (threadIdx.x < (unsigned)a.tile[extra]) best = tile_keys<MAXO, 1>(S, a, k0, round, flag);
            } else {
                for (unsigned j = threadIdx.x; j < (unsigned)a.tile[extra]; j += blockDim.x) {
                    const unsigned k = (unsigned)t * a.tile[extra] + j;
                    float c = __int_as_float(0x7f800000);
                    if (k < (unsigned)a.K) {
                        const SampleResult r = run_candidate<MAXO, false>(S, a.p, a.rk, k, round > 0, flag, nullptr,
                                                                          nullptr, nullptr);
                        const unsigned long long key = make_key(r.feasible || mppi, r.cost, r.viol, k);
                        best = key < best ? key : best;
                        if (fabsf(r.cost) <= 3.402823466e38f) c = r.cost;
                    }
                    if constexpr (MPPI) ((float *)Tl::st())[j] = c;
                }
            }
            best = warp_min_u64(best);
            if (lane == 0) atomicMin(&cta_key, best);
            if constexpr (MPPI) mppi_tile<MAXO>(a, t, ag, R.T);
            if (queue) {
                __syncthreads();
                if (threadIdx.x == 0) atomicMin(cur_slot, cta_key);
                signal_done(a.tdone + ag);
                claim_item(a, q_sh);
            }
        }
        if (!ok) break;
        if (!queue) {
            __syncthreads();
            if (threadIdx.x == 0 && cur_slot) atomicMin(cur_slot, cta_key);
            if (!grid_barrier(a, skip)) break;
        }
        stamp(a, 3 + 3 * round);

        // -------------------------------------------------------- winners (one CTA per vehicle)
        const unsigned long long wbase = base + (unsigned long long)a.items[extra];
        for (int ag = blockIdx.x;; ag += gridDim.x) {
            if (queue) {
                if (q_sh >= wbase + (unsigned long long)a.n_agents) break;
                ag = (int)(q_sh - wbase);
            } else if (ag >= a.n_agents) {
                break;
            }
            const AgentDev A = load_agent(a.agents + ag);
            const RaceDev R = get_race(a, A.race);
            const int i = ag - R.agent_off;
            const int T = R.T;
            const bool active = !extra || i == R.ego;
            const size_t xo = (size_t)R.xi_off + (size_t)i * (T + 1) * 4;
            const size_t uo = (size_t)R.u_off + (size_t)i * T * 2;
            __syncthreads();
            if (queue) {
                // an active winner needs all of its vehicle's tiles so far;
                // the extra round's copies need the race's round-L winners
                const unsigned need = !extra ? (unsigned)((round + 1) * a.tiles[0])
                                     : active ? (unsigned)((a.L + 1) * a.tiles[0] + a.tiles[1])
                                              : (unsigned)(round * R.n_v);
                if (!wait_count(a, active ? a.tdone + ag : a.wdone + A.race, need)) {
                    ok = false;
                    break;
                }
            }
            if (!active) {
                if (a.xi_hist)
                    for (int q = threadIdx.x; q < (T + 1) * 4; q += blockDim.x)
                        a.xi_hist[(size_t)round * a.xi_total + xo + q] = __ldcg(a.xi_out + xo + q);
                if (a.u_hist)
                    for (int q = threadIdx.x; q < T * 2; q += blockDim.x)
                        a.u_hist[(size_t)round * a.u_total + uo + q] = __ldcg(a.U_io + uo + q);
                if (queue) {
                    // (fault injection for tests: the winners never report)
                    if (!(a.debug_flags & SGTP_DEBUG_SKIP_WINNER_SIGNAL)) signal_done(a.wdone + A.race);
                    claim_item(a, q_sh);
                }
                continue;
            }
            const int slot = extra ? (a.L + 1) * R.n_v : round * R.n_v + i;
            const TrackView tv = get_track(a, R.track_id);
            const bool issued = stage_vehicle_window<MAXO>(a, tv, A.j0);
            if (threadIdx.x == 0) {
                const unsigned long long key = __ldcg(a.keys + R.ks_off + slot);
                ks_sh = (unsigned)(key & 0x7fffffffull);
                a.k_star_out[R.ks_off + slot] = (int)ks_sh;
            }
            __syncthreads();
            // controls of the selected sample, one step per thread (same noise,
            // same clipping as its evaluation): warm start U-bar <- U^(k*);
            // GA-IBR-MPPI: U-bar <- the path-integral mean
            const unsigned ks = ks_sh;
            const unsigned ar = (unsigned)i | ((unsigned)round << 16);
            const bool from_prop = a.mlp_wb && ks < (unsigned)a.K_prop;
            if constexpr (MPPI) mppi_update<MAXO>(a, ag, T, uo, round);
            else for (int q = threadIdx.x; q < T; q += blockDim.x) {
                const unsigned sbit = from_prop ? 0x80000000u : 0u;
                const uint4 wv = philox4x32_10(make_uint4(ks, (unsigned)(q >> 1) | sbit, ar, R.race_tag), a.key);
                const float2 z = (q & 1) ? box_muller(wv.z, wv.w) : box_muller(wv.x, wv.y);
                const float4 d = from_prop ? __ldcg(a.prop + (size_t)ag * a.maxT + q)
                                           : make_float4(__ldcg(a.U_io + uo + 2 * q), __ldcg(a.U_io + uo + 2 * q + 1),
                                                         a.p.sigma_a, a.p.sigma_delta);
                const float2 u = sample_control_d(a.p, d, z);
                Tl::ctl()[q] = u;
                a.U_io[uo + 2 * q] = u.x;
                a.U_io[uo + 2 * q + 1] = u.y;
                if (a.u_hist) {
                    a.u_hist[(size_t)round * a.u_total + uo + 2 * q] = u.x;
                    a.u_hist[(size_t)round * a.u_total + uo + 2 * q + 1] = u.y;
                }
            }
            window_ready<MAXO>(a, issued, phase);
            float *xi_final = (round == a.L || extra) ? a.xi_out + xo : nullptr;
            float *xi_h = a.xi_hist ? a.xi_hist + (size_t)round * a.xi_total + xo : nullptr;
            roll_cooperative<MAXO>(a.p, A.x0, A.s_t, A.j0, T, R.n_tail,
                                   extra ? nullptr : a.pos[bout] + R.pos_off + (size_t)i * (T + 1), xi_final, xi_h,
                                   extra ? nullptr : a.summ[bout] + ag, flag,
                                   (extra || !a.ptan[bout]) ? nullptr : a.ptan[bout] + R.pos_off + (size_t)i * (T + 1));
            if (queue) {
                // (fault injection for tests: the winners never report)
                if (!(a.debug_flags & SGTP_DEBUG_SKIP_WINNER_SIGNAL)) signal_done(a.wdone + A.race);
                claim_item(a, q_sh);
            }
        }
        if (!ok) break;
        if (!queue && round <= a.L) ok = grid_barrier(a, skip);
        stamp(a, 4 + 3 * round);
    }
    if (flag) atomicOr(a.status, SGTP_E_DEVICE << 8);
}

// ================================================================ host side
struct Layout {
    size_t bar, keys, agents, ref, pos0, pos1, summ0, summ1, prop, part, tan0, tan1, cnt, total;
    // part_floats: GA-IBR-MPPI partial sums (0 for the SGTP calls)
    Layout(long long n_keys, long long n_agents, long long n_pos, int maxT, long long part_floats = 0,
           long long n_races = 1)
    {
        auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
        bar = 0;
        keys = 256;
        agents = up(keys + sizeof(unsigned long long) * n_keys);
        ref = up(agents + sizeof(AgentDev) * n_agents);
        pos0 = up(ref + sizeof(float4) * n_pos);
        pos1 = up(pos0 + sizeof(float2) * n_pos);
        summ0 = up(pos1 + sizeof(float2) * n_pos);
        summ1 = up(summ0 + sizeof(float2) * n_agents);
        prop = up(summ1 + sizeof(float2) * n_agents);
        part = up(prop + sizeof(float4) * n_agents * maxT);
        tan0 = up(part + sizeof(float) * part_floats);
        tan1 = up(tan0 + sizeof(float2) * n_pos);
        cnt = up(tan1 + sizeof(float2) * n_pos);      // queue head, then wdone, tdone, pdone
        total = up(cnt + sizeof(unsigned long long) + sizeof(unsigned) * (n_races + 2 * n_agents));
    }
};

int maxo_bucket(int n) { return n <= 1 ? 1 : n <= 3 ? 3 : n <= 9 ? 9 : 15; }

template <int MAXO, int MODE, bool MPPI>
const void *plan_kernel_of()
{
    if constexpr (MODE == kIlp) return (const void *)plan_kernel_ilp<MAXO, MPPI>;
    else return (const void *)plan_kernel<MAXO, MODE == kWide3 ? 3 : 2, MPPI>;
}

template <int MAXO, int MODE, bool MPPI>
sgtp_status configure_plan_t()
{
    // the shared-memory opt-in applies to the current device only
    static PerDeviceFlag configured;
    return once_per_device(configured, []() -> sgtp_status {
        SGTP_CUDA(cudaFuncSetAttribute(plan_kernel_of<MAXO, MODE, MPPI>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        return SGTP_OK;
    });
}

template <int MAXO>
sgtp_status configure_plan_maxo()
{
    sgtp_status st;
    if ((st = configure_plan_t<MAXO, kWide3, false>()) || (st = configure_plan_t<MAXO, kWide2, false>()) ||
        (st = configure_plan_t<MAXO, kIlp, false>()) || (st = configure_plan_t<MAXO, kWide3, true>()) ||
        (st = configure_plan_t<MAXO, kWide2, true>()) || (st = configure_plan_t<MAXO, kIlp, true>()))
        return st;
    return SGTP_OK;
}

sgtp_status configure_plan_kernels()
{
    sgtp_status st;
    if ((st = configure_plan_maxo<1>()) || (st = configure_plan_maxo<3>()) || (st = configure_plan_maxo<9>()) ||
        (st = configure_plan_maxo<15>()))
        return st;
    return SGTP_OK;
}

template <int MAXO, int MODE, bool MPPI>
sgtp_status launch_plan_v(PlanArgs &a, int block, int ctas, int spt, cudaStream_t s)
{
    const size_t smem = BRTile<MAXO>::kBytes;
    sgtp_status cst = configure_plan_t<MAXO, MODE, MPPI>();
    if (cst) return cst;
    int dev = 0, sms = 0, per_sm = 0;
    SGTP_CUDA(cudaGetDevice(&dev));
    SGTP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SGTP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_kernel_of<MAXO, MODE, MPPI>(), block, smem));
    SGTP_CHECK(per_sm >= 1, "plan kernel does not fit on an SM (smem %zu)", smem);
    if (ctas > 0 && ctas < per_sm) per_sm = ctas;
    const int grid = sms * per_sm;
    // tiles of each round kind: kIlp rolls out ni samples per thread at once,
    // the fewest that fit the round's samples in one wave of the grid (at
    // most 3); a round of several waves even at 3 takes 2 or 3, whichever
    // pads K less to whole tiles (ties: 3) -- except a plain batch under the
    // queue schedule, which keeps 3 (measured: the dynamic balance and the
    // third interleaved sample repay up to 3 % of padding, while a learned
    // batch's proposal items overlap better with the finer tiles); unless
    // the caller fixed it
    const long long cand[2] = {(long long)a.n_agents * a.K, (long long)a.n_races * a.K};
    for (int e = 0; e < 2; ++e) {
        int ni = 1;
        if (MODE == kIlp && MPPI) {
            ni = 2;                       // a tile is the 256 samples of the partial sums
        } else if (MODE == kIlp) {
            const long long slots = (long long)grid * block;
            ni = spt > 0 ? spt : (int)std::min(3ll, std::max(1ll, (cand[e] + slots - 1) / slots));
            const bool keep3 = a.queue && !(a.mlp_wb || a.feat_out);
            if (spt == 0 && cand[e] > 3 * slots && !keep3) {
                auto padded = [&](int n) { return (long long)((a.K + block * n - 1) / (block * n)) * block * n; };
                if (padded(2) < padded(3)) ni = 2;
            }
        }
        a.ni[e] = ni;
        a.tile[e] = MPPI ? kTileSingle : block * ni;
        // a round that fits twice over in one wave at one sample per thread
        // takes half tiles (one sample for each thread of the CTA's first
        // half): its lone-sample chains then spread over twice the CTAs
        if (!MPPI && ni <= 1 && spt <= 1 && (MODE != kIlp || spt == 0) && 2 * cand[e] <= (long long)grid * block)
            a.tile[e] = block / 2;
        a.tiles[e] = (a.K + a.tile[e] - 1) / a.tile[e];
        a.items[e] = (e ? a.n_races : a.n_agents) * a.tiles[e];
        a.w[e] = (e ? a.w_units_ego : a.w_units_all) * a.tiles[e];
    }
    if (a.timeout_ns <= 0) {
        const double units = a.races ? (double)(a.L + 1) * a.w_units_all + (double)a.w_units_ego
                                     : ((double)(a.L + 1) * a.n_agents + 1.0) * a.maxT;
        a.timeout_ns = default_wait_ns(units * a.K);
    }
    void *args[] = {&a};
    SGTP_CUDA(cudaMemsetAsync(a.bar, 0, 256, s));
    SGTP_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), s));
    SGTP_CUDA(cudaLaunchCooperativeKernel(plan_kernel_of<MAXO, MODE, MPPI>(), grid, block, args, smem, s));
    count_launch();
    return SGTP_OK;
}

// Register budget and shape of one launch.  By default a plain SGTP plan
// or batch runs kIlp (samples per thread chosen per round) unless its
// Jacobi round is at most one 256-thread CTA of samples per SM; a single
// plan with the learned proposal runs 256-thread CTAs (the network's layers
// are split over eight warps, which shortens its proposal phase): kWide2
// when a Jacobi round has fewer 256-sample tiles than three CTAs per SM
// could take at once, else kWide3; a learned batch runs kIlp (its proposal
// items overlap other races' tiles under the queue schedule); GA-IBR-MPPI
// runs kIlp with two samples per thread unless its round is small.  Options override: block 128 (or
// samples_per_thread > 1) selects kIlp, block 256 the wide builds
// (ctas_per_sm <= 2: kWide2).
template <int MAXO>
sgtp_status launch_plan_t(PlanArgs &a, const sgtp_launch_opts *opts, cudaStream_t s)
{
    int block = (opts && opts->block > 0) ? opts->block : 0;
    const int spt = (opts && opts->samples_per_thread > 0) ? opts->samples_per_thread : 0;
    int ctas = opts ? opts->ctas_per_sm : 0;
    int dev = 0, sms = 0;
    SGTP_CUDA(cudaGetDevice(&dev));
    SGTP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const bool mppi = a.mppi_il > 0.f;
    const bool learned = a.mlp_wb != nullptr || a.feat_out != nullptr;
    SGTP_CHECK(!(mppi && (spt == 3 || (block == 128 && spt == 1))),
               "GA-IBR-MPPI rolls two samples per thread with 128-thread CTAs, one with 256");
    // a round of at most one 256-thread CTA's worth of samples per SM runs
    // the wide 128-register build by default (measured faster there)
    const int sched = opts ? opts->schedule : SGTP_SCHEDULE_DEFAULT;
    a.queue = sched == SGTP_SCHEDULE_QUEUE || (sched == SGTP_SCHEDULE_DEFAULT && a.races != nullptr);
    const bool small = (long long)a.n_agents * a.K <= 256ll * sms;
    const bool ilp = mppi ? (block == 128 || spt == 2 || (block == 0 && spt == 0 && !small))
                          : (block == 128 || spt > 1 || (block == 0 && !small && (!learned || a.races)));
    if (ilp && mppi) return launch_plan_v<MAXO, kIlp, true>(a, 128, ctas, 2, s);
    if (ilp) return launch_plan_v<MAXO, kIlp, false>(a, 128, ctas, spt, s);
    block = 256;
    const bool wide2 = ctas > 0 ? ctas <= 2 : (long long)((a.K + 255) / 256) * a.n_agents < 3ll * sms;
    if (wide2 && ctas == 0) ctas = 2;
    if (mppi)
        return wide2 ? launch_plan_v<MAXO, kWide2, true>(a, block, ctas, 1, s)
                     : launch_plan_v<MAXO, kWide3, true>(a, block, ctas, 1, s);
    return wide2 ? launch_plan_v<MAXO, kWide2, false>(a, block, ctas, 1, s)
                 : launch_plan_v<MAXO, kWide3, false>(a, block, ctas, 1, s);
}

sgtp_status launch_plan(PlanArgs &a, int max_opp, const sgtp_launch_opts *opts, cudaStream_t s)
{
    if (opts) {
        SGTP_CHECK(opts->block == 0 || opts->block == 128 || opts->block == 256, "block must be 128 or 256 (got %d)",
                   opts->block);
        SGTP_CHECK(opts->samples_per_thread >= 0 && opts->samples_per_thread <= 3,
                   "samples_per_thread must be 0 .. 3 (got %d)", opts->samples_per_thread);
        SGTP_CHECK(!(opts->block == 256 && opts->samples_per_thread > 1),
                   "256-thread CTAs take one sample per thread");
        SGTP_CHECK(opts->ctas_per_sm >= 0 && opts->window >= 0 && opts->wait_timeout_ns >= 0,
                   "negative launch option");
        SGTP_CHECK(opts->schedule >= SGTP_SCHEDULE_DEFAULT && opts->schedule <= SGTP_SCHEDULE_QUEUE,
                   "schedule must be 0 .. 2 (got %d)", opts->schedule);
    }
    switch (maxo_bucket(max_opp)) {
        case 1: return launch_plan_t<1>(a, opts, s);
        case 3: return launch_plan_t<3>(a, opts, s);
        case 9: return launch_plan_t<9>(a, opts, s);
        default: return launch_plan_t<15>(a, opts, s);
    }
}

void fill_common(PlanArgs &a, const sgtp_track *trk, const sgtp_params *p, int K, int L, const float *X0, float *U_io,
                 const float *vref, uint64_t seed, float *xi_out, int *k_star_out, float *xi_hist, float *u_hist,
                 int *status, const sgtp_launch_opts *opts)
{
    a.tdesc = trk->desc_dev;
    a.A = trk->A; a.B = trk->B; a.W = trk->W; a.S = trk->S; a.C = trk->C;
    a.G0 = trk->G0; a.G1 = trk->G1; a.G2 = trk->G2; a.G3 = trk->G3;
    a.p = *p;
    a.K = K; a.L = L;
    a.X0 = X0; a.U_io = U_io; a.vref = vref;
    a.key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    a.rk = make_round_keys(a.key);
    a.xi_out = xi_out; a.k_star_out = k_star_out; a.xi_hist = xi_hist; a.u_hist = u_hist;
    a.status = status;
    a.Wn = window_len(kWinTile, opts ? opts->window : 0);
    a.back = 48;
    a.timeout_ns = (opts && opts->wait_timeout_ns > 0) ? opts->wait_timeout_ns : 0;   // 0: derived at launch
    a.debug_flags = opts ? opts->debug_flags : 0;
    a.trace = opts ? (long long *)opts->trace_ns : nullptr;
}

void attach_workspace(PlanArgs &a, const Layout &lay, void *ws)
{
    unsigned char *w = (unsigned char *)ws;
    a.bar = (unsigned *)(w + lay.bar);
    a.keys = (unsigned long long *)(w + lay.keys);
    a.agents = (AgentDev *)(w + lay.agents);
    a.ref = (float4 *)(w + lay.ref);
    a.pos[0] = (float2 *)(w + lay.pos0);
    a.pos[1] = (float2 *)(w + lay.pos1);
    a.summ[0] = (float2 *)(w + lay.summ0);
    a.summ[1] = (float2 *)(w + lay.summ1);
    a.prop = (float4 *)(w + lay.prop);
    a.mppi_part = (float *)(w + lay.part);
    if (a.sig_lon != 0.f || a.sig_lat != 0.f) {
        a.ptan[0] = (float2 *)(w + lay.tan0);
        a.ptan[1] = (float2 *)(w + lay.tan1);
    }
    a.qhead = (unsigned long long *)(w + lay.cnt);
    a.wdone = (unsigned *)(w + lay.cnt + sizeof(unsigned long long));
    a.tdone = a.wdone + a.n_races;
    a.pdone = a.tdone + a.n_agents;
}

long long mppi_part_floats(long long n_agents, int K, int maxT)
{
    return n_agents * (long long)((K + kTileSingle - 1) / kTileSingle) * (2ll * maxT + 2);
}

// 1 / lambda of a GA-IBR-MPPI call, or -1 when lambda is not finite and > 0
float mppi_inverse(float lambda)
{
    if (!(lambda > 0.f) || !(lambda <= 3.402823466e38f)) return -1.f;
    const double il = 1.0 / (double)lambda;
    return (float)(il < 3.402823466e38 ? il : 3.402823466e38);
}

}  // namespace

extern "C" size_t sgtp_plan_workspace_bytes(int32_t n_v, int32_t T, int32_t L)
{
    if (n_v < 1 || T < 1 || L < 0) return 0;
    return Layout((long long)(L + 1) * n_v + 1, n_v, (long long)n_v * (T + 1), T).total;
}

static sgtp_status ibr_plan_impl(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                                 const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K, int32_t L,
                                 int32_t ego, uint64_t seed, uint32_t race, float *xi_out, int32_t *k_star_out,
                                 float *xi_hist, float *u_hist, int32_t *status_dev, const sgtp_launch_opts *opts,
                                 const sgtp_mlp *mlp, int32_t K_prop, float *feat_out, float *prop_out,
                                 void *workspace, size_t workspace_bytes, void *stream, float mppi_lambda = 0.f,
                                 float sig_lon = 0.f, float sig_lat = 0.f)
{
    SGTP_CHECK(trk != nullptr, "track is NULL");
    SGTP_CHECK(track_id >= 0 && track_id < trk->n_tracks, "track_id out of range");
    sgtp_status st = check_params(p);
    if (st) return st;
    SGTP_CHECK(n_v >= 1 && n_v <= SGTP_MAX_AGENTS, "n_v=%d out of range [1, %d]", n_v, SGTP_MAX_AGENTS);
    SGTP_CHECK(T >= 1 && T <= SGTP_MAX_T, "T=%d out of range", T);
    SGTP_CHECK(K >= 1 && K <= SGTP_MAX_K, "K=%d out of range", K);
    SGTP_CHECK(L >= 0 && L < 4096, "L=%d out of range", L);
    SGTP_CHECK(ego >= 0 && ego < n_v, "ego out of range");
    SGTP_CHECK(race < (1u << 31), "race tag out of range");
    SGTP_CHECK(X0 && U_io && vref_scale && xi_out && k_star_out && status_dev, "NULL array");
    const bool mppi = mppi_lambda != 0.f;
    const float il = mppi ? mppi_inverse(mppi_lambda) : 0.f;
    SGTP_CHECK(!mppi || il > 0.f, "lambda must be finite and > 0");
    SGTP_CHECK(!(mppi && mlp), "GA-IBR-MPPI takes the plain sampler only");
    const Layout lay((long long)(L + 1) * n_v + 1, n_v, (long long)n_v * (T + 1), T,
                     mppi ? mppi_part_floats(n_v, K, T) : 0);
    SGTP_CHECK(workspace && workspace_bytes >= lay.total, "workspace too small: need %zu bytes", lay.total);
    SGTP_CHECK(((uintptr_t)workspace & 255u) == 0, "workspace must be 256-byte aligned");
    SGTP_CHECK(std::isfinite(sig_lon) && std::isfinite(sig_lat) && sig_lon >= 0.f && sig_lat >= 0.f,
               "prediction sigmas must be finite and >= 0");
    SGTP_CHECK(!(mppi && (sig_lon > 0.f || sig_lat > 0.f)), "perturbed predictions take the SGTP update only");
    PlanArgs a{};
    fill_common(a, trk, p, K, L, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist, status_dev, opts);
    a.mppi_il = il;
    a.sig_lon = sig_lon;
    a.sig_lat = sig_lat;
    RaceDev &R = a.one;
    R = RaceDev{};
    R.track_id = track_id; R.n_v = n_v; R.T = T; R.ego = ego; R.race_tag = race;
    R.n_tail = tail_count(p->mu_tail, T);
    a.races = nullptr;
    a.n_races = 1;
    a.n_agents = n_v;
    a.maxT = T;
    a.xi_total = (long long)n_v * (T + 1) * 4;
    a.u_total = (long long)n_v * T * 2;
    attach_workspace(a, lay, workspace);
    if (mlp) {
        int32_t mT = 0;
        int64_t np = 0;
        const void *wb = nullptr;
        sgtp_status st2 = sgtp_mlp_info(mlp, &mT, &np, nullptr, &wb);
        if (st2) return st2;
        SGTP_CHECK(mT == T, "network horizon %d differs from T=%d", mT, T);
        SGTP_CHECK(K_prop >= 0 && K_prop <= K, "K_prop out of range [0, K]");
        a.mlp_wb = sgtp_mlp_fragments(mlp);
        a.mlp_wf = sgtp_mlp_master(mlp);
        a.K_prop = K_prop;
    }
    SGTP_CHECK(((uintptr_t)prop_out & 15u) == 0, "prop_out must be 16-byte aligned");
    a.feat_out = feat_out;
    a.prop_out = mlp ? (float4 *)prop_out : nullptr;
    return launch_plan(a, n_v - 1, opts, (cudaStream_t)stream);
}

extern "C" sgtp_status sgtp_ibr_plan(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                                     const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K,
                                     int32_t L, int32_t ego, uint64_t seed, uint32_t race, float *xi_out,
                                     int32_t *k_star_out, float *xi_hist, float *u_hist, int32_t *status_dev,
                                     const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                     void *stream)
{
    return ibr_plan_impl(trk, track_id, p, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, xi_out, k_star_out,
                         xi_hist, u_hist, status_dev, opts, nullptr, 0, nullptr, nullptr, workspace, workspace_bytes,
                         stream);
}

extern "C" sgtp_status sgtp_ibr_plan_learned(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                             int32_t n_v, const float *X0, float *U_io, const float *vref_scale,
                                             int32_t T, int32_t K, int32_t L, int32_t ego, uint64_t seed,
                                             uint32_t race, const sgtp_mlp *mlp, int32_t K_prop, float *xi_out,
                                             int32_t *k_star_out, float *xi_hist, float *u_hist, float *feat_out,
                                             float *prop_out, int32_t *status_dev, const sgtp_launch_opts *opts,
                                             void *workspace, size_t workspace_bytes, void *stream)
{
    return ibr_plan_impl(trk, track_id, p, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, xi_out, k_star_out,
                         xi_hist, u_hist, status_dev, opts, mlp, K_prop, feat_out, prop_out, workspace,
                         workspace_bytes, stream);
}



extern "C" size_t sgtp_plan_mppi_workspace_bytes(int32_t n_v, int32_t T, int32_t L, int32_t K)
{
    if (n_v < 1 || T < 1 || L < 0 || K < 1) return 0;
    return Layout((long long)(L + 1) * n_v + 1, n_v, (long long)n_v * (T + 1), T, mppi_part_floats(n_v, K, T)).total;
}

extern "C" sgtp_status sgtp_ibr_plan_mppi(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                                          const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K,
                                          int32_t L, int32_t ego, uint64_t seed, uint32_t race, float lambda,
                                          float *xi_out, int32_t *k_star_out, float *xi_hist, float *u_hist,
                                          int32_t *status_dev, const sgtp_launch_opts *opts, void *workspace,
                                          size_t workspace_bytes, void *stream)
{
    SGTP_CHECK(mppi_inverse(lambda) > 0.f, "lambda must be finite and > 0");
    return ibr_plan_impl(trk, track_id, p, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, xi_out, k_star_out,
                         xi_hist, u_hist, status_dev, opts, nullptr, 0, nullptr, nullptr, workspace, workspace_bytes,
                         stream, lambda);
}

extern "C" sgtp_status sgtp_ibr_plan_perturbed(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                               int32_t n_v, const float *X0, float *U_io, const float *vref_scale,
                                               int32_t T, int32_t K, int32_t L, int32_t ego, uint64_t seed,
                                               uint32_t race, float sigma_lon, float sigma_lat, float *xi_out,
                                               int32_t *k_star_out, float *xi_hist, float *u_hist,
                                               int32_t *status_dev, const sgtp_launch_opts *opts, void *workspace,
                                               size_t workspace_bytes, void *stream)
{
    return ibr_plan_impl(trk, track_id, p, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, xi_out, k_star_out,
                         xi_hist, u_hist, status_dev, opts, nullptr, 0, nullptr, nullptr, workspace, workspace_bytes,
                         stream, 0.f, sigma_lon, sigma_lat);
}

extern "C" sgtp_status sgtp_batch_create(const sgtp_track *trk, const sgtp_race *races, int32_t n_races, int32_t K,
                                         int32_t L, sgtp_batch **out)
{
    SGTP_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    SGTP_CHECK(trk != nullptr && races != nullptr, "NULL argument");
    SGTP_CHECK(n_races >= 1 && n_races <= (1 << 20), "n_races out of range");
    SGTP_CHECK(K >= 1 && K <= SGTP_MAX_K, "K out of range");
    SGTP_CHECK(L >= 0 && L < 4096, "L out of range");
    sgtp_batch *b = new sgtp_batch();
    b->trk = trk; b->n_races = n_races; b->K = K; b->L = L;
    long long ag = 0, u = 0, xi = 0, ks = 0, pos = 0;
    for (int r = 0; r < n_races; ++r) {
        const sgtp_race &q = races[r];
        if (q.track_id < 0 || q.track_id >= trk->n_tracks || q.n_v < 1 || q.n_v > SGTP_MAX_AGENTS || q.T < 1 ||
            q.T > SGTP_MAX_T || q.ego < 0 || q.ego >= q.n_v || q.race_tag >= (1u << 31)) {
            delete b;
            return set_error(SGTP_E_INVALID, "race %d: invalid descriptor", r);
        }
        RaceDev R{};
        R.track_id = q.track_id; R.n_v = q.n_v; R.T = q.T; R.ego = q.ego; R.race_tag = q.race_tag;
        R.n_tail = 0;   // filled per call from mu_tail
        R.agent_off = (int)ag; R.u_off = (int)u; R.xi_off = (int)xi; R.ks_off = (int)ks; R.pos_off = (int)pos;
        R.wcum_all = b->w_all;
        R.wcum_ego = b->w_ego;
        b->w_all += (long long)q.n_v * q.T;
        b->w_ego += q.T;
        b->races.push_back(R);
        ag += q.n_v; u += (long long)q.n_v * q.T * 2; xi += (long long)q.n_v * (q.T + 1) * 4;
        ks += (long long)(L + 1) * q.n_v + 1; pos += (long long)q.n_v * (q.T + 1);
        b->maxT = std::max(b->maxT, q.T);
        b->minT = r == 0 ? q.T : std::min(b->minT, q.T);
        b->max_nv = std::max(b->max_nv, q.n_v);
    }
    if (xi > (1ll << 31) || ag * (long long)K > (1ll << 31) || u > (1ll << 31)) {
        delete b;
        return set_error(SGTP_E_INVALID, "batch too large for 32-bit offsets");
    }
    b->agents = ag; b->u_elems = u; b->xi_elems = xi; b->ks = ks; b->n_pos = pos;
    cudaError_t e = dev_malloc(&b->races_dev, sizeof(RaceDev) * n_races);
    if (e != cudaSuccess) {
        delete b;
        return set_error(SGTP_E_NOMEM, "batch table allocation failed: %s", cudaGetErrorString(e));
    }
    // the table is valid on the device from here on (the simulation entry
    // points read it before any planning call; tail counts follow per call)
    e = cudaMemcpy(b->races_dev, b->races.data(), sizeof(RaceDev) * n_races, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(b->races_dev);
        delete b;
        return set_error(SGTP_E_CUDA, "batch table upload failed: %s", cudaGetErrorString(e));
    }
    *out = b;
    return SGTP_OK;
}

extern "C" void sgtp_batch_destroy(sgtp_batch *b)
{
    if (!b) return;
    cudaFree(b->races_dev);
    delete b;
}

extern "C" sgtp_status sgtp_batch_sizes(const sgtp_batch *b, int64_t *agents, int64_t *u_elems, int64_t *xi_elems,
                                        int64_t *ks, size_t *workspace_bytes)
{
    SGTP_CHECK(b != nullptr, "batch is NULL");
    if (agents) *agents = b->agents;
    if (u_elems) *u_elems = b->u_elems;
    if (xi_elems) *xi_elems = b->xi_elems;
    if (ks) *ks = b->ks;
    if (workspace_bytes) *workspace_bytes = Layout(b->ks, b->agents, b->n_pos, b->maxT, 0, b->n_races).total;
    return SGTP_OK;
}

// The tail counts of the race table depend on mu_tail: refresh the device
// copy when the parameters change it (a blocking copy, never inside a graph
// capture: the capture entry point refreshes before capturing).
static sgtp_status refresh_tail_counts(const sgtp_batch *b, const sgtp_params *p)
{
    sgtp_batch *bm = const_cast<sgtp_batch *>(b);
    bool changed = false;
    for (auto &R : bm->races) {
        const int nt = tail_count(p->mu_tail, R.T);
        if (R.n_tail != nt) { R.n_tail = nt; changed = true; }
    }
    if (changed)
        SGTP_CUDA(cudaMemcpy(bm->races_dev, bm->races.data(), sizeof(RaceDev) * b->n_races, cudaMemcpyHostToDevice));
    return SGTP_OK;
}

static sgtp_status batch_plan_impl(const sgtp_batch *b, const sgtp_params *p, const float *X0, float *U_io,
                                   const float *vref_scale, uint64_t seed, float *xi_out, int32_t *k_star_out,
                                   float *xi_hist, float *u_hist, int32_t *status_dev, const sgtp_launch_opts *opts,
                                   const sgtp_mlp *mlp, int32_t K_prop, float *feat_out, float *prop_out,
                                   void *workspace, size_t workspace_bytes, void *stream, float mppi_lambda = 0.f,
                                   float sig_lon = 0.f, float sig_lat = 0.f)
{
    SGTP_CHECK(b != nullptr, "batch is NULL");
    sgtp_status st = check_params(p);
    if (st) return st;
    SGTP_CHECK(X0 && U_io && vref_scale && xi_out && k_star_out && status_dev, "NULL array");
    const bool mppi = mppi_lambda != 0.f;
    const float il = mppi ? mppi_inverse(mppi_lambda) : 0.f;
    SGTP_CHECK(!mppi || il > 0.f, "lambda must be finite and > 0");
    SGTP_CHECK(!(mppi && mlp), "GA-IBR-MPPI takes the plain sampler only");
    const Layout lay(b->ks, b->agents, b->n_pos, b->maxT, mppi ? mppi_part_floats(b->agents, b->K, b->maxT) : 0,
                     b->n_races);
    SGTP_CHECK(workspace && workspace_bytes >= lay.total, "workspace too small: need %zu bytes", lay.total);
    SGTP_CHECK(((uintptr_t)workspace & 255u) == 0, "workspace must be 256-byte aligned");
    st = refresh_tail_counts(b, p);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    PlanArgs a{};
    SGTP_CHECK(std::isfinite(sig_lon) && std::isfinite(sig_lat) && sig_lon >= 0.f && sig_lat >= 0.f,
               "prediction sigmas must be finite and >= 0");
    SGTP_CHECK(!(mppi && (sig_lon > 0.f || sig_lat > 0.f)), "perturbed predictions take the SGTP update only");
    fill_common(a, b->trk, p, b->K, b->L, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist,
                status_dev, opts);
    a.mppi_il = il;
    a.sig_lon = sig_lon;
    a.sig_lat = sig_lat;
    a.races = b->races_dev;
    a.n_races = b->n_races;
    a.w_units_all = b->w_all;
    a.w_units_ego = b->w_ego;
    a.n_agents = (int)b->agents;
    a.maxT = b->maxT;
    a.xi_total = b->xi_elems;
    a.u_total = b->u_elems;
    attach_workspace(a, lay, workspace);
    if (mlp) {
        int32_t mT = 0;
        sgtp_status st2 = sgtp_mlp_info(mlp, &mT, nullptr, nullptr, nullptr);
        if (st2) return st2;
        for (const auto &R : b->races) SGTP_CHECK(R.T == mT, "race horizon %d differs from the network's %d", R.T, mT);
        SGTP_CHECK(K_prop >= 0 && K_prop <= b->K, "K_prop out of range [0, K]");
        a.mlp_wb = sgtp_mlp_fragments(mlp);
        a.mlp_wf = sgtp_mlp_master(mlp);
        a.K_prop = K_prop;
    }
    SGTP_CHECK(((uintptr_t)prop_out & 15u) == 0, "prop_out must be 16-byte aligned");
    a.feat_out = feat_out;
    a.prop_out = mlp ? (float4 *)prop_out : nullptr;
    return launch_plan(a, b->max_nv - 1, opts, s);
}

extern "C" sgtp_status sgtp_batch_plan(const sgtp_batch *b, const sgtp_params *p, const float *X0, float *U_io,
                                       const float *vref_scale, uint64_t seed, float *xi_out, int32_t *k_star_out,
                                       float *xi_hist, float *u_hist, int32_t *status_dev,
                                       const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                       void *stream)
{
    return batch_plan_impl(b, p, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist, status_dev, opts,
                           nullptr, 0, nullptr, nullptr, workspace, workspace_bytes, stream);
}

extern "C" sgtp_status sgtp_batch_plan_learned(const sgtp_batch *b, const sgtp_params *p, const sgtp_mlp *mlp,
                                               int32_t K_prop, const float *X0, float *U_io,
                                               const float *vref_scale, uint64_t seed, float *xi_out,
                                               int32_t *k_star_out, float *xi_hist, float *u_hist, float *feat_out,
                                               float *prop_out, int32_t *status_dev, const sgtp_launch_opts *opts,
                                               void *workspace, size_t workspace_bytes, void *stream)
{
    return batch_plan_impl(b, p, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist, status_dev, opts,
                           mlp, K_prop, feat_out, prop_out, workspace, workspace_bytes, stream);
}

extern "C" sgtp_status sgtp_batch_mppi_workspace_bytes(const sgtp_batch *b, size_t *workspace_bytes)
{
    SGTP_CHECK(b != nullptr && workspace_bytes != nullptr, "NULL argument");
    *workspace_bytes =
        Layout(b->ks, b->agents, b->n_pos, b->maxT, mppi_part_floats(b->agents, b->K, b->maxT), b->n_races).total;
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_batch_plan_mppi(const sgtp_batch *b, const sgtp_params *p, float lambda, const float *X0,
                                            float *U_io, const float *vref_scale, uint64_t seed, float *xi_out,
                                            int32_t *k_star_out, float *xi_hist, float *u_hist, int32_t *status_dev,
                                            const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                            void *stream)
{
    SGTP_CHECK(mppi_inverse(lambda) > 0.f, "lambda must be finite and > 0");
    return batch_plan_impl(b, p, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist, status_dev, opts,
                           nullptr, 0, nullptr, nullptr, workspace, workspace_bytes, stream, lambda);
}

extern "C" sgtp_status sgtp_batch_plan_perturbed(const sgtp_batch *b, const sgtp_params *p, float sigma_lon,
                                                 float sigma_lat, const float *X0, float *U_io,
                                                 const float *vref_scale, uint64_t seed, float *xi_out,
                                                 int32_t *k_star_out, float *xi_hist, float *u_hist,
                                                 int32_t *status_dev, const sgtp_launch_opts *opts, void *workspace,
                                                 size_t workspace_bytes, void *stream)
{
    return batch_plan_impl(b, p, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist, status_dev, opts,
                           nullptr, 0, nullptr, nullptr, workspace, workspace_bytes, stream, 0.f, sigma_lon,
                           sigma_lat);
}

// ================================================================ CUDA graphs
// A planning call captured once and replayed: the graph holds the two
// memset nodes and the plan kernel node with every pointer fixed, so a
// receding-horizon loop rewrites X0 / U_io in place and relaunches.
struct sgtp_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;   // the plan kernel node
    cudaKernelNodeParams kp{};        // its launch configuration
    PlanArgs args{};                  // its parameter block (seed updates)
};

extern "C" void sgtp_graph_destroy(sgtp_graph *G)
{
    if (!G) return;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    delete G;
}

template <typename F>
static sgtp_status capture_plan_graph(F body, sgtp_graph **out)
{
    SGTP_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    sgtp_status st = configure_plan_kernels();
    if (st) return st;
    cudaStream_t cs = nullptr;
    SGTP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return set_error(SGTP_E_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    }
    st = body(cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st) return st;
        return set_error(SGTP_E_CUDA, "stream capture of the plan failed: %s", cudaGetErrorString(e));
    }
    sgtp_graph *G = new sgtp_graph();
    G->graph = g;
    size_t n = 0;
    if ((e = cudaGraphGetNodes(g, nullptr, &n)) == cudaSuccess) {
        std::vector<cudaGraphNode_t> nodes(n);
        e = cudaGraphGetNodes(g, nodes.data(), &n);
        for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
            cudaGraphNodeType t;
            if ((e = cudaGraphNodeGetType(nodes[i], &t)) == cudaSuccess && t == cudaGraphNodeTypeKernel) G->node = nodes[i];
        }
    }
    if (e == cudaSuccess && G->node) e = cudaGraphKernelNodeGetParams(G->node, &G->kp);
    if (e == cudaSuccess && G->node) std::memcpy(&G->args, G->kp.kernelParams[0], sizeof(PlanArgs));
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, g, 0);
    if (e != cudaSuccess || !G->node) {
        sgtp_graph_destroy(G);
        return set_error(SGTP_E_CUDA, "graph setup failed: %s", e ? cudaGetErrorString(e) : "no kernel node");
    }
    *out = G;
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_graph_capture_plan(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                               int32_t n_v, const float *X0, float *U_io, const float *vref_scale,
                                               int32_t T, int32_t K, int32_t L, int32_t ego, uint64_t seed,
                                               uint32_t race, float *xi_out, int32_t *k_star_out, float *xi_hist,
                                               float *u_hist, int32_t *status_dev, const sgtp_launch_opts *opts,
                                               void *workspace, size_t workspace_bytes, sgtp_graph **out)
{
    return capture_plan_graph(
        [&](cudaStream_t cs) {
            return sgtp_ibr_plan(trk, track_id, p, n_v, X0, U_io, vref_scale, T, K, L, ego, seed, race, xi_out,
                                 k_star_out, xi_hist, u_hist, status_dev, opts, workspace, workspace_bytes, cs);
        },
        out);
}

extern "C" sgtp_status sgtp_graph_capture_batch(const sgtp_batch *b, const sgtp_params *p, const float *X0,
                                                float *U_io, const float *vref_scale, uint64_t seed, float *xi_out,
                                                int32_t *k_star_out, float *xi_hist, float *u_hist,
                                                int32_t *status_dev, const sgtp_launch_opts *opts, void *workspace,
                                                size_t workspace_bytes, sgtp_graph **out)
{
    SGTP_CHECK(b != nullptr, "batch is NULL");
    sgtp_status st = check_params(p);
    if (st) return st;
    st = refresh_tail_counts(b, p);     // any table upload happens before the capture
    if (st) return st;
    return capture_plan_graph(
        [&](cudaStream_t cs) {
            return sgtp_batch_plan(b, p, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist,
                                   status_dev, opts, workspace, workspace_bytes, cs);
        },
        out);
}

extern "C" sgtp_status sgtp_graph_set_seed(sgtp_graph *G, uint64_t seed)
{
    SGTP_CHECK(G != nullptr, "graph is NULL");
    G->args.key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    G->args.rk = make_round_keys(G->args.key);
    void *params[] = {&G->args};
    cudaKernelNodeParams kp = G->kp;
    kp.kernelParams = params;
    kp.extra = nullptr;
    SGTP_CUDA(cudaGraphExecKernelNodeSetParams(G->exec, G->node, &kp));
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_graph_launch(sgtp_graph *G, void *stream)
{
    SGTP_CHECK(G != nullptr, "graph is NULL");
    SGTP_CUDA(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
    count_launch();
    return SGTP_OK;
}
