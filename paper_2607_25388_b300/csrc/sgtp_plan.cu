// sgtp_plan.cu -- the SGTP planning call (Alg. 1) as one persistent
// cooperative kernel, for one race or a batch of independent races.
//
// Phases of the kernel (grid barriers in between):
//   setup   : per vehicle, Frenet of x_{i,t} (global search), reference
//             trajectory (Sec. III-A), nominal rollout of the current U-bar
//             = the opponents' predictions for round 0;
//   round r : every (race, vehicle, sample tile) item evaluates its samples
//             and folds their selection keys into the best response's key;
//   winner r: per vehicle, re-roll of the selected sample k*, warm start
//             U-bar <- U^(k*) (Alg. 1, update step), and the new prediction
//             (positions, progress gain, tail offset) for the next round.
// Rounds 0..L are Jacobi rounds over all vehicles (round 0 without the game
// term); round L+1 is the extra ego response.
#include <cmath>
#include <cstring>

#include "sgtp_host.hpp"
#include "sgtp_rollout.cuh"

using namespace sgtp;

namespace {

constexpr int kMaxMoves = 64;

struct RaceDev {
    int track_id, n_v, T, ego;
    unsigned race_tag;
    int n_tail;
    int agent_off;   // first vehicle of the race in the batch arrays
    int u_off;       // float offset into U_io (n_v * T * 2 per race)
    int xi_off;      // float offset into xi_out (n_v * (T+1) * 4)
    int ks_off;      // offset into k_star_out ((L+1) * n_v + 1)
    int pos_off;     // float2 offset into each prediction buffer (n_v * (T+1))
    int item_all;    // BR items before this race in a Jacobi round
    int item_ego;    // BR items before this race in the extra ego round
    int pad[3];
};

struct AgentDev {
    float4 x0;
    float s_t, d_t;
    int j0, race;
};

struct PlanArgs {
    const TrackDesc *tdesc;
    const float4 *A, *B, *W, *C;
    sgtp_params p;
    const RaceDev *races;     // NULL: single race `one`
    RaceDev one;
    int n_races, n_agents;
    int K, L, tiles;          // tiles of blockDim samples per best response
    int items_all, items_ego; // BR items of a Jacobi round / the extra round
    int maxT;
    const float *X0;
    float *U_io;
    const float *vref;
    uint2 key;
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
};

__device__ __forceinline__ RaceDev get_race(const PlanArgs &a, int r) { return a.races ? a.races[r] : a.one; }

// Workspace written inside the launch by other CTAs is read through L2.
__device__ __forceinline__ AgentDev load_agent(const AgentDev *p)
{
    const float4 *q = (const float4 *)p;
    const float4 u = __ldcg(q), w = __ldcg(q + 1);
    AgentDev A;
    A.x0 = u;
    A.s_t = w.x; A.d_t = w.y; A.j0 = __float_as_int(w.z); A.race = __float_as_int(w.w);
    return A;
}

__device__ __forceinline__ TrackView get_track(const PlanArgs &a, int id)
{
    const TrackDesc d = a.tdesc[id];
    TrackView v;
    v.A = a.A + d.offset; v.B = a.B + d.offset; v.W = a.W + d.offset; v.C = a.C + d.offset;
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

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_status(const int *p)
{
    return *(const volatile int *)p;
}

// Grid-wide barrier of a cooperative launch.  Every wait has a limit: a CTA
// whose wait runs out records SGTP_E_TIMEOUT and returns false, and every
// other waiter stops as soon as it sees a fatal status.
__device__ bool grid_barrier(const PlanArgs &a, bool skip_arrival)
{
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned *count = a.bar, *gen = a.bar + 1;
        const unsigned g = ld_acquire(gen);
        __threadfence();
        bool released = false;
        if (!skip_arrival) {
            const unsigned prev = atomicAdd(count, 1u);
            if (prev == gridDim.x - 1) {
                atomicExch(count, 0u);
                __threadfence();
                atomicAdd(gen, 1u);
                released = true;
            }
        }
        if (!released) {
            const unsigned long long t0 = global_ns();
            while (ld_acquire(gen) == g) {
                if (ld_status(a.status) & 0xff) break;
                if (global_ns() - t0 > (unsigned long long)a.timeout_ns) {
                    atomicOr(a.status, SGTP_E_TIMEOUT);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        ok_sh = (ld_status(a.status) & 0xff) == 0;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Roll out one selected (or nominal) control sequence of a vehicle, from the
// same noise, control and dynamics functions as the sample evaluation, and
// write its states, controls and Frenet summary.  One thread.
__device__ void reroll(const PlanArgs &a, const TrackView &tv, const AgentDev &ag, int T, int n_tail,
                       const float *U, unsigned k, bool zero_noise, unsigned agent_round, unsigned race_tag,
                       float *U_out, float2 *pos_out, float *xi_a, float *xi_b, float *u_hist, float2 *summ_out,
                       int &flag)
{
    const SegWindow nowin{nullptr, nullptr, 0, 0};
    const float invL = 1.0f / tv.L;
    float x = ag.x0.x, y = ag.x0.y, psi = ag.x0.z, v = ag.x0.w;
    float s = ag.s_t, dsum = 0.f;
    int j = ag.j0;
    if (pos_out) pos_out[0] = make_float2(x, y);
    if (xi_a) { xi_a[0] = x; xi_a[1] = y; xi_a[2] = psi; xi_a[3] = v; }
    if (xi_b) { xi_b[0] = x; xi_b[1] = y; xi_b[2] = psi; xi_b[3] = v; }
    for (int m = 0; 2 * m < T; ++m) {
        float2 z[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (!zero_noise) {
            const uint4 w = philox4x32_10(make_uint4(k, (unsigned)m, agent_round, race_tag), a.key);
            z[0] = box_muller(w.x, w.y);
            z[1] = box_muller(w.z, w.w);
        }
        for (int h = 0; h < 2; ++h) {
            const int tau = 2 * m + h;
            if (tau >= T) break;
            const float2 ub = make_float2(__ldcg(U + 2 * tau), __ldcg(U + 2 * tau + 1));
            const float2 u = sample_control(a.p, ub, z[h]);
            if (U_out) { U_out[2 * tau] = u.x; U_out[2 * tau + 1] = u.y; }
            if (u_hist) { u_hist[2 * tau] = u.x; u_hist[2 * tau + 1] = u.y; }
            bicycle_step(a.p, x, y, psi, v, u.x, u.y);
            const FrenetPt f = frenet_walk(tv, nowin, j, x, y, kMaxMoves, flag);
            s = s + wrap_len(f.s - s, tv.L, invL);
            const int st = tau + 1;
            if (st > T - n_tail) dsum = dsum + f.d;
            if (pos_out) pos_out[st] = make_float2(x, y);
            if (xi_a) { xi_a[4 * st] = x; xi_a[4 * st + 1] = y; xi_a[4 * st + 2] = psi; xi_a[4 * st + 3] = v; }
            if (xi_b) { xi_b[4 * st] = x; xi_b[4 * st + 1] = y; xi_b[4 * st + 2] = psi; xi_b[4 * st + 3] = v; }
        }
    }
    if (summ_out) *summ_out = make_float2(s - ag.s_t, dsum / (float)n_tail);
}

struct PlanSmem {
    size_t sA, sB, ref, ubar, opp, osum, odbar, total;
    __host__ __device__ PlanSmem(int Wn, int maxT, int maxO)
    {
        auto up = [](size_t x) { return (x + 15) & ~(size_t)15; };
        sA = 16;
        sB = sA + sizeof(float4) * Wn;
        ref = sB + sizeof(float4) * Wn;
        ubar = up(ref + sizeof(float4) * (maxT + 1));
        opp = up(ubar + sizeof(float2) * maxT);
        osum = up(opp + sizeof(float2) * (size_t)maxT * maxO);
        odbar = up(osum + sizeof(float4) * maxO);
        total = up(odbar + sizeof(float) * maxO);
    }
};

template <int MAXO>
__global__ void __launch_bounds__(256, 2) plan_kernel(PlanArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long cta_key;
    __shared__ int abort_sh;
    const PlanSmem SL(a.Wn, a.maxT, MAXO);
    unsigned long long *mbar = (unsigned long long *)smem;
    float4 *sA = (float4 *)(smem + SL.sA);
    float4 *sB = (float4 *)(smem + SL.sB);
    float4 *sref = (float4 *)(smem + SL.ref);
    float2 *subar = (float2 *)(smem + SL.ubar);
    float2 *sopp = (float2 *)(smem + SL.opp);
    float4 *sosum = (float4 *)(smem + SL.osum);
    float *sodbar = (float *)(smem + SL.odbar);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int gwarp = blockIdx.x * nwarps + warp, total_warps = gridDim.x * nwarps;
    const bool skip = (a.debug_flags & SGTP_DEBUG_SKIP_BARRIER_ARRIVAL) && blockIdx.x == 0;
    int flag = 0;
    unsigned phase = 0;
    bool ok = true;
    if (threadIdx.x == 0) mbar_init(mbar, 1);

    // ------------------------------------------------------------ setup
    for (int ag = gwarp; ag < a.n_agents; ag += total_warps) {
        const int ri = find_race(a, ag, [](const RaceDev &r) { return r.agent_off; });
        const RaceDev R = get_race(a, ri);
        const int i = ag - R.agent_off;
        const TrackView tv = get_track(a, R.track_id);
        const float4 x0 = make_float4(a.X0[4 * ag], a.X0[4 * ag + 1], a.X0[4 * ag + 2], a.X0[4 * ag + 3]);
        const int j0 = nearest_segment_warp(tv, x0.x, x0.y);
        if (lane == 0) {
            const FrenetPt f = frenet_at(tv, j0, x0.x, x0.y);
            AgentDev A;
            A.x0 = x0; A.s_t = f.s; A.d_t = f.d; A.j0 = j0; A.race = ri;
            a.agents[ag] = A;
            // reference progress recursion s^r_{tau+1} = s^r_tau + dt v^r(s^r_tau)
            const float vs = a.vref[ag];
            float4 *ref = a.ref + (size_t)R.pos_off + (size_t)i * (R.T + 1);
            int jr = j0;
            float sr = f.s;
            ref[0] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int tau = 0; tau < R.T; ++tau) {
                const float4 r0 = reference_at(tv, jr, sr);
                sr = __fmaf_rn(a.p.dt, __fmul_rn(vs, r0.w), sr);
                float4 r1 = reference_at(tv, jr, sr);
                r1.w = __fmul_rn(r1.w, vs);
                ref[tau + 1] = r1;
            }
            // nominal rollout: round-0 predictions
            reroll(a, tv, A, R.T, R.n_tail, a.U_io + R.u_off + (size_t)i * R.T * 2, 0u, true, 0u, 0u, nullptr,
                   a.pos[0] + R.pos_off + (size_t)i * (R.T + 1), nullptr, nullptr, nullptr, a.summ[0] + ag, flag);
        }
    }
    {
        // fresh selection keys for every best response of the plan
        const RaceDev last = get_race(a, a.n_races - 1);
        const int n_keys = a.races ? (last.ks_off + (a.L + 1) * last.n_v + 1) : ((a.L + 1) * a.one.n_v + 1);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_keys; i += gridDim.x * blockDim.x)
            a.keys[i] = ~0ull;
    }
    ok = grid_barrier(a, skip);

    for (int round = 0; ok && round <= a.L + 1; ++round) {
        const bool extra = round == a.L + 1;
        const int bin = round & 1, bout = bin ^ 1;
        const int n_items = extra ? a.items_ego : a.items_all;
        const int i0 = (int)((long long)n_items * blockIdx.x / gridDim.x);
        const int i1 = (int)((long long)n_items * (blockIdx.x + 1) / gridDim.x);
        int cur = -1;                 // current vehicle (global index) staged
        unsigned long long *cur_slot = nullptr;
        BRView bv;
        for (int item = i0; item < i1; ++item) {
            int ri, i, t;
            if (!extra) {
                ri = find_race(a, item, [](const RaceDev &r) { return r.item_all; });
                const RaceDev R0 = get_race(a, ri);
                const int local = item - R0.item_all;
                i = local / a.tiles;
                t = local - i * a.tiles;
            } else {
                ri = find_race(a, item, [](const RaceDev &r) { return r.item_ego; });
                const RaceDev R0 = get_race(a, ri);
                i = R0.ego;
                t = item - R0.item_ego;
            }
            const RaceDev R = get_race(a, ri);
            const int ag = R.agent_off + i;
            if (ag != cur) {
                // flush the previous vehicle's key, then stage this one
                __syncthreads();
                if (threadIdx.x == 0 && cur_slot) atomicMin(cur_slot, cta_key);
                const TrackView tv = get_track(a, R.track_id);
                const AgentDev A = load_agent(a.agents + ag);
                const int Wn = min(a.Wn, tv.N);
                const int back = min(a.back, Wn / 4);
                const int w0 = wrap_index(A.j0 - back, tv.N);
                if (threadIdx.x == 0) {
                    cta_key = ~0ull;
                    // track window by bulk copy (TMA)
                    const int n1 = min(Wn, tv.N - w0);
                    mbar_expect_tx(mbar, (unsigned)(2 * Wn * sizeof(float4)));
                    bulk_g2s(sA, tv.A + w0, (unsigned)(n1 * sizeof(float4)), mbar);
                    bulk_g2s(sB, tv.B + w0, (unsigned)(n1 * sizeof(float4)), mbar);
                    if (n1 < Wn) {
                        bulk_g2s(sA + n1, tv.A, (unsigned)((Wn - n1) * sizeof(float4)), mbar);
                        bulk_g2s(sB + n1, tv.B, (unsigned)((Wn - n1) * sizeof(float4)), mbar);
                    }
                }
                const int T = R.T, n_opp = R.n_v - 1;
                const float *U = a.U_io + R.u_off + (size_t)i * T * 2;
                for (int q = threadIdx.x; q < T; q += blockDim.x) subar[q] = make_float2(__ldcg(U + 2 * q), __ldcg(U + 2 * q + 1));
                const float4 *gref = a.ref + (size_t)R.pos_off + (size_t)i * (T + 1);
                for (int q = threadIdx.x; q <= T; q += blockDim.x) sref[q] = __ldcg(gref + q);
                const float2 *pin = a.pos[bin] + R.pos_off;
                for (int q = threadIdx.x; q < T * n_opp; q += blockDim.x) {
                    const int tau = q / n_opp, o = q - tau * n_opp;
                    const int jv = o < i ? o : o + 1;
                    sopp[q] = __ldcg(pin + (size_t)jv * (T + 1) + tau + 1);
                }
                if (threadIdx.x < n_opp) {
                    const int o = threadIdx.x;
                    const int jv = o < i ? o : o + 1;
                    const AgentDev B = load_agent(a.agents + R.agent_off + jv);
                    const float2 sm = __ldcg(a.summ[bin] + R.agent_off + jv);
                    const float ds_t = wrap_len(A.s_t - B.s_t, tv.L, 1.0f / tv.L);
                    const float alpha = 1.0f / (1.0f + fabsf(ds_t) / (a.p.s_contest + a.p.eps_alpha));
                    const float gamma = (ds_t > a.p.s_role && ds_t < a.p.s_contest) ? a.p.w_block : 0.f;
                    sosum[o] = make_float4(ds_t, alpha, gamma, sm.x);
                    sodbar[o] = sm.y;
                }
                bv.tv = tv;
                bv.win = SegWindow{sA, sB, w0, Wn};
                bv.ubar = subar; bv.ref = sref; bv.opp = sopp; bv.osum = sosum; bv.odbar = sodbar;
                bv.x0 = A.x0; bv.s_t = A.s_t; bv.d_t = A.d_t; bv.j0 = A.j0;
                bv.T = T; bv.n_opp = n_opp; bv.n_tail = R.n_tail;
                bv.invL = 1.0f / tv.L;
                bv.max_moves = kMaxMoves;
                bv.key = a.key;
                bv.ctr_agent_round = (unsigned)i | ((unsigned)round << 16);
                bv.ctr_race = R.race_tag;
                bv.stream_bit = 0u;
                cur = ag;
                cur_slot = a.keys + R.ks_off + (extra ? (a.L + 1) * R.n_v : round * R.n_v + i);
                __syncthreads();
                if (threadIdx.x == 0) {
                    if (!mbar_wait_bounded(mbar, phase, (unsigned long long)a.timeout_ns))
                        atomicOr(a.status, SGTP_E_TIMEOUT);
                    abort_sh = (ld_status(a.status) & 0xff) != 0;
                }
                phase ^= 1u;
                __syncthreads();
                if (abort_sh) { ok = false; break; }
            }
            const unsigned k = (unsigned)t * blockDim.x + threadIdx.x;
            unsigned long long best = ~0ull;
            if (k < (unsigned)a.K) {
                const SampleResult r = run_candidate<MAXO, false>(bv, a.p, k, round > 0, false, flag, nullptr,
                                                                  nullptr, nullptr);
                best = make_key(r.feasible, r.cost, r.viol, k);
            }
            best = warp_min_u64(best);
            if (lane == 0) atomicMin(&cta_key, best);
        }
        if (!ok) break;
        __syncthreads();
        if (threadIdx.x == 0 && cur_slot) atomicMin(cur_slot, cta_key);
        if (!grid_barrier(a, skip)) break;

        // -------------------------------------------------------- winners
        for (int ag = gwarp; ag < a.n_agents; ag += total_warps) {
            if (lane != 0) continue;
            const AgentDev A = load_agent(a.agents + ag);
            const RaceDev R = get_race(a, A.race);
            const int i = ag - R.agent_off;
            const int T = R.T;
            const bool active = !extra || i == R.ego;
            const size_t xo = (size_t)R.xi_off + (size_t)i * (T + 1) * 4;
            const size_t uo = (size_t)R.u_off + (size_t)i * T * 2;
            if (!active) {
                if (a.xi_hist) {
                    for (int q = 0; q < (T + 1) * 4; ++q)
                        a.xi_hist[(size_t)round * a.xi_total + xo + q] = __ldcg(a.xi_out + xo + q);
                }
                if (a.u_hist) {
                    for (int q = 0; q < T * 2; ++q)
                        a.u_hist[(size_t)round * a.u_total + uo + q] = __ldcg(a.U_io + uo + q);
                }
                continue;
            }
            const int slot = extra ? (a.L + 1) * R.n_v : round * R.n_v + i;
            const unsigned long long key = __ldcg(a.keys + R.ks_off + slot);
            const unsigned ks = (unsigned)(key & 0x7fffffffull);
            a.k_star_out[R.ks_off + slot] = (int)ks;
            const TrackView tv = get_track(a, R.track_id);
            float *xi_final = (round == a.L || extra) ? a.xi_out + xo : nullptr;
            float *xi_h = a.xi_hist ? a.xi_hist + (size_t)round * a.xi_total + xo : nullptr;
            float *u_h = a.u_hist ? a.u_hist + (size_t)round * a.u_total + uo : nullptr;
            reroll(a, tv, A, T, R.n_tail, a.U_io + uo, ks, false, (unsigned)i | ((unsigned)round << 16),
                   R.race_tag, a.U_io + uo, extra ? nullptr : a.pos[bout] + R.pos_off + (size_t)i * (T + 1),
                   xi_final, xi_h, u_h, extra ? nullptr : a.summ[bout] + ag, flag);
        }
        if (round <= a.L) ok = grid_barrier(a, skip);
    }
    if (flag) atomicOr(a.status, SGTP_E_DEVICE << 8);
}

// ================================================================ host side
struct Layout {
    size_t bar, keys, agents, ref, pos0, pos1, summ0, summ1, total;
    Layout(long long n_keys, long long n_agents, long long n_pos)
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
        total = up(summ1 + sizeof(float2) * n_agents);
    }
};

int maxo_bucket(int n) { return n <= 1 ? 1 : n <= 3 ? 3 : n <= 9 ? 9 : 15; }

template <int MAXO>
sgtp_status launch_plan_t(PlanArgs &a, const sgtp_launch_opts *opts, cudaStream_t s)
{
    const int block = 256;
    const size_t smem = PlanSmem(a.Wn, a.maxT, MAXO).total;
    static int configured = 0;
    if (!configured) {
        SGTP_CUDA(cudaFuncSetAttribute(plan_kernel<MAXO>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        configured = 1;
    }
    int dev = 0, sms = 0, per_sm = 0;
    SGTP_CUDA(cudaGetDevice(&dev));
    SGTP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SGTP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_kernel<MAXO>, block, smem));
    SGTP_CHECK(per_sm >= 1, "plan kernel does not fit on an SM (smem %zu)", smem);
    if (opts && opts->ctas_per_sm > 0 && opts->ctas_per_sm < per_sm) per_sm = opts->ctas_per_sm;
    const int grid = sms * per_sm;
    void *args[] = {&a};
    SGTP_CUDA(cudaMemsetAsync(a.bar, 0, 256, s));
    SGTP_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), s));
    SGTP_CUDA(cudaLaunchCooperativeKernel((const void *)plan_kernel<MAXO>, grid, block, args, smem, s));
    count_launch();
    return SGTP_OK;
}

sgtp_status launch_plan(PlanArgs &a, int max_opp, const sgtp_launch_opts *opts, cudaStream_t s)
{
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
    a.A = trk->A; a.B = trk->B; a.W = trk->W; a.C = trk->C;
    a.p = *p;
    a.K = K; a.L = L;
    a.tiles = (K + 255) / 256;
    a.X0 = X0; a.U_io = U_io; a.vref = vref;
    a.key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    a.xi_out = xi_out; a.k_star_out = k_star_out; a.xi_hist = xi_hist; a.u_hist = u_hist;
    a.status = status;
    a.Wn = (opts && opts->window > 0) ? opts->window : 1024;
    a.back = 64;
    a.timeout_ns = (opts && opts->wait_timeout_ns > 0) ? opts->wait_timeout_ns : 1000000000ll;
    a.debug_flags = opts ? opts->debug_flags : 0;
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
}

}  // namespace

struct sgtp_batch {
    const sgtp_track *trk = nullptr;
    int n_races = 0, K = 0, L = 0;
    std::vector<RaceDev> races;
    RaceDev *races_dev = nullptr;
    long long agents = 0, u_elems = 0, xi_elems = 0, ks = 0, n_pos = 0;
    int items_all = 0, items_ego = 0, maxT = 0, max_nv = 0;
};

extern "C" size_t sgtp_plan_workspace_bytes(int32_t n_v, int32_t T, int32_t L)
{
    if (n_v < 1 || T < 1 || L < 0) return 0;
    return Layout((long long)(L + 1) * n_v + 1, n_v, (long long)n_v * (T + 1)).total;
}

extern "C" sgtp_status sgtp_ibr_plan(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                                     const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K,
                                     int32_t L, int32_t ego, uint64_t seed, uint32_t race, float *xi_out,
                                     int32_t *k_star_out, float *xi_hist, float *u_hist, int32_t *status_dev,
                                     const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                     void *stream)
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
    const Layout lay((long long)(L + 1) * n_v + 1, n_v, (long long)n_v * (T + 1));
    SGTP_CHECK(workspace && workspace_bytes >= lay.total, "workspace too small: need %zu bytes", lay.total);
    SGTP_CHECK(((uintptr_t)workspace & 255u) == 0, "workspace must be 256-byte aligned");
    PlanArgs a{};
    fill_common(a, trk, p, K, L, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist, status_dev, opts);
    RaceDev &R = a.one;
    R = RaceDev{};
    R.track_id = track_id; R.n_v = n_v; R.T = T; R.ego = ego; R.race_tag = race;
    R.n_tail = tail_count(p->mu_tail, T);
    a.races = nullptr;
    a.n_races = 1;
    a.n_agents = n_v;
    a.items_all = n_v * a.tiles;
    a.items_ego = a.tiles;
    a.maxT = T;
    a.xi_total = (long long)n_v * (T + 1) * 4;
    a.u_total = (long long)n_v * T * 2;
    attach_workspace(a, lay, workspace);
    return launch_plan(a, n_v - 1, opts, (cudaStream_t)stream);
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
    const int tiles = (K + 255) / 256;
    long long ag = 0, u = 0, xi = 0, ks = 0, pos = 0, it_all = 0, it_ego = 0;
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
        R.item_all = (int)it_all; R.item_ego = (int)it_ego;
        b->races.push_back(R);
        ag += q.n_v; u += (long long)q.n_v * q.T * 2; xi += (long long)q.n_v * (q.T + 1) * 4;
        ks += (long long)(L + 1) * q.n_v + 1; pos += (long long)q.n_v * (q.T + 1);
        it_all += (long long)q.n_v * tiles; it_ego += tiles;
        b->maxT = std::max(b->maxT, q.T);
        b->max_nv = std::max(b->max_nv, q.n_v);
    }
    if (xi > (1ll << 31) || it_all > (1ll << 31) || u > (1ll << 31)) {
        delete b;
        return set_error(SGTP_E_INVALID, "batch too large for 32-bit offsets");
    }
    b->agents = ag; b->u_elems = u; b->xi_elems = xi; b->ks = ks; b->n_pos = pos;
    b->items_all = (int)it_all; b->items_ego = (int)it_ego;
    cudaError_t e = cudaMalloc(&b->races_dev, sizeof(RaceDev) * n_races);
    if (e != cudaSuccess) {
        delete b;
        return set_error(SGTP_E_NOMEM, "batch table allocation failed: %s", cudaGetErrorString(e));
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
    if (workspace_bytes) *workspace_bytes = Layout(b->ks, b->agents, b->n_pos).total;
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_batch_plan(const sgtp_batch *b, const sgtp_params *p, const float *X0, float *U_io,
                                       const float *vref_scale, uint64_t seed, float *xi_out, int32_t *k_star_out,
                                       float *xi_hist, float *u_hist, int32_t *status_dev,
                                       const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                       void *stream)
{
    SGTP_CHECK(b != nullptr, "batch is NULL");
    sgtp_status st = check_params(p);
    if (st) return st;
    SGTP_CHECK(X0 && U_io && vref_scale && xi_out && k_star_out && status_dev, "NULL array");
    const Layout lay(b->ks, b->agents, b->n_pos);
    SGTP_CHECK(workspace && workspace_bytes >= lay.total, "workspace too small: need %zu bytes", lay.total);
    SGTP_CHECK(((uintptr_t)workspace & 255u) == 0, "workspace must be 256-byte aligned");
    // per-call tail counts depend on mu_tail: refresh the device race table
    sgtp_batch *bm = const_cast<sgtp_batch *>(b);
    bool changed = false;
    for (auto &R : bm->races) {
        const int nt = tail_count(p->mu_tail, R.T);
        if (R.n_tail != nt) { R.n_tail = nt; changed = true; }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (changed) {
        SGTP_CUDA(cudaMemcpy(bm->races_dev, bm->races.data(), sizeof(RaceDev) * b->n_races, cudaMemcpyHostToDevice));
    }
    PlanArgs a{};
    fill_common(a, b->trk, p, b->K, b->L, X0, U_io, vref_scale, seed, xi_out, k_star_out, xi_hist, u_hist,
                status_dev, opts);
    a.races = b->races_dev;
    a.n_races = b->n_races;
    a.n_agents = (int)b->agents;
    a.items_all = b->items_all;
    a.items_ego = b->items_ego;
    a.maxT = b->maxT;
    a.xi_total = b->xi_elems;
    a.u_total = b->u_elems;
    attach_workspace(a, lay, workspace);
    return launch_plan(a, b->max_nv - 1, opts, s);
}
