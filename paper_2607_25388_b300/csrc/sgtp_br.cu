// sgtp_br.cu -- raceline setup and the single best-response entry points.
//
//   sgtp_track_create*   raceline G (Sec. II, Preliminaries) on the device
//   sgtp_rollout_costs   K candidates: cost (Eq. allc), h (Eq. selection), nu
//   sgtp_best_response   the same, plus selection with the least-violation
//                        fallback (Sec. III-B) and the re-rolled winner
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "sgtp_host.hpp"
#include "sgtp_rollout.cuh"

using namespace sgtp;

// ================================================================ host utils
namespace sgtp {

static thread_local std::string g_error;
static std::atomic<long long> g_launches{0};

sgtp_status set_error(sgtp_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return s;
}

void count_launch(int n) { g_launches += n; }

sgtp_status check_params(const sgtp_params *p)
{
    SGTP_CHECK(p != nullptr, "params is NULL");
    SGTP_CHECK(p->dt > 0.f && std::isfinite(p->dt), "dt must be > 0");
    SGTP_CHECK(p->wheelbase > 0.f, "wheelbase must be > 0");
    SGTP_CHECK(p->a_min <= p->a_max, "a_min > a_max");
    SGTP_CHECK(p->delta_max >= 0.f && p->delta_max < 1.5f, "delta_max must be in [0, 1.5)");
    SGTP_CHECK(p->v_min <= p->v_max, "v_min > v_max");
    SGTP_CHECK(p->sigma_a >= 0.f && p->sigma_delta >= 0.f, "negative sigma");
    SGTP_CHECK(p->mu_tail > 0.f && p->mu_tail <= 1.f, "mu_tail must be in (0, 1]");
    SGTP_CHECK(p->s_contest + p->eps_alpha > 0.f, "s_contest + eps must be > 0");
    const float *f = (const float *)p;
    for (size_t i = 0; i < sizeof(sgtp_params) / sizeof(float); ++i)
        SGTP_CHECK(std::isfinite(f[i]), "params field %zu is not finite", i);
    return SGTP_OK;
}

}  // namespace sgtp

extern "C" const char *sgtp_last_error(void) { return g_error.c_str(); }
extern "C" const char *sgtp_version(void) { return "sgtp-b300 0.1 (sm_103a)"; }
extern "C" int64_t sgtp_launch_count(void) { return (int64_t)g_launches.load(); }

extern "C" void sgtp_debug_fail_alloc(int32_t n) { sgtp::fail_alloc_countdown().store(n > 0 ? n : 0); }

// ================================================================ track prep
// One CTA per track: per waypoint the sum of the unit chords meeting there
// (bisector direction), per segment the chord, its inverse squared length,
// width, heading and speed increments, for the ring-extended arrays; then a
// compensated (Kahan) running sum of the segment lengths gives s_j in float32
// to about one ulp of L.
__global__ void track_prep_kernel(const float *xr, const float *wl, const float *wr, const int *src_off,
                                  TrackDesc *desc, float4 *A, float4 *B, float4 *W, float *S, float4 *C, float4 *G0,
                                  float4 *G1, float4 *G2, float2 *G3)
{
    const TrackDesc d = desc[blockIdx.x];
    const int so = src_off[blockIdx.x];
    const int next = ext_len_dev(d.N);
    for (int j = threadIdx.x; j < next; j += blockDim.x) {
        const int g = j % d.N;
        const int gn = g + 1 == d.N ? 0 : g + 1;
        const int gp = g == 0 ? d.N - 1 : g - 1;
        const float *p0 = xr + 4 * (size_t)(so + g), *p1 = xr + 4 * (size_t)(so + gn), *pm = xr + 4 * (size_t)(so + gp);
        const float ex = p1[0] - p0[0], ey = p1[1] - p0[1];
        const float fx = p0[0] - pm[0], fy = p0[1] - pm[1];
        const float l2 = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
        const float len = sqrtf(l2);
        const float lp = sqrtf(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)));
        const int o = d.offset + j;
        A[o] = make_float4(p0[0], p0[1], ex / len + fx / lp, ey / len + fy / lp);
        B[o] = make_float4(ex, ey, 1.0f / l2, len);
        W[o] = make_float4(wl[so + g], wl[so + gn] - wl[so + g], wr[so + g], wr[so + gn] - wr[so + g]);
        C[o] = make_float4(p0[2], wrap_angle(p1[2] - p0[2]), p0[3], p1[3] - p0[3]);
        // projection records (plane offsets in double, then rounded)
        const float ux = ex / len, uy = ey / len;
        const float bx = ux + fx / lp, by = uy + fy / lp;
        const double px = p0[0], py = p0[1];
        G0[o] = make_float4(bx, by, (float)((double)bx * px + (double)by * py), len);
        G1[o] = make_float4(ux, uy, (float)((double)ux * px + (double)uy * py),
                            (float)((double)ux * py - (double)uy * px));
        const float l0 = wl[so + g], r0 = wr[so + g], l1 = wl[so + gn], r1 = wr[so + gn];
        const float h0 = 0.5f * (l0 + r0), h1 = 0.5f * (l1 + r1), c0 = 0.5f * (l0 - r0), c1 = 0.5f * (l1 - r1);
        G2[o] = make_float4(1.0f / len, h0, h1 - h0, c0);
        G3[o] = make_float2(c1 - c0, 0.f);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float sum = 0.f, comp = 0.f;
        for (int j = 0; j < d.N; ++j) {
            const int o = d.offset + j;
            S[o] = sum;
            const float y = B[o].w - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        desc[blockIdx.x].L = sum;
    }
    __syncthreads();
    for (int j = d.N + threadIdx.x; j < next; j += blockDim.x) S[d.offset + j] = S[d.offset + j % d.N];
    __syncthreads();
    for (int j = threadIdx.x; j < next; j += blockDim.x) G3[d.offset + j].y = S[d.offset + j];
}

static sgtp_status track_create_impl(const float *xr, const float *wl, const float *wr, const int32_t *offsets,
                                     int32_t n_tracks, void *stream, sgtp_track **out)
{
    SGTP_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    SGTP_CHECK(xr && wl && wr && offsets, "NULL track array");
    SGTP_CHECK(n_tracks >= 1 && n_tracks <= (1 << 20), "n_tracks out of range");
    SGTP_CHECK(offsets[0] == 0, "offsets[0] must be 0");
    for (int t = 0; t < n_tracks; ++t) {
        const int N = offsets[t + 1] - offsets[t];
        SGTP_CHECK(N >= 3 && N <= (1 << 20), "track %d: N=%d out of range [3, 2^20]", t, N);
    }
    const int total_src = offsets[n_tracks];
    SGTP_CHECK(total_src <= (1 << 26), "too many waypoints");
    for (int t = 0; t < n_tracks; ++t) {
        const int o = offsets[t], N = offsets[t + 1] - o;
        for (int j = 0; j < N; ++j) {
            const int g = o + j, gn = o + (j + 1) % N;
            for (int c = 0; c < 4; ++c) SGTP_CHECK(std::isfinite(xr[4 * g + c]), "track %d: non-finite waypoint", t);
            SGTP_CHECK(std::isfinite(wl[g]) && std::isfinite(wr[g]) && wl[g] > 0.f && wr[g] > 0.f,
                       "track %d: widths must be finite and > 0", t);
            const float ex = xr[4 * gn] - xr[4 * g], ey = xr[4 * gn + 1] - xr[4 * g + 1];
            SGTP_CHECK(ex * ex + ey * ey > 0.f, "track %d: zero-length segment %d", t, j);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    sgtp_track *T = new sgtp_track();
    T->n_tracks = n_tracks;
    cudaGetDevice(&T->device);
    T->desc.resize(n_tracks);
    long long total = 0;
    for (int t = 0; t < n_tracks; ++t) {
        const int N = offsets[t + 1] - offsets[t];
        T->desc[t] = TrackDesc{(int)total, N, 0.f, 0};
        total += ext_len(N);
    }
    T->total = total;
    SGTP_CHECK(total < (1ll << 31), "tracks too large");
    float *d_xr = nullptr, *d_wl = nullptr, *d_wr = nullptr;
    int *d_off = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_xr); cudaFree(d_wl); cudaFree(d_wr); cudaFree(d_off);
    };
    cudaError_t e = cudaSuccess;
    if ((e = dev_malloc(&T->A, sizeof(float4) * total)) || (e = dev_malloc(&T->B, sizeof(float4) * total)) ||
        (e = dev_malloc(&T->W, sizeof(float4) * total)) || (e = dev_malloc(&T->C, sizeof(float4) * total)) ||
        (e = dev_malloc(&T->S, sizeof(float) * total)) || (e = dev_malloc(&T->G0, sizeof(float4) * total)) ||
        (e = dev_malloc(&T->G1, sizeof(float4) * total)) || (e = dev_malloc(&T->G2, sizeof(float4) * total)) ||
        (e = dev_malloc(&T->G3, sizeof(float2) * total)) ||
        (e = dev_malloc(&T->desc_dev, sizeof(TrackDesc) * n_tracks)) ||
        (e = dev_malloc(&d_xr, sizeof(float) * 4 * total_src)) || (e = dev_malloc(&d_wl, sizeof(float) * total_src)) ||
        (e = dev_malloc(&d_wr, sizeof(float) * total_src)) || (e = dev_malloc(&d_off, sizeof(int) * n_tracks))) {
        cleanup();
        sgtp_track_destroy(T);
        return set_error(SGTP_E_NOMEM, "track allocation failed: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(d_xr, xr, sizeof(float) * 4 * total_src, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_wl, wl, sizeof(float) * total_src, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_wr, wr, sizeof(float) * total_src, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(d_off, offsets, sizeof(int) * n_tracks, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(T->desc_dev, T->desc.data(), sizeof(TrackDesc) * n_tracks, cudaMemcpyHostToDevice, s))) {
        cleanup();
        sgtp_track_destroy(T);
        return set_error(SGTP_E_CUDA, "track upload failed: %s", cudaGetErrorString(e));
    }
    track_prep_kernel<<<n_tracks, 256, 0, s>>>(d_xr, d_wl, d_wr, d_off, T->desc_dev, T->A, T->B, T->W, T->S, T->C,
                                               T->G0, T->G1, T->G2, T->G3);
    count_launch();
    if ((e = cudaGetLastError()) ||
        (e = cudaMemcpyAsync(T->desc.data(), T->desc_dev, sizeof(TrackDesc) * n_tracks, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
        cleanup();
        sgtp_track_destroy(T);
        return set_error(SGTP_E_CUDA, "track prep failed: %s", cudaGetErrorString(e));
    }
    cleanup();
    *out = T;
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_track_create(const float *xr, const float *wl, const float *wr, int32_t N, void *stream,
                                         sgtp_track **out)
{
    const int32_t off[2] = {0, N};
    return track_create_impl(xr, wl, wr, off, 1, stream, out);
}

extern "C" sgtp_status sgtp_track_create_many(const float *xr, const float *wl, const float *wr,
                                              const int32_t *offsets, int32_t n_tracks, void *stream,
                                              sgtp_track **out)
{
    return track_create_impl(xr, wl, wr, offsets, n_tracks, stream, out);
}

extern "C" void sgtp_track_destroy(sgtp_track *T)
{
    if (!T) return;
    cudaFree(T->A); cudaFree(T->B); cudaFree(T->W); cudaFree(T->S); cudaFree(T->C); cudaFree(T->desc_dev);
    cudaFree(T->G0); cudaFree(T->G1); cudaFree(T->G2); cudaFree(T->G3);
    delete T;
}

extern "C" sgtp_status sgtp_track_info(const sgtp_track *trk, int32_t track_id, int32_t *n_tracks, int32_t *N,
                                       float *length)
{
    SGTP_CHECK(trk != nullptr, "track is NULL");
    SGTP_CHECK(track_id >= 0 && track_id < trk->n_tracks, "track_id out of range");
    if (n_tracks) *n_tracks = trk->n_tracks;
    if (N) *N = trk->desc[track_id].N;
    if (length) *length = trk->desc[track_id].L;
    return SGTP_OK;
}

// ================================================================ single BR
// Workspace of one best response: a header followed by the per-problem
// arrays (all 256-byte aligned).
struct BRHeader {
    unsigned long long key;     // running minimum selection key
    int flag;                   // device-side check flags
    int j0;                     // nearest segment of x_{i,t}
    float4 x0;
    float s_t, d_t, t0;         // Frenet of x_{i,t}, segment parameter
    int pad;
};

struct BRLayout {
    size_t ref, opp, osum, odbar, total;
    static constexpr size_t up(size_t x) { return (x + 255) & ~(size_t)255; }
    constexpr BRLayout(int n_opp, int T)
        : ref(up(sizeof(BRHeader))),
          opp(up(ref + sizeof(float4) * (T + 1))),
          osum(up(opp + sizeof(float2) * (size_t)T * (n_opp > 0 ? n_opp : 1))),
          odbar(up(osum + sizeof(float4) * (n_opp > 0 ? n_opp : 1))),
          total(up(odbar + sizeof(float) * (n_opp > 0 ? n_opp : 1)))
    {
    }
};

// Per-problem preparation (one CTA): Frenet of x_{i,t} by global search, the
// reference trajectory (Sec. III-A, overall ranking), and for every opponent
// prediction its positions, unwrapped progress and tail-mean offset, then
// the pair terms that do not depend on the candidate: the current gap
// Delta s_{ij,t}, alpha_{ij,t} and gamma_{block,ij}.  The opponents'
// projections run one (opponent, step) pair per thread; the progress is then
// unwrapped in step order by one thread per opponent.
__global__ void __launch_bounds__(256) br_prep_kernel(TrackView tv, sgtp_params p, const float *x0, const float *opp,
                                                      int n_opp, int T, float vscale, int n_tail, unsigned char *ws,
                                                      size_t off_ref, size_t off_opp, size_t off_osum,
                                                      size_t off_odbar)
{
    BRHeader *h = (BRHeader *)ws;
    float4 *ref = (float4 *)(ws + off_ref);
    float2 *opos = (float2 *)(ws + off_opp);
    float4 *osum = (float4 *)(ws + off_osum);
    float *odbar = (float *)(ws + off_odbar);
    float2 *ofr = (float2 *)g_smem;                                 // [T][n_opp] raw (s, d)
    __shared__ float s0_sh[SGTP_MAX_AGENTS], t0_sh[SGTP_MAX_AGENTS], sH_sh[SGTP_MAX_AGENTS];
    __shared__ int j0_sh[SGTP_MAX_AGENTS + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const float invL = 1.0f / tv.L;
    if (threadIdx.x == 0) h->flag = 0;
    // global nearest segment of x_{i,t} (slot 0) and of each opponent's first state
    for (int q = warp; q <= n_opp; q += nwarps) {
        const float *pt = q == 0 ? x0 : opp + (size_t)(q - 1) * (T + 1) * 4;
        const int j = nearest_segment_warp(tv, pt[0], pt[1]);
        if (lane == 0) j0_sh[q] = j;
    }
    __syncthreads();
    const int j0 = j0_sh[0];
    const float4 xs = make_float4(x0[0], x0[1], x0[2], x0[3]);
    if (threadIdx.x < n_opp) {
        const int o = threadIdx.x;
        const float *q = opp + (size_t)o * (T + 1) * 4;
        const FrenetPt f0 = frenet_at(tv, j0_sh[o + 1], q[0], q[1]);
        s0_sh[o] = f0.s;
        t0_sh[o] = f0.t;
    }
    for (int q = threadIdx.x; q < T * n_opp; q += blockDim.x) {
        const int tau = q / n_opp, o = q - tau * n_opp;
        const float *pt = opp + ((size_t)o * (T + 1) + tau + 1) * 4;
        opos[q] = make_float2(pt[0], pt[1]);
    }
    __syncthreads();
    // projections of this one-CTA preparation read the track from global memory
    const SegWindow w{nullptr, nullptr, nullptr, nullptr, 0, 0};
    if (threadIdx.x < 32) {
        const FrenetPt f = frenet_at(tv, j0, xs.x, xs.y);
        if (threadIdx.x == 0) {
            h->key = ~0ull;
            h->x0 = xs;
            h->s_t = f.s;
            h->d_t = f.d;
            h->t0 = f.t;
            h->j0 = j0;
        }
        reference_traj(tv, w, nullptr, j0, f.s, p.dt, vscale, T, ref);
    }
    // every (opponent, step) projection in parallel
    int flag = 0;
    for (int q = threadIdx.x; q < T * n_opp; q += blockDim.x) {
        const int tau = q / n_opp, o = q - tau * n_opp;
        const float *q0 = opp + (size_t)o * (T + 1) * 4;
        const float *pt = q0 + (size_t)(tau + 1) * 4;
        const int jo = j0_sh[o + 1];
        const int guess = jo + chord_guess(pt[0] - q0[0], pt[1] - q0[1], __ldg(tv.B + jo), 4 * kWinTile);
        const FrenetPt f = frenet_search(tv, w, guess, pt[0], pt[1]);
        flag |= f.flag;
        ofr[q] = make_float2(f.s, f.d);
    }
    if (flag) atomicOr(&h->flag, SGTP_E_DEVICE << 8);
    __syncthreads();
    if (threadIdx.x < n_opp) {
        const int o = threadIdx.x;
        float s = s0_sh[o], dsum = 0.f;
        for (int tau = 1; tau <= T; ++tau) {
            const float2 f = ofr[(size_t)(tau - 1) * n_opp + o];
            s = s + wrap_len(f.x - s, tv.L, invL);
            if (tau > T - n_tail) dsum = dsum + f.y;
        }
        sH_sh[o] = s;
        odbar[o] = dsum / (float)n_tail;
        const float st = h->s_t;
        const float ds_t = wrap_len(st - s0_sh[o], tv.L, invL);
        const float alpha = 1.0f / (1.0f + fabsf(ds_t) / (p.s_contest + p.eps_alpha));
        const float gamma = (ds_t > p.s_role && ds_t < p.s_contest) ? p.w_block : 0.f;
        osum[o] = make_float4(ds_t, alpha, gamma, s - s0_sh[o]);
    }
}

struct BRArgs {
    TrackView tv;
    sgtp_params p;
    const unsigned char *ws;
    size_t off_ref, off_opp, off_osum, off_odbar;
    const float *u_nom;
    int T, n_opp, K, n_tail, Wn, back;
    uint2 key;
    RoundKeys rk;                // the key's Weyl schedule
    unsigned agent_round, race;
    int game_on;
    // outputs (costs mode)
    float *cost, *viol, *states, *frenet, *controls;
    unsigned char *feas;
    long long timeout_ns;
    // proposal (learned sampler): per step (mean a, mean delta, sigma a, sigma delta)
    const float *prop;
    int K_prop;
};

// Stage one best response's tile: scalars, track window (TMA) with its lap
// correction, reference, nominal controls, opponent pairs and pair terms.
// Ends with the window ready and a __syncthreads.  Returns false if the
// wait timed out.
template <int MAXO>
__device__ bool br_stage(const BRArgs &a)
{
    using T = Tile<MAXO>;
    __shared__ int ok_sh;
    const BRHeader *h = (const BRHeader *)a.ws;
    if (threadIdx.x == 0) {
        BRScalars &S = T::sc();
        mbar_init(T::bar(), 1);
        const int j0 = h->j0;
        S.tv = a.tv;
        S.x0 = h->x0; S.s_t = h->s_t; S.d_t = h->d_t;
        const float2 hs = heading_split(h->x0.z);
        S.psi0 = hs.x; S.psi_off = hs.y;
        S.Wn = a.Wn;
        S.w0 = window_start(j0, a.back, a.tv.N);
        S.r0 = wrap_index(j0 - S.w0, a.tv.N);
        S.lap0 = S.w0 + S.r0 >= a.tv.N ? 1 : 0;
        S.pos0 = (float)S.r0 + h->t0;
        S.ppred0 = S.pos0 + __fdiv_rn(__fmul_rn(a.p.dt, h->x0.w), __ldg(a.tv.B + j0).w) - 0.5f;
        S.T = a.T; S.n_opp = a.n_opp; S.n_tail = a.n_tail;
        S.invL = 1.0f / a.tv.L;
        S.key = a.key; S.ctr_agent_round = a.agent_round; S.ctr_race = a.race; S.stream_bit = 0u;
        S.K_prop = a.prop ? a.K_prop : 0;
        T::stage_window(a.tv, S.w0, S.Wn);
    }
    const float4 *gref = (const float4 *)(a.ws + a.off_ref);
    for (int i = threadIdx.x; i <= a.T; i += blockDim.x) T::ref()[i] = gref[i];
    for (int i = threadIdx.x; i < a.T; i += blockDim.x) {
        T::dist()[i] = make_float4(a.u_nom[2 * i], a.u_nom[2 * i + 1], a.p.sigma_a, a.p.sigma_delta);
        if (a.prop) T::dist()[SGTP_MAX_T + i] = ((const float4 *)a.prop)[i];
    }
    const float2 *gopp = (const float2 *)(a.ws + a.off_opp);
    const int n_opp = a.n_opp;
    stage_opponents<MAXO>(a.T, n_opp, [&](int tau, int o) { return gopp[(size_t)(tau - 1) * n_opp + o]; });
    const float4 *gosum = (const float4 *)(a.ws + a.off_osum);
    const float *godbar = (const float *)(a.ws + a.off_odbar);
    for (int i = threadIdx.x; i < n_opp; i += blockDim.x) { T::osum()[i] = gosum[i]; T::odbar()[i] = godbar[i]; }
    __syncthreads();
    if (threadIdx.x == 0) ok_sh = mbar_wait_bounded(T::bar(), 0, (unsigned long long)a.timeout_ns) ? 1 : 0;
    __syncthreads();
    if (ok_sh && window_wraps(T::sc())) {
        T::fix_laps(T::sc());
        __syncthreads();
    }
    return ok_sh != 0;
}

template <int MAXO, bool KEY_MODE>
__global__ void __launch_bounds__(256, 3) br_rollout_kernel(BRArgs a)
{
    using T = Tile<MAXO>;
    __shared__ unsigned long long cta_key;
    __shared__ int cta_flag;
    if (threadIdx.x == 0) { cta_key = ~0ull; cta_flag = 0; }
    const bool ok = br_stage<MAXO>(a);
    const BRScalars &S = T::sc();
    int flag = 0;
    unsigned long long best = ~0ull;
    const unsigned k = blockIdx.x * blockDim.x + threadIdx.x;
    if (ok && k < (unsigned)a.K) {
        if (KEY_MODE) {
            const SampleResult r = run_candidate<MAXO, false>(S, a.p, a.rk, k, a.game_on != 0, flag, nullptr, nullptr,
                                                              nullptr);
            best = make_key(r.feasible, r.cost, r.viol, k);
        } else {
            float *st = a.states ? a.states + (size_t)k * (a.T + 1) * 4 : nullptr;
            float *fr = a.frenet ? a.frenet + (size_t)k * (a.T + 1) * 2 : nullptr;
            float *uo = a.controls ? a.controls + (size_t)k * a.T * 2 : nullptr;
            SampleResult r;
            if (st || fr || uo)
                r = run_candidate<MAXO, true>(S, a.p, a.rk, k, a.game_on != 0, flag, st, fr, uo);
            else
                r = run_candidate<MAXO, false>(S, a.p, a.rk, k, a.game_on != 0, flag, nullptr, nullptr, nullptr);
            a.cost[k] = r.cost;
            a.viol[k] = r.viol;
            a.feas[k] = r.feasible ? 1 : 0;
        }
    }
    if (!ok && threadIdx.x == 0) atomicOr(&cta_flag, SGTP_E_TIMEOUT);
    if (flag) atomicOr(&cta_flag, SGTP_E_DEVICE << 8);
    if (KEY_MODE) {
        best = warp_min_u64(best);
        if ((threadIdx.x & 31) == 0) atomicMin(&cta_key, best);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        BRHeader *hw = (BRHeader *)a.ws;
        if (KEY_MODE) atomicMin(&hw->key, cta_key);
        if (cta_flag) atomicOr(&hw->flag, cta_flag);
    }
}

// Value of the ranked float of a selection key (inverse of float_order).
__device__ __forceinline__ float key_value(unsigned long long key)
{
    const unsigned ord = (unsigned)((key >> 31) & 0xffffffffull);
    const unsigned u = (ord & 0x80000000u) ? (ord & 0x7fffffffu) : ~ord;
    return __uint_as_float(u);
}

// Selection result and re-roll of the winner: the selected sample's
// controls one step per thread (same noise and clipping as its evaluation),
// then the bicycle recurrence by one thread (same arithmetic), so the
// returned trajectory is bit-identical to the evaluated one.  cost_star
// (optional) receives the ranked value of the winner: its cost when a
// feasible sample exists, else its violation.
template <int MAXO>
__global__ void br_finalize_kernel(BRArgs a, int *k_star, float *u_star, float *xi_star, int *any_feasible,
                                   float *cost_star)
{
    using Tl = Tile<MAXO>;
    __shared__ unsigned ks_sh;
    const BRHeader *h = (const BRHeader *)a.ws;
    if (threadIdx.x == 0) {
        const unsigned long long key = h->key;
        ks_sh = (unsigned)(key & 0x7fffffffull);
        *k_star = (int)ks_sh;
        *any_feasible = (key >> 63) ? 0 : 1;
        if (cost_star) *cost_star = key_value(key);
    }
    __syncthreads();
    const unsigned k = ks_sh;
    const bool prop = a.prop && k < (unsigned)a.K_prop;
    for (int q = threadIdx.x; q < a.T; q += blockDim.x) {
        const unsigned sbit = prop ? 0x80000000u : 0u;
        const uint4 wv = philox4x32_10(make_uint4(k, (unsigned)(q >> 1) | sbit, a.agent_round, a.race), a.key);
        const float2 z = (q & 1) ? box_muller(wv.z, wv.w) : box_muller(wv.x, wv.y);
        const float4 d = prop ? ((const float4 *)a.prop)[q]
                              : make_float4(a.u_nom[2 * q], a.u_nom[2 * q + 1], a.p.sigma_a, a.p.sigma_delta);
        const float2 u = sample_control_d(a.p, d, z);
        Tl::ctl()[q] = u;
        u_star[2 * q] = u.x;
        u_star[2 * q + 1] = u.y;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const float4 x0 = h->x0;
        const float2 hs = heading_split(x0.z);
        float x = x0.x, y = x0.y, psi = hs.x, v = x0.w;
        ((float4 *)xi_star)[0] = x0;
        for (int tau = 0; tau < a.T; ++tau) {
            const float2 u = Tl::ctl()[tau];
            bicycle_step(a.p, x, y, psi, v, u.x, u.y);
            ((float4 *)xi_star)[tau + 1] = make_float4(x, y, psi + hs.y, v);
        }
    }
}

// ---------------------------------------------------------------- dispatch
template <int MAXO>
static size_t br_smem(const BRArgs &) { return BRTile<MAXO>::kBytes; }

template <int MAXO>
static sgtp_status launch_rollout(const BRArgs &a, bool key_mode, cudaStream_t s, int grid, int block)
{
    // the shared-memory opt-in applies to the current device only
    static PerDeviceFlag configured;
    const sgtp_status cst = once_per_device(configured, []() -> sgtp_status {
        SGTP_CUDA(cudaFuncSetAttribute(br_rollout_kernel<MAXO, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        SGTP_CUDA(cudaFuncSetAttribute(br_rollout_kernel<MAXO, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        SGTP_CUDA(cudaFuncSetAttribute(br_finalize_kernel<MAXO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024));
        return SGTP_OK;
    });
    if (cst) return cst;
    if (key_mode)
        br_rollout_kernel<MAXO, true><<<grid, block, br_smem<MAXO>(a), s>>>(a);
    else
        br_rollout_kernel<MAXO, false><<<grid, block, br_smem<MAXO>(a), s>>>(a);
    return SGTP_OK;
}

static int maxo_bucket(int n) { return n <= 1 ? 1 : n <= 3 ? 3 : n <= 9 ? 9 : 15; }

static sgtp_status br_common(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, const float *x0,
                             const float *u_nom, float vref_scale, const float *opp, int32_t n_opp, int32_t T,
                             int32_t K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                             int32_t game_on, void *ws, size_t ws_bytes, BRArgs &a, int &maxo)
{
    SGTP_CHECK(trk != nullptr, "track is NULL");
    SGTP_CHECK(track_id >= 0 && track_id < trk->n_tracks, "track_id %d out of range", track_id);
    sgtp_status st = check_params(p);
    if (st) return st;
    SGTP_CHECK(x0 && u_nom, "x0 / u_nom is NULL");
    SGTP_CHECK(n_opp >= 0 && n_opp <= SGTP_MAX_AGENTS - 1, "n_opp=%d out of range [0, %d]", n_opp,
               SGTP_MAX_AGENTS - 1);
    SGTP_CHECK(n_opp == 0 || opp != nullptr, "opp is NULL with n_opp > 0");
    SGTP_CHECK(T >= 1 && T <= SGTP_MAX_T, "T=%d out of range [1, %d]", T, SGTP_MAX_T);
    SGTP_CHECK(K >= 1 && K <= SGTP_MAX_K, "K=%d out of range [1, 2^30]", K);
    SGTP_CHECK(agent < (1u << 16) && round < (1u << 16) && race < (1u << 31), "agent/round/race out of range");
    SGTP_CHECK(std::isfinite(vref_scale) && vref_scale >= 0.f, "vref_scale must be finite and >= 0");
    const BRLayout lay(n_opp, T);
    SGTP_CHECK(ws != nullptr && ws_bytes >= lay.total, "workspace too small: need %zu bytes", lay.total);
    SGTP_CHECK(((uintptr_t)ws & 255u) == 0, "workspace must be 256-byte aligned");
    a = BRArgs{};
    a.tv = track_view(trk, track_id);
    a.p = *p;
    a.ws = (const unsigned char *)ws;
    a.off_ref = lay.ref; a.off_opp = lay.opp; a.off_osum = lay.osum; a.off_odbar = lay.odbar;
    a.u_nom = u_nom;
    a.T = T; a.n_opp = n_opp; a.K = K;
    a.n_tail = tail_count(p->mu_tail, T);
    a.Wn = window_len(a.tv.N, kWinTile);
    a.back = a.Wn >= 256 ? 64 : a.Wn / 4;
    a.key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    a.rk = make_round_keys(a.key);
    a.agent_round = agent | (round << 16);
    a.race = race;
    a.game_on = game_on;
    a.timeout_ns = default_wait_ns((double)K * T);
    maxo = maxo_bucket(n_opp);
    return SGTP_OK;
}

static sgtp_status br_launch(const BRArgs &a, int maxo, bool key_mode, const float *x0, const float *opp,
                             float vref_scale, cudaStream_t s)
{
    // a response of at most 128 samples per SM runs 128-thread CTAs: its
    // lone-sample chains then spread over twice the SMs (every sample is
    // computed the same way in either shape)
    int dev = 0, sms = 0;
    SGTP_CUDA(cudaGetDevice(&dev));
    SGTP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int block = (long long)a.K <= 128ll * sms ? 128 : 256;
    const int grid = (a.K + block - 1) / block;
    static PerDeviceFlag prep_configured;
    const sgtp_status cst = once_per_device(prep_configured, []() -> sgtp_status {
        SGTP_CUDA(cudaFuncSetAttribute(br_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        return SGTP_OK;
    });
    if (cst) return cst;
    const size_t prep_smem = sizeof(float2) * (size_t)a.T * (a.n_opp > 0 ? a.n_opp : 1);
    br_prep_kernel<<<1, 256, prep_smem, s>>>(a.tv, a.p, x0, opp, a.n_opp, a.T, vref_scale, a.n_tail,
                                             (unsigned char *)a.ws, a.off_ref, a.off_opp, a.off_osum, a.off_odbar);
    sgtp_status st;
    switch (maxo) {
        case 1: st = launch_rollout<1>(a, key_mode, s, grid, block); break;
        case 3: st = launch_rollout<3>(a, key_mode, s, grid, block); break;
        case 9: st = launch_rollout<9>(a, key_mode, s, grid, block); break;
        default: st = launch_rollout<15>(a, key_mode, s, grid, block); break;
    }
    if (st) return st;
    count_launch(2);
    SGTP_CUDA(cudaGetLastError());
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_sync_status(const int32_t *status_dev, void *stream, int32_t *status_host)
{
    SGTP_CHECK(status_dev != nullptr && status_host != nullptr, "NULL argument");
    SGTP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    SGTP_CUDA(cudaMemcpy(status_host, status_dev, sizeof(int32_t), cudaMemcpyDeviceToHost));
    return SGTP_OK;
}

extern "C" size_t sgtp_br_workspace_bytes(int32_t n_opp, int32_t T)
{
    if (n_opp < 0 || T < 1) return 0;
    return BRLayout(n_opp, T).total;
}

extern "C" sgtp_status sgtp_rollout_costs(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                          const float *x0, const float *u_nom, float vref_scale, const float *opp,
                                          int32_t n_opp, int32_t T, int32_t K, uint64_t seed, uint32_t race,
                                          uint32_t agent, uint32_t round, int32_t game_on, float *cost,
                                          uint8_t *feasible, float *violation, float *states, float *frenet,
                                          float *controls, void *workspace, size_t workspace_bytes, void *stream)
{
    BRArgs a;
    int maxo;
    sgtp_status st = br_common(trk, track_id, p, x0, u_nom, vref_scale, opp, n_opp, T, K, seed, race, agent, round,
                               game_on, workspace, workspace_bytes, a, maxo);
    if (st) return st;
    SGTP_CHECK(cost && feasible && violation, "cost/feasible/violation is NULL");
    a.prop = nullptr;
    a.K_prop = 0;
    a.cost = cost; a.feas = feasible; a.viol = violation;
    a.states = states; a.frenet = frenet; a.controls = controls;
    return br_launch(a, maxo, false, x0, opp, vref_scale, (cudaStream_t)stream);
}

static sgtp_status best_response_impl(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, const float *x0,
                                      const float *u_nom, float vref_scale, const float *opp, int32_t n_opp, int32_t T,
                                      int32_t K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                                      int32_t game_on, const float *prop, int32_t K_prop, int32_t *k_star,
                                      float *u_star, float *xi_star, int32_t *any_feasible, float *cost_star,
                                      void *workspace, size_t workspace_bytes, void *stream)
{
    BRArgs a;
    int maxo;
    sgtp_status st = br_common(trk, track_id, p, x0, u_nom, vref_scale, opp, n_opp, T, K, seed, race, agent, round,
                               game_on, workspace, workspace_bytes, a, maxo);
    if (st) return st;
    SGTP_CHECK(k_star && u_star && xi_star && any_feasible, "NULL output");
    SGTP_CHECK(prop == nullptr || (K_prop >= 0 && K_prop <= K), "K_prop out of range [0, K]");
    a.prop = prop;
    a.K_prop = prop ? K_prop : 0;
    cudaStream_t s = (cudaStream_t)stream;
    st = br_launch(a, maxo, true, x0, opp, vref_scale, s);
    if (st) return st;
    switch (maxo) {
        case 1: br_finalize_kernel<1><<<1, 128, br_smem<1>(a), s>>>(a, k_star, u_star, xi_star, any_feasible, cost_star); break;
        case 3: br_finalize_kernel<3><<<1, 128, br_smem<3>(a), s>>>(a, k_star, u_star, xi_star, any_feasible, cost_star); break;
        case 9: br_finalize_kernel<9><<<1, 128, br_smem<9>(a), s>>>(a, k_star, u_star, xi_star, any_feasible, cost_star); break;
        default:
            br_finalize_kernel<15><<<1, 128, br_smem<15>(a), s>>>(a, k_star, u_star, xi_star, any_feasible, cost_star);
            break;
    }
    count_launch();
    SGTP_CUDA(cudaGetLastError());
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_best_response(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                          const float *x0, const float *u_nom, float vref_scale, const float *opp,
                                          int32_t n_opp, int32_t T, int32_t K, uint64_t seed, uint32_t race,
                                          uint32_t agent, uint32_t round, int32_t game_on, int32_t *k_star,
                                          float *u_star, float *xi_star, int32_t *any_feasible, void *workspace,
                                          size_t workspace_bytes, void *stream)
{
    return best_response_impl(trk, track_id, p, x0, u_nom, vref_scale, opp, n_opp, T, K, seed, race, agent, round,
                              game_on, nullptr, 0, k_star, u_star, xi_star, any_feasible, nullptr, workspace,
                              workspace_bytes, stream);
}

extern "C" sgtp_status sgtp_best_response_mixed(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                                const float *x0, const float *u_nom, float vref_scale,
                                                const float *opp, int32_t n_opp, int32_t T, int32_t K,
                                                uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                                                int32_t game_on, const float *prop, int32_t K_prop, int32_t *k_star,
                                                float *u_star, float *xi_star, int32_t *any_feasible,
                                                float *cost_star, void *workspace, size_t workspace_bytes,
                                                void *stream)
{
    SGTP_CHECK(prop != nullptr, "prop is NULL");
    SGTP_CHECK(((uintptr_t)prop & 15u) == 0, "prop must be 16-byte aligned");
    return best_response_impl(trk, track_id, p, x0, u_nom, vref_scale, opp, n_opp, T, K, seed, race, agent, round,
                              game_on, prop, K_prop, k_star, u_star, xi_star, any_feasible, cost_star, workspace,
                              workspace_bytes, stream);
}

// ================================================================ no-allocation entry point
// The scratch of sgtp_best_response_noalloc: a file-scope device array, so
// the call itself never allocates.  Its callers are control loops that must
// not wait on an allocator and hosts without a device allocator.
static __device__ __align__(256) unsigned char g_br_scratch[SGTP_NOALLOC_SCRATCH_BYTES];
static_assert(BRLayout(SGTP_MAX_AGENTS - 1, SGTP_MAX_T).total <= SGTP_NOALLOC_SCRATCH_BYTES,
              "the static scratch must hold the largest best response the ABI accepts");

namespace {
std::mutex g_scratch_mu;
void *g_scratch_addr[sgtp::kMaxDevices] = {};
}  // namespace

extern "C" sgtp_status sgtp_best_response_noalloc(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                                  const float *x0, const float *u_nom, float vref_scale,
                                                  const float *opp, int32_t n_opp, int32_t T, int32_t K,
                                                  uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                                                  int32_t game_on, int32_t *k_star, float *u_star, float *xi_star,
                                                  int32_t *any_feasible, void *stream)
{
    SGTP_CHECK(n_opp >= 0 && n_opp <= SGTP_MAX_AGENTS - 1, "n_opp=%d out of range [0, %d]", n_opp,
               SGTP_MAX_AGENTS - 1);
    SGTP_CHECK(T >= 1 && T <= SGTP_MAX_T, "T=%d out of range [1, %d]", T, SGTP_MAX_T);
    const size_t need = BRLayout(n_opp, T).total;
    SGTP_CHECK(need <= (size_t)SGTP_NOALLOC_SCRATCH_BYTES,
               "best response needs %zu bytes of scratch; the static scratch holds %d", need,
               SGTP_NOALLOC_SCRATCH_BYTES);
    int dev = -1;
    SGTP_CUDA(cudaGetDevice(&dev));
    SGTP_CHECK(dev >= 0 && dev < kMaxDevices, "device %d out of range [0, %d)", dev, kMaxDevices);
    void *ws = nullptr;
    {
        // one address lookup per device, made with that device current
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *addr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&addr, g_br_scratch);
            if (e != cudaSuccess)
                return set_error(SGTP_E_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                                 cudaGetErrorString(e));
            g_scratch_addr[dev] = addr;
        }
        ws = g_scratch_addr[dev];
    }
    return best_response_impl(trk, track_id, p, x0, u_nom, vref_scale, opp, n_opp, T, K, seed, race, agent, round,
                              game_on, nullptr, 0, k_star, u_star, xi_star, any_feasible, nullptr, ws,
                              SGTP_NOALLOC_SCRATCH_BYTES, stream);
}
