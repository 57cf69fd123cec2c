// sgtp_device.cuh -- device building blocks of the SGTP best-response engine
// (sm_103a).  Everything here runs in float32 registers; nothing calls back to
// the host.  Paper references are to Li et al., "SGTP: Sampling-based
// Game-Theoretic Planning for Real-Time Multi-Vehicle Autonomous Racing".
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sgtp.h"

namespace sgtp {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInvTwoPi = 0.15915494309189533577f;

// Longest shared-memory window of a track (segments); the device arrays of
// every track repeat their first segments after the last one so that any
// window [w0, w0 + Wn) with w0 < N, Wn <= kWinMax is one contiguous copy.
constexpr int kWinMax = 1024;
constexpr int kMaxMoves = 64;

// ---------------------------------------------------------------- track
// Device raceline of one closed track; per segment j (waypoint j to j+1 mod N),
// arrays of length N + kWinMax (entry j >= N repeats entry j mod N):
//   A[j]  = (x_j, y_j, ex_j, ey_j)             chord e_j = P_{j+1} - P_j
//   I[j]  = 1 / |e_j|^2
//   SB[j] = (s_j, |e_j|, wL_j, wL_{j+1} - wL_j)  s_j cumulative arc length
//   SW[j] = (wR_j, wR_{j+1} - wR_j)
//   C[j]  = (psi_j, wrap(psi_{j+1} - psi_j), v_j, v_{j+1} - v_j)
struct TrackView {
    const float4 *A;
    const float *I;
    const float4 *SB;
    const float2 *SW;
    const float4 *C;
    int N;
    float L;
};

// Per-track entry of an sgtp_track object (offsets in elements, multiples of 4).
struct TrackDesc {
    int offset;
    int N;
    float L;
    int pad;
};

// Shared-memory window of a track: local index r <-> segment (w0 + r) mod N.
struct SegWindow {
    const float4 *A;
    const float *I;
    const float4 *SB;
    const float2 *SW;
    int w0, Wn;
};

__host__ __device__ __forceinline__ int ext_len_dev(int N) { return (N + kWinMax + 3) & ~3; }

__device__ __forceinline__ int wrap_index(int j, int N)
{
    j %= N;
    return j < 0 ? j + N : j;
}

// ---------------------------------------------------------------- Frenet
struct FrenetPt {
    float s, d, t;
    float wl, wr;   // widths at the foot point
};

__device__ __forceinline__ float seg_dist2(const float4 &a, float inv_l2, float px, float py, float &t, float &cr)
{
    const float dx = px - a.x, dy = py - a.y;
    float u = __fmul_rn(__fmaf_rn(dx, a.z, __fmul_rn(dy, a.w)), inv_l2);
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    const float ex = __fmaf_rn(-u, a.z, dx), ey = __fmaf_rn(-u, a.w, dy);
    t = u;
    cr = __fmaf_rn(a.z, dy, -__fmul_rn(a.w, dx));
    return __fmaf_rn(ex, ex, __fmul_rn(ey, ey));
}

// Segment data at window-local index r (shared memory inside the window,
// global memory outside it).
__device__ __forceinline__ void seg_at(const TrackView &tv, const SegWindow &w, int r, float4 &a, float &il)
{
    if ((unsigned)r < (unsigned)w.Wn) {
        a = w.A[r];
        il = w.I[r];
    } else {
        const int j = wrap_index(w.w0 + r, tv.N);
        a = __ldg(tv.A + j);
        il = __ldg(tv.I + j);
    }
}

__device__ __forceinline__ void seg_tail(const TrackView &tv, const SegWindow &w, int r, float4 &sb, float2 &sw)
{
    if ((unsigned)r < (unsigned)w.Wn) {
        sb = w.SB[r];
        sw = w.SW[r];
    } else {
        const int j = wrap_index(w.w0 + r, tv.N);
        sb = __ldg(tv.SB + j);
        sw = __ldg(tv.SW + j);
    }
}

// Frenet projection s(x; G), d(x; G) (Sec. II) as a local search from a
// predicted segment c: the nearer of c's neighbours is followed while it is
// strictly nearer (the left one also on ties), so the result is a local
// minimum of the point-to-segment distance over the segment index; for points
// within the track's reach it is the global nearest segment.  r is the
// window-local segment index (updated); dr the last shift (a prediction of
// the next one).  A search longer than kMaxMoves stops and sets flag.
__device__ __forceinline__ FrenetPt frenet_walk(const TrackView &tv, const SegWindow &w, int &r, int &dr, float px,
                                                float py, int &flag)
{
    const int c = r + dr;
    float4 a0, a1, a2;
    float i0, i1, i2;
    if (c >= 1 && c + 1 < w.Wn) {
        a0 = w.A[c - 1]; a1 = w.A[c]; a2 = w.A[c + 1];
        i0 = w.I[c - 1]; i1 = w.I[c]; i2 = w.I[c + 1];
    } else {
        seg_at(tv, w, c - 1, a0, i0);
        seg_at(tv, w, c, a1, i1);
        seg_at(tv, w, c + 1, a2, i2);
    }
    float t0, t1, t2, c0, c1, c2;
    const float d0 = seg_dist2(a0, i0, px, py, t0, c0);
    const float d1 = seg_dist2(a1, i1, px, py, t1, c1);
    const float d2 = seg_dist2(a2, i2, px, py, t2, c2);
    int best = c;
    float bd = d1, bt = t1, bc = c1;
    if (d0 <= d1 && d0 <= d2) {
        best = c - 1; bd = d0; bt = t0; bc = c0;
        // keep walking backward while strictly nearer
        for (int it = 0; it < kMaxMoves; ++it) {
            float4 a; float il, t, cr;
            seg_at(tv, w, best - 1, a, il);
            const float dd = seg_dist2(a, il, px, py, t, cr);
            if (!(dd <= bd)) break;
            best -= 1; bd = dd; bt = t; bc = cr;
            if (it == kMaxMoves - 1) flag = 1;
        }
    } else if (d2 < d1) {
        best = c + 1; bd = d2; bt = t2; bc = c2;
        for (int it = 0; it < kMaxMoves; ++it) {
            float4 a; float il, t, cr;
            seg_at(tv, w, best + 1, a, il);
            const float dd = seg_dist2(a, il, px, py, t, cr);
            if (!(dd < bd)) break;
            best += 1; bd = dd; bt = t; bc = cr;
            if (it == kMaxMoves - 1) flag = 1;
        }
    }
    dr = best - r;
    r = best;
    float4 sb;
    float2 sw;
    seg_tail(tv, w, best, sb, sw);
    const float dist = __fmul_rn(bd, rsqrtf(fmaxf(bd, 1e-30f)));
    FrenetPt f;
    f.s = __fmaf_rn(bt, sb.y, sb.x);
    f.d = bc >= 0.0f ? dist : -dist;
    f.t = bt;
    f.wl = __fmaf_rn(bt, sb.w, sb.z);
    f.wr = __fmaf_rn(bt, sw.y, sw.x);
    return f;
}

// Global nearest segment by brute force over all N segments, cooperatively by
// one warp (lowest index on ties).  Used once per vehicle state x_{i,t}.
__device__ __forceinline__ int nearest_segment_warp(const TrackView &tv, float px, float py)
{
    const int lane = threadIdx.x & 31;
    unsigned long long best = ~0ull;
    for (int j = lane; j < tv.N; j += 32) {
        const float4 a = __ldg(tv.A + j);
        float t, cr;
        const float d2 = seg_dist2(a, __ldg(tv.I + j), px, py, t, cr);
        const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j;
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    return (int)(best & 0xffffffffu);
}

// Projection on a known segment j (global index).
__device__ __forceinline__ FrenetPt frenet_at(const TrackView &tv, int j, float px, float py)
{
    const float4 a = __ldg(tv.A + j);
    float t, cr;
    const float d2 = seg_dist2(a, __ldg(tv.I + j), px, py, t, cr);
    const float4 sb = __ldg(tv.SB + j);
    const float2 sw = __ldg(tv.SW + j);
    const float dist = __fmul_rn(d2, rsqrtf(fmaxf(d2, 1e-30f)));
    FrenetPt f;
    f.s = __fmaf_rn(t, sb.y, sb.x);
    f.d = cr >= 0.0f ? dist : -dist;
    f.t = t;
    f.wl = __fmaf_rn(t, sb.w, sb.z);
    f.wr = __fmaf_rn(t, sw.y, sw.x);
    return f;
}

// Wrap a progress difference into (-L/2, L/2].
__device__ __forceinline__ float wrap_len(float x, float L, float invL)
{
    return __fmaf_rn(-L, ceilf(__fmaf_rn(x, invL, -0.5f)), x);
}

// Wrap an angle into (-pi, pi] (used only squared, so the end choice is moot).
__device__ __forceinline__ float wrap_angle(float a) { return __fmaf_rn(-kTwoPi, rintf(a * kInvTwoPi), a); }

// Reference trajectory (Sec. III-A, overall ranking): s^r_0 = s_{i,t},
// s^r_{tau+1} = s^r_tau + dt * v^r(s^r_tau), x^r_tau = x^r(s^r_tau) with
// x^r(s) linear in s between waypoints (heading along the shorter arc) and
// the agent's speed profile scaled by vscale.  Progress is kept unwrapped and
// accumulated as an unevaluated float pair (hi + lo, Knuth's two-sum); the
// position inside a segment is ((hi - lap L) - s_j) + lo with an exact lap
// subtraction, so the reference stays within a few float ulps of the exact
// recursion however long the track.  One thread.  Segment data comes from
// the shared-memory window (A, SB and C) when it holds the segment, else
// from global memory.  j0 is the global segment of s0 (s0 in [0, L)).
__device__ __forceinline__ void reference_traj(const TrackView &tv, const SegWindow &w, const float4 *Cw, int j0,
                                               float s0, float dt, float vscale, int T, float4 *ref)
{
    float hi = s0, lo = 0.f;
    int q = j0;                         // unwrapped segment index: segment q mod N of lap q div N
    auto fetch = [&](int qq, float4 &a, float4 &sb, float4 &c) {
        const int j = wrap_index(qq, tv.N);
        const int rl = w.Wn > 0 ? wrap_index(qq - w.w0, tv.N) : -1;
        if (rl >= 0 && rl < w.Wn) {
            a = w.A[rl]; sb = w.SB[rl]; c = Cw[rl];
        } else {
            a = __ldg(tv.A + j); sb = __ldg(tv.SB + j); c = __ldg(tv.C + j);
        }
    };
    auto lap_of = [&](int qq) { return (qq - wrap_index(qq, tv.N)) / tv.N; };
    auto locate = [&]() -> float4 {
        float4 a, sb, c;
        for (int it = 0; it < 2 * tv.N + 2; ++it) {
            fetch(q, a, sb, c);
            const int j = wrap_index(q, tv.N);
            const float lapL = (float)lap_of(q) * tv.L;
            const float hm = hi - lapL;                    // exact: hi and lapL within a factor 2
            const float sn = (j + 1 == tv.N) ? tv.L : sb.x + sb.y;
            if (hm < sb.x) { q -= 1; continue; }
            if (hm >= sn) { q += 1; continue; }
            const float u = ((hm - sb.x) + lo) / sb.y;
            float4 o;
            o.x = __fmaf_rn(u, a.z, a.x);
            o.y = __fmaf_rn(u, a.w, a.y);
            o.z = __fmaf_rn(u, c.y, c.x);
            o.w = __fmaf_rn(u, c.w, c.z);
            return o;
        }
        return make_float4(a.x, a.y, c.x, c.z);
    };
    ref[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 r_cur = locate();
    for (int tau = 0; tau < T; ++tau) {
        const float ds = __fmul_rn(dt, __fmul_rn(vscale, r_cur.w));
        const float s = hi + ds;                 // two-sum of hi + ds, error into lo
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (ds - bp);
        hi = s;
        lo = lo + err;
        const float s2 = hi + lo;                // renormalise
        lo = lo - (s2 - hi);
        hi = s2;
        float4 r1 = locate();
        r_cur = r1;
        r1.w = __fmul_rn(r1.w, vscale);
        ref[tau + 1] = r1;
    }
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies with a Weyl
// key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform in (0,1) from the top 23 bits (exact in float32).
__device__ __forceinline__ float uniform_open(unsigned w)
{
    return __fmaf_rn((float)(w >> 9), 1.1920928955078125e-7f, 5.9604644775390625e-8f);
}

// Box-Muller pair from two words: (sqrt(-2 ln u1) cos 2pi u2, ... sin ...).
// The angle is evaluated as 2 pi u2 - pi in (-pi, pi) with the signs folded
// back, keeping __sincosf inside its accurate range.
__device__ __forceinline__ float2 box_muller(unsigned w0, unsigned w1)
{
    const float u1 = uniform_open(w0), u2 = uniform_open(w1);
    const float m = fmaxf(-2.0f * __logf(u1), 1e-30f);   // __logf may overshoot 0 for u1 -> 1
    const float r = m * rsqrtf(m);
    float sn, cs;
    __sincosf(__fmaf_rn(kTwoPi, u2, -kPi), &sn, &cs);
    return make_float2(-r * cs, -r * sn);
}

// ---------------------------------------------------------------- argmin key
// 64-bit selection key: bit 63 = infeasible, bits 62..31 = order-preserving
// image of the float ranked (cost if feasible, violation otherwise; NaN as
// +inf), bits 30..0 = k.  The minimum key is the paper's selection
// (Eq. selection, least-violation fallback) with ties to the lowest k.
__device__ __forceinline__ unsigned float_order(float f)
{
    f = f + 0.0f;                                // -0 -> +0
    unsigned u = __float_as_uint(f);
    if (f != f) u = 0x7f800000u;                  // NaN ranks as +inf
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ unsigned long long make_key(bool feasible, float cost, float viol, unsigned k)
{
    const unsigned ord = float_order(feasible ? cost : viol);
    return ((unsigned long long)(feasible ? 0u : 1u) << 63) | ((unsigned long long)ord << 31) |
           (unsigned long long)(k & 0x7fffffffu);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// ---------------------------------------------------------------- timing / waits
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- TMA (bulk copy)
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk global->shared copy (TMA, no multicast).  dst, src 16-byte aligned;
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the bulk copies of the current phase.  Gives up after limit_ns and
// returns false (the caller records SGTP_E_TIMEOUT); it then keeps waiting up
// to 4x the limit for the copies in flight before returning, so that no copy
// lands in shared memory after the CTA has left.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, unsigned long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        const unsigned long long dt = global_ns() - t0;
        if (dt > limit_ns) {
            while (!mbar_try_wait(bar, parity) && global_ns() - t0 < 4 * limit_ns) {
            }
            return false;
        }
    }
    return true;
}

// Shared-memory layout of a track window (16-byte aligned pieces).
struct WindowSmem {
    unsigned A, I, SB, SW, end;
    __host__ __device__ WindowSmem(unsigned base, int Wn)
    {
        A = base;
        I = A + 16u * Wn;
        SB = I + 4u * Wn;
        SW = SB + 16u * Wn;
        end = SW + 8u * Wn;
    }
};

// Window start for a segment j0: `back` segments behind it, rounded down to a
// multiple of 4 so that every array's copy starts 16-byte aligned.
__device__ __forceinline__ int window_start(int j0, int back, int N)
{
    int w0 = wrap_index(j0 - back, N);
    return w0 & ~3;
}

// Issue the bulk copies of window [w0, w0+Wn) (Wn a multiple of 4) of track
// tv into shared memory at smem + layout; one thread; completes on bar.
__device__ __forceinline__ SegWindow stage_window_issue(const TrackView &tv, int w0, int Wn, unsigned char *smem,
                                                       const WindowSmem &ly, unsigned long long *bar, bool issue)
{
    SegWindow w;
    w.A = (const float4 *)(smem + ly.A);
    w.I = (const float *)(smem + ly.I);
    w.SB = (const float4 *)(smem + ly.SB);
    w.SW = (const float2 *)(smem + ly.SW);
    w.w0 = w0;
    w.Wn = Wn;
    if (issue) {
        mbar_expect_tx(bar, (unsigned)Wn * (16u + 4u + 16u + 8u));
        bulk_g2s(smem + ly.A, tv.A + w0, (unsigned)Wn * 16u, bar);
        bulk_g2s(smem + ly.I, tv.I + w0, (unsigned)Wn * 4u, bar);
        bulk_g2s(smem + ly.SB, tv.SB + w0, (unsigned)Wn * 16u, bar);
        bulk_g2s(smem + ly.SW, tv.SW + w0, (unsigned)Wn * 8u, bar);
    }
    return w;
}

}  // namespace sgtp
