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

// ---------------------------------------------------------------- track
// Device raceline of one closed track, one float4 triple per segment j
// (waypoint j to waypoint j+1 mod N):
//   A[j] = (x_j, y_j, ex_j, ey_j)            chord e_j = P_{j+1} - P_j
//   B[j] = (1/|e_j|^2, s_j, |e_j|, 0)        s_j cumulative arc length
//   W[j] = (wL_j, wL_{j+1}-wL_j, wR_j, wR_{j+1}-wR_j)
//   C[j] = (psi_j, wrap(psi_{j+1}-psi_j), v_j, v_{j+1}-v_j)
struct TrackView {
    const float4 *A, *B, *W, *C;
    int N;
    float L;     // total length
};

// Per-launch track table entry (one per track of an sgtp_track object).
struct TrackDesc {
    int offset;  // first segment in the concatenated arrays
    int N;
    float L;
    int pad;
};

// Shared-memory window of a track: segments w0 .. w0+Wn-1 (mod N) of A and B.
struct SegWindow {
    const float4 *sA, *sB;   // shared memory
    int w0, Wn;
};

__device__ __forceinline__ int wrap_index(int j, int N) { return j >= N ? j - N : (j < 0 ? j + N : j); }

__device__ __forceinline__ void load_seg(const TrackView &tv, const SegWindow &win, int j, float4 &a, float4 &b)
{
    int r = j - win.w0;
    if (r < 0) r += tv.N;
    if (r < win.Wn) {
        a = win.sA[r];
        b = win.sB[r];
    } else {
        a = __ldg(tv.A + j);
        b = __ldg(tv.B + j);
    }
}

// Squared distance from p to segment (a, inv_l2); t is the clamped parameter.
__device__ __forceinline__ float seg_dist2(const float4 &a, float inv_l2, float px, float py, float &t)
{
    const float dx = px - a.x, dy = py - a.y;
    float u = __fmul_rn(__fmaf_rn(dx, a.z, __fmul_rn(dy, a.w)), inv_l2);
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    const float ex = __fmaf_rn(-u, a.z, dx), ey = __fmaf_rn(-u, a.w, dy);
    t = u;
    return __fmaf_rn(ex, ex, __fmul_rn(ey, ey));
}

// Frenet projection s(x; G), d(x; G) (Sec. II) by a local walk over segments
// from the previous nearest segment j: move forward while the next segment
// is strictly nearer, otherwise backward while the previous one is.  For
// points inside the track's reach the local minimum is the global nearest
// segment.  Returns raw progress s in [0, L), signed offset d (left +) and
// the segment parameter t; j is updated.  A walk longer than max_moves
// stops and sets *flag.
struct FrenetPt {
    float s, d, t;
};

__device__ __forceinline__ FrenetPt frenet_walk(const TrackView &tv, const SegWindow &win, int &j, float px, float py,
                                                int max_moves, int &flag)
{
    float4 a, b;
    load_seg(tv, win, j, a, b);
    float t;
    float d2 = seg_dist2(a, b.x, px, py, t);
    bool moved = false;
    for (int it = 0; it < max_moves; ++it) {
        const int jn = wrap_index(j + 1, tv.N);
        float4 an, bn;
        load_seg(tv, win, jn, an, bn);
        float tn;
        const float d2n = seg_dist2(an, bn.x, px, py, tn);
        if (!(d2n < d2)) break;
        j = jn; a = an; b = bn; d2 = d2n; t = tn; moved = true;
        if (it == max_moves - 1) flag = 1;
    }
    if (!moved) {
        for (int it = 0; it < max_moves; ++it) {
            const int jp = wrap_index(j - 1, tv.N);
            float4 ap, bp;
            load_seg(tv, win, jp, ap, bp);
            float tp;
            const float d2p = seg_dist2(ap, bp.x, px, py, tp);
            if (!(d2p < d2)) break;
            j = jp; a = ap; b = bp; d2 = d2p; t = tp;
            if (it == max_moves - 1) flag = 1;
        }
    }
    const float dx = px - a.x, dy = py - a.y;
    const float cr = __fmaf_rn(a.z, dy, -__fmul_rn(a.w, dx));
    const float dist = __fmul_rn(d2, rsqrtf(fmaxf(d2, 1e-30f)));
    FrenetPt r;
    r.s = __fmaf_rn(t, b.z, b.y);
    r.d = cr >= 0.0f ? dist : -dist;
    r.t = t;
    return r;
}

// Global nearest segment by brute force over all N segments, cooperatively by
// one warp (lowest index on ties).  Used once per vehicle state x_{i,t}.
__device__ __forceinline__ int nearest_segment_warp(const TrackView &tv, float px, float py)
{
    const int lane = threadIdx.x & 31;
    unsigned long long best = ~0ull;
    for (int j = lane; j < tv.N; j += 32) {
        const float4 a = __ldg(tv.A + j);
        const float4 b = __ldg(tv.B + j);
        float t;
        const float d2 = seg_dist2(a, b.x, px, py, t);
        const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j;
        best = key < best ? key : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    return (int)(best & 0xffffffffu);
}

// Projection at a known segment (no walk).
__device__ __forceinline__ FrenetPt frenet_at(const TrackView &tv, int j, float px, float py)
{
    const float4 a = __ldg(tv.A + j);
    const float4 b = __ldg(tv.B + j);
    float t;
    const float d2 = seg_dist2(a, b.x, px, py, t);
    const float dx = px - a.x, dy = py - a.y;
    const float cr = __fmaf_rn(a.z, dy, -__fmul_rn(a.w, dx));
    const float dist = __fmul_rn(d2, rsqrtf(fmaxf(d2, 1e-30f)));
    FrenetPt r;
    r.s = __fmaf_rn(t, b.z, b.y);
    r.d = cr >= 0.0f ? dist : -dist;
    r.t = t;
    return r;
}

// Wrap a progress difference into (-L/2, L/2].
__device__ __forceinline__ float wrap_len(float x, float L, float invL)
{
    return __fmaf_rn(-L, ceilf(__fmaf_rn(x, invL, -0.5f)), x);
}

// Wrap an angle into (-pi, pi] (used only squared, so the end choice is moot).
__device__ __forceinline__ float wrap_angle(float a) { return __fmaf_rn(-kTwoPi, rintf(a * kInvTwoPi), a); }

// Reference map x^r(s) (Sec. III-A): s taken modulo L; segment found by
// walking forward from j (s increases monotonically along the reference).
__device__ __forceinline__ float4 reference_at(const TrackView &tv, int &j, float s)
{
    float sm = s - tv.L * floorf(s / tv.L);
    if (sm >= tv.L) sm -= tv.L;
    // walk to the segment with s_j <= sm < s_{j+1}
    for (int it = 0; it < 4 * tv.N; ++it) {
        const float4 b = __ldg(tv.B + j);
        const float s_next = (j + 1 == tv.N) ? tv.L : __ldg(tv.B + j + 1).y;
        if (sm < b.y) { j = wrap_index(j - 1, tv.N); continue; }
        if (sm >= s_next) { j = wrap_index(j + 1, tv.N); continue; }
        break;
    }
    const float4 a = __ldg(tv.A + j);
    const float4 b = __ldg(tv.B + j);
    const float4 c = __ldg(tv.C + j);
    const float u = (sm - b.y) / b.z;
    float4 r;
    r.x = __fmaf_rn(u, a.z, a.x);
    r.y = __fmaf_rn(u, a.w, a.y);
    r.z = __fmaf_rn(u, c.y, c.x);
    r.w = __fmaf_rn(u, c.w, c.z);
    return r;
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
__device__ __forceinline__ float uniform_open(unsigned w) { return __fmaf_rn((float)(w >> 9), 1.1920928955078125e-7f, 5.9604644775390625e-8f); }

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

}  // namespace sgtp
