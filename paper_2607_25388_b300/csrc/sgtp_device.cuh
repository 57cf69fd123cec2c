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
// Device raceline of one closed track; per waypoint/segment j (segment j runs
// from waypoint j to j+1 mod N), arrays of length N + kWinMax (entry j >= N
// repeats entry j mod N):
//   A[j] = (x_j, y_j, bx_j, by_j)   waypoint and the direction u_{j-1} + u_j
//                                   (sum of the unit chords meeting there)
//   B[j] = (ex_j, ey_j, 1/|e_j|^2, |e_j|)   chord e_j = P_{j+1} - P_j
//   W[j] = (wL_j, wL_{j+1} - wL_j, wR_j, wR_{j+1} - wR_j)
//   S[j] = s_j                      cumulative arc length
//   C[j] = (psi_j, wrap(psi_{j+1} - psi_j), v_j, v_{j+1} - v_j)
//
// and the per-segment records of the sample-loop projection (frenet_fast in
// sgtp_rollout.cuh), with u_j = e_j / |e_j| and b_j = u_{j-1} + u_j:
//   G0[j] = (bx_j, by_j, b_j . P_j, |e_j|)   plane of waypoint j's bisector
//   G1[j] = (ux_j, uy_j, u_j . P_j, u_j x P_j)  the segment's line
//   G2[j] = (1/|e_j|, h_j, h_{j+1} - h_j, c_j)  half width h = (wL + wR)/2,
//                                               centre offset c = (wL - wR)/2
//   G3[j] = (c_{j+1} - c_j, s_j)
struct TrackView {
    const float4 *A;
    const float4 *B;
    const float4 *W;
    const float *S;
    const float4 *C;
    const float4 *G0, *G1, *G2;
    const float2 *G3;
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
    const float4 *B;
    const float4 *W;
    const float *S;
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
    int m;          // segment (window-local, or global without a window)
    int flag;       // the search hit its move limit
};

// ---- packed float pairs (Blackwell f32x2 arithmetic)
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk(float a, float b)
{
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(f2p v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b)
{
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b)
{
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c)
{
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Squared distance from p to segment (vertex a.xy, chord b); t is the
// clamped parameter, cr the cross product e x (p - a) (sign of d).
// ---------------------------------------------------------------- hardware approximations
// The special-function unit's approximations with denormal inputs and
// results flushed to zero (PTX .approx.ftz): no denormal handling around the
// instruction.  Every argument in this engine is either zero or a normal
// float (wrapped angles, steering angles, uniforms in [2^-24, 1), squared
// distances clamped to >= 1e-30), so the flush never applies.
__device__ __forceinline__ float sin_ftz(float x)
{
    float r;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float cos_ftz(float x)
{
    float r;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_ftz(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_ftz(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float seg_dist2(const float4 &a, const float4 &b, float px, float py, float &t, float &cr)
{
    const float dx = px - a.x, dy = py - a.y;
    float u = __fmul_rn(__fmaf_rn(dx, b.x, __fmul_rn(dy, b.y)), b.z);
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    const float ex = __fmaf_rn(-u, b.x, dx), ey = __fmaf_rn(-u, b.y, dy);
    t = u;
    cr = __fmaf_rn(b.x, dy, -__fmul_rn(b.y, dx));
    return __fmaf_rn(ex, ex, __fmul_rn(ey, ey));
}

// Segment data at window-local index r (shared memory inside the window,
// global memory outside it).
struct SegData {
    float4 a, b, w;
    float s;
};
__device__ __forceinline__ SegData seg_at(const TrackView &tv, const SegWindow &w, int r)
{
    SegData d;
    if ((unsigned)r < (unsigned)w.Wn) {
        d.a = w.A[r]; d.b = w.B[r]; d.w = w.W[r]; d.s = w.S[r];
    } else {
        const int j = wrap_index(w.w0 + r, tv.N);
        d.a = __ldg(tv.A + j); d.b = __ldg(tv.B + j); d.w = __ldg(tv.W + j); d.s = __ldg(tv.S + j);
    }
    return d;
}

__device__ __forceinline__ FrenetPt frenet_result(const SegData &g, int m, float t, float d2, float cr)
{
    const float dist = __fmul_rn(d2, rsqrt_ftz(fmaxf(d2, 1e-30f)));
    FrenetPt f;
    f.s = __fmaf_rn(t, g.b.w, g.s);
    f.d = cr >= 0.0f ? dist : -dist;
    f.t = t;
    f.wl = __fmaf_rn(t, g.w.y, g.w.x);
    f.wr = __fmaf_rn(t, g.w.w, g.w.z);
    f.m = m;
    f.flag = 0;
    return f;
}

// General local search by distance: starting at segment r, move to the next
// segment while it is strictly nearer, else to the previous one while it is
// at least as near (lowest index on ties); the result is a local minimum of
// the point-to-segment distance over the segment index, which for points
// within the track's reach is the global nearest segment of Sec. II's
// projection.  A search longer than kMaxMoves stops and sets flag.
static __device__ __forceinline__ FrenetPt frenet_search(const TrackView tv, const SegWindow w, int r, float px, float py)
{
    int flag = 0;
    SegData g = seg_at(tv, w, r);
    float t, cr;
    float bd = seg_dist2(g.a, g.b, px, py, t, cr);
    bool moved = false;
    for (int it = 0; it < kMaxMoves; ++it) {
        const SegData gn = seg_at(tv, w, r + 1);
        float tn, cn;
        const float dn = seg_dist2(gn.a, gn.b, px, py, tn, cn);
        if (!(dn < bd)) break;
        r += 1; bd = dn; t = tn; cr = cn; g = gn; moved = true;
        if (it == kMaxMoves - 1) flag = 1;
    }
    if (!moved) {
        for (int it = 0; it < kMaxMoves; ++it) {
            const SegData gp = seg_at(tv, w, r - 1);
            float tp, cp;
            const float dp = seg_dist2(gp.a, gp.b, px, py, tp, cp);
            if (!(dp <= bd)) break;
            r -= 1; bd = dp; t = tp; cr = cp; g = gp;
            if (it == kMaxMoves - 1) flag = 1;
        }
    }
    FrenetPt f = frenet_result(g, r, t, bd, cr);
    f.flag = flag;
    return f;
}

// Start segment offset for frenet_search of a point displaced by (dx, dy)
// from a state whose nearest segment has chord b = B[j]: the displacement's
// length in units of |e_j|, capped at cap, negative when the displacement
// points against the segment's direction (a vehicle that has turned around
// moves back along the track, and an always-forward guess would overshoot by
// twice its travel).  Within the track's reach the walk ends at the same
// segment from any start; the guess only keeps the walk short.
__device__ __forceinline__ int chord_guess(float dx, float dy, float4 b, int cap)
{
    const float ch = sqrtf(dx * dx + dy * dy);
    const int n = min((int)(ch / b.w), cap);
    return __fmaf_rn(dx, b.x, dy * b.y) < 0.0f ? -n : n;
}

// Segments of one brute-force pass that a thread loads before it evaluates
// them: the pass over a cold track then waits for a few memory round trips
// instead of one per segment.
constexpr int kScanBatch = 8;

// This thread's minimum key (squared distance bits, segment) over segments
// j0, j0 + step, ... < N; out-of-range slots of the last batch load segment
// N - 1 and are ignored.
__device__ __forceinline__ unsigned long long nearest_scan(const TrackView &tv, float px, float py, int j0, int step)
{
    unsigned long long best = ~0ull;
    for (int jb = j0; jb < tv.N; jb += kScanBatch * step) {
        float4 va[kScanBatch], vb[kScanBatch];
#pragma unroll
        for (int u = 0; u < kScanBatch; ++u) {
            const int j = min(jb + u * step, tv.N - 1);
            va[u] = __ldg(tv.A + j);
            vb[u] = __ldg(tv.B + j);
        }
#pragma unroll
        for (int u = 0; u < kScanBatch; ++u) {
            const int j = jb + u * step;
            float t, cr;
            const float d2 = seg_dist2(va[u], vb[u], px, py, t, cr);
            const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j;
            if (j < tv.N && key < best) best = key;
        }
    }
    return best;
}

// Global nearest segment by brute force over all N segments, cooperatively by
// one warp (lowest index on ties).  Used once per vehicle state x_{i,t}.
__device__ __forceinline__ int nearest_segment_warp(const TrackView &tv, float px, float py)
{
    const int lane = threadIdx.x & 31;
    unsigned long long best = nearest_scan(tv, px, py, lane, 32);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    return (int)(best & 0xffffffffu);
}

// The same search by every thread of the CTA (lowest index on ties); key_sh
// is one shared 64-bit word.  All threads must call it; all get the result.
__device__ __forceinline__ int nearest_segment_cta(const TrackView &tv, float px, float py, unsigned long long *key_sh)
{
    if (threadIdx.x == 0) *key_sh = ~0ull;
    __syncthreads();
    unsigned long long best = nearest_scan(tv, px, py, threadIdx.x, blockDim.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(key_sh, best);
    __syncthreads();
    return (int)(*key_sh & 0xffffffffu);
}

// Projection on a known segment j (global index).
__device__ __forceinline__ FrenetPt frenet_at(const TrackView &tv, int j, float px, float py)
{
    SegData g;
    g.a = __ldg(tv.A + j); g.b = __ldg(tv.B + j); g.w = __ldg(tv.W + j); g.s = __ldg(tv.S + j);
    float t, cr;
    const float d2 = seg_dist2(g.a, g.b, px, py, t, cr);
    return frenet_result(g, j, t, d2, cr);
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
// recursion however long the track.
//
// One warp (all 32 lanes call it; lane 0 writes ref).  The recursion is
// sequential, so every lane carries the same (hi, lo); the lanes hold 32
// consecutive segments (from the shared-memory window, A, B, S and C, when it
// has them, else from global memory), and each step finds the segment
// holding the progress, s_j <= hm < s_j + |e_j| (the lap's last segment ends
// at L), with one ballot -- the lowest such lane -- instead of a walk of
// dependent loads.  The block moves forward when the progress passes its
// middle.  j0 is the global segment of s0 (s0 in [0, L)).
__device__ __forceinline__ void reference_traj(const TrackView &tv, const SegWindow &w, const float4 *Cw, int j0,
                                               float s0, float dt, float vscale, int T, float4 *ref)
{
    const int lane = threadIdx.x & 31;
    const int N = tv.N, Wn = w.Wn;
    const float L = tv.L;
    float hi = s0, lo = 0.f;
    int jb = j0, lapb = 0;                 // first segment of the lanes' block and its lap
    float4 va, vb, c;
    float sj;
    int lapl;
    bool last;
    auto load_block = [&]() {
        int g = jb + lane, lp = lapb;
        while (g >= N) { g -= N; ++lp; }
        while (g < 0) { g += N; --lp; }
        const int rl = Wn > 0 ? wrap_index(g - w.w0, N) : -1;
        if ((unsigned)rl < (unsigned)Wn) {
            va = w.A[rl]; vb = w.B[rl]; sj = w.S[rl]; c = Cw[rl];
        } else {
            va = __ldg(tv.A + g); vb = __ldg(tv.B + g); sj = __ldg(tv.S + g); c = __ldg(tv.C + g);
        }
        lapl = lp;
        last = g == N - 1;
    };
    load_block();
    auto locate = [&]() -> float4 {
        for (int it = 0; it < 2 * (N / 32) + 8; ++it) {
            const float hm = hi - (float)lapl * L;            // exact: within a factor 2 of lap L
            const float sn = last ? L : sj + vb.w;
            const unsigned bal = __ballot_sync(0xffffffffu, hm >= sj && hm < sn);
            if (bal) {
                const int src = __ffs(bal) - 1;
                const float u = ((hm - sj) + lo) * (vb.w * vb.z);      // / |e_j|, as |e_j| * (1 / |e_j|^2)
                float4 o;
                o.x = __shfl_sync(0xffffffffu, __fmaf_rn(u, vb.x, va.x), src);
                o.y = __shfl_sync(0xffffffffu, __fmaf_rn(u, vb.y, va.y), src);
                o.z = __shfl_sync(0xffffffffu, __fmaf_rn(u, c.y, c.x), src);
                o.w = __shfl_sync(0xffffffffu, __fmaf_rn(u, c.w, c.z), src);
                if (src >= 16) {                               // keep at least 16 segments ahead
                    jb += src;
                    while (jb >= N) { jb -= N; ++lapb; }
                    load_block();
                }
                return o;
            }
            // no lane holds it: move the block by 32 segments toward it
            const bool ahead = __shfl_sync(0xffffffffu, hm >= sn, 31);
            jb += ahead ? 32 : -32;
            while (jb >= N) { jb -= N; ++lapb; }
            while (jb < 0) { jb += N; --lapb; }
            load_block();
        }
        return make_float4(__shfl_sync(0xffffffffu, va.x, 0), __shfl_sync(0xffffffffu, va.y, 0),
                           __shfl_sync(0xffffffffu, c.x, 0), __shfl_sync(0xffffffffu, c.z, 0));
    };
    if (lane == 0) ref[0] = make_float4(0.f, 0.f, 0.f, 0.f);
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
        if (lane == 0) ref[tau + 1] = r1;
    }
}

// Segments of track from a vehicle's own segment that a setup stages in
// shared memory for its reference recursion (vertex, chord, arc length and
// the heading/speed coefficients; 52 bytes each).  A 60-step reference at
// up to 3 m per step spans about 100 segments of 1.8 m, and the recursion's
// block of 32 lanes reaches up to 31 segments past its progress; whatever
// lies beyond the staged stretch is read from global memory.
constexpr int kRefSegs = 152;
constexpr unsigned kRefStretchBytes = 52u * kRefSegs;

// Stage the stretch from segment j0 into dst (16-byte aligned, all threads
// of the CTA; the caller synchronises before the recursion reads it).  The
// copies are the values the recursion would read from global memory, so the
// reference is the same bit for bit.  Returns the window for reference_traj
// and its coefficient array in Cw.
__device__ __forceinline__ SegWindow stage_ref_stretch(const TrackView &tv, int j0, void *dst, const float4 *&Cw)
{
    float4 *A = (float4 *)dst;
    float4 *B = A + kRefSegs;
    float4 *C = B + kRefSegs;
    float *Sv = (float *)(C + kRefSegs);
    const int Wn = min(kRefSegs, tv.N);
    for (int r = threadIdx.x; r < Wn; r += blockDim.x) {
        const int g = wrap_index(j0 + r, tv.N);
        A[r] = __ldg(tv.A + g);
        B[r] = __ldg(tv.B + g);
        C[r] = __ldg(tv.C + g);
        Sv[r] = __ldg(tv.S + g);
    }
    Cw = C;
    return SegWindow{A, B, nullptr, Sv, j0, Wn};
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies with a Weyl
// key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
        c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ k.x, (unsigned)p1, (unsigned)(p0 >> 32) ^ c.w ^ k.y,
                       (unsigned)p0);
    }
    return c;
}

// The ten round keys of the Weyl schedule, computed once per launch on the
// host: a kernel parameter, so every round's key is a constant-bank operand
// of the sample loop instead of two additions per round.
struct RoundKeys {
    uint2 k[10];
};

__host__ __device__ inline RoundKeys make_round_keys(uint2 key)
{
    RoundKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k[r] = key;
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
    }
    return rk;
}

// philox4x32_10 with precomputed round keys (the same bits).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const RoundKeys &rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
        c = make_uint4((unsigned)(p1 >> 32) ^ c.y ^ rk.k[r].x, (unsigned)p1, (unsigned)(p0 >> 32) ^ c.w ^ rk.k[r].y,
                       (unsigned)p0);
    }
    return c;
}

// Uniform in (0,1) from the top 23 bits: ((w >> 9) + 1/2) 2^-23, exact in
// float32.  One funnel shift builds the float 1 + (w >> 9) 2^-23 in [1, 2)
// (exponent bits 0x3f8 above the 23 mantissa bits); subtracting 1 - 2^-24 is
// exact (Sterbenz) and leaves the uniform.
__device__ __forceinline__ float uniform_open(unsigned w)
{
    return __uint_as_float(__funnelshift_r(w, 0x7Fu, 9)) - 0.99999994039535522461f;
}

// Box-Muller pair from two words: (sqrt(-2 ln u1) cos 2pi u2, ... sin ...).
// The angle is evaluated as 2 pi u2 - pi in (-pi, pi) with the signs folded
// back, keeping the sine and cosine approximations inside their accurate range.
__device__ __forceinline__ float2 box_muller(unsigned w0, unsigned w1)
{
    const float u1 = uniform_open(w0), u2 = uniform_open(w1);
    // -2 ln u1 = (-2 ln 2) log2 u1; the approximate log2 may overshoot 0 as
    // u1 -> 1 (u1 <= 1 - 2^-24), where the magnitude stays the right size
    const float r = sqrt_ftz(fabsf(-1.38629436111989061883f * lg2_ftz(u1)));
    const float ang = __fmaf_rn(kTwoPi, u2, -kPi);
    const float sn = sin_ftz(ang), cs = cos_ftz(ang);
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

// Plain arrival (release at CTA scope), no transaction bytes.
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
    if (mbar_try_wait(bar, parity)) return true;         // the common case: no clock read
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

// Window start for a segment j0: `back` segments behind it, rounded down to a
// multiple of 4 so that every array's copy starts 16-byte aligned.
__device__ __forceinline__ int window_start(int j0, int back, int N)
{
    int w0 = wrap_index(j0 - back, N);
    return w0 & ~3;
}

}  // namespace sgtp
