// sgtp_host.hpp -- host-side pieces shared by the ABI translation units:
// the track object, error text, launch counting and argument checks.
#pragma once

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "sgtp.h"
#include "sgtp_device.cuh"

struct sgtp_mlp;
const float *sgtp_mlp_master(const sgtp_mlp *M);
// BF16 weights in mma fragment order: per layer, per 8-row tile and 16-deep
// k-step, 32 lanes x {b0, b1}; rows padded to a multiple of 8.
const __nv_bfloat16 *sgtp_mlp_fragments(const sgtp_mlp *M);

struct sgtp_track {
    int n_tracks = 0;
    long long total = 0;                   // elements over all (ring-extended) tracks
    float4 *A = nullptr, *B = nullptr, *W = nullptr, *C = nullptr;
    float *S = nullptr;
    float4 *G0 = nullptr, *G1 = nullptr, *G2 = nullptr;   // sample-loop projection records
    float2 *G3 = nullptr;
    sgtp::TrackDesc *desc_dev = nullptr;
    std::vector<sgtp::TrackDesc> desc;     // host copy (L filled after prep)
    int device = 0;
};

namespace sgtp {

sgtp_status set_error(sgtp_status s, const char *fmt, ...);
void count_launch(int n = 1);

inline TrackView track_view(const sgtp_track *t, int id)
{
    const TrackDesc &d = t->desc[id];
    TrackView v;
    v.A = t->A + d.offset; v.B = t->B + d.offset; v.W = t->W + d.offset; v.S = t->S + d.offset;
    v.C = t->C + d.offset;
    v.G0 = t->G0 + d.offset; v.G1 = t->G1 + d.offset; v.G2 = t->G2 + d.offset; v.G3 = t->G3 + d.offset;
    v.N = d.N; v.L = d.L;
    return v;
}

// Elements of one ring-extended track (multiple of 4).
inline int ext_len(int N) { return (N + kWinMax + 3) & ~3; }

// Window length for a track of N segments: the requested window (default
// 512), at most kWinMax, at least 8, a multiple of 4.
inline int window_len(int N, int requested)
{
    int w = requested > 0 ? requested : 512;
    if (w > kWinMax) w = kWinMax;
    const int n4 = (N + 3) & ~3;
    if (w > n4) w = n4;
    if (w < 8) w = 8;
    return (w + 3) & ~3;
}

// Per-vehicle tail count of the blocking term: ceil(mu * H - 1e-4) clamped
// to [1, H], evaluated in double on the host so that every kernel sees the
// same integer.
inline int tail_count(float mu, int T)
{
    double v = (double)mu * (double)T - 1e-4;
    int n = (int)v;
    if ((double)n < v) n += 1;
    if (n < 1) n = 1;
    if (n > T) n = T;
    return n;
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

sgtp_status check_params(const sgtp_params *p);

// Devices whose one-time set-up is tracked per device index.
constexpr int kMaxDevices = 64;

// A flag per device for set-up that applies only to the device current when
// it runs (cudaFuncSetAttribute, cudaGetSymbolAddress): zero-initialised in
// static storage.
struct PerDeviceFlag {
    std::atomic<bool> on[kMaxDevices];
};

}  // namespace sgtp

#define SGTP_CUDA(x)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (x);                                                                         \
        if (e_ != cudaSuccess) return sgtp::set_error(SGTP_E_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

#define SGTP_CHECK(cond, ...)                                            \
    do {                                                                 \
        if (!(cond)) return sgtp::set_error(SGTP_E_INVALID, __VA_ARGS__); \
    } while (0)

namespace sgtp {

// Run `step` (which returns sgtp_status) once on the current device: later
// calls on the same device skip it.  Several host threads may run it at
// once on one device, which is harmless because every step used here is
// idempotent.  Devices beyond kMaxDevices run it on every call.
template <typename F>
sgtp_status once_per_device(PerDeviceFlag &flag, F step)
{
    int dev = 0;
    SGTP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return step();
    if (flag.on[dev].load(std::memory_order_acquire)) return SGTP_OK;
    const sgtp_status st = step();
    if (st == SGTP_OK) flag.on[dev].store(true, std::memory_order_release);
    return st;
}

// Default limit of each device-side wait of a launch that rolls out
// `rollout_steps` candidate-steps: 20 times its duration at a pessimistic
// 5e10 rollout-steps/s, at least 100 ms (the measured rate is about 1e11).
inline long long default_wait_ns(double rollout_steps)
{
    const double est_ns = rollout_steps / 5e10 * 1e9;
    const double lim = 20.0 * est_ns;
    return lim > 1e8 ? (long long)lim : 100000000ll;
}

// Every device allocation of the library goes through dev_malloc, so that
// a test can make the n-th next one fail as if the device were out of
// memory (sgtp_debug_fail_alloc; 0 = never, the default).
inline std::atomic<int> &fail_alloc_countdown()
{
    static std::atomic<int> c{0};
    return c;
}

template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes)
{
    int c = fail_alloc_countdown().load();
    while (c > 0 && !fail_alloc_countdown().compare_exchange_weak(c, c - 1)) {
    }
    if (c == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc((void **)p, bytes);
}

}  // namespace sgtp
