// sgtp_probe.cu -- measurement and verification entry points: the FP32 FMA
// throughput of the device (the denominator of the hot path's roofline) and
// the noise generator's raw words and normals, exactly as the sample loop
// computes them.
#include <algorithm>

#include "sgtp_host.hpp"
#include "sgtp_rollout.cuh"

using namespace sgtp;

namespace {

// Eight independent FMA chains per thread, eight steps each per iteration:
// with a few warps per scheduler every issue slot carries an FMA.  The
// result is stored only under a condition no chain meets, so every thread
// must compute it.
template <bool PACKED>
__global__ void __launch_bounds__(256) fma_probe_kernel(float *sink, int iters, float a, float b)
{
    float r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = (float)threadIdx.x * 1e-6f + (float)i;
    if (PACKED) {
        f2p q[4], av = pk(a, a), bv = pk(b, b);
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = pk(r[2 * i], r[2 * i + 1]);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int i = 0; i < 4; ++i) q[i] = fma2(q[i], av, bv);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 v = upk(q[i]);
            r[2 * i] = v.x;
            r[2 * i + 1] = v.y;
        }
    } else {
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int i = 0; i < 8; ++i) r[i] = __fmaf_rn(r[i], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += r[i];
    if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

__global__ void philox_words_kernel(RoundKeys rk, uint2 key, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, int n,
                                    uint32_t *out, int *mismatch)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(k0 + (uint32_t)i, c1, c2, c3);
        const uint4 w = philox4x32_10_rk(c, rk);
        // the key-schedule form used outside the sample loop must agree
        const uint4 v = philox4x32_10(c, key);
        if (w.x != v.x || w.y != v.y || w.z != v.z || w.w != v.w) atomicAdd(mismatch, 1);
        out[4 * (size_t)i + 0] = w.x;
        out[4 * (size_t)i + 1] = w.y;
        out[4 * (size_t)i + 2] = w.z;
        out[4 * (size_t)i + 3] = w.w;
    }
}

// The sample loop's normals of candidates k0 .. k0 + nk - 1, steps 0 .. T-1
// (noise_pair on the counter layout of sgtp.h).
__global__ void noise_normals_kernel(RoundKeys rk, unsigned ar, unsigned race, unsigned sbit, uint32_t k0, int nk,
                                     int T, float *z)
{
    const int pairs = (T + 1) / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nk * pairs; q += gridDim.x * blockDim.x) {
        const int i = q / pairs, m = q - i * pairs;
        const uint4 w = philox4x32_10_rk(make_uint4(k0 + (uint32_t)i, (unsigned)m | sbit, ar, race), rk);
        const float2 z0 = box_muller(w.x, w.y), z1 = box_muller(w.z, w.w);
        float *o = z + ((size_t)i * T + 2 * m) * 2;
        o[0] = z0.x;
        o[1] = z0.y;
        if (2 * m + 1 < T) {
            o[2] = z1.x;
            o[3] = z1.y;
        }
    }
}

}  // namespace

extern "C" sgtp_status sgtp_fma_probe(int32_t ctas_per_sm, int32_t iters, int32_t packed, float *sink, void *stream,
                                      double *flops)
{
    SGTP_CHECK(ctas_per_sm >= 1 && ctas_per_sm <= 8, "ctas_per_sm must be in [1, 8]");
    SGTP_CHECK(iters >= 1 && iters <= (1 << 24), "iters must be in [1, 2^24]");
    SGTP_CHECK(sink != nullptr, "sink is NULL");
    int dev = 0, sms = 0;
    SGTP_CUDA(cudaGetDevice(&dev));
    SGTP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * ctas_per_sm;
    cudaStream_t s = (cudaStream_t)stream;
    if (packed)
        fma_probe_kernel<true><<<grid, 256, 0, s>>>(sink, iters, 1.0000001f, 1e-7f);
    else
        fma_probe_kernel<false><<<grid, 256, 0, s>>>(sink, iters, 1.0000001f, 1e-7f);
    count_launch();
    SGTP_CUDA(cudaGetLastError());
    if (flops) *flops = (double)grid * 256.0 * (double)iters * 64.0 * 2.0;
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, int32_t n,
                                         uint32_t *words, int32_t *mismatch, void *stream)
{
    SGTP_CHECK(n >= 1 && words != nullptr && mismatch != nullptr, "bad arguments");
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    const int grid = (int)std::min<long long>(4096, ((long long)n + 255) / 256);
    philox_words_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(make_round_keys(key), key, c1, c2, c3, k0, n, words,
                                                                mismatch);
    count_launch();
    SGTP_CUDA(cudaGetLastError());
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_noise_normals(uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                                          uint32_t stream_bit, uint32_t k0, int32_t nk, int32_t T, float *z,
                                          void *stream)
{
    SGTP_CHECK(nk >= 1 && T >= 1 && T <= SGTP_MAX_T && z != nullptr, "bad arguments");
    SGTP_CHECK(agent < (1u << 16) && round < (1u << 16) && stream_bit <= 1u, "agent/round/stream out of range");
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    const long long work = (long long)nk * ((T + 1) / 2);
    SGTP_CHECK(work < (1ll << 31), "nk x T too large");
    const int grid = (int)std::min<long long>(4096, (work + 255) / 256);
    noise_normals_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(make_round_keys(key), agent | (round << 16), race,
                                                                 stream_bit << 31, k0, nk, T, z);
    count_launch();
    SGTP_CUDA(cudaGetLastError());
    return SGTP_OK;
}
