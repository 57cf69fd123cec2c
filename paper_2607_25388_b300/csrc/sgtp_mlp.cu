// sgtp_mlp.cu -- the learned proposal: features, BF16 MLP on the tensor
// cores with FP32 accumulation (forward, backward, Adam), and the Gaussian
// NLL loss.  Not part of the paper: a proposal distribution over control
// sequences that seeds part of the sample budget of a best response, while
// the plain Gaussian sampler (Sec. II) keeps the rest.
//
// Network: x (64) -> 256 -> 256 -> 256 -> 4T, ReLU on the hidden layers.
// Output row b: [mu_a(0..T-1), mu_delta(0..T-1), logsig_a(0..T-1),
// logsig_delta(0..T-1)] in units of the plain sampler's sigma per channel.
// Parameters (FP32 master and BF16 working copy) are laid out per layer as
// W_l [out][in] followed by b_l [out].
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>

#include "sgtp_host.hpp"
#include "sgtp_mlp.h"

using namespace sgtp;

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kIn = SGTP_MLP_IN, kHid = SGTP_MLP_HIDDEN;

__host__ __device__ inline int layer_in(int l) { return l == 0 ? kIn : kHid; }
__host__ __device__ inline int layer_out(int l, int out) { return l == 3 ? out : kHid; }
__host__ __device__ inline long long layer_off(int l, int out)
{
    long long o = 0;
    for (int q = 0; q < l; ++q) o += (long long)layer_out(q, out) * layer_in(q) + layer_out(q, out);
    return o;
}

// ---------------------------------------------------------------- tensor-core GEMM
// C[M x N] = A[M x K] * B[K x N] with BF16 operands and FP32 accumulation
// (gemm_kernel below).
enum { EPI_F32 = 0, EPI_BIAS_RELU_BF16 = 1, EPI_BIAS_F32 = 2 };

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldsm_x4(unsigned r[4], const bf16 *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned r[4], const bf16 *p)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// One operand tile of a pipeline stage, copied in the global layout: ROWS
// rows of COLS contiguous elements (row pitch PITCH in shared memory).
// Element (r, c) is global (row0 + r, col0 + c), present when row0 + r <
// row_lim and col0 + c < col_lim, else zero.  Whole 16-byte chunks are
// asynchronous copies (zero-filled outside the matrix); a chunk cut by
// col_lim, or any chunk when the rows are not 16-byte aligned, is copied
// element by element.
template <int ROWS, int COLS, int PITCH>
__device__ __forceinline__ void load_tile(bf16 *dst, const bf16 *g, int ld, int row0, int row_lim, int col0,
                                          int col_lim, bool vec_ok)
{
    constexpr int CPR = COLS / 8;
    for (int q = threadIdx.x; q < ROWS * CPR; q += blockDim.x) {
        const int r = q / CPR, c = (q - r * CPR) * 8;
        bf16 *d = dst + r * PITCH + c;
        const int gr = row0 + r, gc = col0 + c;
        if (gr >= row_lim || gc >= col_lim) {
            cp_async16(d, g, 0);
        } else {
            const bf16 *src = g + (size_t)gr * ld + gc;
            if (vec_ok && gc + 8 <= col_lim) {
                cp_async16(d, src, 16);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) d[e] = gc + e < col_lim ? src[e] : __float2bfloat16(0.f);
            }
        }
    }
}

// C = A B on the tensor cores (mma.sync m16n8k16, BF16 in, FP32 accumulate).
// A is stored [M][K] (TA = false) or [K][M] (TA = true); B is stored [N][K]
// (TB = true) or [K][N] (TB = false).  CTA tile 64 x 64, K step 32, 4 warps
// of 32 x 32; three pipeline stages of 16-byte asynchronous copies keep the
// operands in their global layout in shared memory, and ldmatrix (.trans for
// the M- or N-major operands) builds the mma fragments.  Epilogues: FP32 out
// (optionally + bias), or BF16 out of ReLU(acc + bias).
// Split K: CTA z of a grid with gridDim.z > 1 sums k in [z kchunk,
// (z+1) kchunk) only and writes its FP32 partial product to Cv + z
// part_stride (EPI_F32); splitk_reduce_kernel then adds the partials in z
// order, so the result does not depend on scheduling.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(const bf16 *__restrict__ A, const bf16 *__restrict__ B, void *Cv,
                                                   const float *__restrict__ bias, int M, int N, int K, int lda,
                                                   int ldb, int ldc, int kchunk, long long part_stride)
{
    constexpr int BM = 64, BN = 64, BK = 32, STAGES = 3;
    constexpr int PA = TA ? BM + 8 : BK + 8;          // row pitch of the A tile (elements)
    constexpr int PB = TB ? BK + 8 : BN + 8;          // row pitch of the B tile
    constexpr int SA = TA ? BK * PA : BM * PA, SB = TB ? BN * PB : BK * PB;
    __shared__ __align__(16) bf16 As[STAGES][SA];
    __shared__ __align__(16) bf16 Bs[STAGES][SB];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    if (EPI == EPI_F32) Cv = (float *)Cv + blockIdx.z * part_stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    const bool va = (lda & 7) == 0 && ((uintptr_t)A & 15) == 0;
    const bool vb = (ldb & 7) == 0 && ((uintptr_t)B & 15) == 0;
    auto load_stage = [&](int st, int k0) {
        if (TA) load_tile<BK, BM, PA>(As[st], A, lda, k0, ke, m0, M, va);
        else load_tile<BM, BK, PA>(As[st], A, lda, m0, M, k0, ke, va);
        if (TB) load_tile<BN, BK, PB>(Bs[st], B, ldb, n0, N, k0, ke, vb);
        else load_tile<BK, BN, PB>(Bs[st], B, ldb, k0, ke, n0, N, vb);
    };
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    const int nk = ke > kb ? (ke - kb + BK - 1) / BK : 0;
#pragma unroll
    for (int st = 0; st < STAGES - 1; ++st) {
        if (st < nk) load_stage(st, kb + st * BK);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nt = kt + STAGES - 1;
            if (nt < nk) load_stage(nt % STAGES, kb + nt * BK);
            cp_async_commit();
        }
        const bf16 *as = As[kt % STAGES], *bs = Bs[kt % STAGES];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (TA)
                    ldsm_x4_t(af[i], as + (kk + (lane & 7) + ((lane >> 4) << 3)) * PA + wm + 16 * i +
                                         ((lane >> 3) & 1) * 8);
                else
                    ldsm_x4(af[i], as + (wm + 16 * i + (lane & 15)) * PA + kk + (lane >> 4) * 8);
            }
#pragma unroll
            for (int jp = 0; jp < 2; ++jp) {
                const int nb = wn + 16 * jp;
                unsigned r[4];
                if (TB) ldsm_x4(r, bs + (nb + (lane & 7) + ((lane >> 4) << 3)) * PB + kk + ((lane >> 3) & 1) * 8);
                else ldsm_x4_t(r, bs + (kk + (lane & 15)) * PB + nb + (lane >> 4) * 8);
                bfr[2 * jp][0] = r[0]; bfr[2 * jp][1] = r[1];
                bfr[2 * jp + 1][0] = r[2]; bfr[2 * jp + 1][1] = r[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
    }
    cp_async_wait<0>();
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = m0 + wm + 16 * i + g + (q >= 2 ? 8 : 0);
                const int c = n0 + wn + 8 * j + 2 * t + (q & 1);
                if (r >= M || c >= N) continue;
                float v = acc[i][j][q];
                if (EPI == EPI_F32) {
                    ((float *)Cv)[(size_t)r * ldc + c] = v;
                } else if (EPI == EPI_BIAS_F32) {
                    ((float *)Cv)[(size_t)r * ldc + c] = v + bias[c];
                } else {
                    v = fmaxf(v + bias[c], 0.f);
                    ((bf16 *)Cv)[(size_t)r * ldc + c] = __float2bfloat16(v);
                }
            }
}

template <bool TA, bool TB, int EPI>
void gemm(const bf16 *A, const bf16 *B, void *C, const float *bias, int M, int N, int K, int lda, int ldb, int ldc,
          cudaStream_t s)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_kernel<TA, TB, EPI><<<grid, 128, 0, s>>>(A, B, C, bias, M, N, K, lda, ldb, ldc, K, 0ll);
    count_launch();
}

// C[i] = sum_z part[z][i], z in order.
__global__ void splitk_reduce_kernel(const float *part, int splits, long long n, float *C)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v = part[i];
        for (int z = 1; z < splits; ++z) v += part[(size_t)z * n + i];
        C[i] = v;
    }
}

// Work items (output tiles x K chunks) a split-K product aims at, and the
// FP32 partials it may need: splits x tiles <= kSplitTarget and
// M N <= tiles x 64 x 64.
constexpr int kSplitTarget = 256;
constexpr size_t kSplitPartFloats = (size_t)kSplitTarget * 64 * 64;

// FP32 C [M x N] (row-major, ldc = N) = A B with K split into chunks of a
// multiple of 32 so that the tiles times the chunks reach about
// kSplitTarget CTAs: the weight gradients have K = batch and few output
// tiles.  The split depends on M, N and K only, so results are
// reproducible run to run.
template <bool TA, bool TB>
void gemm_splitk(const bf16 *A, const bf16 *B, float *C, float *part, int M, int N, int K, int lda, int ldb,
                 cudaStream_t s)
{
    const int tiles = ((N + 63) / 64) * ((M + 63) / 64);
    int splits = std::max(1, std::min((K + 31) / 32, kSplitTarget / tiles));
    const int kchunk = ((K + splits - 1) / splits + 31) / 32 * 32;
    splits = (K + kchunk - 1) / kchunk;
    if (splits <= 1) {
        gemm<TA, TB, EPI_F32>(A, B, C, nullptr, M, N, K, lda, ldb, N, s);
        return;
    }
    dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
    const long long n = (long long)M * N;
    gemm_kernel<TA, TB, EPI_F32><<<grid, 128, 0, s>>>(A, B, part, nullptr, M, N, K, lda, ldb, N, kchunk, n);
    count_launch();
    splitk_reduce_kernel<<<(int)std::min<long long>(1024, (n + 255) / 256), 256, 0, s>>>(part, splits, n, C);
    count_launch();
}

// ---------------------------------------------------------------- elementwise
__global__ void f32_to_bf16_kernel(const float *x, bf16 *y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// Gaussian NLL of the target (in sigma units) under N(mu, exp(2 ls)), ls
// clamped to [-5, 2]; mean over B x 2T elements.  Writes d out (FP32, into
// dout), and the loss (atomic sum) into loss.
__global__ void nll_kernel(const float *out, const float *target, int Bsz, int T, float *dout, float *loss)
{
    const int n2 = 2 * T;
    const float inv = 1.0f / ((float)Bsz * (float)n2);
    float lsum = 0.f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Bsz * n2; e += gridDim.x * blockDim.x) {
        const int b = e / n2, q = e - b * n2;
        const float *o = out + (size_t)b * 2 * n2;
        const float mu = o[q];
        const float ls_raw = o[n2 + q];
        const float ls = fminf(fmaxf(ls_raw, -5.f), 2.f);
        const float is = expf(-ls);
        const float z = (target[(size_t)b * n2 + q] - mu) * is;
        lsum += 0.5f * z * z + ls;
        float *d = dout + (size_t)b * 2 * n2;
        d[q] = -z * is * inv;
        d[n2 + q] = (ls_raw > -5.f && ls_raw < 2.f) ? (1.f - z * z) * inv : 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum * inv);
}

// db[n] = sum_b dZ[b][n] (FP32) in a fixed order: a CTA takes 32 columns;
// its thread (g, c) sums rows g, g + 32, ... of column c (the warp reads 32
// consecutive columns of a row), then the 32 partial sums of a column are
// added in g order.
__global__ void __launch_bounds__(1024) colsum_kernel(const float *dz, int Bsz, int N, float *db)
{
    __shared__ float part[32][33];
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + c;
    float acc = 0.f;
    if (n < N)
        for (int b = g; b < Bsz; b += 32) acc += dz[(size_t)b * N + n];
    part[g][c] = acc;
    __syncthreads();
    if (g == 0 && n < N) {
        float t = 0.f;
        for (int q = 0; q < 32; ++q) t += part[q][c];
        db[n] = t;
    }
}

// dZ = dH * (H > 0) as BF16 (the ReLU mask from the BF16 activation), and
// the FP32 copy for the bias gradient.
__global__ void relu_back_kernel(const float *dh, const bf16 *h, long long n, bf16 *dz_b, float *dz_f)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = __bfloat162float(h[i]) > 0.f ? dh[i] : 0.f;
        dz_f[i] = v;
        dz_b[i] = __float2bfloat16(v);
    }
}

// Adam with bias correction on FP32 master weights; refreshes the BF16 copy.
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, bf16 *wb, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}

// Inference copy of the weights in mma fragment order (bias-free): per layer,
// per 8-row tile and 16-deep k-step, 32 lanes x {b0, b1} with lane (g, t)
// holding W[n][k0+2t], W[n][k0+2t+1], W[n][k0+2t+8], W[n][k0+2t+9] for
// n = 8 tile + g, k0 = 16 kstep; rows beyond N are zero.
__host__ __device__ inline long long frag_off(int l, int out)
{
    long long o = 0;
    for (int q = 0; q < l; ++q) o += (long long)((layer_out(q, out) + 7) & ~7) * layer_in(q);
    return o;
}

__global__ void frag_kernel(const float *w, bf16 *frag, int out)
{
    const long long total = frag_off(4, out);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int l = 0;
        while (l < 3 && e >= frag_off(l + 1, out)) ++l;
        const long long r = e - frag_off(l, out);
        const int K = layer_in(l), N = layer_out(l, out), ksteps = K / 16;
        const long long pair = r / 128;
        const int lane = (int)((r % 128) / 4), slot = (int)(r % 4);
        const int tile = (int)(pair / ksteps), ks = (int)(pair % ksteps);
        const int n = tile * 8 + (lane >> 2);
        const int k = ks * 16 + 2 * (lane & 3) + (slot & 1) + 8 * (slot >> 1);
        const float v = n < N ? w[layer_off(l, out) + (long long)n * K + k] : 0.f;
        frag[e] = __float2bfloat16(v);
    }
}

__global__ void init_kernel(float *w, bf16 *wb, long long off, int out, int in, unsigned long long seed)
{
    // Kaiming-uniform weights (bound sqrt(6/in)) from Philox, zero biases
    const long long nw = (long long)out * in;
    const float bound = sqrtf(6.0f / (float)in);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw + out;
         i += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i < nw) {
            const uint4 r = philox4x32_10(make_uint4((unsigned)i, (unsigned)(i >> 32), (unsigned)off, 7u),
                                          make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
            v = (uniform_open(r.x) * 2.f - 1.f) * bound;
        }
        w[off + i] = v;
        wb[off + i] = __float2bfloat16(v);
    }
}

// Per-step Gaussian of each output row: (sigma_a mu_a, sigma_delta mu_delta,
// sigma_a exp(ls_a), sigma_delta exp(ls_delta)), ls clamped to [-5, 2].
// Per-step Gaussian of each row: mean = nominal + sigma_plain mu (a residual
// around the plain sampler's centre; nominal 0 when u_nom is NULL), sigma =
// sigma_plain exp(clamp(logsig, -5, 2)).
__global__ void proposal_kernel(const float *out, const float *u_nom, int Bsz, int T, float sa, float sd,
                                float4 *prop)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Bsz * T; e += gridDim.x * blockDim.x) {
        const int b = e / T, t = e - b * T;
        const float *o = out + (size_t)b * 4 * T;
        const float la = fminf(fmaxf(o[2 * T + t], -5.f), 2.f);
        const float ld = fminf(fmaxf(o[3 * T + t], -5.f), 2.f);
        const float na = u_nom ? u_nom[2 * (size_t)e] : 0.f, nd = u_nom ? u_nom[2 * (size_t)e + 1] : 0.f;
        prop[e] = make_float4(__fmaf_rn(sa, o[t], na), __fmaf_rn(sd, o[T + t], nd), sa * expf(la), sd * expf(ld));
    }
}

}  // namespace

// ================================================================ ABI
struct sgtp_mlp {
    int T = 0, out = 0;
    long long n_params = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    bf16 *wb = nullptr;
    bf16 *wfrag = nullptr;        // inference copy in mma fragment order
    long long step = 0;
    // training scratch (batch-sized, grown on demand at setup time)
    int cap = 0;
    bf16 *xb = nullptr, *h[3] = {nullptr, nullptr, nullptr}, *dzb = nullptr, *dhb = nullptr;
    float *outf = nullptr, *dout = nullptr, *dh = nullptr, *dzf = nullptr, *loss = nullptr;
    float *part = nullptr;        // split-K partial products (kSplitPartFloats)
};

static void refresh_fragments(sgtp_mlp *M, cudaStream_t s)
{
    frag_kernel<<<128, 256, 0, s>>>(M->w, M->wfrag, M->out);
    count_launch();
}

extern "C" size_t sgtp_mlp_param_count(int32_t T)
{
    if (T < 1 || T > SGTP_MAX_T) return 0;
    return (size_t)layer_off(4, 4 * T);
}

extern "C" sgtp_status sgtp_mlp_create(int32_t T, uint64_t seed, void *stream, sgtp_mlp **out)
{
    SGTP_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    SGTP_CHECK(T >= 1 && T <= SGTP_MAX_T, "T out of range");
    sgtp_mlp *M = new sgtp_mlp();
    M->T = T;
    M->out = 4 * T;
    M->n_params = layer_off(4, M->out);
    cudaError_t e;
    if ((e = dev_malloc(&M->w, 4 * M->n_params)) || (e = dev_malloc(&M->m, 4 * M->n_params)) ||
        (e = dev_malloc(&M->v, 4 * M->n_params)) || (e = dev_malloc(&M->g, 4 * M->n_params)) ||
        (e = dev_malloc(&M->wb, 2 * M->n_params)) || (e = dev_malloc(&M->loss, 4)) ||
        (e = dev_malloc(&M->wfrag, 2 * frag_off(4, M->out)))) {
        sgtp_mlp_destroy(M);
        return set_error(SGTP_E_NOMEM, "MLP allocation failed: %s", cudaGetErrorString(e));
    }
    cudaStream_t s = (cudaStream_t)stream;
    SGTP_CUDA(cudaMemsetAsync(M->m, 0, 4 * M->n_params, s));
    SGTP_CUDA(cudaMemsetAsync(M->v, 0, 4 * M->n_params, s));
    for (int l = 0; l < 4; ++l) {
        init_kernel<<<64, 256, 0, s>>>(M->w, M->wb, layer_off(l, M->out), layer_out(l, M->out), layer_in(l), seed);
        count_launch();
    }
    refresh_fragments(M, s);
    SGTP_CUDA(cudaGetLastError());
    SGTP_CUDA(cudaStreamSynchronize(s));
    *out = M;
    return SGTP_OK;
}

static void free_scratch(sgtp_mlp *M)
{
    cudaFree(M->xb); cudaFree(M->h[0]); cudaFree(M->h[1]); cudaFree(M->h[2]); cudaFree(M->dzb); cudaFree(M->dhb);
    cudaFree(M->outf); cudaFree(M->dout); cudaFree(M->dh); cudaFree(M->dzf); cudaFree(M->part);
    M->xb = M->dzb = M->dhb = nullptr;
    M->h[0] = M->h[1] = M->h[2] = nullptr;
    M->outf = M->dout = M->dh = M->dzf = M->part = nullptr;
    M->cap = 0;
}

extern "C" void sgtp_mlp_destroy(sgtp_mlp *M)
{
    if (!M) return;
    free_scratch(M);
    cudaFree(M->w); cudaFree(M->m); cudaFree(M->v); cudaFree(M->g); cudaFree(M->wb); cudaFree(M->loss);
    cudaFree(M->wfrag);
    delete M;
}

extern "C" sgtp_status sgtp_mlp_reserve(sgtp_mlp *M, int32_t batch)
{
    SGTP_CHECK(M != nullptr, "mlp is NULL");
    SGTP_CHECK(batch >= 1 && batch <= (1 << 20), "batch out of range");
    if (batch <= M->cap) return SGTP_OK;
    free_scratch(M);
    const size_t B = (size_t)batch, W = (size_t)(M->out > kHid ? M->out : kHid);
    cudaError_t e;
    if ((e = dev_malloc(&M->xb, 2 * B * kIn)) || (e = dev_malloc(&M->h[0], 2 * B * kHid)) ||
        (e = dev_malloc(&M->h[1], 2 * B * kHid)) || (e = dev_malloc(&M->h[2], 2 * B * kHid)) ||
        (e = dev_malloc(&M->dzb, 2 * B * W)) || (e = dev_malloc(&M->dhb, 2 * B * W)) ||
        (e = dev_malloc(&M->outf, 4 * B * M->out)) || (e = dev_malloc(&M->dout, 4 * B * M->out)) ||
        (e = dev_malloc(&M->dh, 4 * B * W)) || (e = dev_malloc(&M->dzf, 4 * B * W)) ||
        (e = dev_malloc(&M->part, 4 * kSplitPartFloats))) {
        free_scratch(M);
        return set_error(SGTP_E_NOMEM, "MLP scratch allocation failed: %s", cudaGetErrorString(e));
    }
    M->cap = batch;
    return SGTP_OK;
}

static sgtp_status forward_impl(sgtp_mlp *M, const float *x, int B, cudaStream_t s)
{
    f32_to_bf16_kernel<<<(B * kIn + 255) / 256, 256, 0, s>>>(x, M->xb, (long long)B * kIn);
    count_launch();
    const bf16 *in = M->xb;
    for (int l = 0; l < 3; ++l) {
        const long long o = layer_off(l, M->out);
        gemm<false, true, EPI_BIAS_RELU_BF16>(in, M->wb + o, M->h[l], M->w + o + (long long)kHid * layer_in(l), B,
                                               kHid, layer_in(l), layer_in(l), layer_in(l), kHid, s);
        in = M->h[l];
    }
    const long long o3 = layer_off(3, M->out);
    // the output bias is read from the FP32 master copy (as for the hidden layers)
    gemm<false, true, EPI_BIAS_F32>(in, M->wb + o3, M->outf, M->w + o3 + (long long)M->out * kHid, B, M->out, kHid,
                                    kHid, kHid, M->out, s);
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_mlp_forward(sgtp_mlp *M, const float *x, int32_t batch, float *out, void *stream)
{
    SGTP_CHECK(M && x && out, "NULL argument");
    sgtp_status st = sgtp_mlp_reserve(M, batch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    forward_impl(M, x, batch, s);
    SGTP_CUDA(cudaMemcpyAsync(out, M->outf, 4 * (size_t)batch * M->out, cudaMemcpyDeviceToDevice, s));
    SGTP_CUDA(cudaGetLastError());
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_mlp_proposal(sgtp_mlp *M, const float *x, const float *u_nom, int32_t batch,
                                         float sigma_a, float sigma_delta, float *prop, void *stream)
{
    SGTP_CHECK(M && x && prop, "NULL argument");
    SGTP_CHECK(sigma_a > 0.f && sigma_delta > 0.f, "sigmas must be positive");
    sgtp_status st = sgtp_mlp_reserve(M, batch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    forward_impl(M, x, batch, s);
    const int n = batch * M->T;
    proposal_kernel<<<(n + 255) / 256, 256, 0, s>>>(M->outf, u_nom, batch, M->T, sigma_a, sigma_delta,
                                                    (float4 *)prop);
    count_launch();
    SGTP_CUDA(cudaGetLastError());
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_mlp_train_step(sgtp_mlp *M, const float *x, const float *target, int32_t batch, float lr,
                                           float *loss_out, float *grad_out, int32_t apply, void *stream)
{
    SGTP_CHECK(M && x && target, "NULL argument");
    sgtp_status st = sgtp_mlp_reserve(M, batch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int B = batch, OUT = M->out;
    forward_impl(M, x, B, s);
    SGTP_CUDA(cudaMemsetAsync(M->loss, 0, 4, s));
    nll_kernel<<<(B * 2 * M->T + 255) / 256, 256, 0, s>>>(M->outf, target, B, M->T, M->dout, M->loss);
    count_launch();
    // output layer: dW3 = dOut^T H2, db3 = colsum(dOut), dH2 = dOut W3
    f32_to_bf16_kernel<<<(B * OUT + 255) / 256, 256, 0, s>>>(M->dout, M->dzb, (long long)B * OUT);
    count_launch();
    const float *dzf = M->dout;
    int N = OUT;
    for (int l = 3; l >= 0; --l) {
        const long long o = layer_off(l, OUT);
        const int in = layer_in(l);
        const bf16 *act_in = l == 0 ? M->xb : M->h[l - 1];
        // dW_l [N x in] = dZ^T [N x B] * act_in [B x in] (K = B: split)
        gemm_splitk<true, false>(M->dzb, act_in, M->g + o, M->part, N, in, B, N, in, s);
        colsum_kernel<<<(N + 31) / 32, 1024, 0, s>>>(dzf, B, N, M->g + o + (long long)N * in);
        count_launch();
        if (l == 0) break;
        // dH_{l-1} [B x in] = dZ [B x N] * W_l [N x in]
        gemm<false, false, EPI_F32>(M->dzb, M->wb + o, M->dh, nullptr, B, in, N, N, in, in, s);
        relu_back_kernel<<<(B * in + 255) / 256, 256, 0, s>>>(M->dh, M->h[l - 1], (long long)B * in, M->dhb, M->dzf);
        count_launch();
        // swap: the new dZ (BF16 and FP32)
        bf16 *tb = M->dzb; M->dzb = M->dhb; M->dhb = tb;
        dzf = M->dzf;
        N = in;
    }
    if (grad_out) SGTP_CUDA(cudaMemcpyAsync(grad_out, M->g, 4 * M->n_params, cudaMemcpyDeviceToDevice, s));
    if (loss_out) SGTP_CUDA(cudaMemcpyAsync(loss_out, M->loss, 4, cudaMemcpyDeviceToDevice, s));
    if (apply) {
        M->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
        adam_kernel<<<256, 256, 0, s>>>(M->w, M->g, M->m, M->v, M->wb, M->n_params, lr, b1, b2, 1e-8f, c1, c2);
        count_launch();
        refresh_fragments(M, s);
    }
    SGTP_CUDA(cudaGetLastError());
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_mlp_get_params(const sgtp_mlp *M, float *host_out)
{
    SGTP_CHECK(M && host_out, "NULL argument");
    SGTP_CUDA(cudaMemcpy(host_out, M->w, 4 * M->n_params, cudaMemcpyDeviceToHost));
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_mlp_set_params(sgtp_mlp *M, const float *host_in)
{
    SGTP_CHECK(M && host_in, "NULL argument");
    SGTP_CUDA(cudaMemcpy(M->w, host_in, 4 * M->n_params, cudaMemcpyHostToDevice));
    f32_to_bf16_kernel<<<256, 256>>>(M->w, M->wb, M->n_params);
    count_launch();
    refresh_fragments(M, 0);
    SGTP_CUDA(cudaDeviceSynchronize());
    return SGTP_OK;
}

extern "C" sgtp_status sgtp_mlp_info(const sgtp_mlp *M, int32_t *T, int64_t *n_params, int64_t *step,
                                     const void **bf16_params)
{
    SGTP_CHECK(M != nullptr, "mlp is NULL");
    if (T) *T = M->T;
    if (n_params) *n_params = M->n_params;
    if (step) *step = M->step;
    if (bf16_params) *bf16_params = M->wb;
    return SGTP_OK;
}

// FP32 master parameters and the fragment-ordered BF16 weights on the
// device (library-internal accessors).
const float *sgtp_mlp_master(const sgtp_mlp *M) { return M ? M->w : nullptr; }
const __nv_bfloat16 *sgtp_mlp_fragments(const sgtp_mlp *M) { return M ? M->wfrag : nullptr; }
