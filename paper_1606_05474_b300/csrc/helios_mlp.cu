// Learned initialiser: a small multilayer perceptron trained on the solver's own
// radiative-equilibrium solutions (the paper starts the iteration from an arbitrary
// profile, Sect. 2.2.3; a better start saves iterations).
//
// Layers: n_in -> hidden x n_hidden_layers (SiLU) -> n_out (linear).  Parameters are
// FP32 master copies; every matrix product rounds both operands to BF16 and accumulates in
// FP32 on the 5th-generation tensor cores (tcgen05.mma, accumulator in tensor memory).  The
// weights are also kept as BF16, laid out tile by tile as the tensor cores read them from shared
// memory, in both orientations (forward and backward products); those copies are made once from
// the parameters, updated in place by every Adam step, and reach shared memory by one bulk
// asynchronous copy per tile.
// Training minimises the mean squared error with Adam.  All reductions have a fixed order
// (deterministic).
#include "helios.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

// a named range on a profiler's timeline around each call of the boundary (nothing is recorded
// when no tool is attached)
namespace {
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
};
}  // namespace

__attribute__((visibility("hidden"))) void helios_set_error_text(const char* msg);
__attribute__((visibility("hidden"))) int helios_ctx_device(const helios_ctx* ctx);
__attribute__((visibility("hidden"))) const int2* helios_plan_layers_dev(const helios_plan* p, int* A);

namespace {

int mfail(int code, const char* fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    helios_set_error_text(msg);
    return code;
}

#define MLP_CUDA(call)                                                                                \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return mfail(HELIOS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

constexpr int kMaxLayers = 8;
enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_SILU = 2, EPI_DSILU = 3 };

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// ---------------------------------------------------------------------------------------------
// C[M x N] = op(A)[M x K] op(B)[K x N] on the 5th-generation tensor cores (tcgen05), both operands
// rounded to BF16, FP32 accumulation in tensor memory, epilogue fused.
// op(A)[m][k] = TA ? A[k*lda + m] : A[m*lda + k];  op(B)[k][n] = TB ? B[n*ldb + k] : B[k*ldb + n].
// One CTA of 4 warps per 128 x 64 tile of C.  Per K step of 64 the CTA stages both operands as
// BF16 into shared memory in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices: element (r, k) of an R-row tile at ((k/8)(R/8) + r/8) 128 + (r%8) 16 + (k%8) 2 bytes,
// so the byte stride between core matrices along K is 16 R and along the rows 128), one thread
// issues four 128 x 64 x 16 MMAs reading both operands through shared-memory descriptors and
// accumulating into 64 tensor-memory columns, and commits them to an mbarrier.  The tiles are
// double-buffered: the next K step is staged while the MMAs of this one run, and a buffer is
// overwritten only after the MMAs that read it have completed.  Staging issues all of a thread's
// global loads (float4 along the contiguous dimension where the rows are 16-byte aligned) before
// converting and storing any, so their latencies overlap.  With BT the B operand is a weight
// matrix already held as BF16 tiles in that layout (64 x 64, 8 KB each, [n tile][K step]): one
// thread copies a K step's tile with one bulk asynchronous copy (cp.async.bulk, completion
// counted in bytes on a per-buffer mbarrier) and waits for it before issuing the MMAs that read it.
// The epilogue reads the accumulator back
// with tcgen05.ld (warp w holds rows 32w .. 32w+31, a thread one row) and applies the bias / SiLU /
// SiLU-derivative.  Every wait on the mbarrier is bounded: on expiry the kernel records an error
// in *err, stops issuing, waits (bounded again) for what it issued, releases its tensor memory and
// returns.
constexpr int UM_BM = 128, UM_BN = 64, UM_BK = 64;
constexpr uint32_t UM_ABYTES = UM_BM * UM_BK * 2, UM_BBYTES = UM_BN * UM_BK * 2;
constexpr uint32_t UM_STAGE = UM_ABYTES + UM_BBYTES;                 // one buffer: A then B
constexpr uint32_t UM_BAR = 2 * UM_STAGE, UM_SLOT = UM_BAR + 8;   // MMA-commit mbarrier, TMEM address
constexpr uint32_t UM_LDBAR = UM_BAR + 16;                          // two bulk-copy mbarriers (BT)
constexpr size_t UM_SMEM = 72 * 1024;        // 48 KB of tiles, padded so that at most 3 CTAs share an SM
constexpr uint32_t UM_COLS = 64;             // FP32 accumulator columns (a power of two >= 32)
constexpr long UM_WAIT_LIMIT = 1L << 22;     // mbarrier polls before the kernel gives up
// instruction descriptor (kind::f16): F32 accumulator (bits 4-5 = 1), A and B BF16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t UM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UM_BN >> 3) << 17) |
                              ((uint32_t)(UM_BM >> 4) << 24);

template <int R>
__device__ __forceinline__ uint32_t um_core_off(int r, int k)
{
    return (uint32_t)((((k >> 3) * (R / 8) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// shared-memory matrix descriptor: start address, leading-dimension (K) byte offset, stride (row
// group) byte offset, all in 16-byte units; descriptor version 1 at bit 46; no swizzle
__device__ __forceinline__ uint64_t um_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool um_wait(uint32_t bar, uint32_t phase)
{
    for (long it = 0; it < UM_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Stage rows r0 .. r0+R-1 and k0 .. k0+63 of an operand as BF16 into dst (K-major core layout).
// KC: element (r, k) at X[r*ld + k] (contiguous in k); otherwise at X[k*ld + r] (contiguous in r).
// Outside rows x K: zero.  vec: 16-byte aligned rows (float4 loads along the contiguous dimension).
template <int R, bool KC>
__device__ __forceinline__ void um_stage(unsigned char* dst, const float* __restrict__ X, int ld, int r0, int rows,
                                         int k0, int K, int tid, bool vec)
{
    constexpr int NV = R * UM_BK / 4 / 128;              // float4 groups per thread
    float v[NV][4];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e = tid + 128 * i;
        int r, c;                                        // the group's first (row, k)
        if (KC) { r = e / (UM_BK / 4); c = (e % (UM_BK / 4)) * 4; } else { c = e / (R / 4); r = (e % (R / 4)) * 4; }
        const int gr = r0 + r, gk = k0 + c;
        if (vec && (KC ? (gr < rows && gk + 3 < K) : (gk < K && gr + 3 < rows))) {
            const float4 q = *reinterpret_cast<const float4*>(KC ? X + (size_t)gr * ld + gk : X + (size_t)gk * ld + gr);
            v[i][0] = q.x; v[i][1] = q.y; v[i][2] = q.z; v[i][3] = q.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int rr = KC ? gr : gr + j, kk = KC ? gk + j : gk;
                v[i][j] = (rr < rows && kk < K) ? X[KC ? (size_t)rr * ld + kk : (size_t)kk * ld + rr] : 0.0f;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int e = tid + 128 * i;
        int r, c;
        if (KC) { r = e / (UM_BK / 4); c = (e % (UM_BK / 4)) * 4; } else { c = e / (R / 4); r = (e % (R / 4)) * 4; }
        if (KC) {        // four consecutive k of one row: 8 contiguous bytes of a core-matrix row
            __nv_bfloat162 lo = __floats2bfloat162_rn(v[i][0], v[i][1]), hi = __floats2bfloat162_rn(v[i][2], v[i][3]);
            uint2 w;
            w.x = *reinterpret_cast<uint32_t*>(&lo);
            w.y = *reinterpret_cast<uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(dst + um_core_off<R>(r, c)) = w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                *reinterpret_cast<__nv_bfloat16*>(dst + um_core_off<R>(r + j, c)) = __float2bfloat16_rn(v[i][j]);
        }
    }
}

// thread 0: the BF16 tile of K step st of the pre-tiled B operand into the B half of buffer `buf`
__device__ __forceinline__ void um_bulk_b(uint32_t s0, uint32_t buf, const __nv_bfloat16* Bt, int steps, int st)
{
    const uint32_t ldbar = s0 + UM_LDBAR + 8u * (uint32_t)(st & 1);
    const __nv_bfloat16* src = Bt + ((size_t)blockIdx.x * steps + st) * (UM_BN * UM_BK);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ldbar), "r"(UM_BBYTES) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s0 + buf + UM_ABYTES),
                 "l"(src), "r"(UM_BBYTES), "r"(ldbar)
                 : "memory");
}

template <bool TA, bool TB, int EPI, bool BT>
__global__ void __launch_bounds__(128, 1) mlp_umma(int M, int N, int K, const float* __restrict__ A, int lda,
                                                   const float* __restrict__ B, int ldb,
                                                   const __nv_bfloat16* __restrict__ Bt, float* __restrict__ C, int ldc,
                                                   const float* __restrict__ bias, float* __restrict__ Zout,
                                                   const float* __restrict__ Zin, int ldz, float scale, int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * UM_BM, n0 = blockIdx.x * UM_BN;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(sm);
    const uint32_t bar = s0 + UM_BAR;
    const bool va = (lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    const bool vb = (ldb & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s0 + UM_SLOT),
                     "r"(UM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const int steps = (K + UM_BK - 1) / UM_BK;
    int ld_issued = 0, ld_done = 0;          // thread 0: bulk copies issued / waited for (in order)
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        if (BT) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s0 + UM_LDBAR), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s0 + UM_LDBAR + 8), "r"(1) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (BT) {
            um_bulk_b(s0, 0, Bt, steps, 0);
            ld_issued = 1;
        }
    }
    // the first K step's tiles into buffer 0
    um_stage<UM_BM, !TA>(sm, A, lda, m0, M, 0, K, tid, va);
    if (!BT) um_stage<UM_BN, TB>(sm + UM_ABYTES, B, ldb, n0, N, 0, K, tid, vb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");      // visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(sm + UM_SLOT);
    bool ok = true;
    uint32_t gave_up = 0;                    // the parity of the commit a failed wait gave up on
    for (int st = 0; st < steps && ok; ++st) {
        const uint32_t buf = (uint32_t)(st & 1) * UM_STAGE;
        bool lok = true;                     // thread 0: this step's B tile has arrived
        if (tid == 0 && BT) {
            lok = um_wait(s0 + UM_LDBAR + 8u * (uint32_t)(st & 1), (uint32_t)((st >> 1) & 1));
            if (lok) ld_done = st + 1;
        }
        if (tid == 0 && !lok) {
            // no MMAs: complete the commit barrier's phase by hand so that no thread waits for it
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
        } else if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < UM_BK / 16; ++kk) {
                const uint64_t da = um_desc(s0 + buf + kk * 2 * (16 * UM_BM), 16 * UM_BM, 128);
                const uint64_t db = um_desc(s0 + buf + UM_ABYTES + kk * 2 * (16 * UM_BN), 16 * UM_BN, 128);
                const uint32_t acc = (st > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(UM_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        // the next K step into the other buffer while these MMAs run (its MMAs completed last step)
        if (st + 1 < steps) {
            const uint32_t nb = (uint32_t)((st + 1) & 1) * UM_STAGE;
            if (BT && tid == 0 && lok) {
                um_bulk_b(s0, nb, Bt, steps, st + 1);
                ld_issued = st + 2;
            }
            um_stage<UM_BM, !TA>(sm + nb, A, lda, m0, M, (st + 1) * UM_BK, K, tid, va);
            if (!BT) um_stage<UM_BN, TB>(sm + nb + UM_ABYTES, B, ldb, n0, N, (st + 1) * UM_BK, K, tid, vb);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        ok = __syncthreads_and((um_wait(bar, (uint32_t)(st & 1)) && lok) ? 1 : 0) != 0;   // one decision for the CTA
        if (!ok) gave_up = (uint32_t)(st & 1);
        if (!ok && tid == 0) atomicExch(err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok) {
        // ---- epilogue: row m0 + 32 warp + lane, 8 accumulator columns at a time
        const int m = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < UM_BN && n0 + c0 < N; c0 += 8) {
            uint32_t r[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = n0 + c0 + j;
                if (n >= N) break;
                const float v = __uint_as_float(r[j]);
                float out;
                if (EPI == EPI_STORE) {
                    out = scale * v;
                } else if (EPI == EPI_BIAS) {
                    out = v + bias[n];
                } else if (EPI == EPI_BIAS_SILU) {
                    const float z = v + bias[n];
                    Zout[(size_t)m * ldz + n] = z;
                    out = z * sigmoidf_(z);
                } else {
                    const float z = Zin[(size_t)m * ldz + n], sg = sigmoidf_(z);
                    out = v * sg * fmaf(z, 1.0f - sg, 1.0f);      // d SiLU / dz
                }
                C[(size_t)m * ldc + n] = out;
            }
        }
    } else {
        // the commit the wait gave up on (bounded again): its MMAs may still read the tiles
        um_wait(bar, gave_up);
        // and the bulk copies still in flight into the tiles (bounded again)
        if (BT && tid == 0)
            for (int j = ld_done; j < ld_issued; ++j) um_wait(s0 + UM_LDBAR + 8u * (uint32_t)(j & 1), (uint32_t)((j >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UM_COLS) : "memory");
}

// BF16 tiles of a weight matrix as the B operand op(B)[k][n] = trans ? W[n ld + k] : W[k ld + n]
// (K x N): tile (n tile t, K step j) at dst + (t ks + j) 4096, element (r, c) of a tile at the
// K-major core offset of (r, c); zero outside K x N.  One thread per tile element.
__global__ void retile_kernel(const float* __restrict__ W, int ld, int K, int N, int trans, int ks,
                              __nv_bfloat16* __restrict__ dst, long long total)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const long long tile = e / (UM_BN * UM_BK);
    const int w = (int)(e - tile * (UM_BN * UM_BK));
    const int r = w / UM_BK, c = w % UM_BK;                      // row (n) and column (k) in the tile
    const int n = (int)(tile / ks) * UM_BN + r, k = (int)(tile % ks) * UM_BK + c;
    const float v = (n < N && k < K) ? W[trans ? (size_t)n * ld + k : (size_t)k * ld + n] : 0.0f;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(dst + tile * (UM_BN * UM_BK)) +
                                      um_core_off<UM_BN>(r, c)) = __float2bfloat16_rn(v);
}

// dOut = 2 (Y - T) / (B * N); per-block partial sums of the squared error (fixed order)
__global__ void mse_kernel(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                           long long count, float scale, double* __restrict__ part)
{
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.0f * scale * d;
        s += (double)d * (double)d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void loss_kernel(const double* __restrict__ part, int n, double scale, float* __restrict__ loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *loss = (float)(s * scale);
    }
}

// db[n] = sum_m dZ[m][n] (thread per column, fixed order)
__global__ void colsum_kernel(const float* __restrict__ dZ, int M, int N, float* __restrict__ db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int m = 0; m < M; ++m) s += dZ[(size_t)m * N + n];
    db[n] = s;
}

// where the weights of each layer sit in the parameters and in the BF16 tiles
struct TileMap {
    int nl;
    int in[kMaxLayers], out[kMaxLayers];
    long long woff[kMaxLayers], wtf[kMaxLayers], wtb[kMaxLayers];
};

// one Adam step; a weight's new value also goes, as BF16, into its places in the forward tiles
// (row n, column k of op(B) = W) and, beyond the first layer, the backward tiles (row k, column n
// of op(B) = W^T), so the tiles stay current without a separate pass
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2, TileMap tm, __nv_bfloat16* __restrict__ wt)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pn = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pn;
        int l = tm.nl - 1;
        while (l > 0 && i < tm.woff[l]) --l;
        const long long e = i - tm.woff[l];
        const int in = tm.in[l], out = tm.out[l];
        if (e >= (long long)in * out) continue;                  // a bias
        const int k = (int)(e / out), c = (int)(e - (long long)k * out);
        const __nv_bfloat16 h = __float2bfloat16_rn(pn);
        const int ksf = (in + UM_BK - 1) / UM_BK;
        unsigned char* f = reinterpret_cast<unsigned char*>(wt + tm.wtf[l] + ((long long)(c / UM_BN) * ksf + k / UM_BK) * (UM_BN * UM_BK));
        *reinterpret_cast<__nv_bfloat16*>(f + um_core_off<UM_BN>(c % UM_BN, k % UM_BK)) = h;
        if (l > 0) {
            const int ksb = (out + UM_BK - 1) / UM_BK;
            unsigned char* b = reinterpret_cast<unsigned char*>(wt + tm.wtb[l] + ((long long)(k / UM_BN) * ksb + c / UM_BK) * (UM_BN * UM_BK));
            *reinterpret_cast<__nv_bfloat16*>(b + um_core_off<UM_BN>(k % UM_BN, c % UM_BK)) = h;
        }
    }
}

uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

// standardised features: xs[b][j] = (f[b][j] - mu[j]) / sd[j] in IEEE float32 (correctly rounded)
__global__ void standardize_kernel(const float* __restrict__ f, const float* __restrict__ mu, const float* __restrict__ sd,
                                   float* __restrict__ xs, int B, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * n) {
        const int j = i % n;
        xs[i] = __fdiv_rn(__fsub_rn(f[i], mu[j]), sd[j]);
    }
}

// column j = blockIdx.x of x [B][n]: mean and standard deviation (population) in double, fixed-order
// sums (thread-strided partials, then a fixed tree over the block), sd + eps stored
__global__ void column_stats_kernel(const float* __restrict__ x, int B, int n, double eps, float* __restrict__ mu,
                                    float* __restrict__ sd)
{
    __shared__ double red[256];
    const int j = blockIdx.x, t = threadIdx.x;
    double s = 0.0;
    for (int b = t; b < B; b += 256) s += (double)x[(size_t)b * n + j];
    red[t] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    const double m = red[0] / (double)B;
    __syncthreads();
    double q = 0.0;
    for (int b = t; b < B; b += 256) {
        const double d = (double)x[(size_t)b * n + j] - m;
        q += d * d;
    }
    red[t] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) {
        mu[j] = (float)m;
        sd[j] = (float)(sqrt(red[0] / (double)B) + eps);
    }
}

// one block per atmosphere a0 + blockIdx.x: the network's n_out standardised temperatures at the
// evenly spaced normalised log-P positions s_k = k/(n_out - 1) (bottom first), de-standardised and
// interpolated linearly to the atmosphere's n layer centres (evenly spaced in log P: s_i = i/(n-1));
// a profile with a non-finite temperature or one outside (T_min, T_max) takes the fallback
__global__ void profile_kernel(const int2* __restrict__ lay, int a0, const float* __restrict__ y, int n_out,
                               const float* __restrict__ y_mu, const float* __restrict__ y_sd,
                               const double* __restrict__ T_fb, double T_min, double T_max, double* __restrict__ T_out,
                               int32_t* __restrict__ used)
{
    __shared__ int s_bad;
    const int a = a0 + blockIdx.x;
    const int2 nl = lay[a];
    const int n = nl.x, off = nl.y;
    const float* yr = y + (size_t)blockIdx.x * n_out;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double pos = n > 1 ? (double)i * (double)(n_out - 1) / (double)(n - 1) : 0.0;
        const int k = min((int)floor(pos), n_out - 2);
        const double w = pos - (double)k;
        const double t0 = (double)yr[k] * (double)y_sd[k] + (double)y_mu[k];
        const double t1 = (double)yr[k + 1] * (double)y_sd[k + 1] + (double)y_mu[k + 1];
        const double T = t0 + w * (t1 - t0);
        if (!(T > T_min && T < T_max)) atomicOr(&s_bad, 1);      // also catches NaN
        T_out[off + i] = T;
    }
    __syncthreads();
    const int bad = s_bad;
    if (bad)
        for (int i = threadIdx.x; i < n; i += blockDim.x) T_out[off + i] = T_fb[off + i];
    if (threadIdx.x == 0 && used) used[a] = bad ? 0 : 1;
}

struct helios_mlp {
    helios_ctx* ctx;
    int device;
    int nl;                  // linear layers
    int dims[kMaxLayers + 1];
    int64_t woff[kMaxLayers], boff[kMaxLayers], n_params;
    int max_B;
    float *p, *g, *m, *v;
    __nv_bfloat16* wt;       // BF16 weight tiles: forward orientation, then backward (layers >= 1)
    int64_t wtf[kMaxLayers], wtb[kMaxLayers];   // element offsets of each layer's tiles
    bool wt_stale;           // the FP32 parameters changed since the tiles were made
    float* act;              // per layer: Z (hidden layers) and Y, max_B rows
    float *dA, *dB;          // backprop ping-pong buffers
    float* dout;
    float *xin, *yout;       // initial profiles: standardised features and network outputs, max_B rows
    int* err;                // set by a GEMM whose tensor-core wait gave up
    double* part;
    int64_t t;               // Adam step count
    std::vector<void*> allocs;
};

extern "C" {

int helios_mlp_create(helios_ctx* ctx, int n_in, int n_hidden, int hidden_layers, int n_out,
                      unsigned long long seed, int max_batch, helios_mlp** out)
{
    if (!out || !ctx) return mfail(HELIOS_EINVAL, "helios_mlp_create: null argument");
    *out = nullptr;
    const int device = helios_ctx_device(ctx);
    if (n_in < 1 || n_hidden < 1 || n_out < 1 || hidden_layers < 1 || hidden_layers + 1 > kMaxLayers || max_batch < 1)
        return mfail(HELIOS_EINVAL, "helios_mlp_create: invalid shape");
    MLP_CUDA(cudaSetDevice(device));
    helios_mlp* m = new helios_mlp();
    m->ctx = ctx;
    m->device = device;
    m->nl = hidden_layers + 1;
    m->dims[0] = n_in;
    for (int i = 1; i <= hidden_layers; ++i) m->dims[i] = n_hidden;
    m->dims[m->nl] = n_out;
    int64_t off = 0;
    for (int l = 0; l < m->nl; ++l) {
        m->woff[l] = off;
        off += (int64_t)m->dims[l] * m->dims[l + 1];
        m->boff[l] = off;
        off += m->dims[l + 1];
    }
    m->n_params = off;
    m->max_B = max_batch;
    // initial weights: uniform in +-1/sqrt(fan_in) from a counter-based generator
    std::vector<float> h(off);
    const uint64_t key = mix64(seed ^ 0x6d6c7000ULL);
    for (int l = 0; l < m->nl; ++l) {
        const double bound = 1.0 / std::sqrt((double)m->dims[l]);
        for (int64_t i = m->woff[l]; i < m->boff[l] + m->dims[l + 1]; ++i) {
            const double u = (double)(mix64(key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL) >> 11) * 0x1.0p-53;
            h[i] = (float)((2.0 * u - 1.0) * bound);
        }
    }
    // BF16 weight tiles: forward (op(B) = W_l, K = in, N = out) and, for layers >= 1, backward
    // (op(B) = W_l^T, K = out, N = in)
    int64_t wt_elems = 0;
    auto ntiles = [](int K, int N) { return (int64_t)((N + UM_BN - 1) / UM_BN) * ((K + UM_BK - 1) / UM_BK); };
    for (int l = 0; l < m->nl; ++l) {
        m->wtf[l] = wt_elems;
        wt_elems += ntiles(m->dims[l], m->dims[l + 1]) * UM_BN * UM_BK;
    }
    for (int l = 0; l < m->nl; ++l) {
        m->wtb[l] = wt_elems;
        if (l > 0) wt_elems += ntiles(m->dims[l + 1], m->dims[l]) * UM_BN * UM_BK;
    }
    size_t act_floats = 0;
    for (int l = 0; l < m->nl; ++l) act_floats += (size_t)2 * max_batch * m->dims[l + 1];
    int widest = 0;
    for (int l = 0; l <= m->nl; ++l) widest = std::max(widest, m->dims[l]);
    float** bufs[] = {&m->p, &m->g, &m->m, &m->v};
    for (float** b : bufs) {
        if (cudaMalloc((void**)b, sizeof(float) * off) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp params"); }
        m->allocs.push_back(*b);
    }
    if (cudaMalloc((void**)&m->wt, sizeof(__nv_bfloat16) * wt_elems) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp weight tiles"); }
    m->allocs.push_back(m->wt);
    m->wt_stale = true;
    if (cudaMalloc((void**)&m->act, sizeof(float) * act_floats) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp activations"); }
    m->allocs.push_back(m->act);
    const size_t wide = (size_t)max_batch * widest;
    if (cudaMalloc((void**)&m->dA, sizeof(float) * wide) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp grads"); }
    m->allocs.push_back(m->dA);
    if (cudaMalloc((void**)&m->dB, sizeof(float) * wide) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp grads"); }
    m->allocs.push_back(m->dB);
    if (cudaMalloc((void**)&m->dout, sizeof(float) * (size_t)max_batch * n_out) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp out"); }
    m->allocs.push_back(m->dout);
    if (cudaMalloc((void**)&m->part, sizeof(double) * 1024) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp loss"); }
    m->allocs.push_back(m->part);
    if (cudaMalloc((void**)&m->xin, sizeof(float) * (size_t)max_batch * n_in) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp inputs"); }
    m->allocs.push_back(m->xin);
    if (cudaMalloc((void**)&m->yout, sizeof(float) * (size_t)max_batch * n_out) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp outputs"); }
    m->allocs.push_back(m->yout);
    if (cudaMalloc((void**)&m->err, sizeof(int)) != cudaSuccess) { helios_mlp_destroy(m); return mfail(HELIOS_ENOMEM, "mlp flag"); }
    m->allocs.push_back(m->err);
    MLP_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    MLP_CUDA(cudaMemcpy(m->p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice));
    MLP_CUDA(cudaMemset(m->m, 0, sizeof(float) * off));
    MLP_CUDA(cudaMemset(m->v, 0, sizeof(float) * off));
    MLP_CUDA(cudaMemset(m->g, 0, sizeof(float) * off));
    m->t = 0;
    *out = m;
    return HELIOS_OK;
}

int helios_mlp_destroy(helios_mlp* m)
{
    if (!m) return HELIOS_OK;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    for (void* a : m->allocs) cudaFree(a);
    delete m;
    return HELIOS_OK;
}

int helios_mlp_error(helios_mlp* m, int* flag)
{
    if (!m || !flag) return mfail(HELIOS_EINVAL, "helios_mlp_error: null argument");
    MLP_CUDA(cudaSetDevice(m->device));
    MLP_CUDA(cudaMemcpy(flag, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    return HELIOS_OK;
}

int helios_mlp_params(helios_mlp* m, float** params, float** grads, long long* count)
{
    if (!m || !params || !count) return mfail(HELIOS_EINVAL, "helios_mlp_params: null argument");
    *params = m->p;
    if (grads) *grads = m->g;
    *count = m->n_params;
    return HELIOS_OK;
}

int helios_mlp_params_changed(helios_mlp* m)
{
    if (!m) return mfail(HELIOS_EINVAL, "helios_mlp_params_changed: null argument");
    m->wt_stale = true;
    return HELIOS_OK;
}

}  // extern "C"

namespace {

float* Zbuf(helios_mlp* m, int l) { size_t o = 0; for (int k = 0; k < l; ++k) o += (size_t)2 * m->max_B * m->dims[k + 1]; return m->act + o; }
float* Ybuf(helios_mlp* m, int l) { return Zbuf(m, l) + (size_t)m->max_B * m->dims[l + 1]; }

// Bt: the B operand as BF16 tiles (B then unused); null: B staged from FP32
template <bool TA, bool TB, int EPI, bool BT = false>
int gemm(helios_mlp* m, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
         const float* bias, float* Zout, const float* Zin, int ldz, float scale, cudaStream_t s,
         const __nv_bfloat16* Bt = nullptr)
{
    static thread_local int configured[64] = {};          // per device: the dynamic shared-memory limit set
    if (m->device < 0 || m->device >= 64) return mfail(HELIOS_EINVAL, "device %d", m->device);
    if (!configured[m->device]) {
        MLP_CUDA(cudaFuncSetAttribute(mlp_umma<TA, TB, EPI, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)UM_SMEM));
        // shared memory for one CTA per SM, the rest of the SM's 256 KB stays L1: the grids here are
        // a few to a hundred CTAs, and the epilogue's row-wise stores merge in L1 (with the largest
        // carve-out, which the CUDA driver picks when three CTAs could share an SM, the forward products
        // ran 17% slower)
        MLP_CUDA(cudaFuncSetAttribute(mlp_umma<TA, TB, EPI, BT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)((100 * (UM_SMEM + 1024) + 228 * 1024 - 1) / (228 * 1024))));
        configured[m->device] = 1;
    }
    dim3 grid((N + UM_BN - 1) / UM_BN, (M + UM_BM - 1) / UM_BM);
    mlp_umma<TA, TB, EPI, BT><<<grid, 128, UM_SMEM, s>>>(M, N, K, A, lda, B, ldb, Bt, C, ldc, bias, Zout, Zin, ldz,
                                                          scale, m->err);
    MLP_CUDA(cudaGetLastError());
    return HELIOS_OK;
}

// the BF16 weight tiles of every layer from the FP32 parameters, once after they changed
int refresh_tiles(helios_mlp* m, cudaStream_t s)
{
    if (!m->wt_stale) return HELIOS_OK;
    for (int l = 0; l < m->nl; ++l) {
        const int in = m->dims[l], out = m->dims[l + 1];
        for (int dir = 0; dir < 2; ++dir) {
            if (dir == 1 && l == 0) continue;                  // no input gradient of the first layer
            const int K = dir ? out : in, N = dir ? in : out;
            const int ks = (K + UM_BK - 1) / UM_BK;
            const long long total = (long long)((N + UM_BN - 1) / UM_BN) * ks * UM_BN * UM_BK;
            retile_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m->p + m->woff[l], out, K, N, dir, ks,
                                                                         m->wt + (dir ? m->wtb[l] : m->wtf[l]), total);
            MLP_CUDA(cudaGetLastError());
        }
    }
    m->wt_stale = false;
    return HELIOS_OK;
}

// forward pass; hidden activations kept for the backward pass; output to `y`
int forward(helios_mlp* m, const float* x, float* y, int B, cudaStream_t s)
{
    int rc = refresh_tiles(m, s);
    if (rc) return rc;
    const float* in = x;
    for (int l = 0; l < m->nl; ++l) {
        const int K = m->dims[l], N = m->dims[l + 1];
        const float* b = m->p + m->boff[l];
        const __nv_bfloat16* Wt = m->wt + m->wtf[l];
        if (l + 1 < m->nl)
            rc = gemm<false, false, EPI_BIAS_SILU, true>(m, B, N, K, in, K, nullptr, N, Ybuf(m, l), N, b, Zbuf(m, l),
                                                         nullptr, N, 1.0f, s, Wt);
        else
            rc = gemm<false, false, EPI_BIAS, true>(m, B, N, K, in, K, nullptr, N, y, N, b, nullptr, nullptr, N, 1.0f,
                                                    s, Wt);
        if (rc) return rc;
        in = Ybuf(m, l);
    }
    return HELIOS_OK;
}

// gradients of the mean squared error into m->g; loss (float, device) if requested
int backward(helios_mlp* m, const float* x, const float* target, int B, float* loss, cudaStream_t s)
{
    const int nout = m->dims[m->nl];
    int rc = forward(m, x, m->dout, B, s);
    if (rc) return rc;
    const long long count = (long long)B * nout;
    const int blocks = (int)std::min<long long>(1024, (count + 255) / 256);
    mse_kernel<<<blocks, 256, 0, s>>>(m->dout, target, m->dA, count, 1.0f / (float)count, m->part);
    MLP_CUDA(cudaGetLastError());
    if (loss) {
        loss_kernel<<<1, 32, 0, s>>>(m->part, blocks, 1.0 / (double)count, loss);
        MLP_CUDA(cudaGetLastError());
    }
    float* dcur = m->dA;      // dL/dZ of layer l (for the last layer: dL/dOut)
    float* dnext = m->dB;
    for (int l = m->nl - 1; l >= 0; --l) {
        const int K = m->dims[l], N = m->dims[l + 1];
        const float* inp = l ? Ybuf(m, l - 1) : x;
        // dW_l = in^T dZ_l, db_l = colsum dZ_l
        rc = gemm<true, false, EPI_STORE>(m, K, N, B, inp, K, dcur, N, m->g + m->woff[l], N, nullptr, nullptr, nullptr, 0,
                                          1.0f, s);
        if (rc) return rc;
        colsum_kernel<<<(N + 127) / 128, 128, 0, s>>>(dcur, B, N, m->g + m->boff[l]);
        MLP_CUDA(cudaGetLastError());
        if (l > 0) {
            // dZ_{l-1} = (dZ_l W_l^T) * SiLU'(Z_{l-1})
            rc = gemm<false, true, EPI_DSILU, true>(m, B, K, N, dcur, N, nullptr, N, dnext, K, nullptr, nullptr,
                                                    Zbuf(m, l - 1), K, 1.0f, s, m->wt + m->wtb[l]);
            if (rc) return rc;
            std::swap(dcur, dnext);
        }
    }
    return HELIOS_OK;
}

}  // namespace

extern "C" {

int helios_mlp_forward(helios_mlp* m, const float* x, float* y, int B, cudaStream_t s)
{
    CallRange range_("helios_mlp_forward");
    if (!m || !x || !y) return mfail(HELIOS_EINVAL, "helios_mlp_forward: null argument");
    if (B < 1 || B > m->max_B) return mfail(HELIOS_EINVAL, "helios_mlp_forward: batch %d outside [1, %d]", B, m->max_B);
    MLP_CUDA(cudaSetDevice(m->device));
    return forward(m, x, y, B, s);
}

int helios_mlp_grad(helios_mlp* m, const float* x, const float* target, int B, float* loss, cudaStream_t s)
{
    CallRange range_("helios_mlp_grad");
    if (!m || !x || !target) return mfail(HELIOS_EINVAL, "helios_mlp_grad: null argument");
    if (B < 1 || B > m->max_B) return mfail(HELIOS_EINVAL, "helios_mlp_grad: batch %d outside [1, %d]", B, m->max_B);
    MLP_CUDA(cudaSetDevice(m->device));
    return backward(m, x, target, B, loss, s);
}

int helios_mlp_adam(helios_mlp* m, float lr, float beta1, float beta2, float eps, cudaStream_t s)
{
    CallRange range_("helios_mlp_adam");
    if (!m) return mfail(HELIOS_EINVAL, "helios_mlp_adam: null argument");
    MLP_CUDA(cudaSetDevice(m->device));
    m->t += 1;
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)m->t));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)m->t));
    // tiles made first if the parameters changed since (their zero padding is written only there)
    int rc = refresh_tiles(m, s);
    if (rc) return rc;
    TileMap tm;
    std::memset(&tm, 0, sizeof tm);
    tm.nl = m->nl;
    for (int l = 0; l < m->nl; ++l) {
        tm.in[l] = m->dims[l];
        tm.out[l] = m->dims[l + 1];
        tm.woff[l] = m->woff[l];
        tm.wtf[l] = m->wtf[l];
        tm.wtb[l] = m->wtb[l];
    }
    adam_kernel<<<256, 256, 0, s>>>(m->p, m->g, m->m, m->v, m->n_params, lr, beta1, beta2, eps, c1, c2, tm, m->wt);
    MLP_CUDA(cudaGetLastError());
    return HELIOS_OK;
}

int helios_column_stats(const float* x, int B, int n, double eps, float* mu, float* sd, cudaStream_t s)
{
    if (!x || !mu || !sd) return mfail(HELIOS_EINVAL, "helios_column_stats: null argument");
    if (B < 1 || n < 1) return mfail(HELIOS_EINVAL, "helios_column_stats: %d x %d values", B, n);
    column_stats_kernel<<<n, 256, 0, s>>>(x, B, n, eps, mu, sd);
    MLP_CUDA(cudaGetLastError());
    return HELIOS_OK;
}

int helios_standardize(const float* x, const float* mu, const float* sd, int B, int n, float* xs, cudaStream_t s)
{
    if (!x || !mu || !sd || !xs) return mfail(HELIOS_EINVAL, "helios_standardize: null argument");
    if (B < 0 || n < 1) return mfail(HELIOS_EINVAL, "helios_standardize: %d x %d values", B, n);
    if (B == 0) return HELIOS_OK;
    const long long total = (long long)B * n;
    if (total > (1LL << 31) - 256) return mfail(HELIOS_EINVAL, "helios_standardize: too many values");
    standardize_kernel<<<(int)((total + 255) / 256), 256, 0, s>>>(x, mu, sd, xs, B, n);
    MLP_CUDA(cudaGetLastError());
    return HELIOS_OK;
}

int helios_mlp_initial_profiles(helios_mlp* m, const helios_plan* plan, const float* feats, const float* x_mu,
                                const float* x_sd, const float* y_mu, const float* y_sd, const double* T_fallback,
                                double T_min, double T_max, double* T_layer, int32_t* used, cudaStream_t s)
{
    CallRange range_("helios_mlp_initial_profiles");
    if (!m || !plan || !feats || !x_mu || !x_sd || !y_mu || !y_sd || !T_fallback || !T_layer)
        return mfail(HELIOS_EINVAL, "helios_mlp_initial_profiles: null argument");
    if (m->dims[m->nl] < 2) return mfail(HELIOS_EINVAL, "helios_mlp_initial_profiles: the network has fewer than 2 outputs");
    int A = 0;
    const int2* lay = helios_plan_layers_dev(plan, &A);
    MLP_CUDA(cudaSetDevice(m->device));
    const int n_in = m->dims[0], n_out = m->dims[m->nl];
    for (int a0 = 0; a0 < A; a0 += m->max_B) {
        const int B = std::min(m->max_B, A - a0);
        standardize_kernel<<<(B * n_in + 255) / 256, 256, 0, s>>>(feats + (size_t)a0 * n_in, x_mu, x_sd, m->xin, B, n_in);
        MLP_CUDA(cudaGetLastError());
        const int rc = forward(m, m->xin, m->yout, B, s);
        if (rc) return rc;
        profile_kernel<<<B, 128, 0, s>>>(lay, a0, m->yout, n_out, y_mu, y_sd, T_fallback, T_min, T_max, T_layer, used);
        MLP_CUDA(cudaGetLastError());
    }
    return HELIOS_OK;
}

int helios_mlp_train_step(helios_mlp* m, const float* x, const float* target, int B, float lr, float* loss,
                          cudaStream_t s)
{
    CallRange range_("helios_mlp_train_step");
    int rc = helios_mlp_grad(m, x, target, B, loss, s);
    if (rc) return rc;
    return helios_mlp_adam(m, lr, 0.9f, 0.999f, 1e-8f, s);
}

}  // extern "C"
