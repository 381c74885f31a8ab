// Learned-surrogate kernels (declared in include/ternelbm_sur.h): periodic
// 3x3 convolutions as implicit GEMMs on the BF16 tensor cores with FP32
// accumulation, their input and weight gradients, pooling/upsampling, the
// mass-conserving head with its loss, the field packing between the lattice
// update and the network, and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tel_once.cuh"

#include <cstdint>

#include "ternelbm.h"
#include "ternelbm_sur.h"

namespace {

typedef __nv_bfloat16 bf16;

inline cudaStream_t S(void *s) { return (cudaStream_t)s; }
inline int ok(cudaError_t e) { return e == cudaSuccess ? TEL_OK : TEL_ECUDA; }
inline int launched() { return ok(cudaGetLastError()); }
inline bool chan_ok(int c) { return c == 16 || c == 32 || c == 64 || c == 128; }

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t &r0, uint32_t &r1, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(smem_u32(p)));
}

// D (16x8, FP32) += A (16x16 bf16, row) * B (16x8 bf16, col)
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int TAPS = 9;
__device__ __forceinline__ int tap_dy(int t) { return t / 3 - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }

// ---------------------------------------------------------------------------
// Forward conv: implicit GEMM, CTA tile 128 pixels x COUT, K chunk BK input
// channels of one tap per stage, double-buffered cp.async, 8 warps.
// ---------------------------------------------------------------------------
constexpr int CONV_BM = 128;
constexpr int CONV_THREADS = 256;

template <int COUT, int BK>
struct ConvCfg {
    static constexpr int BN = COUT;
    static constexpr int WN = BN >= 64 ? 2 : 1;        // warps along N
    static constexpr int WM = 8 / WN;                  // warps along M
    static constexpr int WROWS = CONV_BM / WM;         // rows per warp (16 or 32)
    static constexpr int MT = WROWS / 16;              // m16 tiles per warp
    static constexpr int WCOLS = BN / WN;              // columns per warp
    static constexpr int NT = WCOLS / 8;               // n8 tiles per warp
    static constexpr int LDA = BK + 8;                 // padded row (bf16): conflict-free ldmatrix
    static constexpr int LDB = BK + 8;
    static constexpr int A_ELEMS = CONV_BM * LDA;
    static constexpr int B_ELEMS = BN * LDB;
    static constexpr size_t SMEM = sizeof(bf16) * 2 * (A_ELEMS + B_ELEMS);
    static constexpr int A_CHUNKS = CONV_BM * BK / 8;  // 16-byte chunks per stage
    static constexpr int A_PER_T = A_CHUNKS / CONV_THREADS;
    static constexpr int B_CHUNKS = BN * BK / 8;
};

template <int COUT, int BK>
__global__ void __launch_bounds__(CONV_THREADS) conv3x3_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w,
                                                               const float *__restrict__ bias, bf16 *__restrict__ y,
                                                               int H, int W, int CIN, int relu)
{
    typedef ConvCfg<COUT, BK> C;
    static_assert(C::A_PER_T >= 1 && C::A_CHUNKS % CONV_THREADS == 0, "A tile split");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *As = reinterpret_cast<bf16 *>(smem_raw);
    bf16 *Bs = As + 2 * C::A_ELEMS;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp % C::WM, wn = warp / C::WM;
    const long long m0 = (long long)blockIdx.x * CONV_BM;
    const int kchunks = CIN / BK;
    const int stages = TAPS * kchunks;

    // the pixel rows this thread loads (fixed over stages)
    int rb[C::A_PER_T], rh[C::A_PER_T], rw[C::A_PER_T], rq[C::A_PER_T], rr[C::A_PER_T];
#pragma unroll
    for (int j = 0; j < C::A_PER_T; ++j) {
        const int c = tid + j * CONV_THREADS;
        rr[j] = c / (BK / 8);
        rq[j] = c % (BK / 8);
        const long long p = m0 + rr[j];
        rw[j] = (int)(p % W);
        rh[j] = (int)((p / W) % H);
        rb[j] = (int)(p / ((long long)W * H));
    }

    auto load_stage = [&](int s, int buf) {
        const int t = s / kchunks, kc = s % kchunks;
        const int dy = tap_dy(t), dx = tap_dx(t);
        bf16 *a = As + buf * C::A_ELEMS;
#pragma unroll
        for (int j = 0; j < C::A_PER_T; ++j) {
            int hs = rh[j] + dy, ws = rw[j] + dx;
            hs = hs < 0 ? hs + H : (hs >= H ? hs - H : hs);
            ws = ws < 0 ? ws + W : (ws >= W ? ws - W : ws);
            const bf16 *src = x + ((((long long)rb[j] * H + hs) * W + ws) * CIN + kc * BK + rq[j] * 8);
            cp_async16(a + rr[j] * C::LDA + rq[j] * 8, src);
        }
        bf16 *b = Bs + buf * C::B_ELEMS;
        for (int c = tid; c < C::B_CHUNKS; c += CONV_THREADS) {
            const int n = c / (BK / 8), q = c % (BK / 8);
            const bf16 *src = w + (((long long)t * COUT + n) * CIN + kc * BK + q * 8);
            cp_async16(b + n * C::LDB + q * 8, src);
        }
    };

    float acc[C::MT][C::NT][4];
#pragma unroll
    for (int i = 0; i < C::MT; ++i)
#pragma unroll
        for (int j = 0; j < C::NT; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    load_stage(0, 0);
    cp_commit();
    for (int s = 0; s < stages; ++s) {
        if (s + 1 < stages) {
            load_stage(s + 1, (s + 1) & 1);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const bf16 *a = As + (s & 1) * C::A_ELEMS;
        const bf16 *b = Bs + (s & 1) * C::B_ELEMS;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[C::MT][4];
#pragma unroll
            for (int mt = 0; mt < C::MT; ++mt) {
                const int row = wm * C::WROWS + mt * 16 + (lane & 15);
                ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], a + row * C::LDA + kk + (lane >> 4) * 8);
            }
#pragma unroll
            for (int nt = 0; nt < C::NT; nt += 2) {
                uint32_t b0, b1, b2, b3;
                if (nt + 1 < C::NT) {
                    const int n = wn * C::WCOLS + nt * 8 + (lane & 7) + (lane >> 4) * 8;
                    ldsm_x4(b0, b1, b2, b3, b + n * C::LDB + kk + ((lane >> 3) & 1) * 8);
                } else {
                    const int n = wn * C::WCOLS + nt * 8 + (lane & 7);
                    ldsm_x2(b0, b1, b + n * C::LDB + kk + ((lane >> 3) & 1) * 8);
                    b2 = b3 = 0u;
                }
#pragma unroll
                for (int mt = 0; mt < C::MT; ++mt) {
                    mma_bf16(acc[mt][nt], af[mt], b0, b1);
                    if (nt + 1 < C::NT) mma_bf16(acc[mt][nt + 1], af[mt], b2, b3);
                }
            }
        }
        __syncthreads();
    }

    // epilogue: bias, ReLU, bf16 pairs
#pragma unroll
    for (int mt = 0; mt < C::MT; ++mt) {
#pragma unroll
        for (int nt = 0; nt < C::NT; ++nt) {
            const int n = wn * C::WCOLS + nt * 8 + (lane & 3) * 2;
            const float b0 = bias ? bias[n] : 0.f, b1 = bias ? bias[n + 1] : 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long p = m0 + wm * C::WROWS + mt * 16 + (lane >> 2) + h * 8;
                float v0 = acc[mt][nt][2 * h] + b0, v1 = acc[mt][nt][2 * h + 1] + b1;
                if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                *reinterpret_cast<__nv_bfloat162 *>(y + p * COUT + n) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

template <int COUT, int BK>
int launch_conv(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, long long P, int H, int W, int cin,
                int relu, cudaStream_t s)
{
    typedef ConvCfg<COUT, BK> C;
    static tel::DeviceOnce once;  // one attribute call per instantiation and device
    const cudaError_t ea = once.run([] {
        return cudaFuncSetAttribute(conv3x3_kernel<COUT, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (ea != cudaSuccess) return TEL_ECUDA;
    const unsigned grid = (unsigned)(P / CONV_BM);
    conv3x3_kernel<COUT, BK><<<grid, CONV_THREADS, C::SMEM, s>>>(x, w, bias, y, H, W, cin, relu);
    return launched();
}

template <int COUT>
int conv_dispatch_k(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, long long P, int H, int W, int cin,
                    int relu, cudaStream_t s)
{
    switch (cin) {
    case 16: return launch_conv<COUT, 16>(x, w, bias, y, P, H, W, cin, relu, s);
    case 32: return launch_conv<COUT, 32>(x, w, bias, y, P, H, W, cin, relu, s);
    default: return launch_conv<COUT, 64>(x, w, bias, y, P, H, W, cin, relu, s);  // 64, 128
    }
}

// ---------------------------------------------------------------------------
// Forward conv on the 5th-generation tensor cores: tcgen05.mma (kind::f16,
// BF16 operands, FP32 accumulator in tensor memory), one 128-pixel x COUT
// tile per CTA of 4 warps.  Operand tiles are staged in shared memory by
// cp.async in the canonical no-swizzle K-major layout: core matrices of 8
// rows x 16 bytes, the K-adjacent core matrices 128 B apart (leading byte
// offset), the 8-row groups BK*16 B apart (stride byte offset).  One thread
// issues the MMAs of a stage and commits them to an mbarrier; the stage's
// buffer is refilled only after that mbarrier completes.  Every wait is
// bounded: on time-out the kernel records an error and skips its output.
// ---------------------------------------------------------------------------
constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN = 1LL << 26;  // bounded mbarrier wait (iterations)

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version (tcgen05)
    // base offset 0, relative LBO, swizzle mode 0 (none)
    return d;
}

// kind::f16 instruction descriptor: F32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// returns false on time-out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < TC_SPIN; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity));
        if (done) return true;
    }
    return false;
}

template <int COUT>
struct TcCfg {
    static constexpr int BM = 128;
    static constexpr int NS = 5;                 // pipeline stages
    static constexpr int KS = 2;                 // k-steps of 16 per stage (K = 32)
    static constexpr int A_BYTES = BM * KS * 32;
    static constexpr int B_BYTES = COUT * KS * 32;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TMEM_COLS = COUT < 32 ? 32 : COUT;  // power of two >= 32
    // enough shared memory that at most 512 / TMEM_COLS CTAs are resident on
    // an SM (228 KB each), so that their tensor-memory allocations never wait
    static constexpr size_t SMEM_OPS = 1024 + NS * (size_t)STAGE;
    static constexpr size_t SMEM_TMEM = (size_t)233472 * TMEM_COLS / 512 + 1024;
    static constexpr size_t SMEM = SMEM_OPS > SMEM_TMEM ? SMEM_OPS : SMEM_TMEM;
    static constexpr uint32_t IDESC = umma_idesc_bf16(BM, COUT);
};

// K runs over (tap, 16-channel group) pairs: k-step j reads tap j / (CIN/16)
// and channels 16 (j % (CIN/16)) .. +15.  A stage holds KS consecutive
// k-steps (the last one possibly fewer); in shared memory k-step kk of a
// stage occupies k-groups 2kk, 2kk+1 of the core-matrix layout.
template <int COUT>
__global__ void __launch_bounds__(TC_THREADS) conv3x3_tc_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w,
                                                                const float *__restrict__ bias, bf16 *__restrict__ y,
                                                                int H, int W, int CIN, int relu, unsigned *err)
{
    typedef TcCfg<COUT> C;
    constexpr int NS = C::NS, KS = C::KS, KG = 2 * KS;  // k-groups (16 B) per stage row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);  // 1024-byte aligned
    __shared__ uint64_t mbar[NS];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long m0 = (long long)blockIdx.x * C::BM;
    const int cg = CIN / 16;               // 16-channel groups per tap
    const int ksteps = TAPS * cg;          // total k-steps
    const int stages = (ksteps + KS - 1) / KS;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int b = 0; b < NS; ++b) mbar_init(&mbar[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = tmem_base;

    const long long p = m0 + tid;  // this thread's pixel: row tid of the A tile
    const int pw = (int)(p % W), ph = (int)((p / W) % H), pb = (int)(p / ((long long)W * H));

    auto load_stage = [&](int st) {
        unsigned char *a = base + (st % NS) * C::STAGE;
        unsigned char *b = a + C::A_BYTES;
        const int j0 = st * KS;
        const int nk = ksteps - j0 < KS ? ksteps - j0 : KS;
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) {
            if (kk < nk) {
                const int j = j0 + kk, t = j / cg, c0 = (j % cg) * 16;
                int hs = ph + tap_dy(t), ws = pw + tap_dx(t);
                hs = hs < 0 ? hs + H : (hs >= H ? hs - H : hs);
                ws = ws < 0 ? ws + W : (ws >= W ? ws - W : ws);
                const bf16 *src = x + ((((long long)pb * H + hs) * W + ws) * CIN + c0);
                unsigned char *dst = a + ((tid >> 3) * KG + 2 * kk) * 128 + (tid & 7) * 16;
                cp_async16(dst, src);
                cp_async16(dst + 128, src + 8);
            }
        }
        for (int c = tid; c < COUT * 2 * nk; c += TC_THREADS) {
            const int n = c / (2 * nk), q = c % (2 * nk);  // q: k-group within the stage
            const int j = j0 + (q >> 1), t = j / cg, c0 = (j % cg) * 16 + (q & 1) * 8;
            cp_async16(b + ((n >> 3) * KG + q) * 128 + (n & 7) * 16, w + (((long long)t * COUT + n) * CIN + c0));
        }
    };

    bool ok = true;
    // Loads run LEAD = NS-3 stages ahead, so the buffer refilled at stage s
    // (that of stage s + LEAD + 1 - NS = s - 2) was consumed by MMA(s-2),
    // issued two stages earlier: the tensor cores' latency overlaps a stage.
    constexpr int LEAD = NS - 3;
#pragma unroll
    for (int st = 0; st <= LEAD; ++st) {
        if (st < stages) load_stage(st);
        cp_commit();
    }
    for (int s = 0; s < stages; ++s) {
        cp_wait<LEAD>();                                       // stage s has landed
        asm volatile("fence.proxy.async.shared::cta;\n" ::);  // visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t a0 = smem_u32(base + (s % NS) * C::STAGE);
            const uint32_t b0 = a0 + C::A_BYTES;
            const int nk = ksteps - s * KS < KS ? ksteps - s * KS : KS;
            for (int kk = 0; kk < nk; ++kk) {
                const uint64_t da = umma_desc(a0 + kk * 256, 128, KG * 128);
                const uint64_t db = umma_desc(b0 + kk * 256, 128, KG * 128);
                const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(C::IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&mbar[s % NS])));
        }
        // refill the buffer of stage s-2 with stage s+LEAD+1 once MMA(s-2) is done
        const int nxt = s + LEAD + 1;
        if (s >= 2 && nxt < stages) {
            ok = __syncthreads_and(mbar_wait(&mbar[(s - 2) % NS], ((s - 2) / NS) & 1) ? 1 : 0) != 0;
            if (!ok) break;
        }
        if (nxt < stages) load_stage(nxt);
        cp_commit();
    }
    // MMA(stages-1) complete implies all earlier ones are (same issuing thread)
    if (ok) ok = __syncthreads_and(mbar_wait(&mbar[(stages - 1) % NS], ((stages - 1) / NS) & 1) ? 1 : 0) != 0;
    cp_wait<0>();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

    if (ok) {
        // epilogue: row m = tid lives in TMEM lane tid (warp w owns lanes 32w..32w+31)
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int n0 = 0; n0 < COUT; n0 += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(lane_addr + n0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
            __align__(16) __nv_bfloat162 o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float v0 = __uint_as_float(r[2 * j]) + (bias ? bias[n0 + 2 * j] : 0.f);
                float v1 = __uint_as_float(r[2 * j + 1]) + (bias ? bias[n0 + 2 * j + 1] : 0.f);
                if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                o[j] = __floats2bfloat162_rn(v0, v1);
            }
            *reinterpret_cast<uint4 *>(y + p * COUT + n0) = *reinterpret_cast<const uint4 *>(o);
        }
    } else if (tid == 0 && err) {
        atomicOr(err, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::TMEM_COLS));
}

template <int COUT>
int launch_conv_tc(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, long long P, int H, int W, int cin,
                   int relu, unsigned *err, cudaStream_t s)
{
    typedef TcCfg<COUT> C;
    static tel::DeviceOnce once;  // one attribute call per instantiation and device
    const cudaError_t ea = once.run([] {
        return cudaFuncSetAttribute(conv3x3_tc_kernel<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (ea != cudaSuccess) return TEL_ECUDA;
    conv3x3_tc_kernel<COUT><<<(unsigned)(P / C::BM), TC_THREADS, C::SMEM, s>>>(x, w, bias, y, H, W, cin, relu, err);
    return launched();
}

// ---------------------------------------------------------------------------
// tcgen05 convolution with a shared halo tile (rows of a multiple of 128
// pixels).  A CTA owns 128 consecutive pixels of one image row.  Per chunk of
// 16 input channels it stages, once, the 3 x 130-pixel halo around them
// (periodic wrap) and the weights of all nine taps; the nine MMAs of the
// chunk then read the halo through shifted descriptors: in the pixel-major
// core-matrix layout (16 B per pixel and 8-channel group, pixels 16 B apart,
// the two channel groups one halo plane apart) the A operand of tap (dy, dx)
// is the same tile started (1+dy) rows and (1+dx) pixels further on.
// ---------------------------------------------------------------------------
constexpr int HALO_C = 130;                      // pixels per halo row

constexpr int pow2_at_least(int v, int p) { return p >= v ? p : pow2_at_least(v, 2 * p); }

// R image rows per CTA (R accumulators of COUT columns side by side in
// tensor memory): the halo holds R + 2 rows and the weights are staged once
// for all R rows.
template <int COUT, int R>
struct TchCfg {
    static constexpr int NS = 2;                 // chunk buffers
    static constexpr int HALO_PLANE = (R + 2) * HALO_C * 16;  // bytes per 8-channel group
    static constexpr int A_BYTES = 2 * HALO_PLANE;
    static constexpr int B_BYTES = TAPS * 2 * COUT * 16;
    static constexpr int STAGE = (A_BYTES + B_BYTES + 127) / 128 * 128;
    static constexpr int TMEM_COLS = pow2_at_least(R * COUT, 32);
    static constexpr size_t SMEM_OPS = 1024 + NS * (size_t)STAGE;
    // shared memory large enough that at most 512 / TMEM_COLS CTAs fit on an
    // SM (228 KB, 1 KB reserved per CTA): their allocations never wait
    static constexpr size_t SMEM_TMEM = (size_t)233472 / (512 / TMEM_COLS + 1) - 1023;
    static constexpr size_t SMEM = SMEM_OPS > SMEM_TMEM ? SMEM_OPS : SMEM_TMEM;
    static constexpr uint32_t IDESC = umma_idesc_bf16(128, COUT);
};

// up: x is the coarse (H/2) x (W/2) grid, read through 2x2 nearest
// upsampling; skip (may be NULL): added to the stored (rounded) output, as a
// separate addition of two BF16 tensors would.
template <int COUT, int R>
__global__ void __launch_bounds__(TC_THREADS) conv3x3_tch_kernel(const bf16 *__restrict__ x,
                                                                 const bf16 *__restrict__ w,
                                                                 const float *__restrict__ bias,
                                                                 bf16 *__restrict__ y, int H, int W, int CIN, int relu,
                                                                 unsigned *err, int up, const bf16 *__restrict__ skip)
{
    typedef TchCfg<COUT, R> C;
    constexpr int NS = C::NS, HP = C::HALO_PLANE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);  // 1024-byte aligned
    __shared__ uint64_t mbar[NS];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int segs = W / 128;
    const long long row = (long long)(blockIdx.x / segs) * R;  // first image row b*H + h of the CTA
    const int w0 = (int)(blockIdx.x % segs) * 128;
    const int h = (int)(row % H);
    const long long b = row / H;
    const int stages = CIN / 16;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(&mbar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = tmem_base;

    auto load_stage = [&](int st) {
        unsigned char *a = base + (st % NS) * C::STAGE;
        unsigned char *bt = a + C::A_BYTES;
        const int c0 = st * 16;
        // halo: [kg][r][c], 16 B per (kg, r, c)
        for (int e = tid; e < 2 * (R + 2) * HALO_C; e += TC_THREADS) {
            const int kg = e / ((R + 2) * HALO_C), rc = e % ((R + 2) * HALO_C), r = rc / HALO_C, c = rc % HALO_C;
            int hs = h + r - 1, ws = w0 + c - 1;
            hs = hs < 0 ? hs + H : (hs >= H ? hs - H : hs);
            ws = ws < 0 ? ws + W : (ws >= W ? ws - W : ws);
            const long long src = up ? ((b * (H >> 1) + (hs >> 1)) * (W >> 1) + (ws >> 1))
                                     : ((b * H + hs) * W + ws);
            cp_async16(a + e * 16, x + (src * CIN + c0 + kg * 8));
        }
        // weights of the nine taps: [t][kg][n], 16 B each
        for (int e = tid; e < TAPS * 2 * COUT; e += TC_THREADS) {
            const int t = e / (2 * COUT), kg = (e / COUT) % 2, n = e % COUT;
            cp_async16(bt + e * 16, w + (((long long)t * COUT + n) * CIN + c0 + kg * 8));
        }
    };

    bool ok = true;
    load_stage(0);
    cp_commit();
    for (int s = 0; s < stages; ++s) {
        if (s + 1 < stages) {
            if (s >= 1) {  // buffer of stage s+1 held stage s-1: wait for its MMAs
                ok = __syncthreads_and(mbar_wait(&mbar[(s - 1) % NS], ((s - 1) / NS) & 1) ? 1 : 0) != 0;
                if (!ok) break;
            }
            load_stage(s + 1);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::);
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t a0 = smem_u32(base + (s % NS) * C::STAGE);
            const uint32_t b0 = a0 + C::A_BYTES;
#pragma unroll
            for (int t = 0; t < TAPS; ++t) {
                const uint64_t db = umma_desc(b0 + t * 2 * COUT * 16, COUT * 16, 128);
                const uint32_t acc = (s > 0 || t > 0) ? 1u : 0u;
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const uint32_t sa = a0 + ((1 + rr + tap_dy(t)) * HALO_C + (1 + tap_dx(t))) * 16;
                    const uint64_t da = umma_desc(sa, HP, 128);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + rr * COUT),
                        "l"(da), "l"(db), "r"(C::IDESC), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&mbar[s % NS])));
        }
    }
    if (ok) ok = __syncthreads_and(mbar_wait(&mbar[(stages - 1) % NS], ((stages - 1) / NS) & 1) ? 1 : 0) != 0;
    cp_wait<0>();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

    if (ok) {
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int rr = 0; rr < R; ++rr) {
        const long long p = (row + rr) * W + w0 + tid;  // output pixel of TMEM lane tid, row rr
#pragma unroll
        for (int n0 = 0; n0 < COUT; n0 += 8) {
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(lane_addr + rr * COUT + n0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
            __align__(16) __nv_bfloat162 o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float v0 = __uint_as_float(r[2 * j]) + (bias ? bias[n0 + 2 * j] : 0.f);
                float v1 = __uint_as_float(r[2 * j + 1]) + (bias ? bias[n0 + 2 * j + 1] : 0.f);
                if (relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                o[j] = __floats2bfloat162_rn(v0, v1);
            }
            if (skip) {
                const uint4 sv = *reinterpret_cast<const uint4 *>(skip + p * COUT + n0);
                const __nv_bfloat162 *sk = reinterpret_cast<const __nv_bfloat162 *>(&sv);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 a2 = __bfloat1622float2(o[j]), s2 = __bfloat1622float2(sk[j]);
                    o[j] = __floats2bfloat162_rn(a2.x + s2.x, a2.y + s2.y);
                }
            }
            *reinterpret_cast<uint4 *>(y + p * COUT + n0) = *reinterpret_cast<const uint4 *>(o);
        }
        }
    } else if (tid == 0 && err) {
        atomicOr(err, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::TMEM_COLS));
}

template <int COUT, int R>
int launch_conv_tch(const bf16 *x, const bf16 *w, const float *bias, bf16 *y, long long P, int H, int W, int cin,
                    int relu, unsigned *err, cudaStream_t s, int up = 0, const bf16 *skip = nullptr)
{
    typedef TchCfg<COUT, R> C;
    static tel::DeviceOnce once;  // one attribute call per instantiation and device
    const cudaError_t ea = once.run([] {
        return cudaFuncSetAttribute(conv3x3_tch_kernel<COUT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (ea != cudaSuccess) return TEL_ECUDA;
    conv3x3_tch_kernel<COUT, R><<<(unsigned)(P / (128 * R)), TC_THREADS, C::SMEM, s>>>(x, w, bias, y, H, W, cin, relu,
                                                                                     err, up, skip);
    return launched();
}

// ---------------------------------------------------------------------------
// Weight gradient: per CTA one tap, a (Cout tile BMO) x (Cin tile BNI)
// block, and a chunk of pixels; each of 4 warps takes 16 of the 64 pixels of
// a stage (its own k16 slice), then the warps' partial sums are added in
// shared memory and once into global memory with FP32 atomics.
// ---------------------------------------------------------------------------
constexpr int WG_THREADS = 128;
constexpr int WG_KP = 64;       // pixels per stage
constexpr int WG_CHUNK = 2048;  // pixels per CTA

template <int BMO, int BNI>
struct WgCfg {
    static constexpr int MT = BMO / 16, NT = BNI / 8;
    static constexpr int LDA = BMO + 8, LDB = BNI + 8;  // rows are pixels
    static constexpr int A_ELEMS = WG_KP * LDA, B_ELEMS = WG_KP * LDB;
    static constexpr size_t SMEM_TILES = sizeof(bf16) * 2 * (A_ELEMS + B_ELEMS);
    static constexpr size_t SMEM_RED = sizeof(float) * 4 * BMO * BNI;
    static constexpr size_t SMEM = SMEM_TILES > SMEM_RED ? SMEM_TILES : SMEM_RED;
};

template <int BMO, int BNI>
__global__ void __launch_bounds__(WG_THREADS) wgrad_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ dz,
                                                           float *__restrict__ dw, int H, int W, int CIN, int COUT,
                                                           long long P)
{
    typedef WgCfg<BMO, BNI> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *As = reinterpret_cast<bf16 *>(smem_raw);  // [buf][pixel][o]
    bf16 *Bs = As + 2 * C::A_ELEMS;                 // [buf][pixel][i]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = blockIdx.y;
    const int dy = tap_dy(t), dx = tap_dx(t);
    const int ntile_i = CIN / BNI;
    const int o0 = (blockIdx.z / ntile_i) * BMO, i0 = (blockIdx.z % ntile_i) * BNI;
    const long long p0 = (long long)blockIdx.x * WG_CHUNK;
    const long long p1 = p0 + WG_CHUNK < P ? p0 + WG_CHUNK : P;
    const int stages = (int)((p1 - p0) / WG_KP);

    auto load_stage = [&](int s, int buf) {
        const long long pb = p0 + (long long)s * WG_KP;
        bf16 *a = As + buf * C::A_ELEMS;
        bf16 *b = Bs + buf * C::B_ELEMS;
        constexpr int AQ = BMO / 8, BQ = BNI / 8;
        for (int c = tid; c < WG_KP * AQ; c += WG_THREADS) {
            const int r = c / AQ, q = c % AQ;
            cp_async16(a + r * C::LDA + q * 8, dz + ((pb + r) * COUT + o0 + q * 8));
        }
        for (int c = tid; c < WG_KP * BQ; c += WG_THREADS) {
            const int r = c / BQ, q = c % BQ;
            const long long p = pb + r;
            const int w_ = (int)(p % W), h_ = (int)((p / W) % H);
            const long long b_ = p / ((long long)W * H);
            int hs = h_ + dy, ws = w_ + dx;
            hs = hs < 0 ? hs + H : (hs >= H ? hs - H : hs);
            ws = ws < 0 ? ws + W : (ws >= W ? ws - W : ws);
            cp_async16(b + r * C::LDB + q * 8, x + (((b_ * H + hs) * W + ws) * CIN + i0 + q * 8));
        }
    };

    float acc[C::MT][C::NT][4];
#pragma unroll
    for (int i = 0; i < C::MT; ++i)
#pragma unroll
        for (int j = 0; j < C::NT; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    if (stages > 0) {
        load_stage(0, 0);
        cp_commit();
    }
    for (int s = 0; s < stages; ++s) {
        if (s + 1 < stages) {
            load_stage(s + 1, (s + 1) & 1);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const bf16 *a = As + (s & 1) * C::A_ELEMS + warp * 16 * C::LDA;  // this warp's 16 pixels
        const bf16 *b = Bs + (s & 1) * C::B_ELEMS + warp * 16 * C::LDB;
        // A = dz^T (rows o, k = pixel) from [pixel][o] via transposing loads;
        // B (k = pixel, n = i) from [pixel][i] via transposing loads.
        uint32_t af[C::MT][4];
#pragma unroll
        for (int mt = 0; mt < C::MT; ++mt) {
            const int j = lane >> 3;
            const int prow = (j >> 1) * 8 + (lane & 7);
            const int ocol = mt * 16 + (j & 1) * 8;
            ldsm_x4_t(af[mt][0], af[mt][1], af[mt][2], af[mt][3], a + prow * C::LDA + ocol);
        }
#pragma unroll
        for (int nt = 0; nt < C::NT; nt += 2) {
            uint32_t b0, b1, b2, b3;
            if (nt + 1 < C::NT) {
                const int j = lane >> 3;
                const int prow = (j & 1) * 8 + (lane & 7);
                const int icol = nt * 8 + (j >> 1) * 8;
                ldsm_x4_t(b0, b1, b2, b3, b + prow * C::LDB + icol);
            } else {
                const int j = (lane >> 3) & 1;
                const int prow = j * 8 + (lane & 7);
                ldsm_x2_t(b0, b1, b + prow * C::LDB + nt * 8);
                b2 = b3 = 0u;
            }
#pragma unroll
            for (int mt = 0; mt < C::MT; ++mt) {
                mma_bf16(acc[mt][nt], af[mt], b0, b1);
                if (nt + 1 < C::NT) mma_bf16(acc[mt][nt + 1], af[mt], b2, b3);
            }
        }
        __syncthreads();
    }

    // cross-warp reduction in shared memory, then one atomic per element
    float *red = reinterpret_cast<float *>(smem_raw);
#pragma unroll
    for (int mt = 0; mt < C::MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < C::NT; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = mt * 16 + (lane >> 2) + (k >> 1) * 8;
                const int i = nt * 8 + (lane & 3) * 2 + (k & 1);
                red[(warp * BMO + o) * BNI + i] = acc[mt][nt][k];
            }
    __syncthreads();
    for (int e = tid; e < BMO * BNI; e += WG_THREADS) {
        const float v = red[e] + red[BMO * BNI + e] + red[2 * BMO * BNI + e] + red[3 * BMO * BNI + e];
        const int o = e / BNI, i = e % BNI;
        atomicAdd(dw + ((long long)t * COUT + o0 + o) * CIN + i0 + i, v);
    }
}

template <int BMO, int BNI>
int launch_wgrad(const bf16 *x, const bf16 *dz, float *dw, long long P, int H, int W, int cin, int cout,
                 cudaStream_t s)
{
    typedef WgCfg<BMO, BNI> C;
    static tel::DeviceOnce once;  // one attribute call per instantiation and device
    const cudaError_t ea = once.run([] {
        return cudaFuncSetAttribute(wgrad_kernel<BMO, BNI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    });
    if (ea != cudaSuccess) return TEL_ECUDA;
    dim3 grid((unsigned)((P + WG_CHUNK - 1) / WG_CHUNK), TAPS, (unsigned)((cout / BMO) * (cin / BNI)));
    wgrad_kernel<BMO, BNI><<<grid, WG_THREADS, C::SMEM, s>>>(x, dz, dw, H, W, cin, cout, P);
    return launched();
}

// db[o] += sum_p dz[p][o]: each thread sums one channel over a strided
// pixel range, one atomic per thread.
__global__ void bias_grad_kernel(const bf16 *__restrict__ dz, float *__restrict__ db, long long P, int C)
{
    const int per = blockDim.x / C;  // pixel lanes per block
    const int c = threadIdx.x % C, lane = threadIdx.x / C;
    if (lane >= per) return;
    float s = 0.f;
    for (long long p = (long long)blockIdx.x * per + lane; p < P; p += (long long)gridDim.x * per)
        s += __bfloat162float(dz[p * C + c]);
    atomicAdd(db + c, s);
}

// ---------------------------------------------------------------------------
// elementwise / layout kernels
// ---------------------------------------------------------------------------
__global__ void flip_kernel(const bf16 *__restrict__ w, bf16 *__restrict__ wt, int CIN, int COUT)
{
    const long long n = (long long)TAPS * CIN * COUT;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        // wt[s][i][o] = w[8 - s][o][i]
        const int o = (int)(e % COUT);
        const int i = (int)((e / COUT) % CIN);
        const int s = (int)(e / ((long long)COUT * CIN));
        wt[e] = w[((long long)(TAPS - 1 - s) * COUT + o) * CIN + i];
    }
}

__global__ void relu_bwd_kernel(const bf16 *__restrict__ y, const bf16 *dy, bf16 *dz, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dz[e] = __bfloat162float(y[e]) > 0.f ? dy[e] : __float2bfloat16(0.f);
}

__global__ void add_kernel(const bf16 *a, const bf16 *b, bf16 *y, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16(__bfloat162float(a[e]) + __bfloat162float(b[e]));
}

// coarse element e = ((b * Hc + hc) * Wc + wc) * C + c, Hc = H/2, Wc = W/2
__device__ __forceinline__ long long fine_index(long long e, int H, int W, int C, int oy, int ox)
{
    const int Hc = H / 2, Wc = W / 2;
    const int c = (int)(e % C);
    const long long q = e / C;
    const int wc = (int)(q % Wc), hc = (int)((q / Wc) % Hc);
    const long long b = q / ((long long)Wc * Hc);
    return ((b * H + 2 * hc + oy) * W + 2 * wc + ox) * C + c;
}

__global__ void pool2_kernel(const bf16 *__restrict__ x, bf16 *__restrict__ y, long long nc, int H, int W, int C)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nc; e += (long long)gridDim.x * blockDim.x) {
        const float s = __bfloat162float(x[fine_index(e, H, W, C, 0, 0)]) + __bfloat162float(x[fine_index(e, H, W, C, 0, 1)]) +
                        __bfloat162float(x[fine_index(e, H, W, C, 1, 0)]) + __bfloat162float(x[fine_index(e, H, W, C, 1, 1)]);
        y[e] = __float2bfloat16(0.25f * s);
    }
}

__global__ void pool2_bwd_kernel(const bf16 *__restrict__ dy, bf16 *__restrict__ dx, long long nc, int H, int W, int C)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nc; e += (long long)gridDim.x * blockDim.x) {
        const bf16 v = __float2bfloat16(0.25f * __bfloat162float(dy[e]));
        dx[fine_index(e, H, W, C, 0, 0)] = v;
        dx[fine_index(e, H, W, C, 0, 1)] = v;
        dx[fine_index(e, H, W, C, 1, 0)] = v;
        dx[fine_index(e, H, W, C, 1, 1)] = v;
    }
}

__global__ void up2_kernel(const bf16 *__restrict__ x, bf16 *__restrict__ y, long long nc, int H, int W, int C)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nc; e += (long long)gridDim.x * blockDim.x) {
        const bf16 v = x[e];
        y[fine_index(e, H, W, C, 0, 0)] = v;
        y[fine_index(e, H, W, C, 0, 1)] = v;
        y[fine_index(e, H, W, C, 1, 0)] = v;
        y[fine_index(e, H, W, C, 1, 1)] = v;
    }
}

__global__ void up2_bwd_kernel(const bf16 *__restrict__ dy, bf16 *__restrict__ dx, long long nc, int H, int W, int C)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nc; e += (long long)gridDim.x * blockDim.x) {
        const float s = __bfloat162float(dy[fine_index(e, H, W, C, 0, 0)]) + __bfloat162float(dy[fine_index(e, H, W, C, 0, 1)]) +
                        __bfloat162float(dy[fine_index(e, H, W, C, 1, 0)]) + __bfloat162float(dy[fine_index(e, H, W, C, 1, 1)]);
        dx[e] = __float2bfloat16(s);
    }
}

__global__ void pack_kernel(const double *__restrict__ rho, const double *__restrict__ phi, const double *__restrict__ u,
                            const float *__restrict__ norm, float *f32, bf16 *x16, int B, long long N)
{
    const long long n = (long long)B * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / N, k = e % N;
        const float v[4] = {(float)(rho[e] * (double)norm[3 * b]), (float)(phi[e] * (double)norm[3 * b + 1]),
                            (float)(u[(2 * b) * N + k] * (double)norm[3 * b + 2]),
                            (float)(u[(2 * b + 1) * N + k] * (double)norm[3 * b + 2])};
        if (f32) *reinterpret_cast<float4 *>(f32 + 4 * e) = make_float4(v[0], v[1], v[2], v[3]);
        if (x16) {
            bf16 *o = x16 + 16 * e;
#pragma unroll
            for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(c < 4 ? v[c] : 0.f);
        }
    }
}

__global__ void unpack_kernel(const float *__restrict__ f32, const float *__restrict__ norm, double *rho, double *phi,
                              double *u, int B, long long N)
{
    const long long n = (long long)B * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / N, k = e % N;
        const float4 v = *reinterpret_cast<const float4 *>(f32 + 4 * e);
        if (rho) rho[e] = (double)v.x / (double)norm[3 * b];
        if (phi) phi[e] = (double)v.y / (double)norm[3 * b + 1];
        if (u) {
            u[(2 * b) * N + k] = (double)v.z / (double)norm[3 * b + 2];
            u[(2 * b + 1) * N + k] = (double)v.w / (double)norm[3 * b + 2];
        }
    }
}

// Symmetry code s of the square lattice's dihedral group: bit 0 mirrors x,
// bit 1 mirrors y, bit 2 transposes (applied first).  Output node (h, w)
// reads source node (hs, ws); velocities transform with the coordinates.
__device__ __forceinline__ long long sym_source(int s, long long k, int H, int W, float &sx, float &sy, bool &swap)
{
    const int h = (int)(k / W), w = (int)(k % W);
    const int w1 = (s & 1) ? W - 1 - w : w;
    const int h1 = (s & 2) ? H - 1 - h : h;
    swap = (s & 4) != 0;
    sx = (s & 1) ? -1.f : 1.f;
    sy = (s & 2) ? -1.f : 1.f;
    return swap ? (long long)w1 * W + h1 : (long long)h1 * W + w1;
}

__global__ void gather_kernel(const float *__restrict__ store, const int *__restrict__ src, const int *__restrict__ dst,
                              const int *__restrict__ sym, const float *__restrict__ scale, float *f32, bf16 *x16,
                              float *target, int B, int H, int W)
{
    const long long N = (long long)H * W;
    const long long n = (long long)B * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / N;
        float sx = 1.f, sy = 1.f;
        bool swap = false;
        const long long k = sym ? sym_source(sym[b] & 7, e % N, H, W, sx, sy, swap) : e % N;
        float4 a = *reinterpret_cast<const float4 *>(store + 4 * ((long long)src[b] * N + k));
        float4 z = dst ? *reinterpret_cast<const float4 *>(store + 4 * ((long long)dst[b] * N + k)) : a;
        if (swap) {
            float t = a.z; a.z = a.w; a.w = t;
            t = z.z; z.z = z.w; z.w = t;
        }
        a.z *= sx; a.w *= sy;
        z.z *= sx; z.w *= sy;
        if (f32) *reinterpret_cast<float4 *>(f32 + 4 * e) = a;
        if (target)
            *reinterpret_cast<float4 *>(target + 4 * e) =
                make_float4((z.x - a.x) / scale[0], (z.y - a.y) / scale[1], (z.z - a.z) / scale[2], (z.w - a.w) / scale[3]);
        if (x16) {
            bf16 *o = x16 + 16 * e;
            o[0] = __float2bfloat16(a.x);
            o[1] = __float2bfloat16(a.y);
            o[2] = __float2bfloat16(a.z);
            o[3] = __float2bfloat16(a.w);
#pragma unroll
            for (int c = 4; c < 16; ++c) o[c] = __float2bfloat16(0.f);
        }
    }
}

// Block-level sum of v into *dst with one atomic per block.
template <typename T>
__device__ __forceinline__ void block_sum_atomic(T v, T *dst)
{
    __shared__ T part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? part[lane] : (T)0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(dst, v);
    }
}

// per-sample sums of output channels 0, 1 (and target channels 0, 1 when
// target != NULL): work[4 b + c] for c = out0, out1, tgt0, tgt1.  Grid
// (blocks per sample, B).
__global__ void head_sums_kernel(const bf16 *__restrict__ out, const float *__restrict__ target, float *work,
                                 long long N)
{
    const int b = blockIdx.y;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
        const long long e = (long long)b * N + k;
        s[0] += __bfloat162float(out[16 * e]);
        s[1] += __bfloat162float(out[16 * e + 1]);
        if (target) { s[2] += target[4 * e]; s[3] += target[4 * e + 1]; }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) block_sum_atomic(s[c], work + 4 * b + c);
}

__global__ void loss_kernel(const bf16 *__restrict__ out, const float *__restrict__ target, bf16 *dout, float *loss,
                            const float *__restrict__ work, int B, long long N)
{
    const long long n = (long long)B * N;
    const float inv_n = 1.f / (float)(4 * n), invN = 1.f / (float)N;
    float l = 0.f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / N;
        const float mo0 = work[4 * b] * invN, mo1 = work[4 * b + 1] * invN;
        const float mt0 = work[4 * b + 2] * invN, mt1 = work[4 * b + 3] * invN;
        float r[4];
        r[0] = (__bfloat162float(out[16 * e]) - mo0) - target[4 * e];
        r[1] = (__bfloat162float(out[16 * e + 1]) - mo1) - target[4 * e + 1];
        r[2] = __bfloat162float(out[16 * e + 2]) - target[4 * e + 2];
        r[3] = __bfloat162float(out[16 * e + 3]) - target[4 * e + 3];
        l += r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3];
        // the mean of r over the sample is -mean(target) for channels 0, 1
        const float g0 = 2.f * inv_n * (r[0] + mt0), g1 = 2.f * inv_n * (r[1] + mt1);
        bf16 *d = dout + 16 * e;
        d[0] = __float2bfloat16(g0);
        d[1] = __float2bfloat16(g1);
        d[2] = __float2bfloat16(2.f * inv_n * r[2]);
        d[3] = __float2bfloat16(2.f * inv_n * r[3]);
#pragma unroll
        for (int c = 4; c < 16; ++c) d[c] = __float2bfloat16(0.f);
    }
    block_sum_atomic(l * inv_n, loss);
}

__global__ void advance_kernel(const float *__restrict__ f32, const bf16 *__restrict__ out, const float *__restrict__ scale,
                               float *f32n, bf16 *x16n, double *mass, const float *__restrict__ work, long long N)
{
    const int b = blockIdx.y;
    const float invN = 1.f / (float)N;
    const float mo0 = work[4 * b] * invN, mo1 = work[4 * b + 1] * invN;
    double m0 = 0.0, m1 = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
        const long long e = (long long)b * N + k;
        const float4 a = *reinterpret_cast<const float4 *>(f32 + 4 * e);
        const float4 v = make_float4(a.x + scale[0] * (__bfloat162float(out[16 * e]) - mo0),
                                     a.y + scale[1] * (__bfloat162float(out[16 * e + 1]) - mo1),
                                     a.z + scale[2] * __bfloat162float(out[16 * e + 2]),
                                     a.w + scale[3] * __bfloat162float(out[16 * e + 3]));
        *reinterpret_cast<float4 *>(f32n + 4 * e) = v;
        m0 += (double)v.x;
        m1 += (double)v.y;
        if (x16n) {
            bf16 *o = x16n + 16 * e;
            o[0] = __float2bfloat16(v.x);
            o[1] = __float2bfloat16(v.y);
            o[2] = __float2bfloat16(v.z);
            o[3] = __float2bfloat16(v.w);
#pragma unroll
            for (int c = 4; c < 16; ++c) o[c] = __float2bfloat16(0.f);
        }
    }
    if (mass) {
        block_sum_atomic(m0, mass + 2 * b);
        block_sum_atomic(m1, mass + 2 * b + 1);
    }
}

__global__ void errors_kernel(const float *__restrict__ pred, const float *__restrict__ ref, double *acc, long long N)
{
    const int b = blockIdx.y;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
        const long long e = (long long)b * N + k;
        const float4 p = *reinterpret_cast<const float4 *>(pred + 4 * e);
        const float4 r = *reinterpret_cast<const float4 *>(ref + 4 * e);
        const double d0 = (double)p.x - r.x, d1 = (double)p.y - r.y, d2 = (double)p.z - r.z, d3 = (double)p.w - r.w;
        s[0] += d0 * d0; s[1] += (double)r.x * r.x;
        s[2] += d1 * d1; s[3] += (double)r.y * r.y;
        s[4] += d2 * d2 + d3 * d3; s[5] += (double)r.z * r.z + (double)r.w * r.w;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) block_sum_atomic(s[c], acc + 6 * b + c);
}

__global__ void sums_kernel(const float *__restrict__ f32, double *sums, long long N)
{
    const int b = blockIdx.y;
    double m0 = 0.0, m1 = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
        const float4 v = *reinterpret_cast<const float4 *>(f32 + 4 * ((long long)b * N + k));
        m0 += (double)v.x;
        m1 += (double)v.y;
    }
    block_sum_atomic(m0, sums + 2 * b);
    block_sum_atomic(m1, sums + 2 * b + 1);
}

__global__ void adam_kernel(float *w32, bf16 *w16, const float *__restrict__ g, float *m, float *v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2, float gs, const float *gs_dev)
{
    if (gs_dev) gs *= *gs_dev;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gi = g[e] * gs;
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        const float wi = w32[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w32[e] = wi;
        if (w16) w16[e] = __float2bfloat16(wi);
    }
}

__global__ void sumsq_kernel(const float *__restrict__ g, long long n, double *out)
{
    double a = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        a += (double)g[e] * (double)g[e];
    block_sum_atomic(a, out);
}

__global__ void clip_scale_kernel(const double *sumsq, float clip, float *scale)
{
    const double nrm = sqrt(*sumsq);
    *scale = nrm > (double)clip ? (float)((double)clip / nrm) : 1.f;
}

__global__ void to_bf16_kernel(const float *__restrict__ w32, bf16 *w16, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        w16[e] = __float2bfloat16(w32[e]);
}

inline unsigned blocks_for(long long n, int threads = 256)
{
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 16;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

inline unsigned blocks_per_sample(long long N, int B)
{
    long long b = (N + 255) / 256;
    const long long cap = (152LL * 8 + B - 1) / B;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

extern "C" int tel_sur_conv3x3(const void *x, const void *w, const float *bias, void *y, int B, int H, int W, int cin,
                               int cout, int relu, void *stream)
{
    const long long P = (long long)B * H * W;
    if (!x || !w || !y || B < 1 || H < 1 || W < 1 || !chan_ok(cin) || !chan_ok(cout) || P % CONV_BM) return TEL_EINVAL;
    const bf16 *xb = (const bf16 *)x, *wb = (const bf16 *)w;
    bf16 *yb = (bf16 *)y;
    switch (cout) {
    case 16: return conv_dispatch_k<16>(xb, wb, bias, yb, P, H, W, cin, relu, S(stream));
    case 32: return conv_dispatch_k<32>(xb, wb, bias, yb, P, H, W, cin, relu, S(stream));
    case 64: return conv_dispatch_k<64>(xb, wb, bias, yb, P, H, W, cin, relu, S(stream));
    default: return conv_dispatch_k<128>(xb, wb, bias, yb, P, H, W, cin, relu, S(stream));
    }
}

extern "C" int tel_sur_flip_weights(const void *w, void *w_t, int cin, int cout, void *stream)
{
    if (!w || !w_t || !chan_ok(cin) || !chan_ok(cout)) return TEL_EINVAL;
    const long long n = (long long)TAPS * cin * cout;
    flip_kernel<<<blocks_for(n), 256, 0, S(stream)>>>((const bf16 *)w, (bf16 *)w_t, cin, cout);
    return launched();
}

extern "C" int tel_sur_relu_bwd(const void *y, const void *dy, void *dz, long long n, void *stream)
{
    if (!y || !dy || !dz || n < 0) return TEL_EINVAL;
    if (n == 0) return TEL_OK;
    relu_bwd_kernel<<<blocks_for(n), 256, 0, S(stream)>>>((const bf16 *)y, (const bf16 *)dy, (bf16 *)dz, n);
    return launched();
}

extern "C" int tel_sur_conv3x3_wgrad(const void *x, const void *dz, float *dw, float *db, int B, int H, int W, int cin,
                                     int cout, void *stream)
{
    const long long P = (long long)B * H * W;
    if (!x || !dz || !dw || B < 1 || H < 1 || W < 1 || !chan_ok(cin) || !chan_ok(cout) || P % WG_KP) return TEL_EINVAL;
    const bf16 *xb = (const bf16 *)x, *zb = (const bf16 *)dz;
    int rc;
    // Cout tile up to 64, Cin tile up to 32 (64 FP32 accumulators per thread)
    const int bmo = cout >= 64 ? 64 : cout, bni = cin >= 32 ? 32 : cin;
    if (bmo == 64 && bni == 32) rc = launch_wgrad<64, 32>(xb, zb, dw, P, H, W, cin, cout, S(stream));
    else if (bmo == 64) rc = launch_wgrad<64, 16>(xb, zb, dw, P, H, W, cin, cout, S(stream));
    else if (bmo == 32 && bni == 32) rc = launch_wgrad<32, 32>(xb, zb, dw, P, H, W, cin, cout, S(stream));
    else if (bmo == 32) rc = launch_wgrad<32, 16>(xb, zb, dw, P, H, W, cin, cout, S(stream));
    else if (bni == 32) rc = launch_wgrad<16, 32>(xb, zb, dw, P, H, W, cin, cout, S(stream));
    else rc = launch_wgrad<16, 16>(xb, zb, dw, P, H, W, cin, cout, S(stream));
    if (rc || !db) return rc;
    const int per = 256 / cout;
    long long nb = (P + per * 64 - 1) / (per * 64);
    if (nb > 152 * 4) nb = 152 * 4;
    bias_grad_kernel<<<(unsigned)nb, per * cout, 0, S(stream)>>>(zb, db, P, cout);
    return launched();
}

#define POOLCHK                                                                                    \
    if (!a || !b || B < 1 || H < 2 || W < 2 || (H & 1) || (W & 1) || C < 1) return TEL_EINVAL;    \
    const long long nc = (long long)B * (H / 2) * (W / 2) * C;

extern "C" int tel_sur_pool2(const void *a, void *b, int B, int H, int W, int C, void *stream)
{
    POOLCHK
    pool2_kernel<<<blocks_for(nc), 256, 0, S(stream)>>>((const bf16 *)a, (bf16 *)b, nc, H, W, C);
    return launched();
}
extern "C" int tel_sur_pool2_bwd(const void *a, void *b, int B, int H, int W, int C, void *stream)
{
    POOLCHK
    pool2_bwd_kernel<<<blocks_for(nc), 256, 0, S(stream)>>>((const bf16 *)a, (bf16 *)b, nc, H, W, C);
    return launched();
}
extern "C" int tel_sur_up2(const void *a, void *b, int B, int H, int W, int C, void *stream)
{
    POOLCHK
    up2_kernel<<<blocks_for(nc), 256, 0, S(stream)>>>((const bf16 *)a, (bf16 *)b, nc, H, W, C);
    return launched();
}
extern "C" int tel_sur_up2_bwd(const void *a, void *b, int B, int H, int W, int C, void *stream)
{
    POOLCHK
    up2_bwd_kernel<<<blocks_for(nc), 256, 0, S(stream)>>>((const bf16 *)a, (bf16 *)b, nc, H, W, C);
    return launched();
}

extern "C" int tel_sur_add(const void *a, const void *b, void *y, long long n, void *stream)
{
    if (!a || !b || !y || n < 0) return TEL_EINVAL;
    if (n == 0) return TEL_OK;
    add_kernel<<<blocks_for(n), 256, 0, S(stream)>>>((const bf16 *)a, (const bf16 *)b, (bf16 *)y, n);
    return launched();
}

extern "C" int tel_sur_pack(const double *rho, const double *phi, const double *u, const float *norm, float *f32,
                            void *x16, int B, int H, int W, void *stream)
{
    if (!rho || !phi || !u || !norm || (!f32 && !x16) || B < 1 || H < 1 || W < 1) return TEL_EINVAL;
    const long long N = (long long)H * W;
    pack_kernel<<<blocks_for((long long)B * N), 256, 0, S(stream)>>>(rho, phi, u, norm, f32, (bf16 *)x16, B, N);
    return launched();
}

extern "C" int tel_sur_unpack(const float *f32, const float *norm, double *rho, double *phi, double *u, int B, int H,
                              int W, void *stream)
{
    if (!f32 || !norm || B < 1 || H < 1 || W < 1) return TEL_EINVAL;
    const long long N = (long long)H * W;
    unpack_kernel<<<blocks_for((long long)B * N), 256, 0, S(stream)>>>(f32, norm, rho, phi, u, B, N);
    return launched();
}

extern "C" int tel_sur_gather(const float *store, const int *src, const int *dst, const int *sym, const float *scale,
                              float *f32, void *x16, float *target, int B, int H, int W, void *stream)
{
    if (!store || !src || (target && (!dst || !scale)) || B < 1 || H < 1 || W < 1) return TEL_EINVAL;
    if (sym && H != W) return TEL_EINVAL;  // transposition needs a square lattice
    gather_kernel<<<blocks_for((long long)B * H * W), 256, 0, S(stream)>>>(store, src, dst, sym, scale, f32,
                                                                           (bf16 *)x16, target, B, H, W);
    return launched();
}

extern "C" int tel_sur_loss(const void *out, const float *target, void *dout, float *loss, float *work, int B, int H,
                            int W, void *stream)
{
    if (!out || !target || !dout || !loss || !work || B < 1 || H < 1 || W < 1) return TEL_EINVAL;
    const long long N = (long long)H * W;
    if (cudaMemsetAsync(work, 0, sizeof(float) * 4 * B, S(stream)) != cudaSuccess) return TEL_ECUDA;
    head_sums_kernel<<<dim3(blocks_per_sample(N, B), B), 256, 0, S(stream)>>>((const bf16 *)out, target, work, N);
    int rc = launched();
    if (rc) return rc;
    loss_kernel<<<blocks_for((long long)B * N), 256, 0, S(stream)>>>((const bf16 *)out, target, (bf16 *)dout, loss,
                                                                     work, B, N);
    return launched();
}

extern "C" int tel_sur_advance(const float *f32, const void *out, const float *scale, float *f32_next, void *x16_next,
                               double *mass, float *work, int B, int H, int W, void *stream)
{
    if (!f32 || !out || !scale || !f32_next || !work || B < 1 || H < 1 || W < 1) return TEL_EINVAL;
    const long long N = (long long)H * W;
    if (cudaMemsetAsync(work, 0, sizeof(float) * 4 * B, S(stream)) != cudaSuccess) return TEL_ECUDA;
    head_sums_kernel<<<dim3(blocks_per_sample(N, B), B), 256, 0, S(stream)>>>((const bf16 *)out, nullptr, work, N);
    int rc = launched();
    if (rc) return rc;
    advance_kernel<<<dim3(blocks_per_sample(N, B), B), 256, 0, S(stream)>>>(f32, (const bf16 *)out, scale, f32_next,
                                                                           (bf16 *)x16_next, mass, work, N);
    return launched();
}

extern "C" int tel_sur_errors(const float *pred, const float *ref, double *acc, int B, int H, int W, void *stream)
{
    if (!pred || !ref || !acc || B < 1 || H < 1 || W < 1) return TEL_EINVAL;
    const long long N = (long long)H * W;
    errors_kernel<<<dim3(blocks_per_sample(N, B), B), 256, 0, S(stream)>>>(pred, ref, acc, N);
    return launched();
}

extern "C" int tel_sur_adam(float *w32, void *w16, const float *g, float *m, float *v, long long n, float lr,
                            float beta1, float beta2, float eps, int t, float grad_scale, void *stream)
{
    if (!w32 || !g || !m || !v || n < 0 || t < 1) return TEL_EINVAL;
    if (n == 0) return TEL_OK;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    adam_kernel<<<blocks_for(n), 256, 0, S(stream)>>>(w32, (bf16 *)w16, g, m, v, n, lr, beta1, beta2, eps, c1, c2,
                                                      grad_scale, nullptr);
    return launched();
}

extern "C" int tel_sur_clip_scale(const float *g, long long n, float clip, double *work, float *scale, void *stream)
{
    if (!g || !work || !scale || n < 1 || !(clip > 0.f)) return TEL_EINVAL;
    if (cudaMemsetAsync(work, 0, sizeof(double), S(stream)) != cudaSuccess) return TEL_ECUDA;
    sumsq_kernel<<<blocks_for(n), 256, 0, S(stream)>>>(g, n, work);
    int rc = launched();
    if (rc) return rc;
    clip_scale_kernel<<<1, 1, 0, S(stream)>>>(work, clip, scale);
    return launched();
}

extern "C" int tel_sur_adam_scaled(float *w32, void *w16, const float *g, float *m, float *v, long long n, float lr,
                                   float beta1, float beta2, float eps, int t, const float *scale, void *stream)
{
    if (!w32 || !g || !m || !v || !scale || n < 0 || t < 1) return TEL_EINVAL;
    if (n == 0) return TEL_OK;
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    adam_kernel<<<blocks_for(n), 256, 0, S(stream)>>>(w32, (bf16 *)w16, g, m, v, n, lr, beta1, beta2, eps, c1, c2, 1.f,
                                                      scale);
    return launched();
}

extern "C" int tel_sur_to_bf16(const float *w32, void *w16, long long n, void *stream)
{
    if (!w32 || !w16 || n < 0) return TEL_EINVAL;
    if (n == 0) return TEL_OK;
    to_bf16_kernel<<<blocks_for(n), 256, 0, S(stream)>>>(w32, (bf16 *)w16, n);
    return launched();
}

extern "C" int tel_sur_zero(float *p, long long n, void *stream)
{
    if (!p || n < 0) return TEL_EINVAL;
    return ok(cudaMemsetAsync(p, 0, sizeof(float) * (size_t)n, S(stream)));
}

extern "C" int tel_sur_sums(const float *f32, double *sums, int B, int H, int W, void *stream)
{
    if (!f32 || !sums || B < 1 || H < 1 || W < 1) return TEL_EINVAL;
    const long long N = (long long)H * W;
    if (cudaMemsetAsync(sums, 0, sizeof(double) * 2 * B, S(stream)) != cudaSuccess) return TEL_ECUDA;
    sums_kernel<<<dim3(blocks_per_sample(N, B), B), 256, 0, S(stream)>>>(f32, sums, N);
    return launched();
}

extern "C" int tel_sur_conv3x3_tc(const void *x, const void *w, const float *bias, void *y, int B, int H, int W,
                                  int cin, int cout, int relu, unsigned *err, void *stream)
{
    const long long P = (long long)B * H * W;
    if (!x || !w || !y || B < 1 || H < 1 || W < 1 || !chan_ok(cin) || !chan_ok(cout) || P % 128) return TEL_EINVAL;
    const bf16 *xb = (const bf16 *)x, *wb = (const bf16 *)w;
    bf16 *yb = (bf16 *)y;
    if (W % 128 == 0 && H % 4 == 0) {  // whole 128-pixel segments, four rows per CTA: shared halo tile
        switch (cout) {
        case 16: return launch_conv_tch<16, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        case 32: return launch_conv_tch<32, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        case 64: return launch_conv_tch<64, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        default: return launch_conv_tch<128, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        }
    }
    if (W % 128 == 0) {  // whole 128-pixel segments, one row per CTA
        switch (cout) {
        case 16: return launch_conv_tch<16, 1>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        case 32: return launch_conv_tch<32, 1>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        case 64: return launch_conv_tch<64, 1>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        default: return launch_conv_tch<128, 1>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
        }
    }
    switch (cout) {
    case 16: return launch_conv_tc<16>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
    case 32: return launch_conv_tc<32>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
    case 64: return launch_conv_tc<64>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
    default: return launch_conv_tc<128>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream));
    }
}

extern "C" int tel_sur_conv3x3_tc_fused(const void *x, const void *w, const float *bias, void *y, int B, int H, int W,
                                        int cin, int cout, int relu, int up_input, const void *skip, unsigned *err,
                                        void *stream)
{
    const long long P = (long long)B * H * W;
    if (!x || !w || !y || B < 1 || H < 4 || W < 128 || !chan_ok(cin) || !chan_ok(cout)) return TEL_EINVAL;
    if (W % 128 || H % 4) return TEL_EINVAL;  // the four-row halo kernel only (H, W even for the upsampled input)
    const bf16 *xb = (const bf16 *)x, *wb = (const bf16 *)w, *sb = (const bf16 *)skip;
    bf16 *yb = (bf16 *)y;
    switch (cout) {
    case 16: return launch_conv_tch<16, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream), up_input, sb);
    case 32: return launch_conv_tch<32, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream), up_input, sb);
    case 64: return launch_conv_tch<64, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream), up_input, sb);
    default: return launch_conv_tch<128, 4>(xb, wb, bias, yb, P, H, W, cin, relu, err, S(stream), up_input, sb);
    }
}
