// Tensor-core complex GEMM for the large pairwise contraction steps
// (tcgen05 MMA with TMEM accumulators, operands staged by TMA), sm_103a.
//
// The paper maps contractions to matrix multiplications on the GPU
// (Sec. IV-A); here a complex product C[M][N] = A[M][K] . B[N][K]^T is run as
// one real product on the tensor cores:
//   * A's interleaved complex storage, read as floats, already is the real
//     matrix A_r[M][2K] = (re a_m0, im a_m0, re a_m1, ...);
//   * B is expanded to B'[2N][2K] with rows 2n = (re b, -im b, ...) and
//     2n+1 = (im b, re b, ...), so that row m of A_r times row 2n (2n+1) of B'
//     is the real (imaginary) part of C[m][n];
//   * the real result C_r[M][2N] is C's interleaved complex storage.
// Precision forms split each real operand into parts and sum part products
// in one FP32 TMEM accumulator:
//   3xTF32:  x = hi + lo (hi = x rounded to TF32); hi.hi + hi.lo + lo.hi
//   BF16x3:  x = b0 + b1 + b2 (each rounded to BF16 in turn);
//            b0b0 + b0b1 + b1b0 + b0b2 + b1b1 + b2b0
//   FP16:    one product of the operands scaled by powers of two (per tensor)
// Tile: 128 rows of A x 128 rows of B' per CTA, one 128-byte K slab per
// pipeline stage, two 128-column TMEM accumulators used in turn.  Warp 0
// issues TMA, warp 1 owns TMEM and issues the MMAs, warps 2-5 add each stage's
// TMEM partial into FP32 register totals and write C at the end.  Every mbarrier
// wait is bounded; on expiry the kernel records QX_ETIMEOUT, waits (bounded)
// for its own copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "qx.h"
#include "qx_internal.h"

namespace qx {

constexpr int TC_BM = 128, TC_ROWB = 128, TC_SMEM_LIMIT = 196608;

template <int FORM>
struct TcForm;
template <>
struct TcForm<TC_FORM_3XTF32> {
    using T = float;
    static constexpr int NPA = 2, NPB = 2, NPROD = 3, EB = 4, FMT = 2, STAGES = 3;
    static __device__ __forceinline__ int pa(int p) { return p == 2 ? 1 : 0; }
    static __device__ __forceinline__ int pb(int p) { return p == 1 ? 1 : 0; }
};
template <>
struct TcForm<TC_FORM_BF16X3> {
    using T = __nv_bfloat16;
    static constexpr int NPA = 3, NPB = 3, NPROD = 6, EB = 2, FMT = 1, STAGES = 2;
    // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
    static __device__ __forceinline__ int pa(int p) { return p < 2 ? 0 : p == 2 ? 1 : p == 3 ? 0 : p == 4 ? 1 : 2; }
    static __device__ __forceinline__ int pb(int p) { return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 2 : p == 4 ? 1 : 0; }
};

template <>
struct TcForm<TC_FORM_FP16> {
    using T = __half;
    static constexpr int NPA = 1, NPB = 1, NPROD = 1, EB = 2, FMT = 0, STAGES = 6;
    static __device__ __forceinline__ int pa(int) { return 0; }
    static __device__ __forceinline__ int pb(int) { return 0; }
};

// FP16 form: a tensor is multiplied by 2^e with e chosen so that its largest
// magnitude lands just below 2^14 (well inside FP16's range, away from its
// subnormals); the epilogue divides by both operands' factors.
__device__ __forceinline__ float fp16_scale(float amax) {
    if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
    int ex;
    frexpf(amax, &ex);  // amax < 2^ex
    return ldexpf(1.f, 14 - ex);
}

// ------------------------------------------------------------------------------------------------
// operand preparation (split into parts, expand B)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int FORM>
__device__ __forceinline__ void split(float x, typename TcForm<FORM>::T* out, int64_t part_stride, float scale) {
    if constexpr (FORM == TC_FORM_FP16) {
        out[0] = __float2half_rn(x * scale);
    } else if constexpr (FORM == TC_FORM_3XTF32) {
        const float hi = tf32_rna(x);
        out[0] = hi;
        out[part_stride] = x - hi;
    } else {
        const __nv_bfloat16 b0 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(b0);
        const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(b1);
        out[0] = b0;
        out[part_stride] = b1;
        out[2 * part_stride] = __float2bfloat16_rn(r2);
    }
}

// A (complex, [R][K] if kmajor else [K][R]) -> parts [P][R][2K]
template <int FORM>
__global__ void k_prep_a(const float2* __restrict__ src, int64_t src_is, bool kmajor, typename TcForm<FORM>::T* dst,
                         int64_t dst_is_elems, int rb, int kb, const float* amax) {
    using T = typename TcForm<FORM>::T;
    const float sc = amax ? fp16_scale(amax[0]) : 1.f;
    const int64_t R = (int64_t)1 << rb, K = (int64_t)1 << kb;
    const int64_t item = blockIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * K) return;
    const int64_t r = idx >> kb, k = idx & (K - 1);
    const float2 v = src[item * src_is + (kmajor ? idx : k * R + r)];
    T* o = dst + item * dst_is_elems + r * 2 * K + 2 * k;
    const int64_t ps = R * 2 * K;
    split<FORM>(v.x, o, ps, sc);
    split<FORM>(v.y, o + 1, ps, sc);
}

// B (complex, [R][K] if kmajor else [K][R]) -> parts [P][2R][2K]:
// row 2r = (re, -im) per k, row 2r+1 = (im, re)
template <int FORM>
__global__ void k_prep_b(const float2* __restrict__ src, int64_t src_is, bool kmajor, typename TcForm<FORM>::T* dst,
                         int64_t dst_is_elems, int rb, int kb, const float* amax) {
    using T = typename TcForm<FORM>::T;
    const float sc = amax ? fp16_scale(amax[1]) : 1.f;
    const int64_t R = (int64_t)1 << rb, K = (int64_t)1 << kb;
    const int64_t item = blockIdx.y;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= R * K) return;
    const int64_t r = idx >> kb, k = idx & (K - 1);
    const float2 v = src[item * src_is + (kmajor ? idx : k * R + r)];
    T* o = dst + item * dst_is_elems + (2 * r) * 2 * K + 2 * k;
    const int64_t ps = 4 * R * K;
    split<FORM>(v.x, o, ps, sc);
    split<FORM>(-v.y, o + 1, ps, sc);
    split<FORM>(v.y, o + 2 * K, ps, sc);
    split<FORM>(v.x, o + 2 * K + 1, ps, sc);
}

// max |re|, |im| over an operand (all items); non-negative floats order like their bit patterns
__global__ void k_absmax(const float2* __restrict__ src, int64_t src_is, int64_t per_item, int64_t n_items,
                         float* out) {
    float m = 0.f;
    const int64_t total = per_item * n_items;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t item = i / per_item, e = i - item * per_item;
        const float2 v = src[item * src_is + e];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned int*)out, __float_as_uint(m));
}

// ------------------------------------------------------------------------------------------------
// PTX wrappers
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(s_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false after `limit` cycles, or early once any CTA of the
// launch has recorded an error (so one expired wait does not make every
// later CTA wait out its own limit)
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long long limit, const int* err) {
    if (mbar_try(b, parity)) return true;  // the common case: no clock read (it costs hundreds of cycles)
    const long long t0 = clock64();
    uint32_t spins = 0;
    while (!mbar_try(b, parity)) {
        if (clock64() - t0 > limit) return false;
        if ((++spins & 1023) == 0 && *(volatile const int*)err) return false;
    }
    return true;
}
// Wait for asynchronous work this CTA issued itself (TMA copies into its shared memory, MMAs into
// its TMEM) before it exits or frees TMEM.  Issued copies and MMAs always complete, so this wait is
// neither cut short by the launch-wide error flag nor by the caller's limit, which may be tiny: only
// by a fixed bound of about two seconds, so that even a stuck unit cannot keep the CTA forever.
constexpr long long kIssuedWaitCycles = 1ll << 32;
__device__ __forceinline__ void mbar_wait_issued(uint64_t* b, uint32_t parity) {
    if (mbar_try(b, parity)) return;
    const long long t0 = clock64();
    while (!mbar_try(b, parity))
        if (clock64() - t0 > kIssuedWaitCycles) return;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(s_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(s_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_addr(b))
                 : "memory");
}
// Partial in-register transpose of a 32 x 32 block held one row per lane (a[i] = element (lane, i)):
// register index bits 2..4 trade places with lane bits 0..2, one exchange with lane ^ 2^t per
// register pair for t = 0, 1, 2.  Afterwards a[4 r + c] of lane l is element (8 (l >> 3) + r,
// 4 (l & 7) + c): each register quad is four consecutive columns of one row, so one 16-byte store
// per quad from the 32 lanes writes four whole 128-byte row runs (three exchange rounds and eight
// stores instead of five rounds and 32 stores of a full transpose).
__device__ __forceinline__ void transpose_q4(float* a, int lane) {
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const int p = 2 + t;
        const bool up = (lane >> t) & 1;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if ((i >> p) & 1) continue;
            const int j = i | (1 << p);
            const float send = up ? a[i] : a[j];
            const float recv = __shfl_xor_sync(0xffffffffu, send, 1 << t);
            if (up) a[i] = recv;
            else a[j] = recv;
        }
    }
}

// 128-byte-swizzled K-major operand tile: rows of 128 B, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}
// the same for ROWB-byte rows: 128 (above) or 64 (64-byte swizzle, 8-row groups 512 B apart)
template <int ROWB>
__device__ __forceinline__ uint64_t sdesc_rows(uint32_t saddr) {
    if constexpr (ROWB == 128) {
        return sdesc(saddr);
    } else {
        static_assert(ROWB == 64, "64- or 128-byte rows");
        uint64_t d = 0;
        d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
        d |= (uint64_t)1 << 16;
        d |= (uint64_t)(512 >> 4) << 32;
        d |= (uint64_t)1 << 46;
        d |= (uint64_t)4 << 61;  // 64-byte swizzle
        return d;
    }
}
template <int FORM>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if constexpr (FORM == TC_FORM_3XTF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}
// tcgen05.st of 16 32-bit columns starting at taddr for this thread's TMEM lane (not waited)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])));
}
// 3xTF32 product with the A operand read from TMEM (row i in lane i, K along columns)
__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a_tmem, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(a_tmem), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcMaps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

// ------------------------------------------------------------------------------------------------
// the GEMM
// ------------------------------------------------------------------------------------------------
// B tile width BN = 128 or 256 rows of B' (64 or 128 complex columns of C): a 256-wide tile reads each A
// slab once for twice the columns (a quarter less operand traffic per flop), with 8 epilogue warps
// (two per TMEM lane quarter, 128 columns each) and two 256-column TMEM accumulators.  A stage holds
// ROWB bytes of K per row (a 128- or 64-byte swizzled slab): the 256-wide 3xTF32 tile takes 64-byte
// slabs, so that four 48 KB stages fit instead of two 96 KB ones and three stages load while the
// tensor core works on the fourth (with two, each load had one stage's MMA time to land).
template <int FORM, int BN, int ROWB = TC_ROWB>
struct TcTile {
    using F = TcForm<FORM>;
    static constexpr int EW = BN / 32;                             // epilogue warps
    static constexpr int THREADS = 64 + 32 * EW;
    static constexpr int NTB = 512 / BN;                          // TMEM accumulator buffers
    static constexpr uint32_t TILE_A = TC_BM * ROWB, TILE_B = BN * ROWB;
    static constexpr uint32_t STAGE_BYTES = F::NPA * TILE_A + F::NPB * TILE_B;
    static constexpr int STAGES = BN == 128 && ROWB == 128 ? F::STAGES : (int)(TC_SMEM_LIMIT / STAGE_BYTES);
};

template <int FORM, int BN, int ROWB>
__global__ void __launch_bounds__(TcTile<FORM, BN, ROWB>::THREADS, 1)
    k_gemm_tc(const __grid_constant__ TcMaps maps, float* __restrict__ C, int64_t c_is, int M, int N2, int K2,
              int tiles_n, int tiles, int64_t n_items, long long limit, int* err, const float* amax, int a_div,
              int b_div) {
    // persistent over (item, tile) jobs: job = blockIdx.x + t * gridDim.x, tiles of an item in order (n
    // fastest, so CTAs working at the same time share A's m tile in L2).  The stages of successive jobs
    // form one sequence for the ring, and the TMEM partials one sequence for the accumulators, so the
    // loads and MMAs of a job start while the epilogue still stores the job before.
    using F = TcForm<FORM>;
    using T = TcTile<FORM, BN, ROWB>;
    constexpr int BK = ROWB / F::EB;                    // K elements per stage
    constexpr int KSTEP = 32 / F::EB;                   // K elements per MMA (32 bytes)
    constexpr int SPD = TC_ROWB / ROWB;                 // stages per TMEM partial (128 bytes of K each)
    constexpr uint32_t TILE_A = T::TILE_A, TILE_B = T::TILE_B, STAGE_BYTES = T::STAGE_BYTES;
    constexpr int STAGES = T::STAGES, EW = T::EW;
    constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)F::FMT << 7) | ((uint32_t)F::FMT << 10) |
                               ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
    extern __shared__ uint8_t dyn[];
    constexpr int NTB = T::NTB;  // TMEM accumulator buffers (NTB x BN columns: all of TMEM)
    __shared__ uint64_t full[STAGES], empty[STAGES], tfull[NTB], tempty[NTB], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    if (*(volatile const int*)err) return;  // an earlier CTA of this contraction gave up
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (K2 + BK - 1) / BK, np = (nk + SPD - 1) / SPD;
    const int64_t jobs = (int64_t)tiles * n_items;
    const int64_t my_jobs = jobs > blockIdx.x ? (jobs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto job_of = [&](int64_t t, int* item, int* m0, int* n0) {
        const int64_t j = blockIdx.x + t * (int64_t)gridDim.x;
        *item = (int)(j / tiles);
        const int tile = (int)(j % tiles);
        *m0 = (tile / tiles_n) * TC_BM;
        *n0 = (tile % tiles_n) * BN;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NTB; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EW);  // one arrival per epilogue warp
        }
        mbar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_slot)),
                     "r"(NTB * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: ring slot s and its phase advance one step per stage across the jobs
        int64_t issued = 0;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int64_t t = 0; t < my_jobs && ok; ++t) {
            int item, m0, n0;
            job_of(t, &item, &m0, &n0);
            for (int it = 0; it < nk; ++it) {
                if (!mbar_wait(&empty[s], ph ^ 1u, limit, err) || *(volatile int*)&abort_flag) {
                    atomicExch(&abort_flag, 1);
                    ok = false;
                    break;
                }
                mbar_expect_tx(&full[s], STAGE_BYTES);
                uint8_t* st = base + s * STAGE_BYTES;
#pragma unroll
                for (int p = 0; p < F::NPA; ++p)
                    tma_load_3d(st + p * TILE_A, &maps.a[p], it * BK, m0, item / a_div, &full[s]);
#pragma unroll
                for (int p = 0; p < F::NPB; ++p)
                    tma_load_3d(st + F::NPA * TILE_A + p * TILE_B, &maps.b[p], it * BK, n0, item / b_div, &full[s]);
                ++issued;
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        // every copy issued lands before the CTA goes away (immediate unless a wait gave up: the
        // consumers then did not see every stage)
        for (int64_t g = (issued > STAGES ? issued - STAGES : 0); g < issued; ++g)
            mbar_wait_issued(&full[g % STAGES], (uint32_t)((g / STAGES) & 1));
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: the SPD stages of a partial accumulate (fresh) into TMEM buffer b; partials of
        // successive jobs take the buffers in turn
        bool ok = true;
        int s = 0;
        uint32_t ph = 0;  // ring slot and phase
        int64_t pj = 0;   // partials so far: the next one goes to buffer pj % NTB, its use pj / NTB
        for (int64_t t = 0; t < my_jobs && ok; ++t)
        for (int it = 0; it < nk && ok; ++it) {
            const bool first = it % SPD == 0, last = it % SPD == SPD - 1 || it == nk - 1;
            const int b = (int)(pj % NTB);
            const int64_t u = pj / NTB;
            if (!mbar_wait(&full[s], ph, limit, err) ||
                (first && u > 0 && !mbar_wait(&tempty[b], (uint32_t)((u - 1) & 1), limit, err)) ||
                *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t st = s_addr(base + s * STAGE_BYTES);
            const uint32_t d = tmem + b * BN;
            // the smallest part products first, the main one (p = 0) last: each MMA joins the FP32
            // accumulator with a truncated alignment, so correction terms summed while it is still
            // small keep their bits, and only the main product's MMAs add at full magnitude
#pragma unroll
            for (int p = F::NPROD - 1; p >= 0; --p) {
#pragma unroll
                for (int kk = 0; kk < BK / KSTEP; ++kk) {
                    const uint64_t ad = sdesc_rows<ROWB>(st + F::pa(p) * TILE_A + kk * 32);
                    const uint64_t bd = sdesc_rows<ROWB>(st + F::NPA * TILE_A + F::pb(p) * TILE_B + kk * 32);
                    mma<FORM>(d, ad, bd, IDESC, (!first || p != F::NPROD - 1 || kk != 0) ? 1u : 0u);
                }
            }
            tc_commit(&empty[s]);
            if (++s == STAGES) {
                s = 0;
                ph ^= 1u;
            }
            if (last) {
                tc_commit(&tfull[b]);
                ++pj;
            }
        }
        // the MMAs this thread issued finish before TMEM is freed, also when the epilogue warps gave
        // up and stopped waiting for them
        tc_commit(&drain);
        mbar_wait_issued(&drain, 0);
    } else if (warp >= 2) {
        // epilogue: TMEM lanes 32 (warp % 4) .. + 31 are rows of the tile, warp w drains columns
        // 128 h .. + 127 (h = (w - 2) / 4).  The tensor cores' FP32 accumulation drifts toward zero over
        // long sums, so each partial over 128 bytes of K (one stage, or two of 64-byte slabs: <= 24 MMAs)
        // is added to an FP32 total in registers with round-to-nearest instead of accumulating K in TMEM.
        const int q = warp & 3, h = (warp - 2) >> 2;
        float tot[128];
        bool ok = true;
        int64_t pj = 0;  // partials so far (buffer pj % NTB, its use pj / NTB)
        for (int64_t t = 0; t < my_jobs && ok; ++t) {
#pragma unroll
            for (int j = 0; j < 128; ++j) tot[j] = 0.f;
            for (int j = 0; j < np; ++j, ++pj) {
                const int b = (int)(pj % NTB);
                const uint32_t par = (uint32_t)((pj / NTB) & 1);
                // one decision per warp: the TMEM loads below are warp-wide (.sync.aligned)
                const bool go = mbar_wait(&tfull[b], par, limit, err) && !*(volatile int*)&abort_flag;
                if (!__all_sync(0xffffffffu, go)) {
                    atomicExch(&abort_flag, 1);
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + b * BN + 128 * h + 32 * c, v);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) tot[32 * c + jj] += v[jj];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&tempty[b])) : "memory");
            }
            if (!ok) break;
            if (amax) {  // undo the FP16 per-tensor scales (powers of two: exact)
                const float inv = 1.f / (fp16_scale(amax[0]) * fp16_scale(amax[1]));
#pragma unroll
                for (int j = 0; j < 128; ++j) tot[j] *= inv;
            }
            // tiles are whole (rows and columns multiples of 128; see tc_shape_ok)
            int item, m0, n0;
            job_of(t, &item, &m0, &n0);
            float* cb = C + (int64_t)item * c_is + (int64_t)(m0 + 32 * q + ((lane >> 3) << 3)) * N2 + n0 + 128 * h +
                        ((lane & 7) << 2);
#pragma unroll
            for (int b32 = 0; b32 < 4; ++b32) {
                float* tt = tot + 32 * b32;
                transpose_q4(tt, lane);
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    *(float4*)(cb + (int64_t)r * N2 + 32 * b32) =
                        make_float4(tt[4 * r], tt[4 * r + 1], tt[4 * r + 2], tt[4 * r + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) atomicExch(err, QX_ETIMEOUT);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NTB * BN) : "memory");
    }
}

// ------------------------------------------------------------------------------------------------
// 3xTF32 straight from the complex64 operands: TMA brings raw 128-byte K slabs
// of A (128 rows) and of B (BN/2 complex rows) into landing slots.  Converter
// warps split A into hi and lo and store both into TMEM (row = lane), and build
// both parts of the expanded B' (rows 2n = (re, -im), 2n+1 = (im, re)) in an
// MMA slot in shared memory; the MMAs read A from TMEM and B' through
// descriptors.  Keeping A out of shared memory halves the tensor core's
// shared-memory reads, which with the split traffic bound this kernel; B' row
// r puts chunk j at (j ^ (r % 8)), the 128-byte swizzle.  No separate split
// pass, no extra HBM traffic.
// Warps: 0 TMA, 1 TMEM + MMA, 2..9 drain TMEM (warp w reads TMEM lanes
// 32 (w % 4) and half of the columns), 10..13 convert slabs ahead of the MMAs
// (warp w writes the A rows of TMEM lanes 32 (w % 4)).
// ------------------------------------------------------------------------------------------------
// warps 0 TMA, 1 and 14 MMA (even / odd stages), 2-9 drain, 10-13 convert
constexpr int TC2_THREADS = 480, TC2_CONV = 128;
// k_gemm_tc2 adds a second converter group (warps 15-18): the groups convert alternate stages
constexpr int TC2_THREADS2 = TC2_THREADS + TC2_CONV;
// Two rings.  Landing slots take the raw TMA slabs: A (16 KB, 128 rows) and B (BN/2 complex
// rows).  MMA slots hold what the tensor core reads: B' hi and B' lo (BN rows each) in shared
// memory, A hi and A lo (2 x 32 columns) in TMEM after the NTB accumulator buffers.  A landing
// slot is free again as soon as it is converted, so several slabs per SM stay in flight while the
// tensor core works on earlier ones.
template <int BN>
struct Tc2 {
    static constexpr uint32_t A = 16384, BRAW = (BN / 2) * 128, BP = BN * 128;
    static constexpr uint32_t LAND = A + BRAW;          // landing slot: raw A, raw B
    static constexpr uint32_t OFF_BLO = BP, MSLOT = 2 * BP;  // MMA slot: B' hi, B' lo
    static constexpr int NL = BN == 128 ? 5 : 8, NM = BN == 128 ? 3 : 4;
    static constexpr uint32_t SMEM = NL * LAND + NM * MSLOT;  // slots are multiples of 1024 bytes
    static constexpr int NTB = 2;                      // accumulator buffers
    static constexpr uint32_t ACOL = NTB * BN;         // first TMEM column of the A parts (64 per MMA slot)
    static constexpr uint32_t TMEM_COLS = 512;
};

__device__ __forceinline__ void split4(float4 v, float4& hi, float4& lo) {
    hi = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
    lo = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
}

// Convert a landed slab pair (`land`) into an MMA slot (`ms`, TMEM columns ahi / ahi + 32) with the
// converter warps: thread (quarter qq, lane) splits row 32 qq + lane of A into TMEM (row = lane),
// then the threads ct = 0 .. TC2_CONV - 1 build B' hi / lo in shared memory.
template <int BN>
__device__ __forceinline__ void tc2_convert(const uint8_t* land, uint8_t* ms, int ct, uint32_t tmem, int qq,
                                            int lane, uint32_t ahi, bool with_a) {
    using L = Tc2<BN>;
    const int r = 32 * qq + lane;
    const uint32_t lanes = (uint32_t)(32 * qq) << 16;
    // every shared-memory load of the slab first (A row and B chunks), then the splits and stores:
    // the loads overlap instead of waiting behind each other's stores
    constexpr int NBC = (BN / 2) * 8 / TC2_CONV;
    float4 va[8], vb[NBC];
    if (with_a) {
#pragma unroll
        for (int j = 0; j < 8; ++j) va[j] = *(const float4*)(land + r * 128 + ((j ^ (r & 7)) << 4));
    }
#pragma unroll
    for (int i = 0; i < NBC; ++i) {
        const int c = ct + TC2_CONV * i;
        const int n = c >> 3, j = c & 7;
        vb[i] = *(const float4*)(land + L::A + n * 128 + ((j ^ (n & 7)) << 4));
    }
#pragma unroll
    for (int h = 0; h < 2 && with_a; ++h) {  // 16 columns (four 16-byte chunks) at a time
        float hi[16], lo[16];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float4 vh, vl;
            split4(va[4 * h + jj], vh, vl);
            hi[4 * jj] = vh.x; hi[4 * jj + 1] = vh.y; hi[4 * jj + 2] = vh.z; hi[4 * jj + 3] = vh.w;
            lo[4 * jj] = vl.x; lo[4 * jj + 1] = vl.y; lo[4 * jj + 2] = vl.z; lo[4 * jj + 3] = vl.w;
        }
        tmem_st16(tmem + lanes + ahi + 16 * h, hi);
        tmem_st16(tmem + lanes + ahi + 32 + 16 * h, lo);
    }
#pragma unroll
    for (int i = 0; i < NBC; ++i) {  // B: BN/2 rows x 8 chunks of 16 bytes
        const int c = ct + TC2_CONV * i;
        const int n = c >> 3, j = c & 7;
        const float4 v = vb[i];
        const float4 r0 = make_float4(v.x, -v.y, v.z, -v.w);  // row 2n: re, -im
        const float4 r1 = make_float4(v.y, v.x, v.w, v.z);    // row 2n+1: im, re
        const int ra = 2 * n, rb = 2 * n + 1;
        const uint32_t oa = ra * 128 + ((j ^ (ra & 7)) << 4), ob = rb * 128 + ((j ^ (rb & 7)) << 4);
        float4 hi, lo;
        split4(r0, hi, lo);
        *(float4*)(ms + oa) = hi;
        *(float4*)(ms + L::OFF_BLO + oa) = lo;
        split4(r1, hi, lo);
        *(float4*)(ms + ob) = hi;
        *(float4*)(ms + L::OFF_BLO + ob) = lo;
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int BN>
__global__ void __launch_bounds__(TC2_THREADS2, 1)
    k_gemm_tc2(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               float* __restrict__ C, int64_t c_is, int M, int N2, int K2, int tiles_n, int tiles, int64_t n_items,
               int a_div, int b_div, int keep_a, int pack2, long long limit, int* err) {
    // persistent over (pair, tile) jobs: job = blockIdx.x + t * gridDim.x; the
    // k-stages of successive jobs form one sequence g = t * nk + it, so both
    // rings stay full across tile boundaries.
    // keep_a (A shared by the a_div items of a slice, all of A's k-stages fit in TMEM after the
    // accumulators): A is split into TMEM at columns ACOL + 64 it for stage it, and a job whose A
    // (slice, m tile) is the one its CTA's previous job used loads and splits only B.  The job order
    // stays the same, so neighbouring CTAs still work on neighbouring items.
    // pack2 (N = BN / 4 complex per item, B dense per item, both items of a job on the same A): a job
    // covers items 2 i and 2 i + 1 side by side, B's rows of both come in one TMA box (B read as one
    // [items x N][2K] matrix), and drain half h writes item 2 i + h.
    using L = Tc2<BN>;
    constexpr int BK = 32;  // TF32 elements per stage (one 128-byte slab)
    constexpr int NL = L::NL, NM = L::NM, NTB = L::NTB;
    constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(TC_BM >> 4) << 24);
    extern __shared__ uint8_t dyn[];
    __shared__ uint64_t full[NL], lfree[NL], mfull[NM], mfree[NM], tfull[NTB], tempty[NTB], drain[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    if (*(volatile const int*)err) return;
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    auto land = [&](int l) { return base + l * L::LAND; };
    auto mslot = [&](int m) { return base + NL * L::LAND + m * L::MSLOT; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K2 / BK;
    const int64_t jobs = (int64_t)tiles * n_items;
    const int64_t my_jobs = jobs > blockIdx.x ? (jobs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_jobs * nk;
    // job t of this CTA: its item, tile origin and the key of its A (its A item and m tile)
    auto job_of = [&](int64_t t, int64_t* item, int* m0, int* n0, int64_t* akey) {
        const int64_t j = blockIdx.x + t * (int64_t)gridDim.x;
        *item = pack2 ? 2 * (j / tiles) : j / tiles;
        const int tile = (int)(j % tiles);
        *m0 = (tile / tiles_n) * TC_BM;
        *n0 = (tile % tiles_n) * BN;  // row of B'; raw B row n0 / 2
        *akey = (*item / a_div) * (tiles / tiles_n) + tile / tiles_n;
    };
    // Every role walks the stages g = 0, 1, ... with counters (ring slot and its phase, stage within
    // the job, job) advanced by one step at a time: 64-bit divisions per stage would cost more
    // cycles than a stage's MMAs.  A job is decoded (job_of) once, at its first or last stage.
    if (threadIdx.x == 0) {
        for (int s = 0; s < NL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&lfree[s], TC2_CONV / 32);
        }
        for (int s = 0; s < NM; ++s) {
            mbar_init(&mfull[s], TC2_CONV / 32);
            mbar_init(&mfree[s], 1);
        }
        for (int b = 0; b < NTB; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(&drain[0], 1);
        mbar_init(&drain[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_slot)),
                     "r"(L::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        int64_t issued = 0, t = 0, item = 0, akey = 0, prev_key = -1;
        int l = 0, it = 0, m0 = 0, n0 = 0, ia = 0, ib = 0;
        uint32_t lph = 0;
        bool with_a = true;
        for (int64_t g = 0; g < total; ++g) {
            if (!mbar_wait(&lfree[l], lph ^ 1u, limit, err) || *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (it == 0) {
                job_of(t, &item, &m0, &n0, &akey);
                with_a = !keep_a || akey != prev_key;
                prev_key = akey;
                ia = (int)(item / a_div);
                ib = (int)(item / b_div);
            }
            mbar_expect_tx(&full[l], with_a ? L::LAND : L::BRAW);  // raw A (unless kept) and raw B
            if (with_a) tma_load_3d(land(l), &mapA, it * BK, m0, ia, &full[l]);
            if (pack2) tma_load_3d(land(l) + L::A, &mapB, it * BK, (int)item * (BN / 4), 0, &full[l]);
            else tma_load_3d(land(l) + L::A, &mapB, it * BK, n0 >> 1, ib, &full[l]);
            ++issued;
            if (++it == nk) {
                it = 0;
                ++t;
            }
            if (++l == NL) {
                l = 0;
                lph ^= 1u;
            }
        }
        // the copies in flight land before the CTA exits (immediate unless a wait gave up)
        for (int64_t g = (issued > NL ? issued - NL : 0); g < issued; ++g)
            mbar_wait_issued(&full[g % NL], (uint32_t)((g / NL) & 1));
    } else if ((warp == 1 || warp == 14) && lane == 0) {
        // two issuers, even and odd stages: while one waits for its next stage (barrier waits, fence,
        // commits cost about as much as issuing the stage's MMAs), the other keeps the tensor pipe busy;
        // stage g accumulates into TMEM buffer g % 2, i.e. each issuer owns one buffer
        const int who = warp == 1 ? 0 : 1;
        static_assert(NTB == 2 && NM > 2, "issuer g owns accumulator buffer g % 2 and steps two MMA slots");
        const int b = who;
        bool ok = true;
        int m = who, it = who % nk;
        uint32_t mph = 0;
        int64_t u = 0;  // g / NTB
        for (int64_t g = who; g < total && ok; g += 2, ++u) {
            if (!mbar_wait(&mfull[m], mph, limit, err) ||
                (u > 0 && !mbar_wait(&tempty[b], (uint32_t)((u - 1) & 1), limit, err)) || *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t st = s_addr(mslot(m));
            const uint32_t d = tmem + b * BN;
            const uint32_t acol = L::ACOL + 64 * (uint32_t)(keep_a ? it : m);
            // the correction products first, the main one last (see k_gemm_tc: each MMA joins the FP32
            // accumulator with a truncated alignment)
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {
                const uint32_t ahi = tmem + acol + 8 * kk, alo = ahi + 32;
                const uint64_t bhi = sdesc(st + kk * 32), blo = sdesc(st + L::OFF_BLO + kk * 32);
                mma_tf32_ta(d, ahi, blo, IDESC, kk != 0);
                mma_tf32_ta(d, alo, bhi, IDESC, 1);
            }
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk)
                mma_tf32_ta(d, tmem + acol + 8 * kk, sdesc(st + kk * 32), IDESC, 1);
            tc_commit(&mfree[m]);
            tc_commit(&tfull[b]);
            m += 2;
            if (m >= NM) {
                m -= NM;
                mph ^= 1u;
            }
            it += 2;
            while (it >= nk) it -= nk;
        }
        // the MMAs this thread issued finish before TMEM is freed, also when the drain or converter
        // warps gave up and stopped waiting for them
        tc_commit(&drain[who]);
        mbar_wait_issued(&drain[who], 0);
    } else if ((warp >= 10 && warp <= 13) || (warp >= 15 && !keep_a)) {
        // converters: landing slot -> MMA slot, ahead of the MMAs; warp w writes the A rows of TMEM
        // lanes 32 (w % 4).  Two groups (warps 10-13 and 15-18) convert the even and the odd stages:
        // one group's conversion of a stage takes about twice its MMAs.  With a kept A only the first
        // group runs (its decision to overwrite the kept A waits on the two stages before, in order).
        const int grp = warp >= 15 ? 1 : 0, ng = keep_a ? 1 : 2;
        const int ct = threadIdx.x - (grp ? 480 : 320);
        int l = grp, m = grp, it = grp % nk;
        uint32_t lph = 0, mph = 0;
        int64_t t = grp / nk, prev_key = -1;
        bool with_a = true;
        for (int64_t g = grp; g < total; g += ng) {
            // one decision per warp: the TMEM stores of the conversion are warp-wide (.sync.aligned)
            const bool go = mbar_wait(&full[l], lph, limit, err) && mbar_wait(&mfree[m], mph ^ 1u, limit, err) &&
                            !*(volatile int*)&abort_flag;
            if (!__all_sync(0xffffffffu, go)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (keep_a && it == 0) {
                int64_t item, akey;
                int m0, n0;
                job_of(t, &item, &m0, &n0, &akey);
                with_a = akey != prev_key;
                prev_key = akey;
                if (with_a && g > 0) {
                    // a new A overwrites the kept one: every MMA of the earlier stages must be done
                    // (each stage's commit to its accumulator buffer covers the MMAs its issuer issued
                    // before it)
                    bool ok = true;
                    for (int64_t p = g - 1; p >= 0 && p >= g - 2 && ok; --p)
                        ok = mbar_wait(&tfull[p & 1], (uint32_t)((p >> 1) & 1), limit, err);
                    if (!__all_sync(0xffffffffu, ok)) {
                        atomicExch(&abort_flag, 1);
                        break;
                    }
                }
            }
            tc_fence_after();  // the MMAs that last read this MMA slot have completed (mfree)
            tc2_convert<BN>(land(l), mslot(m), ct, tmem, warp & 3, lane,
                            L::ACOL + 64 * (uint32_t)(keep_a ? it : m), with_a);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&lfree[l])) : "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&mfull[m])) : "memory");
            }
            it += ng;
            while (it >= nk) {
                it -= nk;
                ++t;
            }
            l += ng;  // ng <= 2 < NL, NM
            if (l >= NL) {
                l -= NL;
                lph ^= 1u;
            }
            m += ng;
            if (m >= NM) {
                m -= NM;
                mph ^= 1u;
            }
        }
    } else if (warp >= 2 && warp <= 9) {
        // drain: TMEM lanes 32 (warp % 4), columns (BN / 2) ((warp - 2) / 4) .. + BN / 2 - 1
        const int q = warp & 3, half = (warp - 2) >> 2;
        float tot[BN / 2];
#pragma unroll
        for (int j = 0; j < BN / 2; ++j) tot[j] = 0.f;
        int64_t g = 0;
        for (int64_t t = 0; t < my_jobs; ++t) {
            bool ok = true;
            for (int it = 0; it < nk; ++it, ++g) {
                const int b = (int)(g & 1);
                // one decision per warp: the TMEM loads below are warp-wide (.sync.aligned)
                const bool go = mbar_wait(&tfull[b], (uint32_t)((g >> 1) & 1), limit, err) &&
                                !*(volatile int*)&abort_flag;
                if (!__all_sync(0xffffffffu, go)) {
                    atomicExch(&abort_flag, 1);
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < BN / 32; ++c) {  // 16 columns at a time (registers: 608 threads)
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + b * BN + (BN / 2) * half + 16 * c, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) tot[16 * c + j] += v[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&tempty[b])) : "memory");
            }
            if (!ok) break;
            // the job's last stage is in: write its tile, start the next total
            int64_t item, akey;
            int m0, n0;
            job_of(t, &item, &m0, &n0, &akey);
            // lane r holds row 32 q + r; each 32-column block is partly transposed across the warp so
            // that every 16-byte store instruction writes whole 128-byte runs of four rows
            float* cb = (pack2 ? C + (item + half) * c_is : C + item * c_is + n0 + (BN / 2) * half) +
                        (int64_t)(m0 + 32 * q + ((lane >> 3) << 3)) * N2 + ((lane & 7) << 2);
#pragma unroll
            for (int b32 = 0; b32 < BN / 64; ++b32) {
                float* t = tot + 32 * b32;
                transpose_q4(t, lane);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    *(float4*)(cb + (int64_t)r * N2 + 32 * b32) =
                        make_float4(t[4 * r], t[4 * r + 1], t[4 * r + 2], t[4 * r + 3]);
                    t[4 * r] = t[4 * r + 1] = t[4 * r + 2] = t[4 * r + 3] = 0.f;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) atomicExch(err, QX_ETIMEOUT);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TMEM_COLS) : "memory");
    }
}

// ------------------------------------------------------------------------------------------------
// The direct 3xTF32 kernel for a B that every item of the launch shares (an invariant operand, such
// as a gate-sized tensor applied to a large per-slice one) and that one 128-column tile covers
// (2N = BN), with at most Tc2Kb::MAXK k-stages: B' (hi and lo) of every stage is built once per CTA
// and stays in shared memory, so per job TMA brings only A and the converter warps only split A into
// TMEM -- half the converter work and no B traffic per job.  Roles and rings otherwise as in
// k_gemm_tc2 with one converter group: warps 0 TMA, 1 and 14 MMA (even / odd stages), 2-9 drain,
// 10-13 convert.
// ------------------------------------------------------------------------------------------------
template <int BN>
struct Tc2Kb {
    static constexpr uint32_t A = 16384, BRAW = (BN / 2) * 128, BP = BN * 128;
    static constexpr uint32_t LAND = A;                      // landing slot: a raw A slab (first: raw B)
    static constexpr uint32_t OFF_BLO = BP, BSLOT = 2 * BP;  // resident B' of one stage: hi, lo
    static constexpr int MAXK = BN == 128 ? 4 : 8;           // k-stages whose B' stays resident
    static constexpr int NL = 5, NM = 3;                     // landing slots; A positions in TMEM
    static constexpr uint32_t SMEM = NL * LAND + MAXK * BSLOT;
    static constexpr int NTB = 2;                            // accumulator buffers
    static constexpr uint32_t ACOL = NTB * BN;               // first TMEM column of the A parts
    static constexpr uint32_t TMEM_COLS = 512;
};

// B' hi / lo of one stage from its raw slab (BN/2 complex rows of 16 K values): row 2n = (re, -im),
// row 2n+1 = (im, re), 128-byte swizzled as the MMA descriptors read it
template <int BN>
__device__ __forceinline__ void tc2kb_build_b(const uint8_t* braw, uint8_t* bs, int ct) {
    using L = Tc2Kb<BN>;
    constexpr int NBC = (BN / 2) * 8 / TC2_CONV;
    float4 vb[NBC];
#pragma unroll
    for (int i = 0; i < NBC; ++i) {
        const int c = ct + TC2_CONV * i;
        const int n = c >> 3, j = c & 7;
        vb[i] = *(const float4*)(braw + n * 128 + ((j ^ (n & 7)) << 4));
    }
#pragma unroll
    for (int i = 0; i < NBC; ++i) {
        const int c = ct + TC2_CONV * i;
        const int n = c >> 3, j = c & 7;
        const float4 v = vb[i];
        const float4 r0 = make_float4(v.x, -v.y, v.z, -v.w);
        const float4 r1 = make_float4(v.y, v.x, v.w, v.z);
        const int ra = 2 * n, rb = 2 * n + 1;
        const uint32_t oa = ra * 128 + ((j ^ (ra & 7)) << 4), ob = rb * 128 + ((j ^ (rb & 7)) << 4);
        float4 hi, lo;
        split4(r0, hi, lo);
        *(float4*)(bs + oa) = hi;
        *(float4*)(bs + L::OFF_BLO + oa) = lo;
        split4(r1, hi, lo);
        *(float4*)(bs + ob) = hi;
        *(float4*)(bs + L::OFF_BLO + ob) = lo;
    }
}

// A hi / lo of one slab into TMEM: thread (quarter qq, lane) splits row 32 qq + lane into TMEM lane
// 32 qq + lane, columns ahi (hi) and ahi + 32 (lo)
__device__ __forceinline__ void tc2kb_split_a(const uint8_t* araw, uint32_t tmem, int qq, int lane, uint32_t ahi) {
    const int r = 32 * qq + lane;
    const uint32_t lanes = (uint32_t)(32 * qq) << 16;
    float4 va[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) va[j] = *(const float4*)(araw + r * 128 + ((j ^ (r & 7)) << 4));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float hi[16], lo[16];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float4 vh, vl;
            split4(va[4 * h + jj], vh, vl);
            hi[4 * jj] = vh.x; hi[4 * jj + 1] = vh.y; hi[4 * jj + 2] = vh.z; hi[4 * jj + 3] = vh.w;
            lo[4 * jj] = vl.x; lo[4 * jj + 1] = vl.y; lo[4 * jj + 2] = vl.z; lo[4 * jj + 3] = vl.w;
        }
        tmem_st16(tmem + lanes + ahi + 16 * h, hi);
        tmem_st16(tmem + lanes + ahi + 32 + 16 * h, lo);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared memory, completing
// on an mbarrier's transaction count
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s_addr(dst)),
                 "l"(src), "r"(bytes), "r"(s_addr(bar))
                 : "memory");
}

// A hi / lo of one gathered slab (GA): row r's 16 K entries sit at entries lrow + lk[j] of the slot
__device__ __forceinline__ void tc2kb_split_a_local(const uint8_t* araw, int lrow, const int16_t* lk, uint32_t tmem,
                                                    int qq, int lane, uint32_t ahi) {
    const uint32_t lanes = (uint32_t)(32 * qq) << 16;
    float2 a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = *(const float2*)(araw + 8 * (lrow + lk[j]));
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float hi[16], lo[16];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float4 vh, vl;
            const int c = 4 * h + jj;
            split4(make_float4(a[2 * c].x, a[2 * c].y, a[2 * c + 1].x, a[2 * c + 1].y), vh, vl);
            hi[4 * jj] = vh.x; hi[4 * jj + 1] = vh.y; hi[4 * jj + 2] = vh.z; hi[4 * jj + 3] = vh.w;
            lo[4 * jj] = vl.x; lo[4 * jj + 1] = vl.y; lo[4 * jj + 2] = vl.z; lo[4 * jj + 3] = vl.w;
        }
        tmem_st16(tmem + lanes + ahi + 16 * h, hi);
        tmem_st16(tmem + lanes + ahi + 32 + 16 * h, lo);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// GA (A gathered in place, ag): the producer thread brings each stage's 128 x 16 tile of A with
// ag.nblk bulk copies of its contiguous blocks (in A's stored order) instead of one TMA box, and the
// converters read row r's entries at ag.lrow[r] + ag.lk[j] of the slot.
template <int BN, bool GA>
__global__ void __launch_bounds__(TC2_THREADS, 1)
    k_gemm_tc2kb(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 float* __restrict__ C, int64_t c_is, int N2, int K2, int tiles, int64_t n_items, int a_div,
                 long long limit, int* err, const float2* __restrict__ ga_base, int64_t ga_is, int ga_mb,
                 const __grid_constant__ AGather ag) {
    // persistent over (item, m tile) jobs: job = blockIdx.x + t * gridDim.x; B' of every k-stage is
    // resident, A's stages of successive jobs form one sequence g = t * nk + it.  The landing ring
    // first takes the nk raw B slabs, then the A slabs: both producer and converters walk that one
    // sequence (q = nk + g for A stage g).
    using L = Tc2Kb<BN>;
    constexpr int BK = 32;
    constexpr int NL = L::NL, NM = L::NM, NTB = L::NTB;
    constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(TC_BM >> 4) << 24);
    extern __shared__ uint8_t dyn[];
    __shared__ uint64_t full[NL], lfree[NL], mfull[NM], mfree[NM], tfull[NTB], tempty[NTB], drain[2], bready;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int16_t s_lrow[GA ? 128 : 1], s_lk[GA ? 16 : 1];  // GA: the slot offsets of rows / K entries
    if (*(volatile const int*)err) return;
    uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    auto land = [&](int l) { return base + l * L::LAND; };
    auto bslot = [&](int it) { return base + NL * L::LAND + it * L::BSLOT; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K2 / BK;  // <= L::MAXK (checked by the host)
    const int64_t jobs = (int64_t)tiles * n_items;
    const int64_t my_jobs = jobs > blockIdx.x ? (jobs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_jobs * nk;
    auto job_of = [&](int64_t t, int64_t* item, int* m0) {
        const int64_t j = blockIdx.x + t * (int64_t)gridDim.x;
        *item = j / tiles;
        *m0 = (int)(j % tiles) * TC_BM;
    };
    if (GA) {
        if (threadIdx.x < 128) s_lrow[threadIdx.x] = ag.lrow[threadIdx.x];
        if (threadIdx.x < 16) s_lk[threadIdx.x] = ag.lk[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < NL; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&lfree[s], TC2_CONV / 32);
        }
        for (int s = 0; s < NM; ++s) {
            mbar_init(&mfull[s], TC2_CONV / 32);
            mbar_init(&mfree[s], 1);
        }
        for (int b = 0; b < NTB; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);
        }
        mbar_init(&drain[0], 1);
        mbar_init(&drain[1], 1);
        mbar_init(&bready, TC2_CONV / 32);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(&tmem_slot)),
                     "r"(L::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (GA && warp == 0 && lane == 0) {
        int64_t issued = 0, t = 0, item = 0;
        int l = 0, it = 0, m0 = 0;
        uint32_t lph = 0;
        bool ok = true;
        for (int s = 0; s < nk && ok; ++s) {  // the raw B slab of every stage (TMA)
            if (!mbar_wait(&lfree[l], lph ^ 1u, limit, err) || *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            mbar_expect_tx(&full[l], L::BRAW);
            tma_load_3d(land(l), &mapB, s * BK, 0, 0, &full[l]);
            ++issued;
            if (++l == NL) {
                l = 0;
                lph ^= 1u;
            }
        }
        const uint32_t blk_bytes = 8u << ag.run;
        int64_t rowb = 0;
        for (int64_t g = 0; g < total && ok; ++g) {
            if (!mbar_wait(&lfree[l], lph ^ 1u, limit, err) || *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (it == 0) {  // the job's tile base in A: its item and row bits 7 and up
                job_of(t, &item, &m0);
                rowb = (item / a_div) * ga_is;
                for (int b = 7; b < ga_mb; ++b)
                    if ((m0 >> b) & 1) rowb += (int64_t)1 << ag.mpos[b];
            }
            int64_t tb = rowb;  // and the stage's K bits 4 and up
            for (int b = 0; (it >> b) > 0; ++b)
                if ((it >> b) & 1) tb += (int64_t)1 << ag.kpos[4 + b];
            mbar_expect_tx(&full[l], L::A);
            for (int b = 0; b < ag.nblk; ++b)
                bulk_load(land(l) + (size_t)b * blk_bytes, ga_base + tb + ag.blk_off[b], blk_bytes, &full[l]);
            ++issued;
            if (++it == nk) {
                it = 0;
                ++t;
            }
            if (++l == NL) {
                l = 0;
                lph ^= 1u;
            }
        }
        // the copies in flight land before the CTA exits (immediate unless a wait gave up)
        for (int64_t q = (issued > NL ? issued - NL : 0); q < issued; ++q)
            mbar_wait_issued(&full[q % NL], (uint32_t)((q / NL) & 1));
    } else if (!GA && warp == 0 && lane == 0) {
        int64_t issued = 0, t = 0, item = 0;
        int l = 0, it = 0, m0 = 0;
        uint32_t lph = 0;
        bool ok = true;
        for (int s = 0; s < nk && ok; ++s) {  // the raw B slab of every stage
            if (!mbar_wait(&lfree[l], lph ^ 1u, limit, err) || *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            mbar_expect_tx(&full[l], L::BRAW);
            tma_load_3d(land(l), &mapB, s * BK, 0, 0, &full[l]);
            ++issued;
            if (++l == NL) {
                l = 0;
                lph ^= 1u;
            }
        }
        for (int64_t g = 0; g < total && ok; ++g) {
            if (!mbar_wait(&lfree[l], lph ^ 1u, limit, err) || *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (it == 0) job_of(t, &item, &m0);
            mbar_expect_tx(&full[l], L::A);
            tma_load_3d(land(l), &mapA, it * BK, m0, (int)(item / a_div), &full[l]);
            ++issued;
            if (++it == nk) {
                it = 0;
                ++t;
            }
            if (++l == NL) {
                l = 0;
                lph ^= 1u;
            }
        }
        // the copies in flight land before the CTA exits (immediate unless a wait gave up)
        for (int64_t q = (issued > NL ? issued - NL : 0); q < issued; ++q)
            mbar_wait_issued(&full[q % NL], (uint32_t)((q / NL) & 1));
    } else if ((warp == 1 || warp == 14) && lane == 0) {
        const int who = warp == 1 ? 0 : 1;
        const int b = who;
        bool ok = mbar_wait(&bready, 0, limit, err) && !*(volatile int*)&abort_flag;
        if (!ok) atomicExch(&abort_flag, 1);
        int m = who, it = who % nk;
        uint32_t mph = 0;
        int64_t u = 0;
        for (int64_t g = who; g < total && ok; g += 2, ++u) {
            if (!mbar_wait(&mfull[m], mph, limit, err) ||
                (u > 0 && !mbar_wait(&tempty[b], (uint32_t)((u - 1) & 1), limit, err)) || *(volatile int*)&abort_flag) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t st = s_addr(bslot(it));
            const uint32_t d = tmem + b * BN;
            const uint32_t acol = L::ACOL + 64 * (uint32_t)m;
            // the correction products first, the main one last (see k_gemm_tc)
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk) {
                const uint32_t ahi = tmem + acol + 8 * kk, alo = ahi + 32;
                const uint64_t bhi = sdesc(st + kk * 32), blo = sdesc(st + L::OFF_BLO + kk * 32);
                mma_tf32_ta(d, ahi, blo, IDESC, kk != 0);
                mma_tf32_ta(d, alo, bhi, IDESC, 1);
            }
#pragma unroll
            for (int kk = 0; kk < BK / 8; ++kk)
                mma_tf32_ta(d, tmem + acol + 8 * kk, sdesc(st + kk * 32), IDESC, 1);
            tc_commit(&mfree[m]);
            tc_commit(&tfull[b]);
            m += 2;
            if (m >= NM) {
                m -= NM;
                mph ^= 1u;
            }
            it += 2;
            while (it >= nk) it -= nk;
        }
        // the MMAs this thread issued finish before TMEM is freed
        tc_commit(&drain[who]);
        mbar_wait_issued(&drain[who], 0);
    } else if (warp >= 10 && warp <= 13) {
        // converters: first B' of every stage into its resident slot, then A of every stage into TMEM
        const int ct = threadIdx.x - 320;
        int l = 0, m = 0;
        uint32_t lph = 0, mph = 0;
        bool ok = true;
        for (int s = 0; s < nk; ++s) {
            const bool go = mbar_wait(&full[l], lph, limit, err) && !*(volatile int*)&abort_flag;
            if (!__all_sync(0xffffffffu, go)) {
                atomicExch(&abort_flag, 1);
                ok = false;
                break;
            }
            tc2kb_build_b<BN>(land(l), bslot(s), ct);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&lfree[l])) : "memory");
            if (++l == NL) {
                l = 0;
                lph ^= 1u;
            }
        }
        if (ok && lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&bready)) : "memory");
        for (int64_t g = 0; g < total && ok; ++g) {
            // one decision per warp: the TMEM stores of the split are warp-wide (.sync.aligned)
            const bool go = mbar_wait(&full[l], lph, limit, err) && mbar_wait(&mfree[m], mph ^ 1u, limit, err) &&
                            !*(volatile int*)&abort_flag;
            if (!__all_sync(0xffffffffu, go)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            tc_fence_after();  // the MMAs that last read this A position have completed (mfree)
            if (GA)
                tc2kb_split_a_local(land(l), s_lrow[32 * (warp & 3) + lane], s_lk, tmem, warp & 3, lane,
                                    L::ACOL + 64 * (uint32_t)m);
            else
                tc2kb_split_a(land(l), tmem, warp & 3, lane, L::ACOL + 64 * (uint32_t)m);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&lfree[l])) : "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&mfull[m])) : "memory");
            }
            if (++l == NL) {
                l = 0;
                lph ^= 1u;
            }
            if (++m == NM) {
                m = 0;
                mph ^= 1u;
            }
        }
    } else if (warp >= 2 && warp <= 9) {
        // drain: TMEM lanes 32 (warp % 4), columns (BN / 2) ((warp - 2) / 4) .. + BN / 2 - 1
        const int q = warp & 3, half = (warp - 2) >> 2;
        float tot[BN / 2];
#pragma unroll
        for (int j = 0; j < BN / 2; ++j) tot[j] = 0.f;
        int64_t g = 0;
        for (int64_t t = 0; t < my_jobs; ++t) {
            bool ok = true;
            for (int it = 0; it < nk; ++it, ++g) {
                const int b = (int)(g & 1);
                // one decision per warp: the TMEM loads below are warp-wide (.sync.aligned)
                const bool go = mbar_wait(&tfull[b], (uint32_t)((g >> 1) & 1), limit, err) &&
                                !*(volatile int*)&abort_flag;
                if (!__all_sync(0xffffffffu, go)) {
                    atomicExch(&abort_flag, 1);
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < BN / 64; ++c) {
                    float v[32];
                    tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + b * BN + (BN / 2) * half + 32 * c, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) tot[32 * c + j] += v[j];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_addr(&tempty[b])) : "memory");
            }
            if (!ok) break;
            int64_t item;
            int m0;
            job_of(t, &item, &m0);
            float* cb = C + item * c_is + (BN / 2) * half + (int64_t)(m0 + 32 * q + ((lane >> 3) << 3)) * N2 +
                        ((lane & 7) << 2);
#pragma unroll
            for (int b32 = 0; b32 < BN / 64; ++b32) {
                float* tt = tot + 32 * b32;
                transpose_q4(tt, lane);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    *(float4*)(cb + (int64_t)r * N2 + 32 * b32) =
                        make_float4(tt[4 * r], tt[4 * r + 1], tt[4 * r + 2], tt[4 * r + 3]);
                    tt[4 * r] = tt[4 * r + 1] = tt[4 * r + 2] = tt[4 * r + 3] = 0.f;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0) atomicExch(err, QX_ETIMEOUT);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TMEM_COLS) : "memory");
    }
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

template <int FORM>
static bool make_map(CUtensorMap* m, const void* base, int64_t k2, int64_t rows, int64_t items, int64_t item_bytes,
                     int box_rows = TC_BM, int rowb = TC_ROWB) {
    using F = TcForm<FORM>;
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)k2, (cuuint64_t)rows, (cuuint64_t)items};
    const cuuint64_t strides[2] = {(cuuint64_t)(k2 * F::EB), (cuuint64_t)item_bytes};
    const cuuint32_t box[3] = {(cuuint32_t)(rowb / F::EB), (cuuint32_t)box_rows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = F::EB == 4                 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : FORM == TC_FORM_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    return fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              rowb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Items of an operand a launch reads: one for an item stride of 0 (the same
// tensor for every item), n_items / div otherwise; and the divisor the kernel
// applies to its item index (INT_MAX turns every index into item 0).
static int64_t distinct_items(int64_t is, int div, int64_t n_items) {
    if (!is) return 1;
    div = div < 1 ? 1 : div;
    return (n_items + div - 1) / div;
}
static int item_div(int64_t is, int div) { return !is ? INT_MAX : div < 1 ? 1 : div; }

int tc_parts_a(int form) { return form == TC_FORM_3XTF32 ? 2 : form == TC_FORM_FP16 ? 1 : 3; }
int tc_parts_b(int form) { return tc_parts_a(form); }
int tc_elem_bytes(int form) { return form == TC_FORM_3XTF32 ? 4 : 2; }
int tc_products(int form) { return form == TC_FORM_3XTF32 ? 3 : form == TC_FORM_FP16 ? 1 : 6; }

template <int FORM>
static cudaError_t run_prep(const TcArgs& g, cudaStream_t st) {
    using F = TcForm<FORM>;
    using T = typename F::T;
    const int64_t M = 1ll << g.mb, N = 1ll << g.nb, K = 1ll << g.kb;
    const float* amax = nullptr;
    if constexpr (FORM == TC_FORM_FP16) {
        if (!g.amax) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(g.amax, 0, 2 * sizeof(float), st);
        if (e != cudaSuccess) return e;
        const int64_t na = distinct_items(g.a_is, g.a_div, g.n_items), nb_ = distinct_items(g.b_is, g.b_div, g.n_items);
        k_absmax<<<(unsigned)std::min<int64_t>((M * K * na + 255) / 256, 4096), 256, 0, st>>>(g.a, g.a_is, M * K, na,
                                                                                               g.amax);
        k_absmax<<<(unsigned)std::min<int64_t>((N * K * nb_ + 255) / 256, 4096), 256, 0, st>>>(g.b, g.b_is, N * K,
                                                                                                nb_, g.amax + 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        amax = g.amax;
    }
    // each distinct operand item is split once
    dim3 grid((unsigned)((M * K + 255) / 256), (unsigned)distinct_items(g.a_is, g.a_div, g.n_items));
    k_prep_a<FORM><<<grid, 256, 0, st>>>(g.a, g.a_is, g.a_kmajor, (T*)g.pa, g.pa_is_bytes / F::EB, g.mb, g.kb, amax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid2((unsigned)((N * K + 255) / 256), (unsigned)distinct_items(g.b_is, g.b_div, g.n_items));
    k_prep_b<FORM><<<grid2, 256, 0, st>>>(g.b, g.b_is, g.b_kmajor, (T*)g.pb, g.pb_is_bytes / F::EB, g.nb, g.kb, amax);
    return cudaGetLastError();
}

template <int FORM, int BN, int ROWB = TC_ROWB>
static cudaError_t run_gemm_bn(const TcArgs& g, cudaStream_t st) {
    using F = TcForm<FORM>;
    using T = TcTile<FORM, BN, ROWB>;
    const int64_t M = 1ll << g.mb, N = 1ll << g.nb, K = 1ll << g.kb;
    const int64_t pa_part = M * 2 * K, pb_part = 4 * N * K;  // elements per part
    TcMaps maps;
    memset(&maps, 0, sizeof maps);
    for (int p = 0; p < F::NPA; ++p)
        if (!make_map<FORM>(&maps.a[p], (const char*)g.pa + p * pa_part * F::EB, 2 * K, M,
                            distinct_items(g.a_is, g.a_div, g.n_items), g.pa_is_bytes, TC_BM, ROWB))
            return cudaErrorInvalidValue;
    for (int p = 0; p < F::NPB; ++p)
        if (!make_map<FORM>(&maps.b[p], (const char*)g.pb + p * pb_part * F::EB, 2 * K, 2 * N,
                            distinct_items(g.b_is, g.b_div, g.n_items), g.pb_is_bytes, BN, ROWB))
            return cudaErrorInvalidValue;
    const int smem = T::STAGES * (int)T::STAGE_BYTES + 1024;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static uint64_t attr_done[4] = {0, 0, 0, 0};  // per device bit
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 256 && !((attr_done[dev >> 6] >> (dev & 63)) & 1)) {
            e = cudaFuncSetAttribute(k_gemm_tc<FORM, BN, ROWB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            attr_done[dev >> 6] |= 1ull << (dev & 63);
        }
    }
    const int tiles_m = (int)(M / TC_BM), tiles_n = (int)(2 * N / BN);
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    const int64_t jobs = (int64_t)tiles_m * tiles_n * g.n_items;
    const unsigned grid = (unsigned)std::min<int64_t>(jobs, sms);  // persistent: one CTA per SM (shared memory)
    k_gemm_tc<FORM, BN, ROWB><<<grid, T::THREADS, smem, st>>>(maps, (float*)g.c, g.c_is * 2, (int)M, (int)(2 * N),
                                                        (int)(2 * K), tiles_n, tiles_m * tiles_n, g.n_items,
                                                        g.limit, g.err,
                                                        FORM == TC_FORM_FP16 ? (const float*)g.amax : nullptr,
                                                        item_div(g.a_is, g.a_div), item_div(g.b_is, g.b_div));
    return cudaGetLastError();
}

// 256-wide B tiles where whole ones cover 2N and two pipeline stages of them fit (3xTF32 with 64-byte
// slabs, FP16), else 128-wide
template <int FORM>
static cudaError_t run_gemm(const TcArgs& g, cudaStream_t st) {
    if (((2ll << g.nb) % 256) == 0) {
        if constexpr (FORM == TC_FORM_3XTF32) return run_gemm_bn<FORM, 256, 64>(g, st);
        else if constexpr (TcTile<FORM, 256>::STAGES >= 2) return run_gemm_bn<FORM, 256>(g, st);
    }
    return run_gemm_bn<FORM, 128>(g, st);
}

static bool map_raw(CUtensorMap* m, const void* base, int64_t k2, int64_t rows, int64_t items, int64_t item_bytes,
                    int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)k2, (cuuint64_t)rows, (cuuint64_t)items};
    const cuuint64_t strides[2] = {(cuuint64_t)(k2 * 4), (cuuint64_t)item_bytes};
    const cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
static cudaError_t run_tc2(const TcArgs& g, cudaStream_t st, bool pack2 = false) {
    using L = Tc2<BN>;
    const int64_t M = 1ll << g.mb, N = 1ll << g.nb, K = 1ll << g.kb;
    const bool abc = g.a_is == 0, bbc = g.b_is == 0;
    CUtensorMap ma, mb;
    if (!map_raw(&ma, g.a, 2 * K, M, distinct_items(g.a_is, g.a_div, g.n_items), abc ? M * K * 8 : g.a_is * 8, TC_BM))
        return cudaErrorInvalidValue;
    if (pack2 ? !map_raw(&mb, g.b, 2 * K, N * g.n_items, 1, N * g.n_items * K * 8, BN / 2)
              : !map_raw(&mb, g.b, 2 * K, N, distinct_items(g.b_is, g.b_div, g.n_items), bbc ? N * K * 8 : g.b_is * 8,
                         BN / 2))
        return cudaErrorInvalidValue;
    const int smem = (int)L::SMEM + 1024;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static uint64_t done[4] = {0, 0, 0, 0};
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 256 && !((done[dev >> 6] >> (dev & 63)) & 1)) {
            e = cudaFuncSetAttribute(k_gemm_tc2<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            done[dev >> 6] |= 1ull << (dev & 63);
        }
    }
    const int tiles_m = (int)(M / TC_BM), tiles_n = pack2 ? 1 : (int)(2 * N / BN);
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    const int64_t job_items = pack2 ? g.n_items / 2 : g.n_items;  // a packed job covers two items
    const int64_t jobs = (int64_t)tiles_m * tiles_n * job_items;
    const unsigned grid = (unsigned)std::min<int64_t>(jobs, sms);  // one CTA per SM (shared memory)
    // A shared by the items of a slice, and all of its k-stages fit in TMEM after the accumulators:
    // keep it across the jobs of a CTA
    const int nk = (int)(2 * K / 32);
    const int keep_a = g.a_is && g.a_div > 1 && L::ACOL + 64 * nk <= L::TMEM_COLS;
    k_gemm_tc2<BN><<<grid, TC2_THREADS2, smem, st>>>(ma, mb, (float*)g.c, g.c_is * 2, (int)M, (int)(2 * N),
                                                    (int)(2 * K), tiles_n, tiles_m * tiles_n, job_items,
                                                    item_div(g.a_is, g.a_div), item_div(g.b_is, g.b_div), keep_a,
                                                    pack2 ? 1 : 0, g.limit, g.err);
    return cudaGetLastError();
}

template <int BN, bool GA>
static cudaError_t run_tc2kb(const TcArgs& g, cudaStream_t st) {
    using L = Tc2Kb<BN>;
    const int64_t M = 1ll << g.mb, N = 1ll << g.nb, K = 1ll << g.kb;
    CUtensorMap ma, mb;
    memset(&ma, 0, sizeof ma);
    if (!GA && !map_raw(&ma, g.a, 2 * K, M, distinct_items(g.a_is, g.a_div, g.n_items),
                        g.a_is ? g.a_is * 8 : M * K * 8, TC_BM))
        return cudaErrorInvalidValue;
    if (!map_raw(&mb, g.b, 2 * K, N, 1, N * K * 8, BN / 2)) return cudaErrorInvalidValue;
    const int smem = (int)L::SMEM + 1024;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static uint64_t done[4] = {0, 0, 0, 0};
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 256 && !((done[dev >> 6] >> (dev & 63)) & 1)) {
            e = cudaFuncSetAttribute(k_gemm_tc2kb<BN, GA>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            done[dev >> 6] |= 1ull << (dev & 63);
        }
    }
    const int tiles = (int)(M / TC_BM);
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    const int64_t jobs = (int64_t)tiles * g.n_items;
    const unsigned grid = (unsigned)std::min<int64_t>(jobs, sms);  // one CTA per SM (shared memory)
    k_gemm_tc2kb<BN, GA><<<grid, TC2_THREADS, smem, st>>>(ma, mb, (float*)g.c, g.c_is * 2, (int)(2 * N),
                                                          (int)(2 * K), tiles, g.n_items, item_div(g.a_is, g.a_div),
                                                          g.limit, g.err, g.a, g.a_is, g.mb, g.ag);
    return cudaGetLastError();
}

bool agather_tile(AGather* g, int mb, int kb) {
    if (mb < 7 || kb < 4) return false;
    int tpos[11];
    for (int i = 0; i < 7; ++i) tpos[i] = g->mpos[i];
    for (int i = 0; i < 4; ++i) tpos[7 + i] = g->kpos[i];
    int sorted[11];
    std::copy(tpos, tpos + 11, sorted);
    std::sort(sorted, sorted + 11);
    int run = 0;
    while (run < 11 && sorted[run] == run) ++run;
    if (run < 8) return false;
    // local position of a tile bit: its own below run, else run + its rank among the others
    int local[11];
    for (int i = 0; i < 11; ++i) {
        if (tpos[i] < run) {
            local[i] = tpos[i];
        } else {
            int rk = 0;
            for (int j = 0; j < 11; ++j) rk += sorted[j] >= run && sorted[j] < tpos[i];
            local[i] = run + rk;
        }
    }
    g->run = run;
    g->nblk = 1 << (11 - run);
    for (int b = 0; b < g->nblk; ++b) {
        int64_t o = 0;
        for (int i = 0; i < 11 - run; ++i)
            if ((b >> i) & 1) o += (int64_t)1 << sorted[run + i];
        g->blk_off[b] = o;
    }
    for (int r = 0; r < 128; ++r) {
        int v = 0;
        for (int i = 0; i < 7; ++i)
            if ((r >> i) & 1) v += 1 << local[i];
        g->lrow[r] = (int16_t)v;
    }
    for (int j = 0; j < 16; ++j) {
        int v = 0;
        for (int i = 0; i < 4; ++i)
            if ((j >> i) & 1) v += 1 << local[7 + i];
        g->lk[j] = (int16_t)v;
    }
    return true;
}

cudaError_t launch_tc2_gemm(const TcArgs& g, cudaStream_t st) {
    if (!(g.mb >= 7 && g.nb >= 5 && g.kb >= 4 && g.n_items > 0 && g.n_items <= 65535)) return cudaErrorInvalidValue;
    if ((!g.a_kmajor && !g.ag.on) || !g.b_kmajor) return cudaErrorInvalidValue;
    if (g.ag.on) {  // A gathered where it is stored: only the resident-B' kernel reads it so
        if (!tc2_resident_b(g) || g.ag.run < 8 || g.ag.run > 11 || g.ag.nblk != 1 << (11 - g.ag.run))
            return cudaErrorInvalidValue;
        return g.nb == 6 ? run_tc2kb<128, true>(g, st) : run_tc2kb<64, true>(g, st);
    }
    // N = 32 complex per item: two items per 128-column tile when their B rows are contiguous and
    // they read the same A (shared, or per slice with an even number of items per slice)
    const int64_t NK = (1ll << g.nb) * (1ll << g.kb);
    const bool pack2 = g.nb == 5 && g.b_is == NK && g.b_div <= 1 && g.n_items % 2 == 0 &&
                       (g.a_is == 0 || (g.a_div > 1 && g.a_div % 2 == 0));
    if (pack2) return run_tc2<128>(g, st, true);
    if (tc2_resident_b(g)) return g.nb == 6 ? run_tc2kb<128, false>(g, st) : run_tc2kb<64, false>(g, st);
    return g.nb >= 6 ? run_tc2<128>(g, st) : run_tc2<64>(g, st);
}

// B shared by every item, one tile wide (2N = BN), its B' small enough to stay resident, and A not
// shared by several items (else the kept-A mode of k_gemm_tc2 saves more): k_gemm_tc2kb builds B' once
// per CTA.  (Never with pack2, which needs a B per item.)
bool tc2_resident_b(const TcArgs& g) {
    const int nk = (int)((2ll << g.kb) / 32);
    const bool a_kept = g.a_is && g.a_div > 1;
    if (g.b_is != 0 || a_kept) return false;
    return (g.nb == 6 && nk <= Tc2Kb<128>::MAXK) || (g.nb == 5 && nk <= Tc2Kb<64>::MAXK);
}

static bool tc_shape_ok(const TcArgs& g) {
    // whole 128 x 128 tiles and whole 128-byte K slabs (see the plan compiler)
    return g.mb >= 7 && g.nb >= 6 && g.kb >= 5 && g.n_items > 0 && g.n_items <= 65535;
}

cudaError_t launch_tc_prep(int form, const TcArgs& g, cudaStream_t st) {
    if (!tc_shape_ok(g)) return cudaErrorInvalidValue;
    if (form == TC_FORM_3XTF32) return run_prep<TC_FORM_3XTF32>(g, st);
    if (form == TC_FORM_BF16X3) return run_prep<TC_FORM_BF16X3>(g, st);
    if (form == TC_FORM_FP16) return run_prep<TC_FORM_FP16>(g, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tc_gemm(int form, const TcArgs& g, cudaStream_t st) {
    if (!tc_shape_ok(g)) return cudaErrorInvalidValue;
    if (form == TC_FORM_3XTF32) return run_gemm<TC_FORM_3XTF32>(g, st);
    if (form == TC_FORM_BF16X3) return run_gemm<TC_FORM_BF16X3>(g, st);
    if (form == TC_FORM_FP16) return run_gemm<TC_FORM_FP16>(g, st);
    return cudaErrorInvalidValue;
}

static_assert(TcTile<TC_FORM_3XTF32, 256, 64>::STAGES == 4 && TcTile<TC_FORM_FP16, 256>::STAGES == 4, "stages");
static_assert(TcTile<TC_FORM_3XTF32, 256, 64>::STAGES * TcTile<TC_FORM_3XTF32, 256, 64>::STAGE_BYTES <= TC_SMEM_LIMIT,
              "smem");
static_assert(TcTile<TC_FORM_FP16, 256>::STAGES * TcTile<TC_FORM_FP16, 256>::STAGE_BYTES <= TC_SMEM_LIMIT, "smem");
static_assert(TcForm<TC_FORM_3XTF32>::STAGES * 4 * TC_BM * TC_ROWB + 1024 <= TC_SMEM_LIMIT + 1024, "smem");
static_assert(TcForm<TC_FORM_BF16X3>::STAGES * 6 * TC_BM * TC_ROWB + 1024 <= TC_SMEM_LIMIT + 1024, "smem");
static_assert(TcForm<TC_FORM_FP16>::STAGES * 2 * TC_BM * TC_ROWB + 1024 <= TC_SMEM_LIMIT + 1024, "smem");
static_assert(Tc2<128>::SMEM + 1024 <= 227 * 1024 - 512, "smem");
static_assert(Tc2<64>::SMEM + 1024 <= 227 * 1024 - 512, "smem");
static_assert(Tc2Kb<128>::SMEM + 1024 <= 227 * 1024 - 512, "smem");
static_assert(Tc2Kb<64>::SMEM + 1024 <= 227 * 1024 - 512, "smem");
static_assert(Tc2Kb<128>::ACOL + Tc2Kb<128>::NM * 64 <= Tc2Kb<128>::TMEM_COLS, "tmem");
static_assert(Tc2Kb<64>::ACOL + Tc2Kb<64>::NM * 64 <= Tc2Kb<64>::TMEM_COLS, "tmem");
static_assert(Tc2Kb<128>::BRAW <= Tc2Kb<128>::LAND && Tc2Kb<64>::BRAW <= Tc2Kb<64>::LAND, "raw B fits a slot");
static_assert(Tc2<128>::ACOL + Tc2<128>::NM * 64 <= Tc2<128>::TMEM_COLS, "tmem");
static_assert(Tc2<64>::ACOL + Tc2<64>::NM * 64 <= Tc2<64>::TMEM_COLS, "tmem");

}  // namespace qx
