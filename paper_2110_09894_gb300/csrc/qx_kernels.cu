// CUDA kernels of the contraction path (sm_103a): the index permutation of
// the TTGT scheme, the complex64 SIMT GEMM, the gather contraction for steps
// with a small operand, and the FP64 compensated cross-slice sum.
//
// Paper background: contracting a network is a sequence of pairwise
// contractions mapped to matrix multiplications on the GPU (Sec. IV-A, the
// three levels of parallelism); the primitives needed are contract, reshape,
// permute, slice and recombine (Sec. III-B).  Slicing (Eq. 2) turns into
// per-item address offsets here, recombination into the FP64 sum.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "qx_internal.h"

namespace qx {

__device__ __forceinline__ int64_t fix_offset(const Operand& op, const ItemCtx& ic, int64_t item) {
    // the items of one launch number fewer than 2^16 (kMaxBatchItems): one 32-bit division splits an
    // item into its slice and bitstring within the batch
    const uint32_t i32 = (uint32_t)item, nb = (uint32_t)ic.n_b;
    const uint32_t sl = (op.per_slice || op.n_fix) ? i32 / nb : 0u;
    int64_t off = (int64_t)(op.per_slice ? sl : i32) * op.item_stride;
    if (op.n_fix) {
        const int64_t s = ic.s0 + sl;
        const int64_t b = ic.b0 + (i32 - sl * nb);
        for (int f = 0; f < op.n_fix; ++f) {
            const int src = op.fix_src[f];
            const int64_t v = src >= 0 ? ((s >> src) & 1) : (int64_t)(ic.bits[b * ic.n_qubits + (-src - 1)] & 1);
            off += v * op.fix_stride[f];
        }
    }
    return off;
}

// address offset of the set bits of v placed at positions pos[0..] (bit b of v -> 2^pos[b])
__device__ __forceinline__ int64_t place_bits(int64_t v, const int8_t* pos) {
    int64_t off = 0;
    while (v) {
        const int b = __ffsll((long long)v) - 1;
        off += (int64_t)1 << pos[b];
        v &= v - 1;
    }
    return off;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------------------------------------
// Bit permutation through a shared-memory tile of up to 2^12 entries.  The
// tile spans the 6 lowest input positions and the 6 lowest output bits (plus
// more output bits up to 12), so reads walk it in input order in contiguous
// runs of 64 entries (512 bytes) and writes walk it in output order in runs of
// 64 again; one float2 of padding per 32 entries.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ int pad32(int j) { return j + (j >> 5); }

void perm_tables(const PermDesc& d, PermTables* tb) {
    constexpr int LO = kPermLoBits;
    const int t = d.t;
    for (int j = 0; j < (1 << LO); ++j) {
        int64_t a = 0, b = 0, c = 0, e = 0;
        int ml = 0, mh = 0;
        for (int i = 0; i < LO; ++i) {
            if (!((j >> i) & 1)) continue;
            if (i < t) {
                a += (int64_t)1 << d.in_pos[d.tile_in[i]];
                c += (int64_t)1 << d.tile_out[i];
            }
            if (i + LO < t) {
                b += (int64_t)1 << d.in_pos[d.tile_in[i + LO]];
                e += (int64_t)1 << d.tile_out[i + LO];
            }
        }
        // where output-ordered tile bit i sits in the input-ordered tile index
        for (int i = 0; i < t; ++i) {
            int r = 0;
            for (int k = 0; k < t; ++k)
                if (d.tile_in[k] == d.tile_out[i]) r = k;
            if (i < LO) {
                if ((j >> i) & 1) ml |= 1 << r;
            } else if ((j >> (i - LO)) & 1) {
                mh |= 1 << r;
            }
        }
        tb->in_lo[j] = a;
        tb->in_hi[j] = b;
        tb->out_lo[j] = c;
        tb->out_hi[j] = e;
        tb->map_lo[j] = ml;
        tb->map_hi[j] = mh;
    }
    for (int i = 0; i < kMaxRank; ++i) {
        tb->outer_in[i] = i < d.n_outer ? (int64_t)1 << d.in_pos[d.outer[i]] : 0;
        tb->outer_out[i] = i < d.n_outer ? (int64_t)1 << d.outer[i] : 0;
    }
}

// Grid-stride over (pair, tile) jobs: the tables are loaded into shared memory
// once per CTA, each job moves one tile.  Software pipeline: the next job's
// tile is loaded into registers while the current one is stored, so every
// thread keeps its loads in flight during its stores.
constexpr int kPermThreads = 256, kPermPer = (1 << kPermTileBits) / kPermThreads;
__global__ void __launch_bounds__(kPermThreads, 4) k_permute(const PermDesc d, const PermTables tb, const ItemCtx ic,
                                                          float2* __restrict__ out, int64_t out_is, int64_t n_items) {
    constexpr int LO = kPermLoBits, LM = (1 << LO) - 1;
    __shared__ float2 tile[(1 << kPermTileBits) + (1 << kPermTileBits) / 32];
    __shared__ int64_t s_in[128], s_out[128];
    __shared__ int s_map[128];
    const int tid = threadIdx.x;
    if (tid < 64) {
        s_in[tid] = tb.in_lo[tid];
        s_in[64 + tid] = tb.in_hi[tid];
        s_out[tid] = tb.out_lo[tid];
        s_out[64 + tid] = tb.out_hi[tid];
        s_map[tid] = tb.map_lo[tid];
        s_map[64 + tid] = tb.map_hi[tid];
    }
    __syncthreads();
    const int n = 1 << d.t;
    const int64_t tiles = (int64_t)1 << d.n_outer;
    const int64_t jobs = tiles * n_items;
    // input and output bases of a job (pair, tile of the outer bits)
    auto bases = [&](int64_t job, int64_t* ib, int64_t* ob) {
        const int64_t item = job >> d.n_outer;
        uint64_t u = (uint64_t)(job & (tiles - 1));
        *ib = fix_offset(d.in, ic, item);
        *ob = item * out_is;
        while (u) {
            const int i = __ffsll((long long)u) - 1;
            *ib += tb.outer_in[i];
            *ob += tb.outer_out[i];
            u &= u - 1;
        }
    };
    float2 v[kPermPer];
    auto load = [&](int64_t job) {
        int64_t ib, ob;
        bases(job, &ib, &ob);
        const float2* __restrict__ src = d.in.base + ib;
#pragma unroll
        for (int k = 0; k < kPermPer; ++k) {
            const int j = tid + kPermThreads * k;
            if (j < n) v[k] = src[s_in[j & LM] + s_in[64 + (j >> LO)]];
        }
    };
    int64_t job = blockIdx.x;
    if (job < jobs) load(job);
    while (job < jobs) {
#pragma unroll
        for (int k = 0; k < kPermPer; ++k) {
            const int j = tid + kPermThreads * k;
            if (j < n) tile[pad32(j)] = v[k];
        }
        __syncthreads();
        int64_t ib, ob;
        bases(job, &ib, &ob);
        const int64_t next = job + gridDim.x;
        if (next < jobs) load(next);
        float2* __restrict__ dst = out + ob;
        for (int j = tid; j < n; j += kPermThreads)
            dst[s_out[j & LM] + s_out[64 + (j >> LO)]] = tile[pad32(s_map[j & LM] | s_map[64 + (j >> LO)])];
        __syncthreads();
        job = next;
    }
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 152;
    }
    return n;
}

cudaError_t launch_permute(const PermDesc& d, const ItemCtx& ic, int64_t n_items, float2* out, int64_t out_is,
                           cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (n_items > kMaxBatchItems || ic.n_items > kMaxBatchItems) return cudaErrorInvalidValue;  // fix_offset
    PermTables tb;
    perm_tables(d, &tb);
    const int64_t jobs = ((int64_t)1 << d.n_outer) * n_items;
    if (d.t > kPermTileBits) return cudaErrorInvalidValue;
    const int64_t grid = std::min<int64_t>(jobs, (int64_t)sm_count() * 4);  // 4 resident CTAs per SM (registers)
    k_permute<<<(unsigned)grid, kPermThreads, 0, st>>>(d, tb, ic, out, out_is, n_items);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Gather contraction against a small operand Y held in shared memory.  One
// thread per free index m of the large operand X: it loads the 2^k entries
// X[m, k] straight from X's native layout (no permute) and writes the 2^n
// outputs C[m, n].  Used for the many steps that absorb a gate-sized tensor.
// ---------------------------------------------------------------------------------------------
template <int KB>
__global__ void __launch_bounds__(256) k_small(const __grid_constant__ SmallDesc d, const ItemCtx ic, float2* __restrict__ out,
                                               int64_t out_is, int64_t n_items, int ppc, int y_shared) {
    // A CTA owns 256 rows of one pair (ppc = 1), or ppc whole pairs of 2^mb < 256 rows each, whose
    // products are then contiguous (out_is = 2^(mb + nb)).  The small operand of each of its pairs
    // (one copy when every pair reads the same one) is staged in shared memory, then the output stage.
    extern __shared__ float4 small_dyn[];  // 16-byte aligned
    float2* ys = (float2*)small_dyn;
    __shared__ int64_t kofs[1 << kSmallMaxK];
    __shared__ int64_t cofs[1 << kSmallMaxN];  // placed product: offset of each column n
    __shared__ int8_t rpos[kMaxRank];          // placed product: position of each row bit
    const int nb = d.nb;
    const int nn = 1 << nb;
    const int yn = (1 << KB) << nb;   // entries of one small operand
    const int yst = (yn + 1) & ~1;    // its stride in shared memory (even: 16-byte aligned pairs)
    const int ny = y_shared ? 1 : ppc;
    const int64_t M = (int64_t)1 << d.mb;
    const int64_t item0 = (int64_t)blockIdx.y * ppc;
    if (d.om.on) {
        for (int n = threadIdx.x; n < nn; n += blockDim.x) cofs[n] = place_bits(n, d.om.pos);
        for (int b = threadIdx.x; b < d.mb; b += blockDim.x) rpos[b] = d.om.pos[nb + b];
    }
    for (int idx = threadIdx.x; idx < ny * yn; idx += blockDim.x) {
        const int p = idx / yn, e = idx - p * yn;
        if (item0 + p >= n_items) continue;
        const int kk = e >> nb, n = e & (nn - 1);
        int64_t a = fix_offset(d.y, ic, item0 + p);
        for (int i = 0; i < KB; ++i)
            if ((kk >> i) & 1) a += (int64_t)1 << d.yk_pos[i];
        for (int i = 0; i < nb; ++i)
            if ((n >> i) & 1) a += (int64_t)1 << d.yn_pos[i];
        ys[p * yst + e] = d.y.base[a];
    }
    if (threadIdx.x < (1 << KB)) {
        int64_t a = 0;
        for (int i = 0; i < KB; ++i)
            if ((threadIdx.x >> i) & 1) a += (int64_t)1 << d.xk_pos[i];
        kofs[threadIdx.x] = a;
    }
    __syncthreads();
    const int p = ppc > 1 ? (int)(threadIdx.x >> d.mb) : 0;
    const int64_t item = item0 + p;
    const int64_t m = ppc > 1 ? (int64_t)(threadIdx.x & (M - 1)) : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float2* __restrict__ yp = ys + (y_shared ? 0 : p * yst);
    // outputs of the CTA's rows form one block: stage them (row stride nn + 1) and store coalesced
    float2* stage = ys + ny * yst;
    const bool staged = !d.om.on && nb <= 4 && blockDim.x == 256;
    if (m < M && item < n_items) {
        int64_t xa = m;
        for (int h = 0; h < d.n_holes; ++h) {
            const int q = d.holes[h];
            xa = ((xa >> q) << (q + 1)) | (xa & (((int64_t)1 << q) - 1));
        }
        const float2* __restrict__ xp = d.x.base + fix_offset(d.x, ic, item) + xa;
        float2 a[1 << KB];
#pragma unroll
        for (int kk = 0; kk < (1 << KB); ++kk) a[kk] = xp[kofs[kk]];
        float2* __restrict__ cp = out + item * out_is + (d.om.on ? place_bits(m, rpos) : (m << nb));
        if (nn >= 2) {
            // two outputs per pass: their Y entries are adjacent, one 16-byte shared load per k; a placed
            // product with column bit 0 at address bit 0 stores both with one 16-byte store (the other
            // address bits of n and m are >= 1, so the pair starts on 16 bytes)
            const bool pair16 = d.om.on && d.om.pos[0] == 0;
            const float4* __restrict__ ys4 = (const float4*)yp;
            for (int n = 0; n < nn; n += 2) {
                float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int kk = 0; kk < (1 << KB); ++kk) {
                    const float4 y = ys4[(kk * nn + n) >> 1];
                    cfma(acc0, a[kk], make_float2(y.x, y.y));
                    cfma(acc1, a[kk], make_float2(y.z, y.w));
                }
                if (staged) {
                    stage[threadIdx.x * (nn + 1) + n] = acc0;
                    stage[threadIdx.x * (nn + 1) + n + 1] = acc1;
                } else if (d.om.on) {
                    if (pair16) {  // column bit 0 at address bit 0: outputs n, n + 1 are adjacent
                        *(float4*)(cp + cofs[n]) = make_float4(acc0.x, acc0.y, acc1.x, acc1.y);
                    } else {
                        cp[cofs[n]] = acc0;
                        cp[cofs[n + 1]] = acc1;
                    }
                } else {
                    *(float4*)(cp + n) = make_float4(acc0.x, acc0.y, acc1.x, acc1.y);
                }
            }
        } else {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < (1 << KB); ++kk) cfma(acc, a[kk], yp[kk]);
            if (staged) stage[threadIdx.x * (nn + 1)] = acc;
            else cp[d.om.on ? cofs[0] : 0] = acc;
        }
    }
    if (!staged) return;
    __syncthreads();
    // the block: rows r0 .. of pair item0 (ppc = 1), or every row of pairs item0 .. (ppc > 1)
    int64_t rows;
    float2* __restrict__ dst;
    if (ppc > 1) {
        const int64_t np = n_items - item0 < ppc ? n_items - item0 : ppc;
        rows = np * M;
        dst = out + item0 * out_is;
    } else {
        const int64_t r0 = (int64_t)blockIdx.x * blockDim.x;
        rows = M - r0 < 256 ? M - r0 : 256;
        dst = out + item0 * out_is + (r0 << nb);
    }
    const int64_t cnt = rows * nn;
    for (int i = threadIdx.x; i < cnt; i += 256) dst[i] = stage[(i >> nb) * (nn + 1) + (i & (nn - 1))];
}

// Two adjacent rows per thread, for a large operand whose address bit 0 is a free row bit (rows 2t
// and 2t + 1 are then neighbouring entries of every row of X): one 16-byte load brings X[m][k] and
// X[m+1][k], and every shared-memory load of the small operand feeds both rows -- half the load
// instructions per output of k_small, whose load/store unit it saturates.  256 threads x 2 rows per
// CTA, one pair per grid.y; outputs staged for coalesced stores as in k_small, or placed.
template <int KB>
__global__ void __launch_bounds__(256) k_small2(const __grid_constant__ SmallDesc d, const ItemCtx ic,
                                                float2* __restrict__ out, int64_t out_is) {
    extern __shared__ float4 small_dyn[];
    float2* ys = (float2*)small_dyn;
    __shared__ int64_t kofs[1 << KB];
    __shared__ int64_t cofs[1 << kSmallMaxN];
    __shared__ int8_t rpos[kMaxRank];
    const int nb = d.nb;
    const int nn = 1 << nb;
    const int yn = (1 << KB) << nb;
    const int64_t M = (int64_t)1 << d.mb;
    const int64_t item = blockIdx.y;
    if (d.om.on) {
        for (int n = threadIdx.x; n < nn; n += blockDim.x) cofs[n] = place_bits(n, d.om.pos);
        for (int b = threadIdx.x; b < d.mb; b += blockDim.x) rpos[b] = d.om.pos[nb + b];
    }
    {
        const int64_t yb = fix_offset(d.y, ic, item);
        for (int e = threadIdx.x; e < yn; e += blockDim.x) {
            const int kk = e >> nb, n = e & (nn - 1);
            int64_t a = yb;
            for (int i = 0; i < KB; ++i)
                if ((kk >> i) & 1) a += (int64_t)1 << d.yk_pos[i];
            for (int i = 0; i < nb; ++i)
                if ((n >> i) & 1) a += (int64_t)1 << d.yn_pos[i];
            ys[e] = d.y.base[a];
        }
    }
    if (threadIdx.x < (1 << KB)) {
        int64_t a = 0;
        for (int i = 0; i < KB; ++i)
            if ((threadIdx.x >> i) & 1) a += (int64_t)1 << d.xk_pos[i];
        kofs[threadIdx.x] = a;
    }
    __syncthreads();
    const int t = threadIdx.x;
    const int64_t m = ((int64_t)blockIdx.x * 256 + t) * 2;  // even: rows m, m + 1
    float2* stage = ys + ((yn + 1) & ~1);
    const bool staged = !d.om.on && nb <= 4;
    if (m < M) {
        int64_t xa = m;
        for (int h = 0; h < d.n_holes; ++h) {
            const int q = d.holes[h];
            xa = ((xa >> q) << (q + 1)) | (xa & (((int64_t)1 << q) - 1));
        }
        const float2* __restrict__ xp = d.x.base + fix_offset(d.x, ic, item) + xa;
        float4 a[1 << KB];
#pragma unroll
        for (int kk = 0; kk < (1 << KB); ++kk) a[kk] = *(const float4*)(xp + kofs[kk]);
        const float4* __restrict__ ys4 = (const float4*)ys;
        float2* __restrict__ cp0 = out + item * out_is + (d.om.on ? place_bits(m, rpos) : (m << nb));
        float2* __restrict__ cp1 = d.om.on ? cp0 + ((int64_t)1 << rpos[0]) : cp0 + nn;
        const bool pair16 = d.om.on && d.om.pos[0] == 0;
        for (int n = 0; n < nn; n += 2) {
            float2 c00 = make_float2(0.f, 0.f), c01 = c00, c10 = c00, c11 = c00;
#pragma unroll
            for (int kk = 0; kk < (1 << KB); ++kk) {
                const float4 y = ys4[(kk * nn + n) >> 1];
                const float2 y0 = make_float2(y.x, y.y), y1 = make_float2(y.z, y.w);
                const float2 a0 = make_float2(a[kk].x, a[kk].y), a1 = make_float2(a[kk].z, a[kk].w);
                cfma(c00, a0, y0);
                cfma(c01, a0, y1);
                cfma(c10, a1, y0);
                cfma(c11, a1, y1);
            }
            if (staged) {
                stage[(2 * t) * (nn + 1) + n] = c00;
                stage[(2 * t) * (nn + 1) + n + 1] = c01;
                stage[(2 * t + 1) * (nn + 1) + n] = c10;
                stage[(2 * t + 1) * (nn + 1) + n + 1] = c11;
            } else if (d.om.on) {
                if (pair16) {  // column bit 0 at address bit 0 (see k_small)
                    *(float4*)(cp0 + cofs[n]) = make_float4(c00.x, c00.y, c01.x, c01.y);
                    *(float4*)(cp1 + cofs[n]) = make_float4(c10.x, c10.y, c11.x, c11.y);
                } else {
                    cp0[cofs[n]] = c00;
                    cp0[cofs[n + 1]] = c01;
                    cp1[cofs[n]] = c10;
                    cp1[cofs[n + 1]] = c11;
                }
            } else {
                *(float4*)(cp0 + n) = make_float4(c00.x, c00.y, c01.x, c01.y);
                *(float4*)(cp1 + n) = make_float4(c10.x, c10.y, c11.x, c11.y);
            }
        }
    }
    if (!staged) return;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * 512;
    const int64_t rows = M - r0 < 512 ? M - r0 : 512;
    float2* __restrict__ dst = out + item * out_is + (r0 << nb);
    const int64_t cnt = rows * nn;
    for (int64_t i = t; i < cnt; i += 256) dst[i] = stage[(i >> nb) * (nn + 1) + (i & (nn - 1))];
}

// Flat variant for small per-pair tensors (2^mb < 256): one thread per
// (pair, m) across the whole batch, the small operand read through L1 with
// per-pair offsets (its entries are shared by the threads of a pair).  The
// 256 threads of a CTA own 256 consecutive (pair, m), whose outputs form one
// contiguous block: they are staged in shared memory (row stride 2^NB + 1
// against bank conflicts) and stored coalesced.
template <int KB, int NB>
__global__ void __launch_bounds__(256) k_small_flat(const __grid_constant__ SmallDesc d, const ItemCtx ic, float2* __restrict__ out,
                                                    int64_t out_is, int64_t n_items) {
    constexpr int NN = 1 << NB, STAGE = NB <= 4;
    __shared__ int64_t yrel[(1 << KB) << NB];
    __shared__ int64_t kofs[1 << KB];
    __shared__ float2 stage[STAGE ? 256 * (NN + 1) : 1];
    __shared__ int64_t cofs[NN];      // placed product: offset of each column n
    __shared__ int8_t rpos[kMaxRank];  // placed product: position of each row bit
    const bool staged = STAGE && !d.om.on;
    if (d.om.on) {
        for (int n = threadIdx.x; n < NN; n += blockDim.x) cofs[n] = place_bits(n, d.om.pos);
        for (int b = threadIdx.x; b < d.mb; b += blockDim.x) rpos[b] = d.om.pos[NB + b];
    }
    for (int i = threadIdx.x; i < ((1 << KB) << NB); i += blockDim.x) {
        const int kk = i >> NB, n = i & (NN - 1);
        int64_t a = 0;
        for (int b = 0; b < KB; ++b)
            if ((kk >> b) & 1) a += (int64_t)1 << d.yk_pos[b];
        for (int b = 0; b < NB; ++b)
            if ((n >> b) & 1) a += (int64_t)1 << d.yn_pos[b];
        yrel[i] = a;
    }
    if (threadIdx.x < (1 << KB)) {
        int64_t a = 0;
        for (int b = 0; b < KB; ++b)
            if ((threadIdx.x >> b) & 1) a += (int64_t)1 << d.xk_pos[b];
        kofs[threadIdx.x] = a;
    }
    __syncthreads();
    const int64_t total = n_items << d.mb;
    for (int64_t t0 = (int64_t)blockIdx.x * 256; t0 < total; t0 += (int64_t)gridDim.x * 256) {
        const int64_t t = t0 + threadIdx.x;
        float2 res[NN];
        if (t < total) {
            const int64_t item = t >> d.mb, m = t & (((int64_t)1 << d.mb) - 1);
            int64_t xa = m;
            for (int h = 0; h < d.n_holes; ++h) {
                const int p = d.holes[h];
                xa = ((xa >> p) << (p + 1)) | (xa & (((int64_t)1 << p) - 1));
            }
            const float2* __restrict__ xp = d.x.base + fix_offset(d.x, ic, item) + xa;
            const float2* __restrict__ yp = d.y.base + fix_offset(d.y, ic, item);
            float2 a[1 << KB];
#pragma unroll
            for (int kk = 0; kk < (1 << KB); ++kk) a[kk] = xp[kofs[kk]];
#pragma unroll
            for (int n = 0; n < NN; ++n) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int kk = 0; kk < (1 << KB); ++kk) cfma(acc, a[kk], __ldg(yp + yrel[(kk << NB) + n]));
                res[n] = acc;
            }
            if (!staged) {
                float2* __restrict__ cp = out + item * out_is + (d.om.on ? place_bits(m, rpos) : (m << NB));
#pragma unroll
                for (int n = 0; n < NN; ++n) cp[d.om.on ? cofs[n] : n] = res[n];
            }
        }
        if (staged) {
            // outputs of (pair, m) = t sit at t * NN (out_is = 2^(mb + NB)): one block per CTA
#pragma unroll
            for (int n = 0; n < NN; ++n) stage[threadIdx.x * (NN + 1) + n] = res[n];
            __syncthreads();
            const int64_t cnt = (total - t0 < 256 ? total - t0 : 256) * NN;
            float2* __restrict__ dst = out + t0 * NN;
            for (int i = threadIdx.x; i < cnt; i += 256) dst[i] = stage[(i / NN) * (NN + 1) + (i % NN)];
            __syncthreads();
        }
    }
}

template <int KB>
static cudaError_t small_flat_nb(const SmallDesc& d, const ItemCtx& ic, int64_t n_items, float2* out, int64_t out_is,
                                 cudaStream_t st, unsigned grid) {
    switch (d.nb) {
        case 0: k_small_flat<KB, 0><<<grid, 256, 0, st>>>(d, ic, out, out_is, n_items); break;
        case 1: k_small_flat<KB, 1><<<grid, 256, 0, st>>>(d, ic, out, out_is, n_items); break;
        case 2: k_small_flat<KB, 2><<<grid, 256, 0, st>>>(d, ic, out, out_is, n_items); break;
        case 3: k_small_flat<KB, 3><<<grid, 256, 0, st>>>(d, ic, out, out_is, n_items); break;
        case 4: k_small_flat<KB, 4><<<grid, 256, 0, st>>>(d, ic, out, out_is, n_items); break;
        default: k_small_flat<KB, 5><<<grid, 256, 0, st>>>(d, ic, out, out_is, n_items); break;
    }
    return cudaGetLastError();
}

static int sm_count();

bool small_is_flat(const SmallDesc& d) { return d.mb < 8 && d.kb + d.nb <= 6; }

cudaError_t launch_small(const SmallDesc& d, const ItemCtx& ic, int64_t n_items, float2* out, int64_t out_is,
                         cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (n_items > kMaxBatchItems || ic.n_items > kMaxBatchItems) return cudaErrorInvalidValue;  // fix_offset
    // flat: short per-pair rows with a small operand light enough to read through L1 per thread;
    // a larger small operand is better staged once per CTA in shared memory (per-pair kernel)
    if (small_is_flat(d)) {
        const int64_t total = n_items << d.mb;
        const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 16);
        switch (d.kb) {
            case 0: return small_flat_nb<0>(d, ic, n_items, out, out_is, st, grid);
            case 1: return small_flat_nb<1>(d, ic, n_items, out, out_is, st, grid);
            case 2: return small_flat_nb<2>(d, ic, n_items, out, out_is, st, grid);
            case 3: return small_flat_nb<3>(d, ic, n_items, out, out_is, st, grid);
            case 4: return small_flat_nb<4>(d, ic, n_items, out, out_is, st, grid);
            default: return small_flat_nb<5>(d, ic, n_items, out, out_is, st, grid);
        }
    }
    // pairs of fewer than 256 rows share a CTA (their products contiguous), within 1536 staged
    // small-operand entries so that with the output stage the CTA stays under 48 KB
    const int64_t m = (int64_t)1 << d.mb;
    const int yst = (((1 << d.kb) << d.nb) + 1) & ~1;
    const int y_shared = d.y.item_stride == 0 && d.y.n_fix == 0;
    int ppc = 1;
    if (m < 256 && (out_is == (m << d.nb) || n_items == 1)) {
        ppc = (int)(256 / m);
        while (ppc > 1 && !y_shared && ppc * yst > 1536) ppc >>= 1;
    }
    // two rows per thread when X's address bit 0 is a row bit (see k_small2)
    if (ppc == 1 && m >= 512 && d.kb <= 4 && d.nb >= 1 && (d.n_holes == 0 || d.holes[0] != 0)) {
        const int yn = (1 << d.kb) << d.nb;
        const bool staged2 = !d.om.on && d.nb <= 4;
        const size_t smem2 = sizeof(float2) * ((size_t)((yn + 1) & ~1) + (staged2 ? 512 * ((1 << d.nb) + 1) : 0));
        dim3 grid2((unsigned)(m / 512), (unsigned)n_items);
        // the staged output of 512 rows needs up to 70 KB: allow 100 KB of dynamic shared memory, once
        // per device and instantiation
        static uint64_t attr_done[5][4] = {};
        static std::mutex mu;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        {
            std::lock_guard<std::mutex> lk(mu);
            const int kb = d.kb;
            if (dev < 256 && !((attr_done[kb][dev >> 6] >> (dev & 63)) & 1)) {
                const void* fn = kb == 0   ? (const void*)k_small2<0>
                                 : kb == 1 ? (const void*)k_small2<1>
                                 : kb == 2 ? (const void*)k_small2<2>
                                 : kb == 3 ? (const void*)k_small2<3>
                                           : (const void*)k_small2<4>;
                e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
                if (e != cudaSuccess) return e;
                attr_done[kb][dev >> 6] |= 1ull << (dev & 63);
            }
        }
        if (smem2 > 100 * 1024) return cudaErrorInvalidValue;
        switch (d.kb) {
            case 0: k_small2<0><<<grid2, 256, smem2, st>>>(d, ic, out, out_is); break;
            case 1: k_small2<1><<<grid2, 256, smem2, st>>>(d, ic, out, out_is); break;
            case 2: k_small2<2><<<grid2, 256, smem2, st>>>(d, ic, out, out_is); break;
            case 3: k_small2<3><<<grid2, 256, smem2, st>>>(d, ic, out, out_is); break;
            default: k_small2<4><<<grid2, 256, smem2, st>>>(d, ic, out, out_is); break;
        }
        return cudaGetLastError();
    }
    const int threads = ppc > 1 ? (int)(ppc * m) : (m < 256 ? (int)((m + 31) / 32 * 32) : 256);
    const bool staged = !d.om.on && d.nb <= 4 && threads == 256;
    dim3 grid(ppc > 1 ? 1u : (unsigned)((m + 255) / 256), (unsigned)((n_items + ppc - 1) / ppc));
    const size_t smem = sizeof(float2) * ((size_t)(y_shared ? 1 : ppc) * yst + (staged ? 256 * ((1 << d.nb) + 1) : 0));
    switch (d.kb) {
        case 0: k_small<0><<<grid, threads, smem, st>>>(d, ic, out, out_is, n_items, ppc, y_shared); break;
        case 1: k_small<1><<<grid, threads, smem, st>>>(d, ic, out, out_is, n_items, ppc, y_shared); break;
        case 2: k_small<2><<<grid, threads, smem, st>>>(d, ic, out, out_is, n_items, ppc, y_shared); break;
        case 3: k_small<3><<<grid, threads, smem, st>>>(d, ic, out, out_is, n_items, ppc, y_shared); break;
        case 4: k_small<4><<<grid, threads, smem, st>>>(d, ic, out, out_is, n_items, ppc, y_shared); break;
        case 5: k_small<5><<<grid, threads, smem, st>>>(d, ic, out, out_is, n_items, ppc, y_shared); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Complex64 SIMT GEMM (the plain reference form).  BM x BN complex output tile
// per CTA (16 x 16 threads, each (BM/16) x (BN/16) outputs at rows ty + 16 i,
// columns tx + 16 j), 16 complex K per stage, register-staged double buffer
// (one barrier per stage), batched over items in grid.y.
//
// Accumulation is blocked: products are summed in FP32 over 64 K (4 stages)
// into a partial that is then added to the running total.  A single running
// FP32 sum over K = 2^15 terms loses about sqrt(K) ulps; blocking keeps the
// error near (sqrt(64) + sqrt(K/64)) ulps at the cost of one add per output
// per 64 K.
// ---------------------------------------------------------------------------------------------
constexpr int GBK = 16;
constexpr int GFOLD = 4;  // stages per partial

template <int BM, int BN>
__global__ void __launch_bounds__(256, (BM * BN >= 8192 ? 1 : 2)) k_gemm_c64(const float2* __restrict__ A, int64_t a_is, bool akm,
                                                  const float2* __restrict__ B, int64_t b_is, bool bkm,
                                                  float2* __restrict__ C, int64_t c_is, int mb, int nb, int kb,
                                                  int tiles_n, const __grid_constant__ OutMap om, int a_div,
                                                  int b_div) {
    constexpr int TM = BM / 16, TN = BN / 16, LA = BM * GBK / 256, LB = BN * GBK / 256;
    extern __shared__ float2 gsm[];  // As[2][GBK][BM + 1], then Bs[2][GBK][BN + 1]
    float2(*As)[GBK][BM + 1] = (float2(*)[GBK][BM + 1])gsm;
    float2(*Bs)[GBK][BN + 1] = (float2(*)[GBK][BN + 1])(gsm + 2 * GBK * (BM + 1));
    const int64_t M = (int64_t)1 << mb, N = (int64_t)1 << nb, K = (int64_t)1 << kb;
    const int64_t item = blockIdx.y;
    const int64_t m0 = (int64_t)(blockIdx.x / tiles_n) * BM;
    const int64_t n0 = (int64_t)(blockIdx.x % tiles_n) * BN;
    const float2* Ap = A + (item / a_div) * a_is;
    const float2* Bp = B + (item / b_div) * b_is;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float2 zero = make_float2(0.f, 0.f);
    float2 ra[LA], rb[LB];

    auto gload = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int idx = tid + 256 * r;
            const int kk = akm ? (idx & (GBK - 1)) : (idx / BM);
            const int mm = akm ? (idx / GBK) : (idx & (BM - 1));
            const int64_t gm = m0 + mm, gk = k0 + kk;
            ra[r] = (gm < M && gk < K) ? (akm ? Ap[gm * K + gk] : Ap[gk * M + gm]) : zero;
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int idx = tid + 256 * r;
            const int kk = bkm ? (idx & (GBK - 1)) : (idx / BN);
            const int nn = bkm ? (idx / GBK) : (idx & (BN - 1));
            const int64_t gn = n0 + nn, gk = k0 + kk;
            rb[r] = (gn < N && gk < K) ? (bkm ? Bp[gn * K + gk] : Bp[gk * N + gn]) : zero;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int idx = tid + 256 * r;
            const int kk = akm ? (idx & (GBK - 1)) : (idx / BM);
            const int mm = akm ? (idx / GBK) : (idx & (BM - 1));
            As[buf][kk][mm] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int idx = tid + 256 * r;
            const int kk = bkm ? (idx & (GBK - 1)) : (idx / BN);
            const int nn = bkm ? (idx / GBK) : (idx & (BN - 1));
            Bs[buf][kk][nn] = rb[r];
        }
    };

    float2 tot[TM][TN], acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) tot[i][j] = acc[i][j] = zero;
    gload(0);
    sstore(0);
    __syncthreads();
    int buf = 0, stage = 0;
    for (int64_t k0 = 0; k0 < K; k0 += GBK) {
        const bool more = k0 + GBK < K;
        if (more) gload(k0 + GBK);
        const int kl = K < GBK ? (int)K : GBK;  // products with K < 16 skip the zero-filled rows
#pragma unroll
        for (int kk = 0; kk < GBK; ++kk) {
            if (kk >= kl) break;
            float2 a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        if (++stage == GFOLD || !more) {
            stage = 0;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    tot[i][j].x += acc[i][j].x;
                    tot[i][j].y += acc[i][j].y;
                    acc[i][j] = zero;
                }
        }
        if (more) sstore(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    float2* Cp = C + item * c_is;
    if (om.on) {  // placed product: row and column offsets from the bit map (columns stay lane-contiguous)
        int64_t co[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) co[j] = place_bits(n0 + tx + 16 * j, om.pos);
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gm = m0 + ty + 16 * i;
            if (gm >= M) continue;
            const int64_t ro = place_bits(gm, om.pos + nb);
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (n0 + tx + 16 * j < N) Cp[ro + co[j]] = tot[i][j];
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gn = n0 + tx + 16 * j;
            if (gn < N) Cp[gm * N + gn] = tot[i][j];
        }
    }
}

// Long dot products (M * N <= 16 outputs, large K): one CTA per item, the 256
// threads stride over K with a private partial per output, then a fixed-order
// tree reduction (deterministic).
template <int MB, int NB>
__global__ void __launch_bounds__(256) k_dot_c64(const float2* __restrict__ A, int64_t a_is, bool akm,
                                                 const float2* __restrict__ B, int64_t b_is, bool bkm,
                                                 float2* __restrict__ C, int64_t c_is, int kb, int a_div, int b_div) {
    constexpr int M = 1 << MB, N = 1 << NB, MN = M * N;
    __shared__ float2 red[MN][256];
    const int64_t K = (int64_t)1 << kb;
    const int64_t item = blockIdx.x;
    const float2* Ap = A + (item / a_div) * a_is;
    const float2* Bp = B + (item / b_div) * b_is;
    const int tid = threadIdx.x;
    float2 acc[MN];
#pragma unroll
    for (int i = 0; i < MN; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int64_t k = tid; k < K; k += 256) {
        float2 a[M], b[N];
#pragma unroll
        for (int m = 0; m < M; ++m) a[m] = akm ? Ap[m * K + k] : Ap[k * M + m];
#pragma unroll
        for (int n = 0; n < N; ++n) b[n] = bkm ? Bp[n * K + k] : Bp[k * N + n];
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int n = 0; n < N; ++n) cfma(acc[m * N + n], a[m], b[n]);
    }
#pragma unroll
    for (int i = 0; i < MN; ++i) red[i][tid] = acc[i];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) {
#pragma unroll
            for (int i = 0; i < MN; ++i) {
                red[i][tid].x += red[i][tid + w].x;
                red[i][tid].y += red[i][tid + w].y;
            }
        }
        __syncthreads();
    }
    if (tid < MN) C[item * c_is + tid] = red[tid][0];
}

// A step that contracts every leg with one operand stored in another leg order: per pair
// C = sum_k A[k] B[p(k)], B read through the permutation's tiles (as k_permute: a tile in input
// order into shared memory, then walked in A's order), so the permuted copy of B never goes to HBM.
// One CTA per pair; per-thread FP32 partials, then a fixed-order tree.
__global__ void __launch_bounds__(256) k_dot_perm(const PermDesc d, const PermTables tb, const ItemCtx ic,
                                                  const float2* __restrict__ A, int64_t a_is, float2* __restrict__ C,
                                                  int64_t c_is, int a_div) {
    constexpr int LO = kPermLoBits, LM = (1 << LO) - 1;
    __shared__ float2 tile[(1 << kPermTileBits) + (1 << kPermTileBits) / 32];
    __shared__ int64_t s_in[128], s_out[128];
    __shared__ int s_map[128];
    __shared__ float2 red[256];
    const int tid = threadIdx.x;
    if (tid < 64) {
        s_in[tid] = tb.in_lo[tid];
        s_in[64 + tid] = tb.in_hi[tid];
        s_out[tid] = tb.out_lo[tid];
        s_out[64 + tid] = tb.out_hi[tid];
        s_map[tid] = tb.map_lo[tid];
        s_map[64 + tid] = tb.map_hi[tid];
    }
    __syncthreads();
    const int64_t item = blockIdx.x;
    const int n = 1 << d.t;
    const int64_t tiles = (int64_t)1 << d.n_outer;
    const int64_t ibase = fix_offset(d.in, ic, item);
    const float2* __restrict__ Ap = A + (item / a_div) * a_is;
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t tj = 0; tj < tiles; ++tj) {
        int64_t ib = ibase, ob = 0;
        uint64_t u = (uint64_t)tj;
        while (u) {
            const int i = __ffsll((long long)u) - 1;
            ib += tb.outer_in[i];
            ob += tb.outer_out[i];
            u &= u - 1;
        }
        for (int j = tid; j < n; j += 256) tile[pad32(j)] = d.in.base[ib + s_in[j & LM] + s_in[64 + (j >> LO)]];
        __syncthreads();
        for (int j = tid; j < n; j += 256)
            cfma(acc, Ap[ob + s_out[j & LM] + s_out[64 + (j >> LO)]], tile[pad32(s_map[j & LM] | s_map[64 + (j >> LO)])]);
        __syncthreads();
    }
    red[tid] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) {
            red[tid].x += red[tid + w].x;
            red[tid].y += red[tid + w].y;
        }
        __syncthreads();
    }
    if (tid == 0) C[item * c_is] = red[0];
}

cudaError_t launch_dot_perm(const PermDesc& d, const ItemCtx& ic, int64_t n_items, const float2* a, int64_t a_is,
                            float2* c, int64_t c_is, cudaStream_t st, int a_div) {
    if (n_items <= 0) return cudaSuccess;
    if (d.t > kPermTileBits || n_items > kMaxBatchItems || ic.n_items > kMaxBatchItems || a_div < 1)
        return cudaErrorInvalidValue;
    PermTables tb;
    perm_tables(d, &tb);
    k_dot_perm<<<(unsigned)n_items, 256, 0, st>>>(d, tb, ic, a, a_is, c, c_is, a_div);
    return cudaGetLastError();
}

// Products with K <= 4 (k <= 2 shared bits): each output reads K entries of A and K of B, so the
// work is writing C.  Threads run along the columns n (whole rows per store, or whole runs of the
// placed columns), each keeps its column of B in registers and walks rows; the A entries of a row
// are the same for the threads of a warp (N >= 32).
template <int KB>
__global__ void __launch_bounds__(256) k_gemm_smallk(const float2* __restrict__ A, int64_t a_is, bool akm,
                                                    const float2* __restrict__ B, int64_t b_is, bool bkm,
                                                    float2* __restrict__ C, int64_t c_is, int mb, int nb,
                                                    int rows_per_cta, const __grid_constant__ OutMap om, int a_div,
                                                    int b_div) {
    constexpr int K = 1 << KB;
    const int64_t item = blockIdx.y;
    const int64_t M = (int64_t)1 << mb, N = (int64_t)1 << nb;
    const int width = N < 256 ? (int)N : 256;            // columns per row pass
    const int passes = 256 / width;                      // rows per pass
    const int64_t col_blocks = N / width;
    const int64_t cb = blockIdx.x % col_blocks, rb = blockIdx.x / col_blocks;
    const int64_t n = cb * width + (threadIdx.x % width);
    const int64_t r0 = rb * rows_per_cta + threadIdx.x / width;
    const int64_t r1 = (rb + 1) * rows_per_cta < M ? (rb + 1) * rows_per_cta : M;
    const float2* __restrict__ Ap = A + (item / a_div) * a_is;
    const float2* __restrict__ Bp = B + (item / b_div) * b_is;
    float2 b[K];
#pragma unroll
    for (int k = 0; k < K; ++k) b[k] = bkm ? Bp[n * K + k] : Bp[(int64_t)k * N + n];
    float2* __restrict__ Cp = C + item * c_is;
    const int64_t co = om.on ? place_bits(n, om.pos) : n;
    for (int64_t r = r0; r < r1; r += passes) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; ++k) cfma(acc, akm ? Ap[r * K + k] : Ap[(int64_t)k * M + r], b[k]);
        Cp[(om.on ? place_bits(r, om.pos + nb) : r * N) + co] = acc;
    }
}

template <int BM, int BN>
static void gemm_tile(dim3 grid, cudaStream_t st, const float2* a, int64_t a_is, bool akm, const float2* b,
                      int64_t b_is, bool bkm, float2* c, int64_t c_is, int mb, int nb, int kb, int tn,
                      const OutMap& om, int a_div, int b_div) {
    constexpr int smem = 2 * GBK * (BM + 1 + BN + 1) * (int)sizeof(float2);
    if (smem > 48 * 1024) {
        // opt in to more than 48 KB of dynamic shared memory, once per device
        static uint64_t done[4] = {0, 0, 0, 0};
        static std::mutex mu;
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 256) {
            std::lock_guard<std::mutex> lk(mu);
            if (!((done[dev >> 6] >> (dev & 63)) & 1) &&
                cudaFuncSetAttribute(k_gemm_c64<BM, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                    cudaSuccess)
                done[dev >> 6] |= 1ull << (dev & 63);
        }
    }
    k_gemm_c64<BM, BN><<<grid, 256, smem, st>>>(a, a_is, akm, b, b_is, bkm, c, c_is, mb, nb, kb, tn, om, a_div,
                                                b_div);
}

cudaError_t launch_gemm_c64(const float2* a, int64_t a_is, bool a_kmajor, const float2* b, int64_t b_is,
                            bool b_kmajor, float2* c, int64_t c_is, int mb, int nb, int kb, int64_t n_items,
                            cudaStream_t st, const OutMap* omp, int a_div, int b_div) {
    if (n_items <= 0) return cudaSuccess;
    if (a_div < 1 || b_div < 1) return cudaErrorInvalidValue;
    OutMap om{};
    if (omp) om = *omp;
    if (kb <= 2 && nb >= 5) {
        // about 4096 outputs per CTA
        const int64_t M = (int64_t)1 << mb, N = (int64_t)1 << nb;
        const int64_t width = N < 256 ? N : 256;
        const int64_t rows = std::max<int64_t>(256 / width, std::min<int64_t>(M, 4096 / width));
        const int64_t blocks = ((M + rows - 1) / rows) * (N / width);
        dim3 grid((unsigned)blocks, (unsigned)n_items);
        switch (kb) {
            case 0: k_gemm_smallk<0><<<grid, 256, 0, st>>>(a, a_is, a_kmajor, b, b_is, b_kmajor, c, c_is, mb, nb, (int)rows, om, a_div, b_div); break;
            case 1: k_gemm_smallk<1><<<grid, 256, 0, st>>>(a, a_is, a_kmajor, b, b_is, b_kmajor, c, c_is, mb, nb, (int)rows, om, a_div, b_div); break;
            default: k_gemm_smallk<2><<<grid, 256, 0, st>>>(a, a_is, a_kmajor, b, b_is, b_kmajor, c, c_is, mb, nb, (int)rows, om, a_div, b_div); break;
        }
        return cudaGetLastError();
    }
    if (mb + nb <= 4 && kb >= 8) {
        if (om.on) return cudaErrorInvalidValue;  // the dot kernel writes the natural layout only
        dim3 grid((unsigned)n_items);
#define QX_DOT_CASE(X, Y)                                                                                   \
    if (mb == X && nb == Y) {                                                                               \
        k_dot_c64<X, Y><<<grid, 256, 0, st>>>(a, a_is, a_kmajor, b, b_is, b_kmajor, c, c_is, kb, a_div, b_div); \
        return cudaGetLastError();                                                                          \
    }
        QX_DOT_CASE(0, 0) QX_DOT_CASE(0, 1) QX_DOT_CASE(0, 2) QX_DOT_CASE(0, 3) QX_DOT_CASE(0, 4)
        QX_DOT_CASE(1, 0) QX_DOT_CASE(1, 1) QX_DOT_CASE(1, 2) QX_DOT_CASE(1, 3)
        QX_DOT_CASE(2, 0) QX_DOT_CASE(2, 1) QX_DOT_CASE(2, 2)
        QX_DOT_CASE(3, 0) QX_DOT_CASE(3, 1) QX_DOT_CASE(4, 0)
#undef QX_DOT_CASE
        return cudaErrorInvalidValue;
    }
    const int bmb = mb >= 7 && nb >= 6 ? 7 : mb >= 6 ? 6 : mb >= 5 ? 5 : 4;  // tile edge 128 / 64 / 32 / 16
    const int bnb = nb >= 6 ? 6 : nb >= 5 ? 5 : 4;
    const int64_t tm = ((1ll << mb) + (1 << bmb) - 1) >> bmb, tn = ((1ll << nb) + (1 << bnb) - 1) >> bnb;
    dim3 grid((unsigned)(tm * tn), (unsigned)n_items);
#define QX_GEMM_CASE(X, Y)                                                                            \
    if (bmb == X && bnb == Y) {                                                                       \
        gemm_tile<(1 << X), (1 << Y)>(grid, st, a, a_is, a_kmajor, b, b_is, b_kmajor, c, c_is, mb, nb, kb, \
                                      (int)tn, om, a_div, b_div);                                     \
        return cudaGetLastError();                                                                    \
    }
    QX_GEMM_CASE(7, 6)
    QX_GEMM_CASE(6, 6) QX_GEMM_CASE(6, 5) QX_GEMM_CASE(6, 4)
    QX_GEMM_CASE(5, 6) QX_GEMM_CASE(5, 5) QX_GEMM_CASE(5, 4)
    QX_GEMM_CASE(4, 6) QX_GEMM_CASE(4, 5) QX_GEMM_CASE(4, 4)
#undef QX_GEMM_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Recombination of slices (Eq. 2) in FP64 with Neumaier compensation.  One
// thread per (bitstring, open index); it walks the batch's slices in order,
// so the result does not depend on thread scheduling.  acc holds
// {sum_re, sum_im, comp_re, comp_im} per amplitude.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

__global__ void k_slice_sum(const SumDesc d, const ItemCtx ic, double* __restrict__ acc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_o = (int64_t)1 << d.open_bits;
    if (idx >= (int64_t)ic.n_b * n_o) return;
    const int64_t bl = idx >> d.open_bits, o = idx & (n_o - 1);
    int64_t rel = 0;
    for (int ob = 0; ob < d.open_bits; ++ob)
        if ((o >> ob) & 1) rel += (int64_t)1 << d.obit_pos[ob];
    double* a = acc + ((ic.b0 + bl) * n_o + o) * 4;
    double sr = a[0], si = a[1], cr = a[2], ci = a[3];
    for (int s = 0; s < d.n_s; ++s) {
        const int64_t item = (int64_t)s * ic.n_b + bl;
        const float2 v = d.root.base[fix_offset(d.root, ic, item) + rel];
        neumaier(sr, cr, (double)v.x);
        neumaier(si, ci, (double)v.y);
    }
    a[0] = sr;
    a[1] = si;
    a[2] = cr;
    a[3] = ci;
}

cudaError_t launch_slice_sum(const SumDesc& d, const ItemCtx& ic, double* acc, cudaStream_t st) {
    const int64_t n = (int64_t)ic.n_b << d.open_bits;
    if (n <= 0) return cudaSuccess;
    if (ic.n_items > kMaxBatchItems) return cudaErrorInvalidValue;  // fix_offset
    k_slice_sum<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, ic, acc);
    return cudaGetLastError();
}

__global__ void k_finalize(const double* __restrict__ acc, double* __restrict__ amps, int64_t n, double sr,
                           double si) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double re = acc[4 * i] + acc[4 * i + 2];
    const double im = acc[4 * i + 1] + acc[4 * i + 3];
    amps[2 * i] = re * sr - im * si;
    amps[2 * i + 1] = re * si + im * sr;
}

cudaError_t launch_finalize(const double* acc, double* amps, int64_t n, double sr, double si, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(acc, amps, n, sr, si);
    return cudaGetLastError();
}

}  // namespace qx
