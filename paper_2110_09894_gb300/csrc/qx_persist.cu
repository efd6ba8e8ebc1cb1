// Persistent slice-batch executor: each CTA takes (slice, bitstring) pairs
// from a work counter and runs the pair's whole contraction -- every plan step
// in order, with __syncthreads() between steps -- in a private scratch region
// that stays in L2, then writes the pair's result vector for the FP64
// cross-slice sum.  This is the slice level of parallelism of Sec. IV-A
// (independent sub-networks, Eq. 2) mapped onto the CTAs of one launch; the
// per-step kernels of qx_kernels.cu instead launch once per step over a batch.
//
// Several programs (networks with their plans) can share one launch: a work
// item names its program, so uneven circuits run side by side.
#include <cuda_runtime.h>

#include "qx.h"
#include "qx_internal.h"

namespace qx {

__device__ __forceinline__ void pcfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

struct PairCtx {
    int64_t s;              // slice index
    const uint8_t* bits;    // this pair's bitstring
    float2* scratch;        // this CTA's scratch
    const PProg* prog;
};

__device__ __forceinline__ const float2* pref_base(const PRef& r, const PairCtx& c) {
    if (r.space == PSPACE_SCRATCH) return c.scratch + r.off;
    int64_t off = r.off;
    for (int f = 0; f < r.n_fix; ++f) {
        const int src = r.fix_src[f];
        const int64_t v = src >= 0 ? ((c.s >> src) & 1) : (int64_t)(c.bits[-src - 1] & 1);
        off += v * r.fix_stride[f];
    }
    return (r.space == PSPACE_LEAF ? c.prog->leaves : c.prog->inv) + off;
}

// ---- bit permutation, tile by tile through shared memory --------------------------------------
__device__ void exec_perm(const POp& op, const PairCtx& c, float2* sm) {
    float2* tile = sm;
    int64_t* tabs = (int64_t*)(sm + 1056);  // in_lo, in_hi, out_lo, out_hi
    int* maps = (int*)(tabs + 128);         // map_lo, map_hi
    const int tid = threadIdx.x, t = op.t;
    if (tid < 32) {
        int64_t a = 0, b = 0, cc = 0, e = 0;
        int ml = 0, mh = 0;
        for (int i = 0; i < 5; ++i) {
            if ((tid >> i) & 1) {
                if (i < t) {
                    a += (int64_t)1 << op.in_pos[op.tile_in[i]];
                    cc += (int64_t)1 << op.tile_out[i];
                }
                if (i + 5 < t) {
                    b += (int64_t)1 << op.in_pos[op.tile_in[i + 5]];
                    e += (int64_t)1 << op.tile_out[i + 5];
                }
            }
        }
        for (int i = 0; i < t; ++i) {
            int r = 0;
            for (int j = 0; j < t; ++j)
                if (op.tile_in[j] == op.tile_out[i]) r = j;
            if (i < 5) {
                if ((tid >> i) & 1) ml |= 1 << r;
            } else if ((tid >> (i - 5)) & 1) {
                mh |= 1 << r;
            }
        }
        tabs[tid] = a;
        tabs[32 + tid] = b;
        tabs[64 + tid] = cc;
        tabs[96 + tid] = e;
        maps[tid] = ml;
        maps[32 + tid] = mh;
    }
    __syncthreads();
    const float2* src = pref_base(op.x, c);
    float2* dst = c.scratch + op.dst;
    const int n = 1 << t;
    const int64_t n_tiles = (int64_t)1 << op.n_outer;
    for (int64_t u = 0; u < n_tiles; ++u) {
        int64_t ib = 0, ob = 0;
        for (int i = 0; i < op.n_outer; ++i)
            if ((u >> i) & 1) {
                ib += (int64_t)1 << op.in_pos[op.outer[i]];
                ob += (int64_t)1 << op.outer[i];
            }
        for (int j = tid; j < n; j += blockDim.x) tile[j + (j >> 5)] = src[ib + tabs[j & 31] + tabs[32 + (j >> 5)]];
        __syncthreads();
        for (int j = tid; j < n; j += blockDim.x) {
            const int q = maps[j & 31] | maps[32 + (j >> 5)];
            dst[ob + tabs[64 + (j & 31)] + tabs[96 + (j >> 5)]] = tile[q + (q >> 5)];
        }
        __syncthreads();
    }
}

// ---- gather contraction with a small operand in shared memory ---------------------------------
template <int KB>
__device__ void exec_small_k(const POp& op, const PairCtx& c, float2* sm) {
    float2* ys = sm;
    int64_t* kofs = (int64_t*)(sm + 1024);
    const int nb = op.nb, nn = 1 << nb;
    const float2* y = pref_base(op.y, c);
    for (int idx = threadIdx.x; idx < ((1 << KB) << nb); idx += blockDim.x) {
        const int kk = idx >> nb, n = idx & (nn - 1);
        int64_t a = 0;
        for (int i = 0; i < KB; ++i)
            if ((kk >> i) & 1) a += (int64_t)1 << op.yk_pos[i];
        for (int i = 0; i < nb; ++i)
            if ((n >> i) & 1) a += (int64_t)1 << op.yn_pos[i];
        ys[idx] = y[a];
    }
    if (threadIdx.x < (1 << KB)) {
        int64_t a = 0;
        for (int i = 0; i < KB; ++i)
            if ((threadIdx.x >> i) & 1) a += (int64_t)1 << op.xk_pos[i];
        kofs[threadIdx.x] = a;
    }
    __syncthreads();
    const float2* x = pref_base(op.x, c);
    float2* out = c.scratch + op.dst;
    const int64_t M = (int64_t)1 << op.mb;
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) {
        int64_t xa = m;
        for (int h = 0; h < op.n_holes; ++h) {
            const int p = op.holes[h];
            xa = ((xa >> p) << (p + 1)) | (xa & (((int64_t)1 << p) - 1));
        }
        float2 a[1 << KB];
#pragma unroll
        for (int kk = 0; kk < (1 << KB); ++kk) a[kk] = x[xa + kofs[kk]];
        float2* cp = out + (m << nb);
        for (int n = 0; n < nn; ++n) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < (1 << KB); ++kk) pcfma(acc, a[kk], ys[kk * nn + n]);
            cp[n] = acc;
        }
    }
}

__device__ void exec_small(const POp& op, const PairCtx& c, float2* sm) {
    switch (op.kb) {
        case 0: exec_small_k<0>(op, c, sm); break;
        case 1: exec_small_k<1>(op, c, sm); break;
        case 2: exec_small_k<2>(op, c, sm); break;
        case 3: exec_small_k<3>(op, c, sm); break;
        case 4: exec_small_k<4>(op, c, sm); break;
        default: exec_small_k<5>(op, c, sm); break;
    }
}

// ---- SIMT complex GEMM over the whole output, tile by tile -------------------------------------
// Same tiling and blocked accumulation as the per-step kernel: 16 x 16 threads,
// (BM/16) x (BN/16) outputs each, 16 complex K per stage, partials folded
// every 64 K.
template <int BM, int BN>
__device__ void exec_gemm_t(const POp& op, const PairCtx& c, float2* sm) {
    constexpr int BK = 16, TM = BM / 16, TN = BN / 16, LA = BM * BK / 256, LB = BN * BK / 256;
    float2(*As)[BM + 1] = (float2(*)[BM + 1])sm;
    float2(*Bs)[BN + 1] = (float2(*)[BN + 1])(sm + BK * (BM + 1));
    const int64_t M = (int64_t)1 << op.mb, N = (int64_t)1 << op.nb, K = (int64_t)1 << op.kb;
    const float2* A = pref_base(op.x, c);
    const float2* B = pref_base(op.y, c);
    float2* Cp = c.scratch + op.dst;
    const bool akm = op.a_km, bkm = op.b_km;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float2 zero = make_float2(0.f, 0.f);
    const int64_t tiles_n = (N + BN - 1) / BN, tiles = ((M + BM - 1) / BM) * tiles_n;
    for (int64_t tile = 0; tile < tiles; ++tile) {
        const int64_t m0 = (tile / tiles_n) * BM, n0 = (tile % tiles_n) * BN;
        float2 tot[TM][TN], acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) tot[i][j] = acc[i][j] = zero;
        int stage = 0;
        for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
            for (int r = 0; r < LA; ++r) {
                const int idx = tid + 256 * r;
                const int kk = akm ? (idx & (BK - 1)) : (idx / BM);
                const int mm = akm ? (idx / BK) : (idx & (BM - 1));
                const int64_t gm = m0 + mm, gk = k0 + kk;
                As[kk][mm] = (gm < M && gk < K) ? (akm ? A[gm * K + gk] : A[gk * M + gm]) : zero;
            }
#pragma unroll
            for (int r = 0; r < LB; ++r) {
                const int idx = tid + 256 * r;
                const int kk = bkm ? (idx & (BK - 1)) : (idx / BN);
                const int nn = bkm ? (idx / BK) : (idx & (BN - 1));
                const int64_t gn = n0 + nn, gk = k0 + kk;
                Bs[kk][nn] = (gn < N && gk < K) ? (bkm ? B[gn * K + gk] : B[gk * N + gn]) : zero;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float2 a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) pcfma(acc[i][j], a[i], b[j]);
            }
            __syncthreads();
            if (++stage == 4 || k0 + BK >= K) {
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
}

__device__ void exec_gemm(const POp& op, const PairCtx& c, float2* sm) {
    const int bm = op.mb >= 6 ? 64 : op.mb >= 5 ? 32 : 16;
    const int bn = op.nb >= 6 ? 64 : op.nb >= 5 ? 32 : 16;
    if (bm == 64 && bn == 64) exec_gemm_t<64, 64>(op, c, sm);
    else if (bm == 64 && bn == 32) exec_gemm_t<64, 32>(op, c, sm);
    else if (bm == 32 && bn == 64) exec_gemm_t<32, 64>(op, c, sm);
    else if (bm == 32 && bn == 32) exec_gemm_t<32, 32>(op, c, sm);
    else if (bm == 64) exec_gemm_t<64, 16>(op, c, sm);
    else if (bn == 64) exec_gemm_t<16, 64>(op, c, sm);
    else if (bm == 32) exec_gemm_t<32, 16>(op, c, sm);
    else if (bn == 32) exec_gemm_t<16, 32>(op, c, sm);
    else exec_gemm_t<16, 16>(op, c, sm);
}

// ---- long dot products (M * N <= 16): strided partials + fixed-order tree ----------------------
__device__ void exec_dot(const POp& op, const PairCtx& c, float2* sm) {
    const int64_t M = (int64_t)1 << op.mb, N = (int64_t)1 << op.nb, K = (int64_t)1 << op.kb;
    const int mn = (int)(M * N);
    const float2* A = pref_base(op.x, c);
    const float2* B = pref_base(op.y, c);
    float2* Cp = c.scratch + op.dst;
    const int tid = threadIdx.x;
    for (int o = 0; o < mn; ++o) {
        const int64_t m = o / N, n = o % N;
        float2 acc = make_float2(0.f, 0.f);
        for (int64_t k = tid; k < K; k += blockDim.x)
            pcfma(acc, op.a_km ? A[m * K + k] : A[k * M + m], op.b_km ? B[n * K + k] : B[k * N + n]);
        sm[tid] = acc;
        __syncthreads();
        for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
            if (tid < w) {
                sm[tid].x += sm[tid + w].x;
                sm[tid].y += sm[tid + w].y;
            }
            __syncthreads();
        }
        if (tid == 0) Cp[o] = sm[0];
        __syncthreads();
    }
}

// ---- the persistent kernel ---------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_persist(const PLaunch L) {
    extern __shared__ float2 psm[];
    __shared__ int64_t cur;
    float2* scratch = L.scratch + (int64_t)blockIdx.x * L.scratch_entries;
    for (;;) {
        if (threadIdx.x == 0) cur = (int64_t)atomicAdd((unsigned long long*)L.counter, 1ull);
        __syncthreads();
        const int64_t w = cur;
        __syncthreads();
        if (w >= L.n_work) break;
        // work item -> program and pair (programs are laid out back to back)
        int p = 0, hi = L.n_progs - 1;  // last program with work0 <= w
        while (p < hi) {
            const int mid = (p + hi + 1) >> 1;
            if (L.progs[mid].work0 <= w) p = mid;
            else hi = mid - 1;
        }
        const PProg& prog = L.n_progs ? L.progs[p] : L.single;
        const int64_t local = w - prog.work0;
        const int64_t sl = local / prog.n_b, bl = local % prog.n_b;
        PairCtx c;
        c.s = prog.s0 + sl;
        c.bits = prog.bits + (prog.b0 + bl) * prog.n_qubits;
        c.scratch = prog.scratch_override ? prog.scratch_override : scratch;
        c.prog = &prog;
        for (int i = 0; i < prog.n_ops; ++i) {
            const POp& op = prog.ops[i];
            switch (op.type) {
                case POP_PERM: exec_perm(op, c, psm); break;
                case POP_SMALL: exec_small(op, c, psm); break;
                case POP_GEMM: exec_gemm(op, c, psm); break;
                default: exec_dot(op, c, psm); break;
            }
            __syncthreads();
        }
        if (!prog.results) continue;  // a prologue program leaves its tensors in place
        // result vector of the pair, canonical open order
        const float2* root = pref_base(prog.root, c);
        const int64_t n_o = (int64_t)1 << prog.open_bits;
        float2* res = prog.results + local * n_o;
        for (int64_t o = threadIdx.x; o < n_o; o += blockDim.x) {
            int64_t rel = 0;
            for (int ob = 0; ob < prog.open_bits; ++ob)
                if ((o >> ob) & 1) rel += (int64_t)1 << prog.root.pos[prog.obit_leg[ob]];
            res[o] = root[rel];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
}

__device__ __forceinline__ void gsum_one(const GSum& g, int64_t local) {
    const int64_t n_o = (int64_t)1 << g.open_bits;
    const int64_t b = local >> g.open_bits, o = local & (n_o - 1);
    double sr = 0, si = 0, cr = 0, ci = 0;
    for (int s = 0; s < g.n_s; ++s) {
        const float2 v = g.results[((int64_t)s * g.n_b + b) * n_o + o];
        neumaier_add(sr, cr, (double)v.x);
        neumaier_add(si, ci, (double)v.y);
    }
    const double re = sr + cr, im = si + ci;
    g.amps[2 * local] = re * g.sr - im * g.si;
    g.amps[2 * local + 1] = re * g.si + im * g.sr;
}

__global__ void k_group_sum(const GSum* __restrict__ sums, int32_t n, int64_t total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int lo = 0, hi = n - 1;  // last program with t0 <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sums[mid].t0 <= t) lo = mid;
        else hi = mid - 1;
    }
    gsum_one(sums[lo], t - sums[lo].t0);
}

__global__ void k_single_sum(const GSum g, int64_t total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < total) gsum_one(g, t);
}

cudaError_t launch_single_sum(const GSum& g, int64_t total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    k_single_sum<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g, total);
    return cudaGetLastError();
}

cudaError_t launch_group_sum(const GSum* d_sums, int32_t n, int64_t total, cudaStream_t st) {
    if (total <= 0 || n <= 0) return cudaSuccess;
    k_group_sum<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(d_sums, n, total);
    return cudaGetLastError();
}

// ---- the invariant steps in one launch -----------------------------------------------------------
// The steps that no slice or bitstring touches are mostly tiny (gate-sized tensors).  The plan
// compiler splits them into chains that share no storage (their dependency trees, with the
// invariant region given no reuse): CTA c runs the steps of chain c in plan order with the code of
// the persistent executor, a block barrier between steps, and waits for no other CTA.
__global__ void __launch_bounds__(256, 2) k_chain(const POp* __restrict__ ops, const int32_t* __restrict__ idx,
                                                  const int32_t* __restrict__ starts, const PProg prog) {
    extern __shared__ float2 psm[];
    PairCtx c;
    c.s = 0;
    c.bits = prog.bits;
    c.scratch = prog.scratch_override;
    c.prog = &prog;
    const int i1 = starts[blockIdx.x + 1];
    for (int i = starts[blockIdx.x]; i < i1; ++i) {
        const POp& op = ops[idx[i]];
        switch (op.type) {
            case POP_PERM: exec_perm(op, c, psm); break;
            case POP_SMALL: exec_small(op, c, psm); break;
            case POP_GEMM: exec_gemm(op, c, psm); break;
            default: exec_dot(op, c, psm); break;
        }
        __syncthreads();  // this step's results (global and shared) before the next step reads them
    }
}

cudaError_t launch_chains(const POp* ops, const int32_t* idx, const int32_t* starts, int n_chains, const PProg& prog,
                          cudaStream_t st) {
    if (n_chains <= 0) return cudaSuccess;
    k_chain<<<n_chains, 256, kPersistSmem, st>>>(ops, idx, starts, prog);
    return cudaGetLastError();
}

cudaError_t launch_persist(const PLaunch& L, int grid, cudaStream_t st) {
    if (L.n_work <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_persist<<<grid, 256, kPersistSmem, st>>>(L);
    return cudaGetLastError();
}

}  // namespace qx
