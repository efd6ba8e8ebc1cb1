// Empirical-supremum rejection sampling of output bitstrings (Sec. III-B).
//
// The sampler's law is p(x) = |<x|C|0>|^2 over the N = 2^n bitstrings, its
// proposal is uniform, and candidate x has density ratio w = p(x) N.  Each
// iteration accepts its candidate X when U < w(X) / M and afterwards sets
// M = max(M, w(X)); M starts at 1 and a warm-up of iterations only moves M.
//
// The iterations look sequential, but the candidates and uniforms are drawn
// independently of the outcomes, so a whole batch is known in advance.  The
// bound an iteration tests against is then an exclusive prefix maximum of
// the batch's w (joined with the bound carried in), and the accepted
// iterations are a stream compaction of the tests: both are scans, done
// here by one CTA that walks the batch in chunks.  The result equals the
// one-at-a-time algorithm's exactly: max is exact in any order, and every
// rounded operation (re*re, im*im, their sum, the product by N, U*M) is
// evaluated as written with no contraction into an FMA.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "qx.h"
#include "qx_internal.h"

namespace {

constexpr int kThreads = 1024;
constexpr int kPer = 8;  // consecutive candidates per thread in a chunk
constexpr int kChunk = kThreads * kPer;

struct EsupResult {
    double m;            // bound after the last consumed iteration
    long long accepted;  // accepted candidates written
    long long consumed;  // iterations consumed
    long long pad;
};

// max(a, b) in the update's sense: a NaN b never replaces a
__device__ __forceinline__ double sup(double a, double b) { return b > a ? b : a; }

__global__ void __launch_bounds__(kThreads)
    k_esup(const double2* __restrict__ amps, const double* __restrict__ uni, int64_t n, double n_total,
           int64_t n_warmup, int64_t max_out, double m_in, int64_t idx_base, int64_t* __restrict__ accepted,
           EsupResult* __restrict__ res) {
    __shared__ double s_wmax[kThreads / 32];
    __shared__ int s_wcnt[kThreads / 32];
    __shared__ long long s_stop;
    __shared__ double s_mstop;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const double kNone = -INFINITY;
    if (t == 0) s_stop = -1;
    double carry = m_in;  // bound before the chunk
    long long done = 0;   // accepted before the chunk
    for (int64_t c0 = 0; c0 < n; c0 += kChunk) {
        // density ratios of this thread's candidates and their running max
        double w[kPer], ex[kPer];
        double run = kNone;
        const int64_t i0 = c0 + (int64_t)t * kPer;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t i = i0 + k;
            double wk = kNone;
            if (i < n) {
                const double2 a = amps[i];
                wk = __dmul_rn(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)), n_total);
            }
            w[k] = wk;
            ex[k] = run;
            run = sup(run, wk);
        }
        // exclusive prefix max over the threads of the block
        double inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = sup(v, inc);
        }
        if (lane == 31) s_wmax[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            double v = s_wmax[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double x = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v = sup(x, v);
            }
            s_wmax[lane] = v;  // inclusive over warps
        }
        __syncthreads();
        double before = __shfl_up_sync(0xffffffffu, inc, 1);
        if (lane == 0) before = kNone;
        if (warp > 0) before = sup(s_wmax[warp - 1], before);
        const double m_thread = sup(carry, before);
        const double chunk_max = s_wmax[kThreads / 32 - 1];

        // the rejection tests, against the bound before each iteration
        unsigned hits = 0;
        double m_at[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t i = i0 + k;
            const double m = sup(m_thread, ex[k]);
            m_at[k] = m;
            if (i < n && i >= n_warmup && __dmul_rn(uni[i], m) < w[k]) hits |= 1u << k;
        }
        // exclusive prefix count of the hits
        const int cnt = __popc(hits);
        int cinc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, cinc, o);
            if (lane >= o) cinc += v;
        }
        if (lane == 31) s_wcnt[warp] = cinc;
        __syncthreads();
        if (warp == 0) {
            int v = s_wcnt[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += x;
            }
            s_wcnt[lane] = v;
        }
        __syncthreads();
        long long pos = done + (cinc - cnt) + (warp > 0 ? s_wcnt[warp - 1] : 0);
        const int chunk_cnt = s_wcnt[kThreads / 32 - 1];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (!(hits >> k & 1u)) continue;
            if (pos < max_out) accepted[pos] = idx_base + i0 + k;
            if (pos == max_out - 1) {  // the run stops right after this iteration
                s_stop = i0 + k + 1;
                s_mstop = sup(m_at[k], w[k]);
            }
            ++pos;
        }
        carry = sup(carry, chunk_max);
        done += chunk_cnt;
        __syncthreads();
        if (s_stop >= 0) break;
    }
    if (t == 0) {
        if (s_stop >= 0) {
            res->m = s_mstop;
            res->accepted = max_out;
            res->consumed = s_stop;
        } else {
            res->m = carry;
            res->accepted = done;
            res->consumed = n;
        }
    }
}

int run_accept(qx_ctx* h, const double* d_amps, const double* d_uniforms, int64_t n, int32_t n_qubits,
               int64_t n_warmup, int64_t max_out, double* m_io, int64_t idx_base, int64_t* d_accepted,
               int64_t* n_accepted, int64_t* n_consumed) {
    EsupResult* d_res = (EsupResult*)qx_internal_small(h);
    if (!d_res) return qx_internal_fail(h, QX_ECUDA, "cudaMalloc of the sampler's result buffer failed");
    cudaStream_t st = qx_internal_stream(h);
    k_esup<<<1, kThreads, 0, st>>>((const double2*)d_amps, d_uniforms, n, std::ldexp(1.0, n_qubits), n_warmup,
                                   max_out, *m_io, idx_base, d_accepted, d_res);
    if (cudaGetLastError() != cudaSuccess) return qx_internal_fail(h, QX_ECUDA, "sampler kernel launch failed");
    EsupResult r;
    if (cudaMemcpyAsync(&r, d_res, sizeof r, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return qx_internal_fail(h, QX_ECUDA, "sampler result copy failed");
    *m_io = r.m;
    *n_accepted = r.accepted;
    *n_consumed = r.consumed;
    return QX_OK;
}

}  // namespace

extern "C" {

int qx_esup_accept(qx_handle h, const double* d_amps, const double* d_uniforms, int64_t n_cand, int32_t n_qubits,
                   int64_t n_warmup, int64_t max_out, double* m_inout, int64_t* d_accepted, int64_t* n_accepted,
                   int64_t* n_consumed) {
    if (!h) return QX_EINVAL;
    if (!m_inout || !n_accepted || !n_consumed) return qx_internal_fail(h, QX_EINVAL, "null result pointer");
    if (n_cand < 0 || n_warmup < 0 || max_out < 0) return qx_internal_fail(h, QX_EINVAL, "negative count");
    if (n_qubits < 1 || n_qubits > 62) return qx_internal_fail(h, QX_EINVAL, "n_qubits out of range [1, 62]");
    *n_accepted = 0;
    *n_consumed = 0;
    if (n_cand == 0 || max_out == 0) return QX_OK;
    if (!d_amps || !d_uniforms || !d_accepted) return qx_internal_fail(h, QX_EINVAL, "null device buffer");
    const int dev = qx_internal_device(h);
    if (dev < 0) return qx_internal_fail(h, QX_ESTATE, "host-only handle has no device");
    if (cudaSetDevice(dev) != cudaSuccess) return qx_internal_fail(h, QX_ECUDA, "cudaSetDevice failed");
    return run_accept(h, d_amps, d_uniforms, n_cand, n_qubits, n_warmup, max_out, m_inout, 0, d_accepted, n_accepted,
                      n_consumed);
}

int qx_esup_sample(qx_handle h, const uint8_t* d_candidates, const double* d_uniforms, int64_t n_cand,
                   int64_t n_warmup, int64_t max_out, double* m_inout, double* d_amps, int64_t* d_accepted,
                   int64_t* n_accepted, int64_t* n_consumed) {
    if (!h) return QX_EINVAL;
    if (!m_inout || !n_accepted || !n_consumed) return qx_internal_fail(h, QX_EINVAL, "null result pointer");
    if (n_cand < 0 || n_warmup < 0 || max_out < 0) return qx_internal_fail(h, QX_EINVAL, "negative count");
    int nq = 0, ready = 0;
    int64_t n_open = 0, max_bits = 0;
    qx_internal_shape(h, &nq, &n_open, &max_bits, &ready);
    if (!nq) return qx_internal_fail(h, QX_ESTATE, "sampling before qx_build_network");
    if (n_open) return qx_internal_fail(h, QX_EINVAL, "sampling needs every output closed (no open qubits)");
    if (!ready) return qx_internal_fail(h, QX_ESTATE, "sampling needs a plan and a bound workspace");
    *n_accepted = 0;
    *n_consumed = 0;
    if (n_cand == 0 || max_out == 0) return QX_OK;
    if (!d_candidates || !d_uniforms || !d_amps || !d_accepted)
        return qx_internal_fail(h, QX_EINVAL, "null device buffer");
    int64_t used = 0, acc = 0;
    while (used < n_cand && acc < max_out) {
        const int64_t cnt = n_cand - used < max_bits ? n_cand - used : max_bits;
        int rc = qx_contract_device(h, d_candidates + used * nq, cnt, d_amps + 2 * used);
        if (rc != QX_OK) return rc;
        if ((rc = qx_device_status(h)) != QX_OK) return rc;
        int64_t a = 0, c = 0;
        const int64_t warm = n_warmup > used ? n_warmup - used : 0;
        rc = run_accept(h, d_amps + 2 * used, d_uniforms + used, cnt, nq, warm, max_out - acc, m_inout, used,
                        d_accepted + acc, &a, &c);
        if (rc != QX_OK) return rc;
        acc += a;
        used += c;
        if (c < cnt) break;  // stopped at the max_out-th acceptance
    }
    *n_accepted = acc;
    *n_consumed = used;
    return QX_OK;
}

}  // extern "C"
