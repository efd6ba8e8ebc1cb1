// Internal interface between the host orchestration (qx_host.cpp) and the
// CUDA kernels (qx_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qx {

constexpr int kMaxRank = 48;   // effective legs of one operand
constexpr int kMaxFix = 8;     // fixed (sliced / output) legs of one leaf
constexpr int kSmallMaxK = 5;  // shared bits handled by the gather kernel
constexpr int kSmallMaxN = 5;  // free bits of its small operand
constexpr int kMaxBatchItems = 65535;

// The (slice, bitstring) pairs of one batch: item = s_local * n_b + b_local.
struct ItemCtx {
    int64_t s0;            // first slice of the batch
    int64_t b0;            // first bitstring of the batch
    int64_t n_items;       // pairs in the batch
    int32_t n_b;           // bitstrings per slice in the batch
    int32_t n_qubits;      // bytes per bitstring
    const uint8_t* bits;   // device bitstrings [n_bits][n_qubits]
};

// Address of entry (leg bits) of an operand for item i:
//   base + i' * item_stride + sum_f value_f * fix_stride[f] + sum_j bit_j << pos[j]
// where i' = i, or i / n_b (the item's slice within the batch) for a per-slice
// tensor read by per-pair work (per_slice = 1; in launches over slices n_b = 1).
// value_f is bit fix_src[f] of the slice index (fix_src >= 0) or the byte of
// output qubit -(fix_src+1) of the bitstring (fix_src < 0).  Leg 0 is the
// most significant; positions are strictly decreasing in leg order.
struct Operand {
    const float2* base;
    int64_t item_stride;
    int32_t n_fix;
    int32_t rank;
    int32_t per_slice;
    int32_t pad;
    int32_t fix_src[kMaxFix];
    int64_t fix_stride[kMaxFix];
    int8_t pos[kMaxRank];
};

// Bit permutation out[y] = in[x]: output bit ob (0 = least significant) is
// taken from input address position in_pos[ob].  The tile holds `t` bits
// (at most kPermTileBits): tile_in lists them (as output-bit ids) by
// increasing input position, tile_out by increasing output bit; `outer` lists
// the remaining output bits.
constexpr int kPermTileBits = 12;  // batched kernel: 2^12-entry tiles, 6 + 6 index bits
constexpr int kPermLoBits = 6;
struct PermDesc {
    Operand in;
    int32_t rank;
    int32_t t;
    int32_t n_outer;
    int8_t in_pos[kMaxRank];
    int8_t tile_in[kPermTileBits];
    int8_t tile_out[kPermTileBits];
    int8_t outer[kMaxRank];
};

// Address tables of a permutation tile, computed once on the host: entry j
// of the tile (input order) sits at in_lo[j & 63] + in_hi[j >> 6] from the
// tile's input base; entry j (output order) goes to out_lo[..] + out_hi[..]
// from the output base and is read from tile slot map_lo[..] | map_hi[..];
// outer bit i moves the bases by outer_in[i] / outer_out[i].
struct PermTables {
    int64_t in_lo[64], in_hi[64], out_lo[64], out_hi[64];
    int32_t map_lo[64], map_hi[64];
    int64_t outer_in[kMaxRank], outer_out[kMaxRank];
};

// Gather contraction with one small operand Y (<= 2^10 entries):
//   C[m * 2^nb + n] = sum_k X[m, k] * Y[k, n]
// m enumerates X's free legs (bit i = i-th lowest free position), k the
// shared legs, n Y's free legs (in Y's leg order, last leg = bit 0).
// Placement of a product in memory: bit i of the kernel's natural product index (the column bits
// first, bit 0 lowest, then the row bits) goes to address position pos[i].  on = 0: the natural
// row-major layout.  Chosen by the plan compiler so that the next GEMM reads the product without a
// permute; the lowest positions always come from the side the kernel's lanes run along.
struct OutMap {
    int8_t pos[kMaxRank];
    int32_t on;
};

struct SmallDesc {
    Operand x, y;
    int32_t mb, kb, nb;
    int32_t n_holes;           // X positions that are not free (shared + fixed), ascending
    int8_t holes[kMaxRank];
    int8_t xk_pos[kSmallMaxK]; // X position of shared bit i of k
    int8_t yk_pos[kSmallMaxK]; // Y position of shared bit i of k
    int8_t yn_pos[kSmallMaxN]; // Y position of bit i of n
    OutMap om;                 // product placement (natural bits: n, then m)
};

// Cross-slice FP64 compensated sum of the root tensor into accumulators.
struct SumDesc {
    Operand root;
    int32_t open_bits;
    int32_t n_s;               // slices in the batch
    int8_t obit_pos[kMaxRank]; // root position of canonical open bit ob (0 = least significant)
};

// Launchers; each returns the launch error (cudaSuccess on success).
cudaError_t launch_permute(const PermDesc& d, const ItemCtx& ic, int64_t n_items, float2* out,
                           int64_t out_item_stride, cudaStream_t st);
void perm_tables(const PermDesc& d, PermTables* tb);
// per pair C = sum_k A[k] B[p(k)]: B = d.in read through the permutation d, A in the target order
// a_div / b_div: item i reads operand item i / div (n_b for a per-slice tensor
// read by per-pair work, else 1)
cudaError_t launch_dot_perm(const PermDesc& d, const ItemCtx& ic, int64_t n_items, const float2* a, int64_t a_is,
                            float2* c, int64_t c_is, cudaStream_t st, int a_div = 1);
// whether launch_small runs this gather as k_small_flat (short per-pair rows, small operand read
// through L1) rather than k_small (small operand staged in shared memory)
bool small_is_flat(const SmallDesc& d);
cudaError_t launch_small(const SmallDesc& d, const ItemCtx& ic, int64_t n_items, float2* out,
                         int64_t out_item_stride, cudaStream_t st);
// Batched complex GEMM, C[M][N] = A . B with A stored [M][K] (a_kmajor) or
// [K][M], B stored [N][K] (b_kmajor) or [K][N]; M = 2^mb etc.
cudaError_t launch_gemm_c64(const float2* a, int64_t a_is, bool a_kmajor, const float2* b, int64_t b_is,
                            bool b_kmajor, float2* c, int64_t c_is, int mb, int nb, int kb, int64_t n_items,
                            cudaStream_t st, const OutMap* om = nullptr, int a_div = 1, int b_div = 1);
cudaError_t launch_slice_sum(const SumDesc& d, const ItemCtx& ic, double* acc, cudaStream_t st);

// Persistent executor (qx_persist.cu): one launch runs whole contractions of
// (slice, bitstring) pairs, one pair per CTA at a time, steps in order.
enum { PSPACE_LEAF = 0, PSPACE_INV = 1, PSPACE_SCRATCH = 2 };
enum { POP_PERM = 0, POP_SMALL = 1, POP_GEMM = 2, POP_DOT = 3 };
struct PRef {                  // an operand: leaf (with fixed legs), invariant tensor or CTA scratch
    int64_t off;               // entries into the leaf buffer / invariant region / CTA scratch
    int32_t space;
    int32_t rank;
    int32_t n_fix;
    int32_t fix_src[kMaxFix];
    int64_t fix_stride[kMaxFix];
    int8_t pos[kMaxRank];
};
struct POp {
    int32_t type, mb, kb, nb, a_km, b_km;
    int64_t dst;               // CTA scratch offset of the result (contiguous)
    PRef x, y;                 // PERM: x; SMALL: x large, y small; GEMM / DOT: x = A, y = B (contiguous)
    int32_t t, n_outer, n_holes;
    int8_t in_pos[kMaxRank], tile_in[10], tile_out[10], outer[kMaxRank];
    int8_t holes[kMaxRank], xk_pos[kSmallMaxK], yk_pos[kSmallMaxK], yn_pos[kSmallMaxN];
};
struct PProg {
    const POp* ops;            // device
    int32_t n_ops;
    int32_t n_qubits;
    const float2* leaves;      // device
    const float2* inv;         // device
    const uint8_t* bits;       // device [n_bits][n_qubits]
    int64_t s0, b0;            // first slice / bitstring of this program's work
    int64_t n_b;               // bitstrings per slice: pair = s_local * n_b + b_local
    int64_t work0;             // first global work index of this program
    PRef root;
    int32_t open_bits;
    int8_t obit_leg[kMaxRank]; // root leg of canonical open bit ob (0 = least significant)
    float2* results;           // device [pairs][2^open_bits]; null: no result (prologue programs)
    float2* scratch_override;  // non-null: results of the ops go here (prologue programs: the invariant region)
};
struct PLaunch {
    PProg single;              // used when n_progs == 0
    const PProg* progs;        // device, ordered by work0
    int32_t n_progs;
    int64_t n_work;
    float2* scratch;           // grid x scratch_entries
    int64_t scratch_entries;
    unsigned long long* counter;
};
constexpr int kPersistSmem = 17408;
cudaError_t launch_persist(const PLaunch& L, int grid, cudaStream_t st);
// one launch of n independent invariant steps: CTA i runs ops[idx[i]] (device arrays)
// n_chains CTAs; CTA c runs ops[idx[starts[c]]], ops[idx[starts[c] + 1]], ... up to starts[c + 1], in
// order, with a block barrier between steps (device arrays idx and starts)
cudaError_t launch_chains(const POp* ops, const int32_t* idx, const int32_t* starts, int n_chains, const PProg& prog,
                          cudaStream_t st);

// FP64 compensated slice sum of persistent results, for many programs in one
// launch, written straight to the amplitudes (times the leaf scale).
struct GSum {
    const float2* results;     // [n_s * n_b][2^open_bits], pair = s * n_b + b
    double* amps;              // [n_b][2^open_bits] complex128
    int64_t n_b;
    int64_t t0;                // first global thread of this program
    int32_t n_s;
    int32_t open_bits;
    double sr, si;             // leaf scale
};
cudaError_t launch_group_sum(const GSum* d_sums, int32_t n, int64_t total, cudaStream_t st);
cudaError_t launch_single_sum(const GSum& g, int64_t total, cudaStream_t st);

// Tensor-core complex GEMM (qx_tc.cu).  Operands are contiguous complex64
// per item, [R][K] (kmajor) or [K][R]; pa / pb receive the split real parts
// (prep), then the tcgen05 kernel writes C [M][N] complex64.
constexpr int TC_FORM_3XTF32 = 1, TC_FORM_BF16X3 = 2, TC_FORM_FP16 = 3;
constexpr int TC_FORM_3XTF32_DIRECT = 4;  // 3xTF32 split in shared memory (launch_tc2_gemm)
// A read where it is stored by the resident-B' direct kernel (no permuted copy): bit i of the row
// index sits at address position mpos[i], bit i of the complex K index at kpos[i].  The tile of one
// stage (row bits 0..6 of a 128-row job, K bits 0..3 of its 16 K entries) covers address positions
// 0 .. run - 1 and nblk - 1 = 2^(11 - run) - 1 combinations of its other bits: nblk contiguous blocks
// of 2^run entries, block b at blk_off[b] from the tile's base, copied to entries b * 2^run of the
// landing slot, where row r / K entry j of the stage sit at lrow[r] + lk[j].
struct AGather {
    int32_t on;
    int32_t run, nblk;
    int8_t mpos[kMaxRank];
    int8_t kpos[16];
    int64_t blk_off[8];
    int16_t lrow[128];
    int16_t lk[16];
};
// fills run, nblk, blk_off, lrow and lk from mpos / kpos (mb >= 7, kb >= 4); false when the stage tile
// is not made of at most 8 contiguous blocks
bool agather_tile(AGather* g, int mb, int kb);

struct TcArgs {
    const float2* a;
    int64_t a_is;
    bool a_kmajor;
    const float2* b;
    int64_t b_is;
    bool b_kmajor;
    float2* c;
    int64_t c_is;
    void* pa;
    int64_t pa_is_bytes;
    void* pb;
    int64_t pb_is_bytes;
    int mb, nb, kb;
    int64_t n_items;
    int a_div, b_div;  // item i reads operand item i / div (0 taken as 1); ignored for an item stride of 0
    long long limit;  // clock cycles per bounded wait
    int* err;         // device error flag (QX_ETIMEOUT on expiry)
    float* amax;      // FP16 form: device max |x| of A and B (2 floats), sets the per-tensor scales
    AGather ag;       // direct kernel: A gathered in place (on = 1; only with B' resident, tc2_resident_b)
};
int tc_parts_a(int form);
int tc_parts_b(int form);
int tc_elem_bytes(int form);
int tc_products(int form);
cudaError_t launch_tc_prep(int form, const TcArgs& g, cudaStream_t st);
cudaError_t launch_tc_gemm(int form, const TcArgs& g, cudaStream_t st);
// 3xTF32 directly on the complex64 operands (split in shared memory; no pa / pb)
cudaError_t launch_tc2_gemm(const TcArgs& g, cudaStream_t st);
// whether launch_tc2_gemm runs g on the kernel with B' resident per CTA (k_gemm_tc2kb)
bool tc2_resident_b(const TcArgs& g);
// amps[i] = (sum + compensation) * (scale_re + i scale_im), all in FP64
cudaError_t launch_finalize(const double* acc, double* amps, int64_t n, double scale_re, double scale_im,
                            cudaStream_t st);

}  // namespace qx

// Contract every slice with `buf` (device, 256-byte aligned, buf_bytes long)
// standing in for the bound workspace; the bound workspace, if any, is left
// untouched.  Defined in qx_host.cpp for entry points that bring their own
// device memory.
struct qx_ctx;
int qx_internal_contract_in(qx_ctx* h, char* buf, int64_t buf_bytes, const uint8_t* d_bits, int64_t n_bits,
                            double* d_amps);
int qx_internal_device(const qx_ctx* h);
int qx_internal_fail(qx_ctx* h, int code, const char* msg);
cudaStream_t qx_internal_stream(const qx_ctx* h);
// 256 bytes of device memory owned by the handle (NULL if the allocation fails)
void* qx_internal_small(qx_ctx* h);
// qubits and open outputs of the built network (0 without one), the
// bitstrings per call the bound workspace takes (0 unbound), and whether a
// plan and a workspace are both in place
int qx_internal_shape(const qx_ctx* h, int* n_qubits, int64_t* n_open, int64_t* max_bits, int* ready);
