// Host side of libqx: the circuit network (Sec. II), plan validation and
// compilation (Sec. III-A order and slicing), the workspace plan, and the
// batched executor that drives the kernels in qx_kernels.cu.
//
// Execution model.  The contraction of every (slice, bitstring) pair follows
// the same plan, so the pairs of a batch are contracted together: each plan
// step is one kernel launch over all pairs of the batch (the slice-parallel
// and bitstring-parallel levels of Sec. IV-A inside one launch).  Sliced
// bonds and the closed output wires are "fixed" bonds: a leaf tensor touching
// one is read at the offset that the pair's slice bit or bitstring byte
// selects, so slicing never copies data.  Intermediates that depend on no
// fixed bond are the same for every pair; they are computed once per call
// (prologue) and read by every pair with item stride 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <limits>
#include <map>
#include <string>
#include <vector>

#include "qx.h"
#include "qx_internal.h"

using namespace qx;

namespace {

constexpr int64_t kAlignEntries = 32;  // 256 bytes
constexpr int64_t kLive = std::numeric_limits<int64_t>::max() / 4;

int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

struct Node {
    std::vector<int> legs;  // bond ids, leg 0 most significant
    std::vector<int> pos;   // address bit of each leg
    std::vector<std::pair<int32_t, int64_t>> fix;  // (source, stride) of fixed legs
    bool const_one = false;
    bool variant = false;   // level > 0
    int level = 0;          // 0: invariant, 1: depends on the slice only, 2: on the bitstring (and slice)
    bool leaf = false;
    int64_t leaf_off = 0;   // entries into the leaf buffer
    int storage = -1;       // intermediate storage id
    int under_rank = 0;     // rank of the stored tensor
};

struct Storage {
    int64_t entries = 0;
    bool variant = false;   // level > 0
    int level = 0;          // region: 0 invariant, 1 per slice, 2 per pair
    int64_t def = 0, last = 0;
    int64_t off = 0;        // entries within its region (per pair for the item region)
};

enum OpType { OP_PERM, OP_SMALL, OP_GEMM };

struct Op {
    OpType type;
    bool variant;           // level > 0
    int level = 0;          // runs once (0), per slice (1) or per pair (2)
    int64_t step;
    // OP_PERM: node -> storage
    int src = -1;
    std::vector<int> target_legs;
    // OP_SMALL: x, y nodes
    int x = -1, y = -1;
    std::vector<int> shared;
    std::vector<int> fy;    // Y's free legs in the order they take in the product
    // output position of each bit of the kernel's natural product index (columns low, then rows);
    // empty: the natural layout
    std::vector<int8_t> out_pos;
    // a step contracting every leg with one operand in another order: that operand (perm_src) is
    // read through the permutation to perm_legs (the other operand's order) inside the dot kernel
    bool dot_perm = false;
    int perm_src = -1;
    std::vector<int> perm_legs;
    // OP_GEMM: operand storages, shapes
    int sa = -1, sb = -1;
    bool a_km = true, b_km = true;
    int mb = 0, nb = 0, kb = 0;
    int dst = -1;           // output storage
    int tc = 0;             // tensor-core form (0: SIMT)
    int spa = -1, spb = -1; // split-part storages of the tensor-core form
    // direct 3xTF32 step on the resident-B' kernel that reads A where it is stored (no permute): address
    // position of each row bit and of each complex K bit of A
    bool a_gather = false;
    std::vector<int8_t> ag_mpos, ag_kpos;
    double flops = 0;
};

}  // namespace

struct qx_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    void* d_small = nullptr;  // 256 device bytes for small results (sampler counts), allocated on first use
    qx_options opt{};
    std::string err;

    // network
    bool have_net = false;
    int nq = 0;
    std::vector<qx_gate> gates;
    std::vector<uint8_t> open_mask;
    int64_t n_tensors = 0, n_bonds = 0;
    std::vector<std::vector<int>> tensor_legs;   // canonical legs of each leaf tensor
    std::vector<int64_t> tensor_vals_off;        // offset of its values in leaf_vals (-1: output)
    std::vector<float2> leaf_vals;
    std::vector<int> final_wire;                 // per qubit
    std::vector<int> open_wires;                 // final wires of open qubits, increasing qubit
    std::vector<int> bond_deg;                   // tensors touching each bond
    double leaf_scale[2] = {1.0, 0.0};           // product over leaves of alpha (complex, FP64)

    // plan
    bool have_plan = false;
    std::vector<int64_t> sliced;
    std::vector<Node> nodes;
    std::vector<Storage> stor;
    std::vector<Op> ops;
    int root = -1;
    int64_t peak_entries = 0;
    int64_t item_entries = 0;  // per pair
    int64_t slice_entries = 0; // per slice (intermediates that no output bit touches)
    int64_t inv_entries = 0;
    int64_t n_slices = 1;
    double flops_inv = 0, flops_slice = 0, flops_item = 0;

    // persistent executor program (variant ops, in order)
    bool persist_ok = false;
    std::vector<POp> pops;      // per-pair ops
    std::vector<POp> pops_inv;  // invariant ops (prologue program)
    PRef proot{};
    std::vector<int8_t> pobit_leg;
    int persist_grid = 0;
    bool pops_on_device = false;

    // batched executor prologue: the invariant steps as chains that share no storage, one launch,
    // one CTA per chain (only when every invariant step is small)
    bool wave_ok = false;
    std::vector<POp> wave_ops;          // one per invariant op, grouped by chain
    std::vector<int32_t> wave_idx;      // 0 .. n-1 (positions into wave_ops)
    std::vector<int32_t> wave_start;    // chain c: wave_ops[wave_start[c] .. wave_start[c + 1])
    std::vector<int> wave_of;           // per op: 0 if the prologue launch runs it, else -1
    std::vector<int> chain_of_op;       // per op: its prologue chain, -1 if none
    std::vector<double> wave_flops, wave_bytes;
    bool waves_on_device = false;
    std::vector<cudaEvent_t> wave_ev;

    // workspace
    char* ws = nullptr;
    int64_t ws_bytes = 0;
    bool ws_owned = false;
    int64_t max_bits = 0;
    int64_t off_err = 0, off_leaf = 0, off_bits = 0, off_acc = 0, off_amps = 0, off_inv = 0, off_item = 0;
    int64_t off_slice = 0, slices_cap = 0;  // per-slice region: room for slices_cap slices
    int64_t off_pops = 0, off_counter = 0, off_results = 0, off_pscratch = 0, off_pops_inv = 0, off_wave = 0;
    int64_t items_cap = 0;
    bool leaves_on_device = false;

    // stats
    double last_flops = 0;
    int64_t last_launches = 0, last_batches = 0;

    // CUDA graph of a repeated contraction (same buffers, sizes and slice range)
    bool graphs = true;
    bool memo = false;       // keep the invariant intermediates across calls (qx_set_memo)
    bool inv_ready = false;  // the bound workspace holds them
    char* static_err = nullptr;  // error flag of the last static-scratch call, until qx_device_status reads it
    char* wb = nullptr;          // qx_bind_workspace_parts: the batch regions' own buffer (else inside ws)
    // Parts of one compensated slice sum (qx_submit_part): the next contraction clears the FP64
    // accumulators first (part_clear) and writes the amplitudes at the end (part_final); a sum left
    // open continues at slice part_next with the same bitstrings.
    bool part_clear = true, part_final = true, part_open = false;
    const uint8_t* part_bits = nullptr;
    int64_t part_nbits = 0, part_next = 0;
    struct {
        const uint8_t* bits = nullptr;
        double* amps = nullptr;
        int64_t n_bits = -1, s0 = -1, s1 = -1;
        bool clear = true, final_ = true;
        int seen = 0;
        cudaGraphExec_t exec = nullptr;
        double flops = 0;
        int64_t launches = 0, batches = 0;
    } gc;

    // Concurrent issue: op j follows the earlier ops in deps[j] (data and space-reuse hazards), so
    // independent branches of the contraction tree run side by side on the handle's extra streams
    // (their order in a captured graph becomes graph edges).  n_streams 1: all on `stream`, in order.
    // asynchronous requests (qx_submit / qx_poll): completion events by request number
    std::map<int64_t, cudaEvent_t> reqs;
    std::vector<cudaEvent_t> req_pool;
    int64_t next_req = 1;

    int n_streams = 8;
    bool fuse_layouts = true;  // products stored in the layout their consuming GEMM reads (batched executor)
    std::vector<std::vector<int>> deps;
    std::vector<cudaStream_t> dstreams;
    std::vector<cudaEvent_t> op_ev;    // one per op
    std::vector<cudaEvent_t> join_ev;  // one per extra stream
    cudaEvent_t fork_ev = nullptr;

    // profiling: an event pair around every launch, folded per kernel kind on read
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Rec { int kind; size_t e0; double flops, bytes; };
    std::vector<Rec> recs;
    double prof_ms[QX_KERNEL_KINDS] = {0}, prof_flops[QX_KERNEL_KINDS] = {0}, prof_bytes[QX_KERNEL_KINDS] = {0};
    int64_t prof_launches[QX_KERNEL_KINDS] = {0};
};

static int fail(qx_ctx* h, int code, const char* fmt, ...);
static void drop_graph(qx_ctx* h) {
    if (h->gc.exec) cudaGraphExecDestroy(h->gc.exec);
    h->gc.exec = nullptr;
    h->gc.seen = 0;
    h->gc.bits = nullptr;
    h->gc.amps = nullptr;
    h->gc.n_bits = h->gc.s0 = h->gc.s1 = -1;
}


static cudaError_t prof_begin(qx_ctx* h, int kind, double flops, double bytes, size_t* slot) {
    *slot = SIZE_MAX;
    if (!h->profiling) return cudaSuccess;
    while (h->ev_used + 2 > h->ev_pool.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        h->ev_pool.push_back(e);
    }
    *slot = h->ev_used;
    h->ev_used += 2;
    h->recs.push_back({kind, *slot, flops, bytes});
    return cudaEventRecord(h->ev_pool[*slot], h->stream);
}

static cudaError_t prof_end(qx_ctx* h, size_t slot) {
    if (slot == SIZE_MAX) return cudaSuccess;
    return cudaEventRecord(h->ev_pool[slot + 1], h->stream);
}

// fold recorded event pairs into the per-kind totals (synchronises the stream)
static int prof_collect(qx_ctx* h) {
    if (h->recs.empty()) return QX_OK;
    cudaError_t r = cudaStreamSynchronize(h->stream);
    if (r != cudaSuccess) return fail(h, QX_ECUDA, "profile sync: %s", cudaGetErrorString(r));
    for (const auto& rc : h->recs) {
        float ms = 0;
        r = cudaEventElapsedTime(&ms, h->ev_pool[rc.e0], h->ev_pool[rc.e0 + 1]);
        if (r != cudaSuccess) return fail(h, QX_ECUDA, "profile events: %s", cudaGetErrorString(r));
        h->prof_ms[rc.kind] += ms;
        h->prof_flops[rc.kind] += rc.flops;
        h->prof_bytes[rc.kind] += rc.bytes;
        h->prof_launches[rc.kind] += 1;
    }
    h->recs.clear();
    h->ev_used = 0;
    return QX_OK;
}

static int fail(qx_ctx* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    h->err = buf;
    return code;
}

#define CUDA_TRY(h, expr)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) return fail(h, QX_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------------------------------------
// Network (Sec. II)
// ------------------------------------------------------------------------------------------------
static int build_network(qx_ctx* h, int32_t n, const qx_gate* gates, int64_t ng, const uint8_t* open_mask) {
    if (n < 1 || n > 62) return fail(h, QX_EINVAL, "n_qubits %d out of range [1, 62]", n);
    if (ng < 0 || (ng > 0 && !gates)) return fail(h, QX_EINVAL, "bad gate list");
    for (int64_t g = 0; g < ng; ++g) {
        const qx_gate& gt = gates[g];
        if (gt.nq != 1 && gt.nq != 2) return fail(h, QX_EINVAL, "gate %lld: nq = %d", (long long)g, gt.nq);
        for (int j = 0; j < gt.nq; ++j)
            if (gt.q[j] < 0 || gt.q[j] >= n)
                return fail(h, QX_EINVAL, "gate %lld: qubit %d out of range", (long long)g, gt.q[j]);
        if (gt.nq == 2 && gt.q[0] == gt.q[1]) return fail(h, QX_EINVAL, "gate %lld: repeated qubit", (long long)g);
    }
    h->have_net = false;
    h->have_plan = false;
    h->nq = n;
    h->gates.assign(gates, gates + ng);
    h->open_mask.assign(n, 0);
    if (open_mask)
        for (int q = 0; q < n; ++q) h->open_mask[q] = open_mask[q] ? 1 : 0;
    h->tensor_legs.clear();
    h->tensor_vals_off.clear();
    h->leaf_vals.clear();
    h->leaf_scale[0] = 1.0;
    h->leaf_scale[1] = 0.0;
    std::vector<int> wire(n);
    for (int q = 0; q < n; ++q) {
        wire[q] = q;
        h->tensor_legs.push_back({q});
        h->tensor_vals_off.push_back((int64_t)h->leaf_vals.size());
        h->leaf_vals.push_back(make_float2(1.f, 0.f));  // |0>
        h->leaf_vals.push_back(make_float2(0.f, 0.f));
    }
    int next = n;
    for (int64_t g = 0; g < ng; ++g) {
        const qx_gate& gt = gates[g];
        std::vector<int> legs;
        for (int j = 0; j < gt.nq; ++j) legs.push_back(next++);
        for (int j = 0; j < gt.nq; ++j) legs.push_back(wire[gt.q[j]]);
        for (int j = 0; j < gt.nq; ++j) wire[gt.q[j]] = legs[j];
        h->tensor_legs.push_back(legs);
        h->tensor_vals_off.push_back((int64_t)h->leaf_vals.size());
        const int d = gt.nq == 1 ? 2 : 4;
        // T[o.., i..] = U[row(o), col(i)], row-major: entry index = row * d + col.
        // Rounding U to complex64 scales it slightly (every entry of a Sycamore
        // one-qubit gate is 1/sqrt(2) in modulus and rounds the same way), and
        // an amplitude is a product over all gates, so those scales add up to a
        // bias of (number of gates) x 2^-25.  The complex least-squares factor
        // alpha = <Uf, U> / <Uf, Uf> (FP64) restores U ~ alpha Uf; every leaf
        // enters every contraction exactly once, so the product of the alphas
        // multiplies the final FP64 amplitudes exactly.
        double num_re = 0, num_im = 0, den = 0;
        for (int e = 0; e < d * d; ++e) {
            const float fr = (float)gt.re[e], fi = (float)gt.im[e];
            h->leaf_vals.push_back(make_float2(fr, fi));
            num_re += (double)fr * gt.re[e] + (double)fi * gt.im[e];
            num_im += (double)fr * gt.im[e] - (double)fi * gt.re[e];
            den += (double)fr * fr + (double)fi * fi;
        }
        if (den > 0) {
            const double ar = num_re / den, ai = num_im / den;
            const double pr = h->leaf_scale[0] * ar - h->leaf_scale[1] * ai;
            const double pi = h->leaf_scale[0] * ai + h->leaf_scale[1] * ar;
            h->leaf_scale[0] = pr;
            h->leaf_scale[1] = pi;
        }
    }
    h->final_wire = wire;
    h->open_wires.clear();
    for (int q = 0; q < n; ++q) {
        if (h->open_mask[q]) {
            h->open_wires.push_back(wire[q]);
        } else {
            h->tensor_legs.push_back({wire[q]});
            h->tensor_vals_off.push_back(-1);  // output <x_q|
        }
    }
    h->n_tensors = (int64_t)h->tensor_legs.size();
    h->n_bonds = next;
    h->bond_deg.assign(next, 0);
    for (auto& l : h->tensor_legs)
        for (int e : l) h->bond_deg[e]++;
    h->have_net = true;
    h->leaves_on_device = false;
    return QX_OK;
}

// ------------------------------------------------------------------------------------------------
// Plan compilation
// ------------------------------------------------------------------------------------------------
static Operand make_operand(const qx_ctx* h, int node) {
    const Node& nd = h->nodes[node];
    Operand op{};
    op.rank = (int32_t)nd.legs.size();
    for (int j = 0; j < op.rank; ++j) op.pos[j] = (int8_t)nd.pos[j];
    op.n_fix = (int32_t)nd.fix.size();
    for (int f = 0; f < op.n_fix; ++f) {
        op.fix_src[f] = nd.fix[f].first;
        op.fix_stride[f] = nd.fix[f].second;
    }
    return op;
}

static int64_t node_entries(const Node& n) { return (int64_t)1 << n.legs.size(); }

static int new_storage(qx_ctx* h, int64_t entries, int level, int64_t def) {
    Storage s;
    s.entries = entries;
    s.variant = level > 0;
    s.level = level;
    s.def = def;
    s.last = def;
    h->stor.push_back(s);
    return (int)h->stor.size() - 1;
}

static void use_node(qx_ctx* h, int node, int64_t step) {
    const Node& nd = h->nodes[node];
    if (nd.storage >= 0) h->stor[nd.storage].last = std::max(h->stor[nd.storage].last, step);
}

static Node contiguous_node(const std::vector<int>& legs, int level, int storage) {
    Node n;
    n.legs = legs;
    const int r = (int)legs.size();
    n.pos.resize(r);
    for (int j = 0; j < r; ++j) n.pos[j] = r - 1 - j;
    n.variant = level > 0;
    n.level = level;
    n.storage = storage;
    n.under_rank = r;
    return n;
}

// First-fit offsets for storages of one region (intervals [def, last] inclusive).
static int64_t assign_offsets(qx_ctx* h, int level) {
    std::vector<int> ids;
    for (int i = 0; i < (int)h->stor.size(); ++i)
        if (h->stor[i].level == level) ids.push_back(i);
    std::sort(ids.begin(), ids.end(), [&](int a, int b) {
        if (h->stor[a].def != h->stor[b].def) return h->stor[a].def < h->stor[b].def;
        return a < b;
    });
    std::vector<int> placed;
    int64_t top = 0;
    for (int id : ids) {
        Storage& s = h->stor[id];
        const int64_t need = align_up(s.entries, kAlignEntries);
        std::vector<std::pair<int64_t, int64_t>> busy;
        for (int p : placed) {
            const Storage& o = h->stor[p];
            if (o.last >= s.def && s.last >= o.def) busy.push_back({o.off, o.off + align_up(o.entries, kAlignEntries)});
        }
        std::sort(busy.begin(), busy.end());
        int64_t cand = 0;
        for (auto& b : busy) {
            if (cand + need <= b.first) break;
            cand = std::max(cand, b.second);
        }
        s.off = cand;
        top = std::max(top, cand + need);
        placed.push_back(id);
    }
    return top;
}

static void build_persistent_program(qx_ctx* h);
static void build_waves(qx_ctx* h);

// Storages an op reads and writes (leaves are read-only and not listed), and whether it uses the
// per-tensor scale words of the workspace (prep-based tensor-core steps).
static void op_access(const qx_ctx* h, const Op& op, std::vector<int>* rd, std::vector<int>* wr, bool* scale) {
    auto node_st = [&](int node) { return h->nodes[node].leaf ? -1 : h->nodes[node].storage; };
    std::vector<int> r;
    if (op.type == OP_PERM) r = {node_st(op.src)};
    else if (op.type == OP_SMALL) r = {node_st(op.x), node_st(op.y)};
    else if (op.dot_perm) r = {op.sa, node_st(op.perm_src)};
    else r = {op.sa, op.sb};
    rd->clear();
    for (int x : r)
        if (x >= 0) rd->push_back(x);
    *wr = {op.dst};
    if (op.spa >= 0) wr->push_back(op.spa);  // split parts: written by the prep, read by the GEMM
    if (op.spb >= 0) wr->push_back(op.spb);
    *scale = op.type == OP_GEMM && op.tc && op.tc != TC_FORM_3XTF32_DIRECT;
}

// Hazards between ops, in plan order: op j follows op i < j when j reads storage that i writes,
// writes storage that i reads, or writes storage that i writes.  Storages of the same region
// (per-pair, per-slice or invariant) conflict when their entry ranges overlap, since the liveness allocator
// gives the space of dead tensors to later ones.  Ops using the scale words follow one another.
static void compute_deps(qx_ctx* h) {
    const size_t n = h->ops.size();
    std::vector<std::vector<int>> rd(n), wr(n);
    std::vector<char> scale(n, 0);
    for (size_t j = 0; j < n; ++j) {
        bool sc;
        op_access(h, h->ops[j], &rd[j], &wr[j], &sc);
        scale[j] = sc;
    }
    auto overlap = [&](int a, int b) {
        const Storage& A = h->stor[a];
        const Storage& B = h->stor[b];
        if (A.level != B.level) return false;
        return A.off < B.off + align_up(B.entries, kAlignEntries) && B.off < A.off + align_up(A.entries, kAlignEntries);
    };
    auto any = [&](const std::vector<int>& x, const std::vector<int>& y) {
        for (int a : x)
            for (int b : y)
                if (overlap(a, b)) return true;
        return false;
    };
    h->deps.assign(n, {});
    for (size_t j = 0; j < n; ++j)
        for (size_t i = 0; i < j; ++i)
            if ((scale[i] && scale[j]) || any(wr[i], rd[j]) || any(rd[i], wr[j]) || any(wr[i], wr[j]))
                h->deps[j].push_back((int)i);
}

static int compile_plan(qx_ctx* h, const int64_t* order, int64_t n_steps, const int64_t* sliced, int32_t n_sliced) {
    const int64_t N = h->n_tensors;
    if (n_steps != N - 1)
        return fail(h, QX_EINVAL, "plan has %lld steps, a full contraction of %lld tensors needs %lld",
                    (long long)n_steps, (long long)N, (long long)(N - 1));
    if (n_sliced < 0 || n_sliced > 40) return fail(h, QX_EINVAL, "n_sliced %d out of range [0, 40]", n_sliced);
    // Intermediates that depend on the slice but on no output bit are computed once per slice and
    // shared by every bitstring of it (batched executor only).
    const bool slice_level = h->opt.executor < 2 && !h->opt.no_slice_level;
    std::vector<int> fixsrc(h->n_bonds, INT32_MIN);  // source of each fixed bond
    for (int j = 0; j < n_sliced; ++j) {
        const int64_t e = sliced[j];
        if (e < 0 || e >= h->n_bonds) return fail(h, QX_EINVAL, "sliced bond %lld out of range", (long long)e);
        if (h->bond_deg[e] != 2) return fail(h, QX_EINVAL, "sliced bond %lld is open", (long long)e);
        if (fixsrc[e] != INT32_MIN) return fail(h, QX_EINVAL, "sliced bond %lld repeated", (long long)e);
        for (int q = 0; q < h->nq; ++q)
            if (h->final_wire[q] == e)
                return fail(h, QX_EINVAL, "sliced bond %lld is the final wire of qubit %d", (long long)e, q);
        fixsrc[e] = j;
    }
    for (int q = 0; q < h->nq; ++q)
        if (!h->open_mask[q]) fixsrc[h->final_wire[q]] = -(q + 1);

    h->nodes.clear();
    h->stor.clear();
    h->ops.clear();
    h->sliced.assign(sliced, sliced + n_sliced);
    h->n_slices = (int64_t)1 << n_sliced;

    // leaves
    for (int64_t t = 0; t < N; ++t) {
        Node nd;
        nd.leaf = true;
        if (h->tensor_vals_off[t] < 0) {
            nd.const_one = true;  // <x_q| with its bond fixed to x_q is the scalar 1
        } else {
            const auto& L = h->tensor_legs[t];
            const int R = (int)L.size();
            nd.under_rank = R;
            nd.leaf_off = h->tensor_vals_off[t];
            for (int j = 0; j < R; ++j) {
                const int p = R - 1 - j;
                if (fixsrc[L[j]] != INT32_MIN) {
                    nd.fix.push_back({fixsrc[L[j]], (int64_t)1 << p});
                } else {
                    nd.legs.push_back(L[j]);
                    nd.pos.push_back(p);
                }
            }
            // a fixed output leg makes a leaf depend on the bitstring, a sliced leg on the slice; with
            // the slice level off (persistent executors) anything fixed is per pair
            bool by_bits = false;
            for (auto& f : nd.fix) by_bits |= f.first < 0;
            nd.level = nd.fix.empty() ? 0 : (by_bits || !slice_level) ? 2 : 1;
            nd.variant = nd.level > 0;
        }
        h->nodes.push_back(nd);
    }
    // Leg sets, closed-output status and consuming step of every node, known before any layout is
    // chosen, so that a step can lay out its product the way the step that consumes it reads it.
    std::vector<char> used(N + n_steps, 0);
    std::vector<std::vector<int>> lset(N + n_steps);
    std::vector<char> lone(N + n_steps, 0);
    std::vector<int64_t> consumer(N + n_steps, -1);
    for (int64_t t = 0; t < N; ++t) {
        lset[t] = h->nodes[t].legs;
        lone[t] = h->nodes[t].const_one;
    }
    for (int64_t t = 0; t < n_steps; ++t) {
        const int64_t ia = order[2 * t], ib = order[2 * t + 1];
        if (ia < 0 || ib < 0 || ia >= N + t || ib >= N + t || ia == ib || used[ia] || used[ib])
            return fail(h, QX_EINVAL, "plan step %lld uses an invalid or consumed id (%lld, %lld)", (long long)t,
                        (long long)ia, (long long)ib);
        used[ia] = used[ib] = 1;
        consumer[ia] = consumer[ib] = t;
        if (lone[ia] || lone[ib]) {
            lset[N + t] = lone[ia] ? lset[ib] : lset[ia];
            lone[N + t] = lone[ia] && lone[ib];
            continue;
        }
        for (int e : lset[ia])
            if (std::find(lset[ib].begin(), lset[ib].end(), e) == lset[ib].end()) lset[N + t].push_back(e);
        for (int e : lset[ib])
            if (std::find(lset[ia].begin(), lset[ia].end(), e) == lset[ia].end()) lset[N + t].push_back(e);
    }
    const int gemm_bits = h->opt.gemm_min_bits > 0 ? h->opt.gemm_min_bits : 5;
    auto has = [](const std::vector<int>& v, int e) { return std::find(v.begin(), v.end(), e) != v.end(); };
    // Legs of node x that the GEMM consuming it contracts (empty when no GEMM step consumes x: the root,
    // or a gather step, which reads its operands at any strides).  Re-labelling steps are followed.
    // *other is the node x is contracted with.
    const int plan_tc = h->opt.precision == QX_PREC_3XTF32       ? TC_FORM_3XTF32
                        : h->opt.precision == QX_PREC_SPLIT_BF16  ? TC_FORM_BF16X3
                        : h->opt.precision == QX_PREC_FP16_SCALED ? TC_FORM_FP16
                                                                  : 0;
    // the tensor-core kernels take products with these free / shared bits; both read their operands
    // K-major (the direct kernel through TMA, the prep-based one best: an M-major operand makes its
    // split pass a transpose)
    auto tc_shape = [&](int fa, int fb, int kb) {
        if (plan_tc && fa < 7 && fb >= 7) std::swap(fa, fb);
        const bool direct = plan_tc == TC_FORM_3XTF32 && fa >= 7 && fb >= 5 && kb >= 4 && (fa <= 8 || fb <= 8);
        return direct || (plan_tc && fa >= 7 && fb >= 6 && kb >= 5);
    };
    // *kmajor_only: the consuming GEMM runs on a tensor-core kernel
    auto next_shared = [&](int64_t x, int64_t* other, bool* kmajor_only = nullptr) {
        std::vector<int> s2;
        int64_t c = consumer[x];
        while (c >= 0 && (lone[order[2 * c]] || lone[order[2 * c + 1]])) {
            x = N + c;
            c = consumer[x];
        }
        if (c < 0) return s2;
        const int64_t d = order[2 * c] == x ? order[2 * c + 1] : order[2 * c];
        *other = d;
        for (int e : lset[x])
            if (has(lset[d], e)) s2.push_back(e);
        const int k2 = (int)s2.size(), fx = (int)(lset[x].size() - k2), fd = (int)(lset[d].size() - k2);
        const bool big = k2 >= gemm_bits && fx >= gemm_bits && fd >= gemm_bits;
        const bool small = (lset[x].size() <= 10 && k2 <= kSmallMaxK && fx <= kSmallMaxN) ||
                           (lset[d].size() <= 10 && k2 <= kSmallMaxK && fd <= kSmallMaxN);
        if (small && !big) s2.clear();
        if (kmajor_only) *kmajor_only = order[2 * c] == x ? tc_shape(fx, fd, k2) : tc_shape(fd, fx, k2);
        return s2;
    };
    // The product of step t is stored as [f1 | f2].  Where a block's legs can be put in any order at no
    // cost (the operand is permuted anyway, or the kernel addresses it per bit), order them to leave the
    // legs that the next GEMM contracts at the end of the product (read K-major there, no permute),
    // else at its start (M-major).
    auto lay_out = [&](int64_t t, std::vector<int>& f1, bool r1, std::vector<int>& f2, bool r2) {
        int64_t d = -1;
        const std::vector<int> s2 = next_shared(N + t, &d);
        if (s2.empty()) return;
        // a block's contracted legs follow the partner's stored order when the partner exists
        auto rank_in_d = [&](int e) {
            if (d < 0 || d >= N + t) return 0;
            const auto& dl = h->nodes[d].legs;
            return (int)(std::find(dl.begin(), dl.end(), e) - dl.begin());
        };
        auto arrange = [&](std::vector<int>& blk, bool last) {
            std::vector<int> in, out;
            for (int e : blk) (has(s2, e) ? in : out).push_back(e);
            std::stable_sort(in.begin(), in.end(), [&](int x, int y) { return rank_in_d(x) < rank_in_d(y); });
            blk = last ? out : in;
            const std::vector<int>& tail = last ? in : out;
            blk.insert(blk.end(), tail.begin(), tail.end());
        };
        auto count_in = [&](const std::vector<int>& blk) {
            int n = 0;
            for (int e : blk) n += has(s2, e);
            return n;
        };
        auto edge_ok = [&](const std::vector<int>& blk, bool last) {  // s2 legs already at that end
            const int n = count_in(blk), m = (int)blk.size();
            for (int i = 0; i < n; ++i)
                if (!has(s2, blk[last ? m - 1 - i : i])) return false;
            return true;
        };
        const int i1 = count_in(f1), i2 = count_in(f2);
        if (i1 == 0 && (r2 || edge_ok(f2, true))) {
            if (r2) arrange(f2, true);
        } else if (i2 == (int)f2.size() && i1 > 0 && (r1 || edge_ok(f1, true))) {
            if (r1) arrange(f1, true);
        } else if (i2 == 0 && (r1 || edge_ok(f1, false))) {
            if (r1) arrange(f1, false);
        } else if (i1 == (int)f1.size() && i2 > 0 && (r2 || edge_ok(f2, false))) {
            if (r2) arrange(f2, false);
        }
    };
    // A product with natural index [R | Cl] (row legs, then column legs, most significant first) can
    // be written by its kernel straight into another leg order D, when D's lowest L positions hold the
    // lowest L bits of one side (the kernel's lanes run along that side, so each store run stays
    // whole); modes lists the (side is rows, L) pairs the kernel supports, best first.  A side whose
    // order is free (rR / rC: its operand is permuted anyway, or addressed per bit) may be reordered
    // to make this work.  D is the order the consuming GEMM reads without a permute: [free' | S2]
    // (K-major), or [S2 | free'] (M-major) unless that GEMM runs on the direct kernel.  Returns D
    // (empty: keep the natural layout) and updates R / Cl where their order was chosen here.
    auto fused_layout = [&](int64_t t, std::vector<int>& R, bool rR, std::vector<int>& Cl, bool rC,
                            std::initializer_list<std::pair<bool, int>> modes) -> std::vector<int> {
        if (!h->fuse_layouts || h->opt.executor >= 2) return {};  // the persistent kernels store natural layouts
        int64_t d = -1;
        bool konly = false;
        const std::vector<int> s2 = next_shared(N + t, &d, &konly);
        if (s2.empty()) return {};
        const int k = (int)s2.size();
        // S2 order (lowest first) of a partner that is stored already in a layout the consumer reads
        std::vector<int> fixed;
        if (d >= 0 && d < N + t) {
            const Node& P = h->nodes[d];
            if (!P.leaf && P.fix.empty()) {
                const int r = (int)P.legs.size();
                bool suf = true, pre = true;
                for (int i = 0; i < k; ++i) {
                    suf = suf && has(s2, P.legs[r - 1 - i]);
                    pre = pre && has(s2, P.legs[i]);
                }
                if (suf)
                    for (int i = 0; i < k; ++i) fixed.push_back(P.legs[r - 1 - i]);
                else if (pre && !konly)
                    for (int i = 0; i < k; ++i) fixed.push_back(P.legs[k - 1 - i]);
            }
        }
        for (int kmaj = 1; kmaj >= (konly ? 1 : 0); --kmaj) {
            for (const auto& md : modes) {
                std::vector<int> X = md.first ? R : Cl;
                const bool rx = md.first ? rR : rC;
                const int L = md.second;
                if ((int)X.size() < L) continue;
                std::vector<int> low;  // the side's lowest L legs, lowest first
                std::vector<int> s2low, freelow;
                if (kmaj) {
                    // lowest positions: S2 (all of it if k < L, then free legs of X)
                    std::vector<int> want;
                    if (!fixed.empty()) {
                        want.assign(fixed.begin(), fixed.begin() + std::min(k, L));
                    } else {
                        for (auto it = X.rbegin(); it != X.rend() && (int)want.size() < std::min(k, L); ++it)
                            if (has(s2, *it)) want.push_back(*it);
                        if ((int)want.size() < std::min(k, L)) continue;
                    }
                    bool ok = true;
                    for (int e : want) ok = ok && has(X, e);
                    if (!ok) continue;
                    if (rx) {
                        low = want;
                        for (auto it = X.rbegin(); it != X.rend() && (int)low.size() < L; ++it)
                            if (!has(s2, *it)) low.push_back(*it);
                        if ((int)low.size() < L) continue;
                    } else {
                        low.assign(X.rbegin(), X.rbegin() + L);
                        for (int i = 0; i < (int)want.size(); ++i) ok = ok && low[i] == want[i];
                        for (int i = (int)want.size(); i < L; ++i) ok = ok && !has(s2, low[i]);
                        if (!ok) continue;
                    }
                    if (!fixed.empty()) {
                        s2low = fixed;
                    } else {
                        s2low.assign(low.begin(), low.begin() + std::min(k, L));
                        std::vector<int> nat = R;
                        nat.insert(nat.end(), Cl.begin(), Cl.end());
                        for (auto it = nat.rbegin(); it != nat.rend(); ++it)
                            if (has(s2, *it) && !has(s2low, *it)) s2low.push_back(*it);
                    }
                    if (k < L) freelow.assign(low.begin() + k, low.end());
                } else {
                    // lowest positions: free legs of X; S2 on top
                    if (rx) {
                        for (auto it = X.rbegin(); it != X.rend() && (int)low.size() < L; ++it)
                            if (!has(s2, *it)) low.push_back(*it);
                        if ((int)low.size() < L) continue;
                    } else {
                        low.assign(X.rbegin(), X.rbegin() + L);
                        bool ok = true;
                        for (int e : low) ok = ok && !has(s2, e);
                        if (!ok) continue;
                    }
                    freelow = low;
                    if (!fixed.empty()) {
                        s2low = fixed;
                    } else {
                        std::vector<int> nat = R;
                        nat.insert(nat.end(), Cl.begin(), Cl.end());
                        for (auto it = nat.rbegin(); it != nat.rend(); ++it)
                            if (has(s2, *it)) s2low.push_back(*it);
                    }
                }
                // the chosen side order: its other legs keep their order, `low` at the bottom
                if (rx) {
                    std::vector<int> nx;
                    for (int e : X)
                        if (!has(low, e)) nx.push_back(e);
                    for (auto it = low.rbegin(); it != low.rend(); ++it) nx.push_back(*it);
                    (md.first ? R : Cl) = nx;
                }
                std::vector<int> nat = R;
                nat.insert(nat.end(), Cl.begin(), Cl.end());
                std::vector<int> D;
                if (kmaj) {
                    for (int e : nat)
                        if (!has(s2, e) && !has(freelow, e)) D.push_back(e);
                    for (auto it = freelow.rbegin(); it != freelow.rend(); ++it) D.push_back(*it);
                    for (auto it = s2low.rbegin(); it != s2low.rend(); ++it) D.push_back(*it);
                } else {
                    for (auto it = s2low.rbegin(); it != s2low.rend(); ++it) D.push_back(*it);
                    for (int e : nat)
                        if (!has(s2, e) && !has(freelow, e)) D.push_back(e);
                    for (auto it = freelow.rbegin(); it != freelow.rend(); ++it) D.push_back(*it);
                }
                return D == nat ? std::vector<int>{} : D;
            }
        }
        return {};
    };
    // output position of every natural bit (columns low, then rows) of [R | Cl] stored as D
    auto out_positions = [&](const std::vector<int>& R, const std::vector<int>& Cl, const std::vector<int>& D) {
        std::vector<int8_t> pos;
        const int r = (int)D.size();
        auto at = [&](int e) { return (int8_t)(r - 1 - (int)(std::find(D.begin(), D.end(), e) - D.begin())); };
        for (auto it = Cl.rbegin(); it != Cl.rend(); ++it) pos.push_back(at(*it));
        for (auto it = R.rbegin(); it != R.rend(); ++it) pos.push_back(at(*it));
        return pos;
    };
    h->peak_entries = 1;
    for (int64_t t = 0; t < n_steps; ++t) {
        const int a = (int)order[2 * t], b = (int)order[2 * t + 1];
        const Node A = h->nodes[a], B = h->nodes[b];
        if (A.const_one || B.const_one) {  // contracting with a closed output is a re-labelling
            Node c = A.const_one ? B : A;
            use_node(h, a, t);
            use_node(h, b, t);
            h->nodes.push_back(c);
            continue;
        }
        std::vector<int> shared, freeA, freeB;
        for (int e : A.legs) {
            if (std::find(B.legs.begin(), B.legs.end(), e) != B.legs.end()) shared.push_back(e);
            else freeA.push_back(e);
        }
        for (int e : B.legs)
            if (std::find(A.legs.begin(), A.legs.end(), e) == A.legs.end()) freeB.push_back(e);
        const int kb = (int)shared.size();
        const int level = std::max(A.level, B.level);
        const bool variant = level > 0;
        const int rc = (int)(freeA.size() + freeB.size());
        if (rc > kMaxRank) return fail(h, QX_EINVAL, "step %lld: intermediate rank %d too large", (long long)t, rc);
        h->peak_entries = std::max(h->peak_entries, (int64_t)1 << rc);
        use_node(h, a, t);
        use_node(h, b, t);

        // gather path: one operand small enough for shared memory, few shared and free bits
        int small_y = -1;
        for (int cand : {0, 1}) {
            const Node& Y = cand ? A : B;
            const int ny = (int)(cand ? freeA.size() : freeB.size());
            if (node_entries(Y) <= 1024 && kb <= kSmallMaxK && ny <= kSmallMaxN) {
                if (small_y < 0 || node_entries(Y) < node_entries(small_y ? A : B)) small_y = cand;
            }
        }
        const bool big_gemm = kb >= gemm_bits && (int)freeA.size() >= gemm_bits && (int)freeB.size() >= gemm_bits;
        if (small_y >= 0 && !big_gemm) {
            const int xn = small_y ? b : a, yn = small_y ? a : b;
            const Node& X = h->nodes[xn];
            const Node& Y = h->nodes[yn];
            std::vector<int> fx, fy;
            for (int e : X.legs)
                if (std::find(shared.begin(), shared.end(), e) == shared.end()) fx.push_back(e);
            for (int e : Y.legs)
                if (std::find(shared.begin(), shared.end(), e) == shared.end()) fy.push_back(e);
            lay_out(t, fx, false, fy, true);
            // gathers: lanes run along rows (X's free index); a thread's own outputs along Y's columns
            const std::vector<int> D =
                variant ? fused_layout(t, fx, false, fy, true, {{true, 4}, {false, 2}, {true, 2}}) : std::vector<int>{};
            std::vector<int> cl = fx;
            cl.insert(cl.end(), fy.begin(), fy.end());
            const int st = new_storage(h, (int64_t)1 << cl.size(), level, t);
            Op op{};
            op.type = OP_SMALL;
            op.fy = fy;
            if (!D.empty()) {
                op.out_pos = out_positions(fx, fy, D);
                cl = D;
            }
            op.variant = variant;
            op.level = level;
            op.step = t;
            op.x = xn;
            op.y = yn;
            op.shared = shared;
            op.dst = st;
            op.mb = (int)fx.size();
            op.kb = kb;
            op.nb = (int)fy.size();
            op.flops = 8.0 * std::ldexp(1.0, op.mb + op.kb + op.nb);
            h->ops.push_back(op);
            h->nodes.push_back(contiguous_node(cl, level, st));
            continue;
        }

        // TTGT path: operands as matrices [M][K] / [K][M] and [N][K] / [K][N], C = [M][N].
        // The tensor-core kernel tiles M by 128, so the larger free side becomes M.
        const int tc_form = h->opt.precision == QX_PREC_3XTF32       ? TC_FORM_3XTF32
                            : h->opt.precision == QX_PREC_SPLIT_BF16  ? TC_FORM_BF16X3
                            : h->opt.precision == QX_PREC_FP16_SCALED ? TC_FORM_FP16
                                                                      : 0;
        int ga = a, gb = b;
        std::vector<int> fA = freeA, fB = freeB;
        if (tc_form && (int)fA.size() < 7 && (int)fB.size() >= 7) {
            std::swap(ga, gb);
            std::swap(fA, fB);
        }
        const Node GA = h->nodes[ga], GB = h->nodes[gb];
        auto contiguous_is = [&](const Node& X, const std::vector<int>& want) {
            return !X.leaf && X.fix.empty() && X.legs == want;
        };
        struct Choice { std::vector<int> S; bool pa, pb, akm, bkm; double cost; };
        // the contracted legs in either operand's stored order
        std::vector<std::vector<int>> cands(1);
        for (int e : GA.legs)
            if (has(shared, e)) cands[0].push_back(e);
        {
            std::vector<int> sB;
            for (int e : GB.legs)
                if (has(shared, e)) sB.push_back(e);
            if (sB != cands[0]) cands.push_back(sB);
        }
        // The direct 3xTF32 kernel splits operands in shared memory and reads them K-major through TMA;
        // the prep-based kernel streams pre-split parts (about (40 M + 72 N) K extra bytes) but leaves
        // shared-memory bandwidth to the MMAs.  Measured on GB300: direct wins for the short products of
        // small per-pair tensors (M or N <= 256), the prep-based kernel for large tensors.
        const bool direct = tc_form == TC_FORM_3XTF32 && (int)fA.size() >= 7 && (int)fB.size() >= 5 && kb >= 4 &&
                            ((int)fA.size() <= 8 || (int)fB.size() <= 8);
        Choice best{};
        best.cost = -1;
        for (auto& S : cands) {
            Choice c{S, true, true, true, true, 0};
            std::vector<int> ak = fA, am = S, bk = fB, bm = S;
            ak.insert(ak.end(), S.begin(), S.end());
            am.insert(am.end(), fA.begin(), fA.end());
            bk.insert(bk.end(), S.begin(), S.end());
            bm.insert(bm.end(), fB.begin(), fB.end());
            if (contiguous_is(GA, ak)) { c.pa = false; c.akm = true; }
            else if (contiguous_is(GA, am)) { c.pa = false; c.akm = false; }
            if (contiguous_is(GB, bk)) { c.pb = false; c.bkm = true; }
            else if (contiguous_is(GB, bm)) { c.pb = false; c.bkm = false; }
            if (direct && !c.akm) c.pa = c.akm = true;
            if (direct && !c.bkm) c.pb = c.bkm = true;
            c.cost = (c.pa ? (double)node_entries(GA) : 0.0) + (c.pb ? (double)node_entries(GB) : 0.0);
            if (best.cost < 0 || c.cost < best.cost) best = c;
        }
        // The resident-B' direct kernel (B invariant and one tile wide, every K stage of B' resident, A
        // per item; the conditions of tc2_resident_b) gathers A where it is stored, row and K bits at
        // their positions, instead of reading a copy permuted to K-major: the permute is left out.
        // The stage tile must be a few contiguous blocks of A (agather_tile).
        const int fa_n = (int)fA.size(), fb_n = (int)fB.size();
        const bool kb_fits = (fb_n == 6 && kb <= 6) || (fb_n == 5 && kb <= 7);
        bool a_gather = direct && best.pa && kb_fits && GB.level == 0 && GA.level == level && !GA.leaf &&
                        GA.fix.empty() && fa_n + kb == (int)GA.legs.size() && fa_n <= kMaxRank;
        std::vector<int8_t> ag_m, ag_k;
        if (a_gather) {
            auto pos_of = [&](int leg) {
                return (int8_t)GA.pos[std::find(GA.legs.begin(), GA.legs.end(), leg) - GA.legs.begin()];
            };
            for (int i = 0; i < fa_n; ++i) ag_m.push_back(pos_of(fA[fa_n - 1 - i]));
            for (int i = 0; i < kb; ++i) ag_k.push_back(pos_of(best.S[kb - 1 - i]));
            AGather probe{};
            for (int i = 0; i < fa_n; ++i) probe.mpos[i] = ag_m[i];
            for (int i = 0; i < kb; ++i) probe.kpos[i] = ag_k[i];
            a_gather = agather_tile(&probe, fa_n, kb);
        }
        if (a_gather) {
            best.pa = false;
            best.akm = true;
        }
        lay_out(t, fA, best.pa, fB, best.pb);
        // the SIMT GEMM places its product with whole 128-byte runs along columns (16 complex); the
        // tensor-core kernels and the dot kernel store their natural layout (measured on GB300: placed
        // tensor-core stores and shorter SIMT runs cost more than the permutes they save)
        std::vector<int> D;
        {
            const int mb = (int)fA.size(), nb = (int)fB.size();
            const bool dot = mb + nb <= 4 && kb >= 8;
            const bool tc = direct || (tc_form && mb >= 7 && nb >= 6 && kb >= 5);
            if (!tc && !dot && variant) D = fused_layout(t, fA, best.pa, fB, best.pb, {{false, 4}});
        }
        Op g{};
        g.type = OP_GEMM;
        g.variant = variant;
        g.level = level;
        g.step = t;
        g.mb = (int)fA.size();
        g.nb = (int)fB.size();
        g.kb = kb;
        g.a_km = best.akm;
        g.b_km = best.bkm;
        if (a_gather) {
            g.a_gather = true;
            g.ag_mpos = ag_m;
            g.ag_kpos = ag_k;
        }
        // a full contraction (scalar per pair) with exactly one operand to permute: the dot kernel
        // reads that operand through the permutation instead (no permuted copy in HBM)
        const bool fuse_dot = fA.empty() && fB.empty() && kb >= 8 && best.pa != best.pb && h->opt.executor < 2;
        for (int side = 0; side < 2; ++side) {
            const int nid = side ? gb : ga;
            const bool perm = side ? best.pb : best.pa;
            const std::vector<int>& fr = side ? fB : fA;
            int sid;
            if (perm && fuse_dot) {
                g.dot_perm = true;
                g.perm_src = nid;
                g.perm_legs = best.S;
                continue;
            }
            if (perm) {
                std::vector<int> tl = fr;
                tl.insert(tl.end(), best.S.begin(), best.S.end());
                const Node& X = h->nodes[nid];
                // an operand of a lower level is permuted at its own level (an invariant one once in the
                // prologue, and kept; a per-slice one once per slice)
                const bool keep = X.level == 0 && variant;
                sid = new_storage(h, node_entries(X), X.level, t);
                if (keep) h->stor[sid].last = kLive;
                Op p{};
                p.type = OP_PERM;
                p.variant = X.variant;
                p.level = X.level;
                p.step = t;
                p.src = nid;
                p.target_legs = tl;
                p.dst = sid;
                h->ops.push_back(p);
            } else {
                sid = h->nodes[nid].storage;
            }
            (side ? g.sb : g.sa) = sid;
        }
        if (g.dot_perm && g.sa < 0) std::swap(g.sa, g.sb);  // the stored operand is A
        std::vector<int> cl = fA;
        cl.insert(cl.end(), fB.begin(), fB.end());
        const int st = new_storage(h, (int64_t)1 << cl.size(), level, t);
        g.dst = st;
        if (!D.empty()) {
            g.out_pos = out_positions(fA, fB, D);
            cl = D;
        }
        if (direct) {
            g.tc = TC_FORM_3XTF32_DIRECT;
        } else if (tc_form && g.mb >= 7 && g.nb >= 6 && g.kb >= 5) {
            // split real parts of A [M][2K] and of the expanded B' [2N][2K], live for this step only
            const int eb = tc_elem_bytes(tc_form);
            const int64_t mk = (int64_t)1 << (g.mb + g.kb), nk = (int64_t)1 << (g.nb + g.kb);
            g.tc = tc_form;
            g.spa = new_storage(h, tc_parts_a(tc_form) * mk * 2 * eb / 8, level, t);
            g.spb = new_storage(h, tc_parts_b(tc_form) * nk * 4 * eb / 8, level, t);
        }
        g.flops = 8.0 * std::ldexp(1.0, g.mb + g.kb + g.nb);
        h->ops.push_back(g);
        h->nodes.push_back(contiguous_node(cl, level, st));
    }
    h->root = (int)h->nodes.size() - 1;
    const Node& R = h->nodes[h->root];
    {
        std::vector<int> rl = R.legs, ow = h->open_wires;
        std::sort(rl.begin(), rl.end());
        std::sort(ow.begin(), ow.end());
        if (R.const_one ? !ow.empty() : rl != ow)
            return fail(h, QX_EINVAL, "plan result legs do not match the open qubits");
    }
    if (R.storage >= 0) h->stor[R.storage].last = kLive;
    // invariant storages read by per-pair work stay resident
    for (const Op& op : h->ops) {
        if (!op.variant) continue;
        auto keep = [&](int node) {
            const Node& nd = h->nodes[node];
            if (nd.storage >= 0 && !nd.variant) h->stor[nd.storage].last = kLive;
        };
        if (op.type == OP_PERM) keep(op.src);
        if (op.type == OP_SMALL) { keep(op.x); keep(op.y); }
        if (op.type == OP_GEMM) {
            if (!h->stor[op.sa].variant) h->stor[op.sa].last = kLive;
            if (op.dot_perm) keep(op.perm_src);
            else if (!h->stor[op.sb].variant) h->stor[op.sb].last = kLive;
        }
    }
    if (!R.variant && R.storage >= 0) h->stor[R.storage].last = kLive;
    // per-slice storages read by per-pair work stay resident too, so that when a slice's bitstrings
    // need several batches of the per-pair region, the later batches run only the per-pair steps
    for (const Op& op : h->ops) {
        if (op.level != 2) continue;
        auto keep_node = [&](int node) {
            const Node& nd = h->nodes[node];
            if (nd.storage >= 0 && h->stor[nd.storage].level == 1) h->stor[nd.storage].last = kLive;
        };
        auto keep_stor = [&](int sid) {
            if (sid >= 0 && h->stor[sid].level == 1) h->stor[sid].last = kLive;
        };
        if (op.type == OP_PERM) keep_node(op.src);
        if (op.type == OP_SMALL) { keep_node(op.x); keep_node(op.y); }
        if (op.type == OP_GEMM) {
            keep_stor(op.sa);
            if (op.dot_perm) keep_node(op.perm_src);
            else keep_stor(op.sb);
        }
    }
    h->item_entries = std::max<int64_t>(assign_offsets(h, 2), kAlignEntries);
    h->slice_entries = assign_offsets(h, 1);
    if (h->opt.executor < 2) {
        // a small invariant region gets no reuse: then the only hazards between invariant steps are
        // their data dependencies, which form trees the prologue runs one CTA per tree
        int64_t tot = 0;
        for (const Storage& st : h->stor)
            if (st.level == 0) tot += align_up(st.entries, kAlignEntries);
        if (tot <= ((int64_t)1 << 22))
            for (Storage& st : h->stor)
                if (st.level == 0) {
                    st.def = 0;
                    st.last = kLive;
                }
    }
    h->inv_entries = assign_offsets(h, 0);
    h->flops_inv = h->flops_slice = h->flops_item = 0;
    for (const Op& op : h->ops) (op.level == 2 ? h->flops_item : op.level == 1 ? h->flops_slice : h->flops_inv) += op.flops;
    compute_deps(h);
    build_persistent_program(h);
    build_waves(h);
    h->have_plan = true;
    return QX_OK;
}

// ------------------------------------------------------------------------------------------------
// Workspace layout: leaves | bitstrings | accumulators | amplitudes | invariant | programs |
// per-slice region | per-pair region
// ------------------------------------------------------------------------------------------------
static int64_t n_open(const qx_ctx* h) { return (int64_t)h->open_wires.size(); }

// persistent executor regions: executor 2 runs this handle alone (own CTA
// scratch and work counter); executor 3 only prepares the handle for a group
// launch (programs and per-pair results; scratch comes from the group)
static bool persist_active(const qx_ctx* h) {
    return h->persist_ok && h->persist_grid > 0 && h->opt.executor == 2;
}
static bool persist_member(const qx_ctx* h) { return h->persist_ok && h->opt.executor >= 2; }

static void layout(qx_ctx* h, int64_t max_bits, int64_t* fixed_bytes) {
    int64_t off = 0;
    h->off_err = off;  // device error flag (int)
    off += 256;
    h->off_leaf = off;
    off += align_up((int64_t)h->leaf_vals.size() * 8, 256);
    h->off_bits = off;
    off += align_up(max_bits * h->nq, 256);
    h->off_acc = off;
    off += align_up((max_bits << n_open(h)) * 32, 256);
    h->off_amps = off;
    off += align_up((max_bits << n_open(h)) * 16, 256);
    h->off_inv = off;
    off += align_up(h->inv_entries * 8, 256);
    h->off_pops = h->off_counter = h->off_results = h->off_pscratch = h->off_pops_inv = off;
    if (persist_member(h)) {
        off += align_up((int64_t)(h->pops.size() * sizeof(POp)), 256);
        h->off_pops_inv = off;
        off += align_up((int64_t)(h->pops_inv.size() * sizeof(POp)), 256);
        h->off_results = off;
        off += align_up((max_bits * h->n_slices << n_open(h)) * 8, 256);
        h->off_counter = h->off_pscratch = off;
    }
    if (persist_active(h)) {
        off += 256;
        h->off_pscratch = off;
        off += align_up((int64_t)h->persist_grid * h->item_entries * 8, 256);
    }
    h->off_wave = off;  // prologue programs: the POps, their index list, the chain boundaries
    if (h->wave_ok)
        off += align_up((int64_t)(h->wave_ops.size() * sizeof(POp)), 256) +
               align_up((int64_t)(h->wave_idx.size() * sizeof(int32_t)), 256) +
               align_up((int64_t)(h->wave_start.size() * sizeof(int32_t)), 256);
    h->off_slice = h->off_item = off;
    *fixed_bytes = off;
}

// Split the bytes after the fixed part between the per-slice and the per-pair region: as many
// (slice, bitstring) pairs per batch as fit, with room for the slices such a batch can span.
// Returns false when not even one pair (and its slice) fits.
static bool fit_regions(const qx_ctx* h, int64_t avail, int64_t max_bits, int64_t* items_out, int64_t* slices_out) {
    const int64_t per_item = h->item_entries * 8, per_slice = h->slice_entries * 8;
    auto cap = [&](int64_t v) {
        if (h->opt.max_items > 0) v = std::min<int64_t>(v, h->opt.max_items);
        v = std::min<int64_t>(v, kMaxBatchItems);
        return std::min<int64_t>(v, h->n_slices * max_bits);
    };
    if (avail <= 0) return false;
    // a batch spans at most as many slices as it has pairs
    int64_t items = cap(avail / (per_item + per_slice));
    if (items < 1) return false;
    const int64_t slices = per_slice ? std::min<int64_t>(h->n_slices, items) : 0;
    const int64_t rest = avail - align_up(slices * per_slice, 256);
    items = std::max<int64_t>(items, cap(rest / per_item));
    *items_out = items;
    *slices_out = slices;
    return true;
}

// Region offsets for a workspace whose fixed part ends at `fixed`.
static void place_regions(qx_ctx* h, int64_t fixed, int64_t items, int64_t slices) {
    h->off_slice = fixed;
    h->off_item = fixed + align_up(slices * h->slice_entries * 8, 256);
    h->items_cap = items;
    h->slices_cap = slices;
}

static float2* item_base(const qx_ctx* h) { return (float2*)((h->wb ? h->wb : h->ws) + h->off_item); }
static float2* slice_base(const qx_ctx* h) { return (float2*)((h->wb ? h->wb : h->ws) + h->off_slice); }
static float2* inv_base(const qx_ctx* h) { return (float2*)(h->ws + h->off_inv); }

// device address and item stride of a storage
static void storage_addr(const qx_ctx* h, int sid, float2** p, int64_t* is) {
    const Storage& s = h->stor[sid];
    if (s.level == 2) {
        *p = item_base(h) + s.off * h->items_cap;
        *is = s.entries;
    } else if (s.level == 1) {
        *p = slice_base(h) + s.off * h->slices_cap;
        *is = s.entries;
    } else {
        *p = inv_base(h) + s.off;
        *is = 0;
    }
}

static Operand node_operand(const qx_ctx* h, int node) {
    Operand op = make_operand(h, node);
    const Node& nd = h->nodes[node];
    if (nd.leaf) {
        op.base = (const float2*)(h->ws + h->off_leaf) + nd.leaf_off;
        op.item_stride = 0;
    } else {
        float2* p;
        int64_t is;
        storage_addr(h, nd.storage, &p, &is);
        op.base = p;
        op.item_stride = is;
        op.per_slice = h->stor[nd.storage].level == 1;
    }
    return op;
}

// lo: lowest input positions and output bits the tile must hold; max_t: tile bits
static PermDesc perm_desc(const qx_ctx* h, const Op& op, int lo = kPermLoBits, int max_t = kPermTileBits) {
    PermDesc d{};
    d.in = node_operand(h, op.src);
    const Node& X = h->nodes[op.src];
    const int r = (int)op.target_legs.size();
    d.rank = r;
    for (int ob = 0; ob < r; ++ob) {
        const int leg = op.target_legs[r - 1 - ob];
        const int j = (int)(std::find(X.legs.begin(), X.legs.end(), leg) - X.legs.begin());
        d.in_pos[ob] = (int8_t)X.pos[j];
    }
    const int L = std::min(lo, r);
    std::vector<char> in_tile(r, 0);
    for (int ob = 0; ob < L; ++ob) in_tile[ob] = 1;
    std::vector<int> by_in(r);
    for (int i = 0; i < r; ++i) by_in[i] = i;
    std::sort(by_in.begin(), by_in.end(), [&](int a, int b) { return d.in_pos[a] < d.in_pos[b]; });
    for (int i = 0; i < L; ++i) in_tile[by_in[i]] = 1;
    int t = 0;
    for (int ob = 0; ob < r; ++ob) t += in_tile[ob];
    for (int ob = 0; ob < r && t < std::min(r, max_t); ++ob)
        if (!in_tile[ob]) { in_tile[ob] = 1; ++t; }
    d.t = t;
    int k = 0;
    for (int i = 0; i < r; ++i)
        if (in_tile[by_in[i]]) d.tile_in[k++] = (int8_t)by_in[i];
    k = 0;
    for (int ob = 0; ob < r; ++ob)
        if (in_tile[ob]) d.tile_out[k++] = (int8_t)ob;
    k = 0;
    for (int ob = 0; ob < r; ++ob)
        if (!in_tile[ob]) d.outer[k++] = (int8_t)ob;
    d.n_outer = k;
    return d;
}

static OutMap out_map(const Op& op) {
    OutMap m{};
    m.on = !op.out_pos.empty();
    for (size_t i = 0; i < op.out_pos.size() && i < (size_t)kMaxRank; ++i) m.pos[i] = op.out_pos[i];
    return m;
}

static SmallDesc small_desc(const qx_ctx* h, const Op& op) {
    SmallDesc d{};
    d.x = node_operand(h, op.x);
    d.y = node_operand(h, op.y);
    const Node& X = h->nodes[op.x];
    const Node& Y = h->nodes[op.y];
    d.mb = op.mb;
    d.kb = op.kb;
    d.nb = op.nb;
    std::vector<char> freepos(X.under_rank, 0);
    for (size_t j = 0; j < X.legs.size(); ++j)
        if (std::find(op.shared.begin(), op.shared.end(), X.legs[j]) == op.shared.end()) freepos[X.pos[j]] = 1;
    int nh = 0;
    for (int p = 0; p < X.under_rank; ++p)
        if (!freepos[p]) d.holes[nh++] = (int8_t)p;
    d.n_holes = nh;
    for (int i = 0; i < op.kb; ++i) {
        const int e = op.shared[i];
        d.xk_pos[i] = (int8_t)X.pos[std::find(X.legs.begin(), X.legs.end(), e) - X.legs.begin()];
        d.yk_pos[i] = (int8_t)Y.pos[std::find(Y.legs.begin(), Y.legs.end(), e) - Y.legs.begin()];
    }
    for (int i = 0; i < op.nb; ++i) {
        const int e = op.fy[op.nb - 1 - i];
        d.yn_pos[i] = (int8_t)Y.pos[std::find(Y.legs.begin(), Y.legs.end(), e) - Y.legs.begin()];
    }
    d.om = out_map(op);
    return d;
}

// ------------------------------------------------------------------------------------------------
// Persistent program: the variant ops with operands named by space and offset
// ------------------------------------------------------------------------------------------------
static PRef pref_node(const qx_ctx* h, int node) {
    const Node& nd = h->nodes[node];
    PRef r{};
    r.rank = (int32_t)nd.legs.size();
    for (int j = 0; j < r.rank; ++j) r.pos[j] = (int8_t)nd.pos[j];
    r.n_fix = (int32_t)nd.fix.size();
    for (int f = 0; f < r.n_fix; ++f) {
        r.fix_src[f] = nd.fix[f].first;
        r.fix_stride[f] = nd.fix[f].second;
    }
    if (nd.leaf) {
        r.space = PSPACE_LEAF;
        r.off = nd.leaf_off;
    } else {
        const Storage& st = h->stor[nd.storage];
        r.space = st.variant ? PSPACE_SCRATCH : PSPACE_INV;
        r.off = st.off;
    }
    return r;
}

static PRef pref_storage(const qx_ctx* h, int sid) {
    const Storage& st = h->stor[sid];
    PRef r{};
    r.space = st.variant ? PSPACE_SCRATCH : PSPACE_INV;
    r.off = st.off;
    return r;
}

static POp to_pop(const qx_ctx* h, const Op& op) {
    POp p{};
    p.mb = op.mb;
    p.kb = op.kb;
    p.nb = op.nb;
    p.dst = h->stor[op.dst].off;
    if (op.type == OP_PERM) {
        const PermDesc d = perm_desc(h, op, 5, 10);  // the persistent kernel's tiles: 2^10 entries, 5 + 5 bits
        p.type = POP_PERM;
        p.x = pref_node(h, op.src);
        p.t = d.t;
        p.n_outer = d.n_outer;
        memcpy(p.in_pos, d.in_pos, sizeof p.in_pos);
        memcpy(p.tile_in, d.tile_in, sizeof p.tile_in);
        memcpy(p.tile_out, d.tile_out, sizeof p.tile_out);
        memcpy(p.outer, d.outer, sizeof p.outer);
    } else if (op.type == OP_SMALL) {
        const SmallDesc d = small_desc(h, op);
        p.type = POP_SMALL;
        p.x = pref_node(h, op.x);
        p.y = pref_node(h, op.y);
        p.n_holes = d.n_holes;
        memcpy(p.holes, d.holes, sizeof p.holes);
        memcpy(p.xk_pos, d.xk_pos, sizeof p.xk_pos);
        memcpy(p.yk_pos, d.yk_pos, sizeof p.yk_pos);
        memcpy(p.yn_pos, d.yn_pos, sizeof p.yn_pos);
    } else {
        p.type = (op.mb + op.nb <= 4 && op.kb >= 8) ? POP_DOT : POP_GEMM;
        p.x = pref_storage(h, op.sa);
        p.y = pref_storage(h, op.sb);
        p.a_km = op.a_km;
        p.b_km = op.b_km;
    }
    return p;
}

static void build_persistent_program(qx_ctx* h) {
    h->persist_ok = false;
    h->pops.clear();
    h->pops_inv.clear();
    for (const Op& op : h->ops)
        if (op.tc || !op.out_pos.empty() || op.dot_perm || op.level == 1) return;  // these run batched only
    const Node& R = h->nodes[h->root];
    if (!R.variant) return;  // nothing depends on the pair
    // invariant ops write the invariant region: their program runs with that region as scratch
    for (const Op& op : h->ops) (op.variant ? h->pops : h->pops_inv).push_back(to_pop(h, op));
    h->proot = pref_node(h, h->root);
    const int ob_n = (int)h->open_wires.size();
    h->pobit_leg.assign(kMaxRank, 0);
    for (int ob = 0; ob < ob_n; ++ob) {
        const int wire = h->open_wires[ob_n - 1 - ob];
        h->pobit_leg[ob] = (int8_t)(std::find(R.legs.begin(), R.legs.end(), wire) - R.legs.begin());
    }
    h->persist_ok = true;
}

static double op_bytes(const qx_ctx* h, const Op& op, int64_t n_items, int64_t n_b = 1);

// The invariant steps grouped into chains for the one prologue launch: steps joined by a dependency
// (data, or space reuse where the invariant region reuses space) share a chain, which one CTA runs in
// plan order.  Used when every invariant step is small enough for one CTA: at most 2^12 entries in
// and out, no tensor cores, natural layouts.
static void build_waves(qx_ctx* h) {
    h->wave_ok = false;
    h->wave_ops.clear();
    h->wave_idx.clear();
    h->wave_start.clear();
    h->wave_flops.clear();
    h->wave_bytes.clear();
    h->wave_of.assign(h->ops.size(), -1);
    h->chain_of_op.assign(h->ops.size(), -1);
    if (h->opt.executor >= 2) return;  // the persistent executors run their own prologue program
    constexpr int64_t kWaveEntries = 4096;
    std::vector<int> inv;
    for (size_t j = 0; j < h->ops.size(); ++j) {
        const Op& op = h->ops[j];
        if (op.variant) continue;
        if (op.tc || !op.out_pos.empty() || op.dot_perm || h->stor[op.dst].entries > kWaveEntries) return;
        auto small_node = [&](int n) { return node_entries(h->nodes[n]) <= kWaveEntries; };
        if (op.type == OP_PERM && !small_node(op.src)) return;
        if (op.type == OP_SMALL && !(small_node(op.x) && small_node(op.y))) return;
        if (op.type == OP_GEMM &&
            !(h->stor[op.sa].entries <= kWaveEntries && h->stor[op.sb].entries <= kWaveEntries))
            return;
        inv.push_back((int)j);
    }
    if (inv.empty()) return;
    // chains: invariant steps joined by a dependency (data, or space reuse when the region is
    // reused) go to one chain, which one CTA runs in plan order; different chains touch no common
    // storage, so the CTAs need no synchronisation
    std::vector<int> root(h->ops.size());
    for (size_t j = 0; j < root.size(); ++j) root[j] = (int)j;
    std::function<int(int)> find = [&](int x) { return root[x] == x ? x : root[x] = find(root[x]); };
    for (int j : inv)
        for (int i : h->deps[j])
            if (!h->ops[i].variant) root[find(i)] = find(j);
    std::vector<int> chain_of(h->ops.size(), -1), order;
    for (int j : inv) {
        const int r = find(j);
        if (chain_of[r] < 0) {
            chain_of[r] = (int)order.size();
            order.push_back(r);
        }
    }
    const int n_chains = (int)order.size();
    h->wave_start.assign(n_chains + 1, 0);
    h->wave_flops.assign(1, 0.0);
    h->wave_bytes.assign(1, 0.0);
    for (int c = 0; c < n_chains; ++c) {
        h->wave_start[c] = (int32_t)h->wave_ops.size();
        for (int j : inv)
            if (chain_of[find(j)] == c) {
                h->wave_of[j] = 0;  // one launch: every dependant waits for its end
                h->chain_of_op[j] = c;
                h->wave_ops.push_back(to_pop(h, h->ops[j]));
                h->wave_flops[0] += h->ops[j].flops;
                h->wave_bytes[0] += op_bytes(h, h->ops[j], 1);
            }
    }
    h->wave_start[n_chains] = (int32_t)h->wave_ops.size();
    h->wave_idx.resize(h->wave_ops.size());
    for (size_t i = 0; i < h->wave_idx.size(); ++i) h->wave_idx[i] = (int32_t)i;
    h->wave_ok = true;
}

// how many distinct copies of a tensor of level `level` a launch of op over n_items items (n_b
// bitstrings per slice) reads or writes
static double copies(const Op& op, int level, int64_t n_items, int64_t n_b) {
    if (level == 0) return 1.0;
    if (level == 1 && op.level == 2) return (double)((n_items + n_b - 1) / n_b);
    return (double)n_items;
}

static double op_bytes(const qx_ctx* h, const Op& op, int64_t n_items, int64_t n_b) {
    // algorithmic bytes of one launch over n_items items: each operand read once (a tensor shared by
    // several items once per launch), the result written once per item
    auto node_b = [&](int node) {
        return 8.0 * (double)node_entries(h->nodes[node]) * copies(op, h->nodes[node].level, n_items, n_b);
    };
    auto stor_b = [&](int sid) { return 8.0 * (double)h->stor[sid].entries * copies(op, h->stor[sid].level, n_items, n_b); };
    const double c = stor_b(op.dst);
    if (op.type == OP_PERM) return c + node_b(op.src);
    if (op.type == OP_SMALL) return c + node_b(op.x) + node_b(op.y);
    if (op.dot_perm) return c + stor_b(op.sa) + node_b(op.perm_src);
    return c + stor_b(op.sa) + stor_b(op.sb);
}

static int run_op(qx_ctx* h, const Op& op, const ItemCtx& ic, int64_t n_items, cudaStream_t st) {
    float2* dp;
    int64_t dis;
    storage_addr(h, op.dst, &dp, &dis);
    const bool direct = op.tc == TC_FORM_3XTF32_DIRECT, prep = op.tc && !direct;
    SmallDesc sdesc{};
    if (op.type == OP_SMALL) sdesc = small_desc(h, op);
    // item i of a per-pair launch reads a per-slice operand at its slice i / n_b
    const int64_t n_b = op.level == 2 ? ic.n_b : 1;
    auto div = [&](int sid) { return h->stor[sid].level == 1 && op.level == 2 ? (int)n_b : 1; };
    TcArgs dg{};  // the direct kernel's arguments (its variant decides the profiling kind)
    if (direct) {
        float2 *ap, *bp;
        int64_t ais, bis;
        storage_addr(h, op.sa, &ap, &ais);
        storage_addr(h, op.sb, &bp, &bis);
        dg.a = ap;
        dg.a_is = ais;
        dg.a_kmajor = op.a_km;
        dg.b = bp;
        dg.b_is = bis;
        dg.b_kmajor = op.b_km;
        dg.c = dp;
        dg.c_is = dis;
        dg.mb = op.mb;
        dg.nb = op.nb;
        dg.kb = op.kb;
        dg.n_items = n_items;
        dg.a_div = div(op.sa);
        dg.b_div = div(op.sb);
        dg.limit = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : 2000000000ll;
        dg.err = (int*)(h->ws + h->off_err);
        if (op.a_gather) {
            dg.ag.on = 1;
            for (size_t i = 0; i < op.ag_mpos.size() && i < (size_t)kMaxRank; ++i) dg.ag.mpos[i] = op.ag_mpos[i];
            for (size_t i = 0; i < op.ag_kpos.size() && i < 16; ++i) dg.ag.kpos[i] = op.ag_kpos[i];
            if (!agather_tile(&dg.ag, op.mb, op.kb)) return fail(h, QX_EINVAL, "step %lld: A tile not gatherable",
                                                                 (long long)op.step);
        }
    }
    const int kind = op.type == OP_PERM    ? QX_KERNEL_PERMUTE
                     : op.type == OP_SMALL ? (small_is_flat(sdesc) ? QX_KERNEL_SMALL_FLAT : QX_KERNEL_SMALL)
                     : direct              ? (tc2_resident_b(dg) ? QX_KERNEL_TC_DIRECT_KB : QX_KERNEL_TC_DIRECT)
                     : prep                ? QX_KERNEL_TC_PREP
                                           : QX_KERNEL_GEMM;
    size_t slot;
    auto stor_b = [&](int sid) { return 8.0 * (double)h->stor[sid].entries * copies(op, h->stor[sid].level, n_items, n_b); };
    // the split parts hold one copy per distinct operand item
    const double prep_bytes = prep ? stor_b(op.sa) + stor_b(op.sb) + 8.0 * (double)h->stor[op.spa].entries *
                                                                          copies(op, h->stor[op.sa].level, n_items, n_b) +
                                         8.0 * (double)h->stor[op.spb].entries * copies(op, h->stor[op.sb].level, n_items, n_b)
                                   : 0.0;
    cudaError_t e = prof_begin(h, kind, prep ? 0.0 : op.flops * (double)n_items,
                               prep ? prep_bytes : op_bytes(h, op, n_items, n_b), &slot);
    if (e != cudaSuccess) return fail(h, QX_ECUDA, "profiling event: %s", cudaGetErrorString(e));
    if (op.type == OP_PERM) {
        e = launch_permute(perm_desc(h, op), ic, n_items, dp, dis, st);
    } else if (op.type == OP_SMALL) {
        e = launch_small(sdesc, ic, n_items, dp, dis, st);
    } else if (op.dot_perm) {
        float2* ap;
        int64_t ais;
        storage_addr(h, op.sa, &ap, &ais);
        Op pv{};
        pv.type = OP_PERM;
        pv.src = op.perm_src;
        pv.target_legs = op.perm_legs;
        e = launch_dot_perm(perm_desc(h, pv), ic, n_items, ap, ais, dp, dis, st, div(op.sa));
    } else if (!op.tc) {
        float2 *ap, *bp;
        int64_t ais, bis;
        storage_addr(h, op.sa, &ap, &ais);
        storage_addr(h, op.sb, &bp, &bis);
        const OutMap om = out_map(op);
        // A per-slice matrix times a per-pair vector (N = 1): the pairs of a slice are consecutive items
        // and share the matrix, so g of them (the largest power of two dividing the bitstrings per slice,
        // at most 256) form one product C'[g][M] = B'[g][K] A[M][K]^T, their vectors as the rows of B'
        // (items dense) and their results as the rows of C' (results dense): one GEMM with M = g per
        // g pairs instead of g matrix-vector products.  Each output is the same K-ordered sum.
        const int ad = div(op.sa), bd = div(op.sb);
        int g = 1, gb = 0;
        if (op.nb == 0 && !om.on && ad > 1 && bd == 1 && bis == ((int64_t)1 << op.kb) && dis == ((int64_t)1 << op.mb))
            while (g < 256 && ad % (2 * g) == 0) g *= 2, ++gb;
        if (g >= 16)
            e = launch_gemm_c64(bp, g * bis, true, ap, ais, op.a_km, dp, g * dis, gb, op.mb, op.kb, n_items / g, st,
                                nullptr, 1, ad / g);
        else
            e = launch_gemm_c64(ap, ais, op.a_km, bp, bis, op.b_km, dp, dis, op.mb, op.nb, op.kb, n_items, st, &om,
                                ad, bd);
    } else if (direct) {
        e = launch_tc2_gemm(dg, st);
    } else {
        TcArgs g{};
        float2 *ap, *bp, *pa, *pb;
        int64_t ais, bis, pais, pbis;
        storage_addr(h, op.sa, &ap, &ais);
        storage_addr(h, op.sb, &bp, &bis);
        storage_addr(h, op.spa, &pa, &pais);
        storage_addr(h, op.spb, &pb, &pbis);
        g.a = ap;
        g.a_is = ais;
        g.a_kmajor = op.a_km;
        g.b = bp;
        g.b_is = bis;
        g.b_kmajor = op.b_km;
        g.c = dp;
        g.c_is = dis;
        g.pa = pa;
        g.pb = pb;
        // an item stride of 0 (one item) still needs a valid tensor-map stride
        g.pa_is_bytes = 8 * (pais ? pais : h->stor[op.spa].entries);
        g.pb_is_bytes = 8 * (pbis ? pbis : h->stor[op.spb].entries);
        g.mb = op.mb;
        g.nb = op.nb;
        g.kb = op.kb;
        g.n_items = n_items;
        g.a_div = div(op.sa);
        g.b_div = div(op.sb);
        g.limit = h->opt.timeout_cycles > 0 ? h->opt.timeout_cycles : 2000000000ll;
        g.err = (int*)(h->ws + h->off_err);
        g.amax = (float*)(h->ws + h->off_err + 16);
        e = launch_tc_prep(op.tc, g, st);
        if (e == cudaSuccess) e = prof_end(h, slot);
        if (e == cudaSuccess)
            e = prof_begin(h, QX_KERNEL_TC_GEMM, op.flops * (double)n_items, op_bytes(h, op, n_items, n_b), &slot);
        if (e == cudaSuccess) e = launch_tc_gemm(op.tc, g, st);
        h->last_launches += 2;
    }
    if (e != cudaSuccess) return fail(h, QX_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    e = prof_end(h, slot);
    if (e != cudaSuccess) return fail(h, QX_ECUDA, "profiling event: %s", cudaGetErrorString(e));
    h->last_launches++;
    h->last_flops += op.flops * (double)n_items;
    return QX_OK;
}

static int upload_programs(qx_ctx* h) {
    if (h->pops_on_device) return QX_OK;
    if (!h->pops.empty())
        CUDA_TRY(h, cudaMemcpyAsync(h->ws + h->off_pops, h->pops.data(), h->pops.size() * sizeof(POp),
                                    cudaMemcpyHostToDevice, h->stream));
    if (!h->pops_inv.empty())
        CUDA_TRY(h, cudaMemcpyAsync(h->ws + h->off_pops_inv, h->pops_inv.data(), h->pops_inv.size() * sizeof(POp),
                                    cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->pops_on_device = true;
    return QX_OK;
}

// the pair program (inv = true: the prologue program) of a handle, for slices [s_begin, s_end)
static PProg make_prog(const qx_ctx* h, bool inv, const uint8_t* d_bits, int64_t n_bits, int64_t s_begin) {
    PProg g{};
    g.ops = (const POp*)(h->ws + (inv ? h->off_pops_inv : h->off_pops));
    g.n_ops = (int32_t)(inv ? h->pops_inv.size() : h->pops.size());
    g.n_qubits = h->nq;
    g.leaves = (const float2*)(h->ws + h->off_leaf);
    g.inv = inv_base(h);
    g.bits = d_bits;
    g.s0 = inv ? 0 : s_begin;
    g.b0 = 0;
    g.n_b = inv ? 1 : n_bits;
    g.root = h->proot;
    g.open_bits = (int32_t)n_open(h);
    for (int i = 0; i < g.open_bits; ++i) g.obit_leg[i] = h->pobit_leg[i];
    g.results = inv ? nullptr : (float2*)(h->ws + h->off_results);
    g.scratch_override = inv ? inv_base(h) : nullptr;
    return g;
}

static GSum make_gsum(const qx_ctx* h, int64_t n_bits, int64_t n_s, double* d_amps, int64_t t0) {
    GSum g{};
    g.results = (const float2*)(h->ws + h->off_results);
    g.amps = d_amps;
    g.n_b = n_bits;
    g.t0 = t0;
    g.n_s = (int32_t)n_s;
    g.open_bits = (int32_t)n_open(h);
    g.sr = h->leaf_scale[0];
    g.si = h->leaf_scale[1];
    return g;
}

static int contract_persistent(qx_ctx* h, const uint8_t* d_bits, int64_t n_bits, int64_t s_begin, int64_t s_end,
                               double* d_amps) {
    int rc = upload_programs(h);
    if (rc) return rc;
    const int64_t pairs = (s_end - s_begin) * n_bits;
    PLaunch L{};
    L.n_progs = 0;
    L.scratch = (float2*)(h->ws + h->off_pscratch);
    L.scratch_entries = h->item_entries;
    L.counter = (unsigned long long*)(h->ws + h->off_counter);
    size_t slot;
    cudaError_t e = cudaSuccess;
    if (!h->pops_inv.empty()) {  // prologue: one CTA runs the invariant ops in order
        L.single = make_prog(h, true, d_bits, n_bits, s_begin);
        L.n_work = 1;
        e = prof_begin(h, QX_KERNEL_PERSIST, h->flops_inv, 0.0, &slot);
        if (e == cudaSuccess) e = launch_persist(L, 1, h->stream);
        if (e == cudaSuccess) e = prof_end(h, slot);
        if (e != cudaSuccess) return fail(h, QX_ECUDA, "persistent prologue failed: %s", cudaGetErrorString(e));
        h->last_launches += 1;
        h->last_flops += h->flops_inv;
    }
    L.single = make_prog(h, false, d_bits, n_bits, s_begin);
    L.n_work = pairs;
    double bytes = 0;
    for (const Op& op : h->ops)
        if (op.variant) bytes += op_bytes(h, op, pairs);
    e = prof_begin(h, QX_KERNEL_PERSIST, h->flops_item * (double)pairs, bytes, &slot);
    if (e == cudaSuccess) e = launch_persist(L, h->persist_grid, h->stream);
    if (e == cudaSuccess) e = prof_end(h, slot);
    if (e != cudaSuccess) return fail(h, QX_ECUDA, "persistent launch failed: %s", cudaGetErrorString(e));
    h->last_launches += 1;
    h->last_flops += h->flops_item * (double)pairs;
    // deterministic FP64 sum over the slices of each bitstring, straight into the amplitudes
    const int64_t n_o = (int64_t)1 << n_open(h);
    const GSum g = make_gsum(h, n_bits, s_end - s_begin, d_amps, 0);
    e = prof_begin(h, QX_KERNEL_SUM, 0.0, (double)pairs * n_o * 8.0 + (double)n_bits * n_o * 16.0, &slot);
    if (e == cudaSuccess) e = launch_single_sum(g, n_bits * n_o, h->stream);
    if (e == cudaSuccess) e = prof_end(h, slot);
    if (e != cudaSuccess) return fail(h, QX_ECUDA, "slice sum launch failed: %s", cudaGetErrorString(e));
    h->last_launches++;
    h->last_batches = 1;
    return QX_OK;
}

// Issues the ops of one batch over the handle's streams.  An op goes to the stream whose last op
// is one of its dependencies (the chain continues without a wait), else to the stream idle the
// longest; it waits on the event of its latest dependency on every other stream.  Streams join the
// handle's stream lazily at first use and all rejoin it at the end.  With one stream, or while
// profiling (events around each launch on the handle's stream), everything runs on that stream.
struct Dag {
    qx_ctx* h;
    bool on = false;
    std::vector<int> stream_of, last_on;  // per op: stream this batch (-1 none); per stream: last op
    std::vector<std::vector<int>> seen;   // seen[s][t]: latest op of stream t that stream s waited for
    std::vector<char> forked;
    std::vector<int> wave_seen;          // per stream: 0 once it waited for the prologue launch
    bool waves_now = false;              // the prologue launch was issued in this batch
    explicit Dag(qx_ctx* hh) : h(hh) {}
    int init() {
        on = h->n_streams > 1 && !h->profiling && !h->ops.empty();
        if (!on) return QX_OK;
        const int S = h->n_streams - 1;  // extra streams next to the handle's own
        while ((int)h->dstreams.size() < S) {
            cudaStream_t st;
            CUDA_TRY(h, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            h->dstreams.push_back(st);
            cudaEvent_t e;
            CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            h->join_ev.push_back(e);
        }
        if (!h->fork_ev) CUDA_TRY(h, cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
        while (h->op_ev.size() < h->ops.size()) {
            cudaEvent_t e;
            CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            h->op_ev.push_back(e);
        }
        while (h->wave_ok && h->wave_ev.empty()) {
            cudaEvent_t e;
            CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            h->wave_ev.push_back(e);
        }
        return QX_OK;
    }
    // the invariant steps, one launch on the handle's stream: one CTA per chain
    int waves(const uint8_t* d_bits) {
        if (!h->wave_ok) return QX_OK;
        const size_t n = h->wave_ops.size(), nc = h->wave_start.size() - 1;
        char* wbase = h->ws + h->off_wave;
        const int32_t* idx = (const int32_t*)(wbase + align_up((int64_t)(n * sizeof(POp)), 256));
        const int32_t* starts = idx + align_up((int64_t)(n * sizeof(int32_t)), 256) / (int64_t)sizeof(int32_t);
        if (!h->waves_on_device) {
            CUDA_TRY(h, cudaMemcpyAsync(wbase, h->wave_ops.data(), n * sizeof(POp), cudaMemcpyHostToDevice, h->stream));
            CUDA_TRY(h, cudaMemcpyAsync((void*)idx, h->wave_idx.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice,
                                        h->stream));
            CUDA_TRY(h, cudaMemcpyAsync((void*)starts, h->wave_start.data(), (nc + 1) * sizeof(int32_t),
                                        cudaMemcpyHostToDevice, h->stream));
            CUDA_TRY(h, cudaStreamSynchronize(h->stream));
            h->waves_on_device = true;
        }
        PProg prog{};
        prog.ops = (const POp*)wbase;
        prog.n_ops = (int32_t)n;
        prog.n_qubits = h->nq;
        prog.leaves = (const float2*)(h->ws + h->off_leaf);
        prog.inv = inv_base(h);
        prog.bits = d_bits;
        prog.n_b = 1;
        prog.scratch_override = inv_base(h);
        size_t slot;
        cudaError_t e = prof_begin(h, QX_KERNEL_WAVE, h->wave_flops[0], h->wave_bytes[0], &slot);
        if (e == cudaSuccess) e = launch_chains(prog.ops, idx, starts, (int)nc, prog, h->stream);
        if (e == cudaSuccess) e = prof_end(h, slot);
        if (e == cudaSuccess && on) e = cudaEventRecord(h->wave_ev[0], h->stream);
        if (e != cudaSuccess) return fail(h, QX_ECUDA, "prologue launch failed: %s", cudaGetErrorString(e));
        h->last_launches++;
        h->last_flops += h->wave_flops[0];
        waves_now = true;
        if (on) last_on[0] = INT32_MAX / 2;  // per-pair steps go to the other streams first
        return QX_OK;
    }
    cudaStream_t stream(int s) const { return s == 0 ? h->stream : h->dstreams[s - 1]; }
    int fork() {
        if (!on) return QX_OK;
        const int S = h->n_streams;
        stream_of.assign(h->ops.size(), -1);
        last_on.assign(S, -1);
        seen.assign(S, std::vector<int>(S, -1));
        forked.assign(S, 0);
        forked[0] = 1;
        wave_seen.assign(S, -1);
        waves_now = false;
        CUDA_TRY(h, cudaEventRecord(h->fork_ev, h->stream));
        return QX_OK;
    }
    int issue(int j, const ItemCtx& ic, int64_t n_items) {
        if (h->wave_ok && h->wave_of[j] >= 0) return QX_OK;  // ran in the prologue launch
        if (!on) return run_op(h, h->ops[j], ic, n_items, h->stream);
        const int S = h->n_streams;
        int s = -1, wneed = -1;
        for (int i : h->deps[j]) {
            if (h->wave_ok && h->wave_of[i] >= 0) {
                if (waves_now) wneed = std::max(wneed, h->wave_of[i]);
                continue;
            }
            const int t = stream_of[i];
            if (t >= 0 && last_on[t] == i && (s < 0 || i > last_on[s])) s = t;
        }
        if (s < 0)
            for (int t = 0; t < S; ++t)
                if (s < 0 || last_on[t] < last_on[s]) s = t;
        if (!forked[s]) {
            CUDA_TRY(h, cudaStreamWaitEvent(stream(s), h->fork_ev, 0));
            forked[s] = 1;
        }
        if (wneed >= 0 && s != 0 && wave_seen[s] < wneed) {
            CUDA_TRY(h, cudaStreamWaitEvent(stream(s), h->wave_ev[wneed], 0));
            wave_seen[s] = wneed;
        }
        std::vector<int> latest(S, -1);
        for (int i : h->deps[j]) {
            if (h->wave_ok && h->wave_of[i] >= 0) continue;
            const int t = stream_of[i];
            if (t >= 0 && t != s) latest[t] = std::max(latest[t], i);
        }
        for (int t = 0; t < S; ++t)
            if (latest[t] > seen[s][t]) {
                CUDA_TRY(h, cudaStreamWaitEvent(stream(s), h->op_ev[latest[t]], 0));
                seen[s][t] = latest[t];
            }
        int rc = run_op(h, h->ops[j], ic, n_items, stream(s));
        if (rc) return rc;
        CUDA_TRY(h, cudaEventRecord(h->op_ev[j], stream(s)));
        stream_of[j] = s;
        last_on[s] = j;
        return QX_OK;
    }
    int join() {
        if (!on) return QX_OK;
        for (int s = 1; s < h->n_streams; ++s)
            if (forked[s]) {
                CUDA_TRY(h, cudaEventRecord(h->join_ev[s - 1], stream(s)));
                CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->join_ev[s - 1], 0));
            }
        return QX_OK;
    }
};

static int contract_impl(qx_ctx* h, const uint8_t* d_bits, int64_t n_bits, int64_t s_begin, int64_t s_end,
                         double* d_amps) {
    const int64_t n_o = (int64_t)1 << n_open(h);
    h->last_flops = 0;
    h->last_launches = 0;
    h->last_batches = 0;
    if (h->part_clear) h->part_open = false;  // any whole contraction ends an open sum of parts
    if (!h->leaves_on_device) {
        CUDA_TRY(h, cudaMemcpyAsync(h->ws + h->off_leaf, h->leaf_vals.data(), h->leaf_vals.size() * sizeof(float2),
                                    cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        h->leaves_on_device = true;
    }
    double* acc = (double*)(h->ws + h->off_acc);
    CUDA_TRY(h, cudaMemsetAsync(h->ws + h->off_err, 0, sizeof(int), h->stream));
    const int mode = h->opt.executor;
    if (mode >= 2 && !persist_active(h))
        return fail(h, QX_EINVAL, mode == 3 ? "a group member contracts only through qx_group_run"
                                            : "the persistent executor does not apply to this plan and precision form");
    if (mode == 2) {
        if (!h->part_clear || !h->part_final)
            return fail(h, QX_EINVAL, "parts of a slice sum need the batched executor");
        return contract_persistent(h, d_bits, n_bits, s_begin, s_end, d_amps);
    }
    if (h->part_clear) CUDA_TRY(h, cudaMemsetAsync(acc, 0, (size_t)(n_bits * n_o * 32), h->stream));
    ItemCtx ic{};
    ic.n_qubits = h->nq;
    ic.bits = d_bits;
    ic.n_b = 1;
    ic.n_items = 1;
    const ItemCtx ic_inv = ic;
    Dag dag(h);
    int rc = dag.init();
    if (rc) return rc;
    // batches of (slice, bitstring) pairs
    int64_t nb_batch, ns_batch;
    if (h->items_cap >= n_bits) {
        nb_batch = n_bits;
        ns_batch = std::min<int64_t>(h->n_slices, h->items_cap / n_bits);
    } else {
        nb_batch = h->items_cap;
        ns_batch = 1;
    }
    if (h->slice_entries) ns_batch = std::max<int64_t>(1, std::min<int64_t>(ns_batch, h->slices_cap));
    SumDesc sd{};
    sd.root = node_operand(h, h->root);
    sd.open_bits = (int32_t)n_open(h);
    {
        const Node& R = h->nodes[h->root];
        for (int ob = 0; ob < sd.open_bits; ++ob) {
            const int wire = h->open_wires[sd.open_bits - 1 - ob];
            const int j = (int)(std::find(R.legs.begin(), R.legs.end(), wire) - R.legs.begin());
            sd.obit_pos[ob] = (int8_t)R.pos[j];
        }
    }
    // The prologue (everything that no slice or bitstring touches) is issued together with the first
    // batch of (slice, bitstring) pairs, so independent branches of both overlap; every batch ends with
    // all streams joined before its slice sum, and the next batch reuses the per-slice and per-pair
    // space.  Steps that no output bit touches run once per slice of the batch (one item per slice),
    // the others once per pair.
    // with qx_set_memo, the invariant intermediates of an earlier call are still in the workspace
    bool prologue = !(h->memo && h->inv_ready);
    for (int64_t s0 = s_begin; s0 < s_end; s0 += ns_batch) {
        const int64_t ns = std::min(ns_batch, s_end - s0);
        for (int64_t b0 = 0; b0 < n_bits; b0 += nb_batch) {
            const int64_t nb = std::min(nb_batch, n_bits - b0);
            ic.s0 = s0;
            ic.b0 = b0;
            ic.n_b = (int32_t)nb;
            ic.n_items = ns * nb;
            if ((rc = dag.fork())) return rc;
            if (prologue && (rc = dag.waves(d_bits))) return rc;
            ItemCtx ic_s = ic;
            ic_s.n_b = 1;
            ic_s.n_items = ns;
            for (size_t j = 0; j < h->ops.size(); ++j) {
                const Op& op = h->ops[j];
                if (!op.variant && !prologue) continue;
                // a later batch of the same slices' bitstrings: the per-slice results are still there
                if (op.level == 1 && b0 > 0) continue;
                const ItemCtx& c = op.level == 2 ? ic : op.level == 1 ? ic_s : ic_inv;
                if ((rc = dag.issue((int)j, c, c.n_items))) return rc;
            }
            prologue = false;
            if ((rc = dag.join())) return rc;
            sd.n_s = (int32_t)ns;
            size_t slot;
            const double sum_bytes = (double)(ns * nb << sd.open_bits) * 8.0 + (double)(nb << sd.open_bits) * 64.0;
            cudaError_t e = prof_begin(h, QX_KERNEL_SUM, 0.0, sum_bytes, &slot);
            if (e == cudaSuccess) e = launch_slice_sum(sd, ic, acc, h->stream);
            if (e == cudaSuccess) e = prof_end(h, slot);
            if (e != cudaSuccess) return fail(h, QX_ECUDA, "slice sum launch failed: %s", cudaGetErrorString(e));
            h->last_launches++;
            h->last_batches++;
        }
    }
    if (h->part_final) {
        cudaError_t e = launch_finalize(acc, d_amps, n_bits * n_o, h->leaf_scale[0], h->leaf_scale[1], h->stream);
        if (e != cudaSuccess) return fail(h, QX_ECUDA, "finalize launch failed: %s", cudaGetErrorString(e));
        h->last_launches++;
    }
    if (h->memo) h->inv_ready = true;
    return QX_OK;
}

// Repeated calls with the same buffers, sizes and slice range replay a CUDA graph of the whole
// contraction (hundreds of short launches become one graph launch).  The first such call runs
// eagerly (it also uploads tensors and programs), the second captures and launches the graph.
static int contract_graph(qx_ctx* h, const uint8_t* d_bits, int64_t n_bits, int64_t s0, int64_t s1, double* d_amps) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (h->stream) CUDA_TRY(h, cudaStreamIsCapturing(h->stream, &cap));
    // the caller may be capturing this stream into a graph of its own: then just enqueue
    const bool usable = h->graphs && !h->profiling && h->stream != nullptr && cap == cudaStreamCaptureStatusNone;
    if (!usable) return contract_impl(h, d_bits, n_bits, s0, s1, d_amps);
    const bool same = h->gc.bits == d_bits && h->gc.amps == d_amps && h->gc.n_bits == n_bits && h->gc.s0 == s0 &&
                      h->gc.s1 == s1 && h->gc.clear == h->part_clear && h->gc.final_ == h->part_final;
    if (same && h->gc.exec) {
        CUDA_TRY(h, cudaGraphLaunch(h->gc.exec, h->stream));
        h->last_flops = h->gc.flops;
        h->last_launches = h->gc.launches;
        h->last_batches = h->gc.batches;
        return QX_OK;
    }
    if (!same) {
        drop_graph(h);
        h->gc.bits = d_bits;
        h->gc.amps = d_amps;
        h->gc.n_bits = n_bits;
        h->gc.s0 = s0;
        h->gc.s1 = s1;
        h->gc.clear = h->part_clear;
        h->gc.final_ = h->part_final;
        return contract_impl(h, d_bits, n_bits, s0, s1, d_amps);
    }
    cudaGraph_t graph = nullptr;
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = contract_impl(h, d_bits, n_bits, s0, s1, d_amps);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        h->graphs = false;  // this plan needs host work inside a contraction: stay eager
        return rc;
    }
    if (e != cudaSuccess) return fail(h, QX_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->gc.exec = nullptr;
        return fail(h, QX_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    h->gc.flops = h->last_flops;
    h->gc.launches = h->last_launches;
    h->gc.batches = h->last_batches;
    CUDA_TRY(h, cudaGraphLaunch(h->gc.exec, h->stream));
    return QX_OK;
}

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
extern "C" {

int qx_create(qx_handle* out, int device, void* stream, const qx_options* opt) {
    if (!out) return QX_EINVAL;
    *out = nullptr;
    if (device != -1) {  // -1: host-only handle (network, plan and sizes; no contraction)
        int n = 0;
        if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return QX_ECUDA;
    }
    qx_ctx* h = new qx_ctx();
    h->device = device;
    h->persist_grid = 2 * 152;  // two CTAs per SM; the real SM count below
    if (device >= 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
            h->persist_grid = 2 * sms;
    }
    h->stream = (cudaStream_t)stream;
    if (opt) h->opt = *opt;
    if (h->opt.precision < QX_PREC_C64 || h->opt.precision > QX_PREC_FP16_SCALED || h->opt.max_items < 0 ||
        h->opt.executor < 0 || h->opt.executor > 3 || h->opt.no_slice_level < 0 || h->opt.no_slice_level > 1) {
        delete h;
        return QX_EINVAL;
    }
    *out = h;
    return QX_OK;
}

void qx_destroy(qx_handle h) {
    if (!h) return;
    drop_graph(h);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : h->op_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->join_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->wave_ev) cudaEventDestroy(e);
    for (auto& kv : h->reqs) cudaEventDestroy(kv.second);
    for (cudaEvent_t e : h->req_pool) cudaEventDestroy(e);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    for (cudaStream_t st : h->dstreams) cudaStreamDestroy(st);
    if (h->ws_owned && h->ws) {
        cudaSetDevice(h->device);
        cudaFree(h->ws);
    }
    if (h->d_small) {
        cudaSetDevice(h->device);
        cudaFree(h->d_small);
    }
    delete h;
}

const char* qx_last_error(qx_handle h) { return h ? h->err.c_str() : "null handle"; }

int qx_set_options(qx_handle h, const qx_options* opt) {
    if (!h || !opt) return QX_EINVAL;
    if (opt->precision < QX_PREC_C64 || opt->precision > QX_PREC_FP16_SCALED)
        return fail(h, QX_EINVAL, "precision form %d is not available", opt->precision);
    if (h->have_plan && opt->precision != h->opt.precision)
        return fail(h, QX_ESTATE, "set the precision form before qx_set_plan");
    if (opt->max_items < 0) return fail(h, QX_EINVAL, "max_items < 0");
    if (opt->executor < 0 || opt->executor > 3) return fail(h, QX_EINVAL, "executor %d out of range", opt->executor);
    if (opt->no_slice_level < 0 || opt->no_slice_level > 1) return fail(h, QX_EINVAL, "no_slice_level must be 0 or 1");
    h->opt = *opt;
    drop_graph(h);  // a captured graph holds the old options' launch parameters (e.g. the wait limit)
    return QX_OK;
}

int qx_build_network(qx_handle h, int32_t n_qubits, const qx_gate* gates, int64_t n_gates, const uint8_t* open_mask) {
    if (!h) return QX_EINVAL;
    h->have_plan = false;
    return build_network(h, n_qubits, gates, n_gates, open_mask);
}

int qx_network_info(qx_handle h, int64_t* n_tensors, int64_t* n_bonds) {
    if (!h) return QX_EINVAL;
    if (!h->have_net) return fail(h, QX_ESTATE, "no network");
    if (n_tensors) *n_tensors = h->n_tensors;
    if (n_bonds) *n_bonds = h->n_bonds;
    return QX_OK;
}

static void unbind(qx_ctx* h) {
    drop_graph(h);
    if (h->ws_owned && h->ws) {
        cudaSetDevice(h->device);
        cudaFree(h->ws);
    }
    h->ws = nullptr;
    h->wb = nullptr;
    h->ws_bytes = 0;
    h->ws_owned = false;
    h->items_cap = 0;
    h->leaves_on_device = false;
    h->pops_on_device = false;
    h->waves_on_device = false;
    h->inv_ready = false;
}

int qx_set_plan(qx_handle h, const int64_t* order, int64_t n_steps, const int64_t* sliced, int32_t n_sliced,
                int64_t* peak_entries_out) {
    if (!h) return QX_EINVAL;
    if (!h->have_net) return fail(h, QX_ESTATE, "qx_set_plan before qx_build_network");
    if ((n_steps > 0 && !order) || (n_sliced > 0 && !sliced)) return fail(h, QX_EINVAL, "null plan arrays");
    unbind(h);
    h->have_plan = false;
    int rc = compile_plan(h, order, n_steps, sliced, n_sliced);
    if (rc) return rc;
    if (peak_entries_out) *peak_entries_out = h->peak_entries;
    return QX_OK;
}

int qx_workspace_size(qx_handle h, int64_t max_bits, int64_t items, int64_t* bytes_out) {
    if (!h || !bytes_out) return QX_EINVAL;
    if (!h->have_plan) return fail(h, QX_ESTATE, "qx_workspace_size before qx_set_plan");
    if (max_bits < 1) return fail(h, QX_EINVAL, "max_bits < 1");
    if (items < 1) items = 1;
    int64_t fixed;
    layout(h, max_bits, &fixed);
    const int64_t slices = h->slice_entries ? std::min<int64_t>(h->n_slices, items) : 0;
    *bytes_out = fixed + align_up(slices * h->slice_entries * 8, 256) + items * h->item_entries * 8;
    return QX_OK;
}

int qx_bind_workspace(qx_handle h, void* dptr, int64_t bytes, int64_t max_bits) {
    if (!h) return QX_EINVAL;
    if (h->device < 0) return fail(h, QX_ESTATE, "host-only handle has no device");
    if (!h->have_plan) return fail(h, QX_ESTATE, "qx_bind_workspace before qx_set_plan");
    if (max_bits < 1) return fail(h, QX_EINVAL, "max_bits < 1");
    if (((uintptr_t)dptr) % 256) return fail(h, QX_EINVAL, "workspace must be 256-byte aligned");
    unbind(h);
    int64_t fixed, items = 0, slices = 0;
    layout(h, max_bits, &fixed);
    if (!fit_regions(h, bytes - fixed, max_bits, &items, &slices))
        return fail(h, QX_ENOMEM, "workspace of %lld bytes holds no (slice, bitstring) pair; need %lld", (long long)bytes,
                    (long long)(fixed + 256 + (h->item_entries + h->slice_entries) * 8));
    CUDA_TRY(h, cudaSetDevice(h->device));
    if (!dptr) {
        CUDA_TRY(h, cudaMalloc(&dptr, (size_t)bytes));
        h->ws_owned = true;
    }
    h->ws = (char*)dptr;
    h->ws_bytes = bytes;
    h->max_bits = max_bits;
    place_regions(h, fixed, items, slices);
    h->leaves_on_device = false;
    h->pops_on_device = false;
    h->waves_on_device = false;
    return QX_OK;
}

int qx_workspace_parts(qx_handle h, int64_t max_bits, int64_t items, int64_t* fixed_bytes, int64_t* batch_bytes) {
    if (!h || !fixed_bytes || !batch_bytes) return QX_EINVAL;
    if (!h->have_plan) return fail(h, QX_ESTATE, "qx_workspace_parts before qx_set_plan");
    if (max_bits < 1) return fail(h, QX_EINVAL, "max_bits < 1");
    if (items < 1) items = 1;
    int64_t fixed;
    layout(h, max_bits, &fixed);
    const int64_t slices = h->slice_entries ? std::min<int64_t>(h->n_slices, items) : 0;
    *fixed_bytes = fixed;
    *batch_bytes = align_up(slices * h->slice_entries * 8, 256) + items * h->item_entries * 8;
    return QX_OK;
}

int qx_bind_workspace_parts(qx_handle h, void* d_fixed, int64_t fixed_bytes, void* d_batch, int64_t batch_bytes,
                            int64_t max_bits) {
    if (!h) return QX_EINVAL;
    if (h->device < 0) return fail(h, QX_ESTATE, "host-only handle has no device");
    if (!h->have_plan) return fail(h, QX_ESTATE, "qx_bind_workspace_parts before qx_set_plan");
    if (max_bits < 1) return fail(h, QX_EINVAL, "max_bits < 1");
    if (!d_fixed || !d_batch) return fail(h, QX_EINVAL, "null buffer");
    if (((uintptr_t)d_fixed) % 256 || ((uintptr_t)d_batch) % 256)
        return fail(h, QX_EINVAL, "workspace parts must be 256-byte aligned");
    if (persist_member(h) || persist_active(h))
        return fail(h, QX_EINVAL, "a split workspace is for the batched executor");
    unbind(h);
    int64_t fixed, items = 0, slices = 0;
    layout(h, max_bits, &fixed);
    if (fixed_bytes < fixed)
        return fail(h, QX_ENOMEM, "fixed part of %lld bytes; need %lld", (long long)fixed_bytes, (long long)fixed);
    if (!fit_regions(h, batch_bytes, max_bits, &items, &slices))
        return fail(h, QX_ENOMEM, "batch part of %lld bytes holds no (slice, bitstring) pair; need %lld",
                    (long long)batch_bytes, (long long)(256 + (h->item_entries + h->slice_entries) * 8));
    h->ws = (char*)d_fixed;
    h->wb = (char*)d_batch;
    h->ws_bytes = fixed_bytes;
    h->max_bits = max_bits;
    place_regions(h, 0, items, slices);
    h->leaves_on_device = false;
    h->pops_on_device = false;
    h->waves_on_device = false;
    return QX_OK;
}

static int check_range(qx_ctx* h, int64_t s_begin, int64_t s_end) {
    if (s_begin < 0 || s_end > h->n_slices || s_begin >= s_end)
        return fail(h, QX_EINVAL, "slice range [%lld, %lld) not within [0, %lld)", (long long)s_begin,
                    (long long)s_end, (long long)h->n_slices);
    return QX_OK;
}

static int check_ready(qx_ctx* h, int64_t n_bits) {
    if (!h->have_plan) return fail(h, QX_ESTATE, "contract before qx_set_plan");
    if (!h->ws) return fail(h, QX_ESTATE, "contract before qx_bind_workspace");
    if (n_bits < 1) return fail(h, QX_EINVAL, "n_bits < 1");
    if (n_bits > h->max_bits)
        return fail(h, QX_ENOMEM, "%lld bitstrings exceed the workspace's %lld", (long long)n_bits, (long long)h->max_bits);
    return QX_OK;
}

int qx_contract_slices(qx_handle h, const uint8_t* bits, int64_t n_bits, int64_t s_begin, int64_t s_end,
                       double* amps_out) {
    if (!h) return QX_EINVAL;
    int rc = check_ready(h, n_bits);
    if (rc) return rc;
    rc = check_range(h, s_begin, s_end);
    if (rc) return rc;
    if (!bits || !amps_out) return fail(h, QX_EINVAL, "null buffer");
    for (int64_t i = 0; i < n_bits * h->nq; ++i)
        if (bits[i] > 1) return fail(h, QX_EINVAL, "bitstring %lld has a byte that is not 0/1", (long long)(i / h->nq));
    CUDA_TRY(h, cudaSetDevice(h->device));
    uint8_t* d_bits = (uint8_t*)(h->ws + h->off_bits);
    double* d_amps = (double*)(h->ws + h->off_amps);
    CUDA_TRY(h, cudaMemcpyAsync(d_bits, bits, (size_t)(n_bits * h->nq), cudaMemcpyHostToDevice, h->stream));
    rc = contract_graph(h, d_bits, n_bits, s_begin, s_end, d_amps);
    if (rc) return rc;
    const size_t out_bytes = (size_t)((n_bits << n_open(h)) * 16);
    CUDA_TRY(h, cudaMemcpyAsync(amps_out, d_amps, out_bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return qx_device_status(h);
}

int qx_contract(qx_handle h, const uint8_t* bits, int64_t n_bits, double* amps_out) {
    if (!h) return QX_EINVAL;
    return qx_contract_slices(h, bits, n_bits, 0, h->n_slices, amps_out);
}

int qx_contract_slices_device(qx_handle h, const uint8_t* d_bits, int64_t n_bits, int64_t s_begin, int64_t s_end,
                              double* d_amps) {
    if (!h) return QX_EINVAL;
    int rc = check_ready(h, n_bits);
    if (rc) return rc;
    rc = check_range(h, s_begin, s_end);
    if (rc) return rc;
    if (!d_bits || !d_amps) return fail(h, QX_EINVAL, "null buffer");
    CUDA_TRY(h, cudaSetDevice(h->device));
    return contract_graph(h, d_bits, n_bits, s_begin, s_end, d_amps);
}

static int enqueue_request(qx_ctx* h, int64_t* req_out) {
    cudaEvent_t e;
    if (!h->req_pool.empty()) {
        e = h->req_pool.back();
        h->req_pool.pop_back();
    } else {
        CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    cudaError_t r = cudaEventRecord(e, h->stream);
    if (r != cudaSuccess) {
        h->req_pool.push_back(e);
        return fail(h, QX_ECUDA, "request event: %s", cudaGetErrorString(r));
    }
    const int64_t id = h->next_req++;
    h->reqs[id] = e;
    *req_out = id;
    return QX_OK;
}

int qx_submit_part(qx_handle h, const uint8_t* d_bits, int64_t n_bits, int64_t s_begin, int64_t s_end,
                   int32_t first, int32_t last, double* d_amps, double* h_amps, int64_t* req_out) {
    if (!h || !req_out) return QX_EINVAL;
    int rc = check_ready(h, n_bits);
    if (rc) return rc;
    rc = check_range(h, s_begin, s_end);
    if (rc) return rc;
    if (!d_bits || !d_amps) return fail(h, QX_EINVAL, "null buffer");
    if (h->opt.executor == 2) return fail(h, QX_EINVAL, "parts of a slice sum need the batched executor");
    if (!first && (!h->part_open || d_bits != h->part_bits || n_bits != h->part_nbits || s_begin != h->part_next))
        return fail(h, QX_ESTATE, "a continuing part must follow the open sum's last part: same bitstrings, slices "
                                  "from %lld", (long long)(h->part_open ? h->part_next : -1));
    CUDA_TRY(h, cudaSetDevice(h->device));
    h->part_clear = first != 0;
    h->part_final = last != 0;
    rc = contract_graph(h, d_bits, n_bits, s_begin, s_end, d_amps);
    h->part_clear = h->part_final = true;
    if (rc) {
        h->part_open = false;
        return rc;
    }
    h->part_open = !last;
    h->part_bits = d_bits;
    h->part_nbits = n_bits;
    h->part_next = s_end;
    if (last && h_amps)
        CUDA_TRY(h, cudaMemcpyAsync(h_amps, d_amps, (size_t)(n_bits << n_open(h)) * 16, cudaMemcpyDeviceToHost,
                                    h->stream));
    return enqueue_request(h, req_out);
}

int qx_submit(qx_handle h, const uint8_t* d_bits, int64_t n_bits, int64_t s_begin, int64_t s_end, double* d_amps,
              double* h_amps, int64_t* req_out) {
    if (!h || !req_out) return QX_EINVAL;
    int rc = qx_contract_slices_device(h, d_bits, n_bits, s_begin, s_end, d_amps);
    if (rc) return rc;
    if (h_amps)
        CUDA_TRY(h, cudaMemcpyAsync(h_amps, d_amps, (size_t)(n_bits << n_open(h)) * 16, cudaMemcpyDeviceToHost,
                                    h->stream));
    return enqueue_request(h, req_out);
}

int qx_poll(qx_handle h, int64_t req, int32_t* done) {
    if (!h || !done) return QX_EINVAL;
    auto it = h->reqs.find(req);
    if (it == h->reqs.end()) return fail(h, QX_EINVAL, "request %lld is unknown or was reported done", (long long)req);
    const cudaError_t r = cudaEventQuery(it->second);
    if (r == cudaErrorNotReady) {
        *done = 0;
        return QX_OK;
    }
    h->req_pool.push_back(it->second);
    h->reqs.erase(it);
    if (r != cudaSuccess) return fail(h, QX_ECUDA, "request %lld: %s", (long long)req, cudaGetErrorString(r));
    *done = 1;
    return QX_OK;
}

int qx_contract_device(qx_handle h, const uint8_t* d_bits, int64_t n_bits, double* d_amps) {
    if (!h) return QX_EINVAL;
    return qx_contract_slices_device(h, d_bits, n_bits, 0, h->n_slices, d_amps);
}

int qx_describe_plan(qx_handle h, char* buf, int64_t len, int64_t* needed) {
    if (!h) return QX_EINVAL;
    if (!h->have_plan) return fail(h, QX_ESTATE, "no plan");
    std::string out;
    char line[256];
    for (size_t i = 0; i < h->ops.size(); ++i) {
        const Op& op = h->ops[i];
        const char* kind = op.type == OP_PERM    ? "permute"
                           : op.type == OP_SMALL ? "gather"
                           : op.dot_perm                    ? "dot_perm"
                           : op.tc == TC_FORM_3XTF32_DIRECT ? "tc_direct"
                           : op.tc                          ? "tc_prep"
                                                            : "gemm";
        if (op.type == OP_PERM) {
            snprintf(line, sizeof line, "%zu step=%lld %s %s rank=%zu", i, (long long)op.step, kind,
                     op.level == 2 ? "pair" : op.level == 1 ? "slice" : "shared", op.target_legs.size());
            out += line;
            // source address position of each target bit, lowest target bit first
            const PermDesc pd = perm_desc(h, op);
            out += " from=";
            for (int ob = 0; ob < pd.rank; ++ob) {
                snprintf(line, sizeof line, "%s%d", ob ? "," : "", (int)pd.in_pos[ob]);
                out += line;
            }
            snprintf(line, sizeof line, "\n");
        } else {
            snprintf(line, sizeof line,
                     "%zu step=%lld %s %s m=%d k=%d n=%d a_kmajor=%d b_kmajor=%d scatter=%d a_gather=%d\n", i,
                     (long long)op.step, kind, op.level == 2 ? "pair" : op.level == 1 ? "slice" : "shared", op.mb, op.kb,
                     op.nb, (int)op.a_km, (int)op.b_km, (int)!op.out_pos.empty(), (int)op.a_gather);
        }
        out += line;
        if (op.type == OP_SMALL) {  // address positions in X of the contracted legs
            const SmallDesc sd = small_desc(h, op);
            out.pop_back();
            out += " xk=";
            for (int i = 0; i < op.kb; ++i) {
                snprintf(line, sizeof line, "%s%d", i ? "," : "", (int)sd.xk_pos[i]);
                out += line;
            }
            out += "\n";
        }
        if (op.a_gather) {  // A read in place: address positions of its K bits, then of its row bits
            out.pop_back();
            out += " ak=";
            for (size_t i = 0; i < op.ag_kpos.size(); ++i) {
                snprintf(line, sizeof line, "%s%d", i ? "," : "", (int)op.ag_kpos[i]);
                out += line;
            }
            out += " am=";
            for (size_t i = 0; i < op.ag_mpos.size(); ++i) {
                snprintf(line, sizeof line, "%s%d", i ? "," : "", (int)op.ag_mpos[i]);
                out += line;
            }
            out += "\n";
        }
        if (!op.out_pos.empty()) {  // placed product: address position of each natural bit (columns, then rows)
            out.pop_back();
            out += " place=";
            for (size_t i = 0; i < op.out_pos.size(); ++i) {
                snprintf(line, sizeof line, "%s%d", i ? "," : "", (int)op.out_pos[i]);
                out += line;
            }
            out += "\n";
        }
        // storages as region:offset+entries (entries rounded up as allocated), then the dependencies
        std::vector<int> rd, wr;
        bool sc;
        op_access(h, op, &rd, &wr, &sc);
        for (int pass = 0; pass < 2; ++pass) {
            out.pop_back();
            out += pass ? " writes=" : " reads=";
            const std::vector<int>& v = pass ? wr : rd;
            for (size_t k = 0; k < v.size(); ++k) {
                const Storage& st = h->stor[v[k]];
                snprintf(line, sizeof line, "%s%s:%lld+%lld", k ? "," : "", st.level == 2 ? "pair" : st.level == 1 ? "slice" : "shared",
                         (long long)st.off, (long long)align_up(st.entries, kAlignEntries));
                out += line;
            }
            out += "\n";
        }
        out.pop_back();
        out += sc ? " scale=1 after=" : " scale=0 after=";
        for (size_t k = 0; k < h->deps[i].size(); ++k) {
            snprintf(line, sizeof line, "%s%d", k ? "," : "", h->deps[i][k]);
            out += line;
        }
        if (h->wave_ok && h->chain_of_op[i] >= 0) {  // run by the prologue launch, in this chain
            snprintf(line, sizeof line, " chain=%d", h->chain_of_op[i]);
            out += line;
        }
        out += "\n";
    }
    if (needed) *needed = (int64_t)out.size() + 1;
    if (buf && len > 0) {
        const size_t n = std::min<size_t>(out.size(), (size_t)len - 1);
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return QX_OK;
}

int qx_set_graphs(qx_handle h, int enable) {
    if (!h) return QX_EINVAL;
    drop_graph(h);
    h->graphs = enable != 0;
    return QX_OK;
}

int qx_set_memo(qx_handle h, int enable) {
    if (!h) return QX_EINVAL;
    if (enable != 0 && enable != 1) return fail(h, QX_EINVAL, "enable must be 0 or 1");
    drop_graph(h);
    h->memo = enable != 0;
    h->inv_ready = false;
    return QX_OK;
}

int qx_set_streams(qx_handle h, int32_t n_streams) {
    if (!h) return QX_EINVAL;
    if (n_streams < 1 || n_streams > 32) return fail(h, QX_EINVAL, "n_streams %d out of range [1, 32]", n_streams);
    drop_graph(h);
    h->n_streams = n_streams;
    return QX_OK;
}

int qx_set_profiling(qx_handle h, int enable) {
    if (!h) return QX_EINVAL;
    int rc = prof_collect(h);
    if (rc) return rc;
    h->profiling = enable != 0;
    for (int k = 0; k < QX_KERNEL_KINDS; ++k) {
        h->prof_ms[k] = h->prof_flops[k] = h->prof_bytes[k] = 0;
        h->prof_launches[k] = 0;
    }
    return QX_OK;
}

int qx_profile_read(qx_handle h, int kind, double* ms, int64_t* launches, double* flops, double* bytes) {
    if (!h) return QX_EINVAL;
    if (kind < 0 || kind >= QX_KERNEL_KINDS) return fail(h, QX_EINVAL, "kernel kind %d out of range", kind);
    int rc = prof_collect(h);
    if (rc) return rc;
    if (ms) *ms = h->prof_ms[kind];
    if (launches) *launches = h->prof_launches[kind];
    if (flops) *flops = h->prof_flops[kind];
    if (bytes) *bytes = h->prof_bytes[kind];
    return QX_OK;
}

int qx_device_status(qx_handle h) {
    if (!h) return QX_EINVAL;
    if (!h->ws && !h->static_err) return QX_OK;
    int flag = 0, sflag = 0;
    CUDA_TRY(h, cudaSetDevice(h->device));
    if (h->ws)
        CUDA_TRY(h, cudaMemcpyAsync(&flag, h->ws + h->off_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    // the flag of a static-scratch call lives in the shared array, not in the handle's workspace
    if (h->static_err)
        CUDA_TRY(h, cudaMemcpyAsync(&sflag, h->static_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->static_err = nullptr;
    if (flag) {
        h->inv_ready = false;  // the kept intermediates may be incomplete
        return fail(h, flag, "a bounded device wait expired; the result is invalid");
    }
    if (sflag) return fail(h, sflag, "a bounded device wait expired in a static-scratch call; the result is invalid");
    return QX_OK;
}

int qx_last_stats(qx_handle h, double* flops, int64_t* launches, int64_t* batches) {
    if (!h) return QX_EINVAL;
    if (flops) *flops = h->last_flops;
    if (launches) *launches = h->last_launches;
    if (batches) *batches = h->last_batches;
    return QX_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Contraction into a caller-chosen device buffer (used by the static-scratch entry point)
// ------------------------------------------------------------------------------------------------
int qx_internal_device(const qx_ctx* h) { return h->device; }

int qx_internal_fail(qx_ctx* h, int code, const char* msg) { return fail(h, code, "%s", msg); }

cudaStream_t qx_internal_stream(const qx_ctx* h) { return h->stream; }

void* qx_internal_small(qx_ctx* h) {
    if (!h->d_small && cudaMalloc(&h->d_small, 256) != cudaSuccess) {
        h->d_small = nullptr;
        cudaGetLastError();
    }
    return h->d_small;
}

int qx_internal_shape(const qx_ctx* h, int* n_qubits, int64_t* n_open_out, int64_t* max_bits, int* ready) {
    *n_qubits = h->have_net ? h->nq : 0;
    *n_open_out = h->have_net ? n_open(h) : 0;
    *max_bits = h->ws ? h->max_bits : 0;
    *ready = h->have_plan && h->ws != nullptr;
    return QX_OK;
}

int qx_internal_contract_in(qx_ctx* h, char* buf, int64_t buf_bytes, const uint8_t* d_bits, int64_t n_bits,
                            double* d_amps) {
    if (!h->have_plan) return fail(h, QX_ESTATE, "contract before qx_set_plan");
    if (h->device < 0) return fail(h, QX_ESTATE, "host-only handle has no device");
    if (n_bits < 1) return fail(h, QX_EINVAL, "n_bits < 1");
    if (!d_bits || !d_amps || !buf) return fail(h, QX_EINVAL, "null buffer");
    struct {
        char* ws;
        int64_t ws_bytes;
        bool ws_owned;
        int64_t max_bits, off_err, off_leaf, off_bits, off_acc, off_amps, off_inv, off_item, items_cap, off_slice,
            slices_cap;
        bool leaves_on_device;
        int64_t off_pops, off_counter, off_results, off_pscratch, off_pops_inv, off_wave;
        bool pops_on_device, waves_on_device, inv_ready;
    } const saved = {h->ws,        h->ws_bytes, h->ws_owned,    h->max_bits,    h->off_err,    h->off_leaf,
                     h->off_bits,  h->off_acc,  h->off_amps,    h->off_inv,     h->off_item,   h->items_cap,
                     h->off_slice, h->slices_cap, h->leaves_on_device, h->off_pops, h->off_counter, h->off_results, h->off_pscratch,
                     h->off_pops_inv, h->off_wave, h->pops_on_device, h->waves_on_device, h->inv_ready};
    int64_t fixed, items = 0, slices = 0;
    layout(h, n_bits, &fixed);
    const bool fits = fit_regions(h, buf_bytes - fixed, n_bits, &items, &slices);
    auto restore = [&]() {
        h->ws = saved.ws;
        h->ws_bytes = saved.ws_bytes;
        h->ws_owned = saved.ws_owned;
        h->max_bits = saved.max_bits;
        h->off_err = saved.off_err;
        h->off_leaf = saved.off_leaf;
        h->off_bits = saved.off_bits;
        h->off_acc = saved.off_acc;
        h->off_amps = saved.off_amps;
        h->off_inv = saved.off_inv;
        h->off_item = saved.off_item;
        h->items_cap = saved.items_cap;
        h->off_slice = saved.off_slice;
        h->slices_cap = saved.slices_cap;
        h->leaves_on_device = saved.leaves_on_device;
        h->off_pops = saved.off_pops;
        h->off_counter = saved.off_counter;
        h->off_results = saved.off_results;
        h->off_pscratch = saved.off_pscratch;
        h->off_pops_inv = saved.off_pops_inv;
        h->pops_on_device = saved.pops_on_device;
        h->off_wave = saved.off_wave;
        h->waves_on_device = saved.waves_on_device;
        h->inv_ready = saved.inv_ready;
    };
    if (!fits) {
        restore();
        return fail(h, QX_ENOMEM, "this plan and %lld bitstrings need %lld bytes of scratch; %lld are available",
                    (long long)n_bits, (long long)(fixed + 256 + (h->item_entries + h->slice_entries) * 8),
                    (long long)buf_bytes);
    }
    char* const saved_wb = h->wb;
    h->wb = nullptr;
    h->ws = buf;
    h->ws_bytes = buf_bytes;
    h->ws_owned = false;
    h->max_bits = n_bits;
    place_regions(h, fixed, items, slices);
    h->leaves_on_device = false;
    h->pops_on_device = false;
    h->waves_on_device = false;
    h->inv_ready = false;  // the shared scratch array holds whatever the last call left
    int rc = QX_OK;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) rc = fail(h, QX_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    if (rc == QX_OK) rc = contract_impl(h, d_bits, n_bits, 0, h->n_slices, d_amps);
    if (rc == QX_OK) h->static_err = buf + h->off_err;  // read by the next qx_device_status
    restore();
    h->wb = saved_wb;
    return rc;
}

// ------------------------------------------------------------------------------------------------
// Groups: many networks contracted by one persistent launch (uneven circuits side by side)
// ------------------------------------------------------------------------------------------------
struct qx_group {
    std::vector<qx_ctx*> hs;
    std::vector<const uint8_t*> bits;
    std::vector<int64_t> n_bits;
    std::vector<double*> amps;
    int device = 0;
    cudaStream_t stream = nullptr;
    int grid = 0;
    std::vector<PProg> inv_progs, pair_progs;
    std::vector<GSum> sums;
    int64_t n_pair_work = 0, total_sum = 0, max_entries = 0;
    char* scratch = nullptr;
    int64_t scratch_bytes = 0;
    int64_t off_inv = 0, off_pair = 0, off_sum = 0, off_sc = 0;
    std::string err;
    bool bound = false;
};

static int gfail(qx_group* g, int code, const char* msg) {
    g->err = msg;
    return code;
}

static void group_layout(qx_group* g, int64_t* bytes) {
    int64_t off = 256;  // work counter
    g->off_inv = off;
    off += align_up((int64_t)(g->hs.size() * sizeof(PProg)), 256);
    g->off_pair = off;
    off += align_up((int64_t)(g->hs.size() * sizeof(PProg)), 256);
    g->off_sum = off;
    off += align_up((int64_t)(g->hs.size() * sizeof(GSum)), 256);
    g->off_sc = off;
    off += align_up((int64_t)g->grid * g->max_entries * 8, 256);
    *bytes = off;
}

extern "C" {

int qx_group_create(qx_group_t* out, qx_handle* hs, int32_t n, const uint8_t* const* d_bits, const int64_t* n_bits,
                    double* const* d_amps, int32_t ctas_per_sm) {
    if (!out) return QX_EINVAL;
    *out = nullptr;
    if (!hs || n < 1 || !d_bits || !n_bits || !d_amps) return QX_EINVAL;
    if (ctas_per_sm < 0 || ctas_per_sm > 4) return QX_EINVAL;
    qx_group* g = new qx_group();
    for (int i = 0; i < n; ++i) {
        qx_ctx* h = hs[i];
        const char* why = nullptr;
        if (!h) why = "null handle";
        else if (!h->have_plan || !h->ws) why = "every handle needs a plan and a bound workspace";
        else if (h->opt.executor != 3 || !h->persist_ok)
            why = "every handle must be created with executor 3 and a plan without tensor-core steps";
        else if (h->device != hs[0]->device) why = "handles on different devices";
        else if (n_bits[i] < 1 || n_bits[i] > h->max_bits) why = "bitstring count outside the handle's workspace";
        else if (!d_bits[i] || !d_amps[i]) why = "null buffer";
        if (why) {
            g->err = why;
            *out = g;
            return QX_EINVAL;
        }
        g->hs.push_back(h);
        g->bits.push_back(d_bits[i]);
        g->n_bits.push_back(n_bits[i]);
        g->amps.push_back(d_amps[i]);
        g->max_entries = std::max(g->max_entries, h->item_entries);
    }
    g->device = hs[0]->device;
    g->stream = hs[0]->stream;
    g->grid = (ctas_per_sm ? ctas_per_sm : 2) * (hs[0]->persist_grid / 2);
    *out = g;
    return QX_OK;
}

const char* qx_group_last_error(qx_group_t g) { return g ? g->err.c_str() : "null group"; }

int qx_group_scratch_size(qx_group_t g, int64_t* bytes) {
    if (!g || !bytes) return QX_EINVAL;
    if (g->hs.empty()) return gfail(g, QX_ESTATE, "group creation failed");
    group_layout(g, bytes);
    return QX_OK;
}

int qx_group_bind(qx_group_t g, void* d_scratch, int64_t bytes) {
    if (!g) return QX_EINVAL;
    if (g->hs.empty()) return gfail(g, QX_ESTATE, "group creation failed");
    int64_t need;
    group_layout(g, &need);
    if (!d_scratch || bytes < need || ((uintptr_t)d_scratch) % 256) return gfail(g, QX_ENOMEM, "scratch too small or misaligned");
    if (cudaSetDevice(g->device) != cudaSuccess) return gfail(g, QX_ECUDA, "cudaSetDevice failed");
    g->scratch = (char*)d_scratch;
    g->scratch_bytes = bytes;
    // each member's tensors and programs on its own workspace
    for (qx_ctx* h : g->hs) {
        if (!h->leaves_on_device) {
            if (cudaMemcpyAsync(h->ws + h->off_leaf, h->leaf_vals.data(), h->leaf_vals.size() * sizeof(float2),
                                cudaMemcpyHostToDevice, g->stream) != cudaSuccess)
                return gfail(g, QX_ECUDA, "leaf upload failed");
            h->leaves_on_device = true;
        }
        if (upload_programs(h) != QX_OK) return gfail(g, QX_ECUDA, h->err.c_str());
    }
    // programs ordered by per-pair work, largest first, so the long pairs start early
    std::vector<int> order(g->hs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return g->hs[a]->flops_item > g->hs[b]->flops_item; });
    g->inv_progs.clear();
    g->pair_progs.clear();
    g->sums.clear();
    int64_t w = 0, t = 0;
    for (int i : order) {
        qx_ctx* h = g->hs[i];
        if (!h->pops_inv.empty()) {
            PProg p = make_prog(h, true, g->bits[i], 1, 0);
            p.work0 = (int64_t)g->inv_progs.size();
            g->inv_progs.push_back(p);
        }
        PProg p = make_prog(h, false, g->bits[i], g->n_bits[i], 0);
        p.work0 = w;
        w += h->n_slices * g->n_bits[i];
        g->pair_progs.push_back(p);
    }
    for (size_t i = 0; i < g->hs.size(); ++i) {
        qx_ctx* h = g->hs[i];
        g->sums.push_back(make_gsum(h, g->n_bits[i], h->n_slices, g->amps[i], t));
        t += g->n_bits[i] << n_open(h);
    }
    g->n_pair_work = w;
    g->total_sum = t;
    cudaError_t e = cudaSuccess;
    if (!g->inv_progs.empty())
        e = cudaMemcpyAsync(g->scratch + g->off_inv, g->inv_progs.data(), g->inv_progs.size() * sizeof(PProg),
                            cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->scratch + g->off_pair, g->pair_progs.data(), g->pair_progs.size() * sizeof(PProg),
                            cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->scratch + g->off_sum, g->sums.data(), g->sums.size() * sizeof(GSum),
                            cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return gfail(g, QX_ECUDA, cudaGetErrorString(e));
    g->bound = true;
    return QX_OK;
}

int qx_group_run(qx_group_t g) {
    if (!g) return QX_EINVAL;
    if (!g->bound) return gfail(g, QX_ESTATE, "qx_group_run before qx_group_bind");
    if (cudaSetDevice(g->device) != cudaSuccess) return gfail(g, QX_ECUDA, "cudaSetDevice failed");
    PLaunch L{};
    L.scratch = (float2*)(g->scratch + g->off_sc);
    L.scratch_entries = g->max_entries;
    L.counter = (unsigned long long*)g->scratch;
    cudaError_t e = cudaSuccess;
    if (!g->inv_progs.empty()) {
        L.progs = (const PProg*)(g->scratch + g->off_inv);
        L.n_progs = (int32_t)g->inv_progs.size();
        L.n_work = L.n_progs;
        e = launch_persist(L, std::min<int>(g->grid, L.n_progs), g->stream);
    }
    if (e == cudaSuccess) {
        L.progs = (const PProg*)(g->scratch + g->off_pair);
        L.n_progs = (int32_t)g->pair_progs.size();
        L.n_work = g->n_pair_work;
        e = launch_persist(L, g->grid, g->stream);
    }
    if (e == cudaSuccess)
        e = launch_group_sum((const GSum*)(g->scratch + g->off_sum), (int32_t)g->sums.size(), g->total_sum, g->stream);
    if (e != cudaSuccess) return gfail(g, QX_ECUDA, cudaGetErrorString(e));
    return QX_OK;
}

void qx_group_destroy(qx_group_t g) { delete g; }

}  // extern "C"
