// tn_internal.h -- structures shared by the host planner and the CUDA kernels
// of libtn.so.  Not part of the public C-ABI (include/tn.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tn {

// Maximum number of index digits (labels) handled by one generic node launch
// in each of its output and summed label sets.
constexpr int kMaxDigits = 40;
// Maximum number of sliced labels present in one leaf operand.
constexpr int kMaxSliceDigits = 16;
// Maximum number of bits per index group of the tiled kernels.
constexpr int kMaxBits = 40;
// Largest tensor (leaf or intermediate of a sliced tree), as log2 of its
// entry count: 2^40 entries are far beyond any device memory, so every size,
// offset and byte count derived from one stays well inside int64.
constexpr int kMaxLog2Entries = 40;
// Largest number of multiply-adds of one node (log2): summed-entry counts
// stay inside int64.
constexpr int kMaxLog2Work = 62;

// Device-side control block of one contraction call (one per plan).
struct Control {
    int64_t slice;        // current slice id
    int64_t slice_begin;  // first slice id of the call
    int64_t acc_exp[2];   // double-buffered exponent of the FP64 accumulator
    int64_t final_exp;    // exponent of the result after the last slice
    int32_t status;       // 0 ok; TN_ETIMEOUT etc. set by device code
    int32_t pad;
    int64_t slice_end;    // instances whose slice id reaches this are idle
};

// Instances: one launch runs n_inst copies of a node.  Instance i reads
// A + i*a_is, B + i*b_is, writes C + i*c_is (elements), uses the
// renormalisation slots offset by i*s?_is, and works on slice
// ctl->slice + i*slice_step (instances beyond ctl->slice_end are idle).
struct InstanceInfo {
    int32_t n_inst;
    int32_t slice_step;
    int64_t a_is, b_is, c_is, p_is;
    int32_t sa_is, sb_is, sc_is;
    int32_t pad;
};

// Offset of a sliced leaf: sum over its sliced labels of
// ((slice / div) % dim) * stride.
struct SliceDigits {
    int n;
    int64_t div[kMaxSliceDigits];
    int64_t dim[kMaxSliceDigits];
    int64_t stride[kMaxSliceDigits];
};

// Power-of-two renormalisation bookkeeping of a node (Sec. 4.2 of the
// paper): the stored tensor times 2^exps[slot] is the true tensor; maxabs
// holds the largest |component| of the stored tensor (float bits).
struct ScaleIO {
    const unsigned* max_a;   // nullptr for a leaf operand (scale 1)
    const unsigned* max_b;
    const int64_t* exp_a;    // nullptr for a leaf operand (exponent 0)
    const int64_t* exp_b;
    unsigned* max_c;
    int64_t* exp_c;
};

// Generic node: out[o] = sum_k A[offA(o,k)] * B[offB(o,k)] with mixed-radix
// digits; handles any label sizes, batch (hyper) labels and labels summed
// in one operand only (stride 0 in the other).
struct GenericArgs {
    const void* A;
    const void* B;
    void* C;
    int64_t n_out;
    int64_t n_sum;
    int n_od;                       // output digits, fastest first
    int n_kd;                       // summed digits, fastest first
    int32_t od_dim[kMaxDigits];
    int64_t od_sa[kMaxDigits];
    int64_t od_sb[kMaxDigits];
    int32_t kd_dim[kMaxDigits];
    int64_t kd_sa[kMaxDigits];
    int64_t kd_sb[kMaxDigits];
    SliceDigits sla, slb;
    const Control* ctl;
    ScaleIO sc;
    int conj_a, conj_b;  // read the operand complex-conjugated (reverse sweep)
    unsigned long long* t_done;  // root of a batched network: completion time (ns)
    InstanceInfo in;
};

// Tiled node (power-of-two label sizes): every index group is a set of bits.
// offset(group index g) = sum_i bit_i(g) << shift_i ; shift 255 = absent.
struct BitGroup {
    int nbits;
    uint8_t sh[kMaxBits];
};

// Tiled node (power-of-two label sizes).  Each index group is a list of
// bits; bit i of a group index contributes 1 << sh[i] to an operand offset
// (kNoBit: the operand lacks that label).  Output layout [batch][M][N].
constexpr uint8_t kNoBit = 255;
enum TileCfg { kTile64x64 = 1, kTile16x256 = 2, kTile4x1024 = 3, kTile256x16 = 4, kTileDot = 5, kTile128x64 = 6 };

struct alignas(16) TileArgs {
    const void* A;
    const void* B;
    void* C;
    void* P;              // K-split partials [split][batch][M][N] (split > 1)
    int nb, nm, nn, nk;   // bits per group
    int64_t nbatch;       // 1 << nb
    uint8_t a_b[kMaxBits], a_m[kMaxBits], a_k[kMaxBits];
    uint8_t b_b[kMaxBits], b_n[kMaxBits], b_k[kMaxBits];
    int a_mfast;          // A's fastest tile bit is an M bit: load A along m
    int b_nfast;          // B's fastest tile bit is an N bit: load B along n
    int cfg;              // TileCfg
    int split;            // K splits (grid.z = nbatch * split)
    int64_t kchunk;       // K entries per split
    SliceDigits sla, slb;
    const Control* ctl;
    ScaleIO sc;
    int a_leaf, b_leaf;   // leaf index of an operand (its pointer comes from the
                          // leaf pointer table in wave launches), else -1
    int conj_a, conj_b;   // read the operand complex-conjugated (reverse sweep)
    unsigned long long* t_done;  // root of a batched network: completion time (ns)
    int tc_swap;          // tensor-core node: B plays the row role (see TcGeom)
    int tc_bn128;         // tensor-core node: 128-column GEMM tiles even where 256 fit
    int tc_planar;        // tensor-core node: planar complex layout (see TcGeom)
    int tc_nopair;        // tensor-core node: single-CTA GEMM even where CTA pairs apply
    InstanceInfo in;
};

// Packed operands of a tensor-core node, in the shared P buffer (per
// instance, p_is elements of the node's dtype apart).  The "row" operand R
// (A, or B when tc_swap) holds [batch x rows] x KR and the "column" operand
// Q (the other one) [batch x cols] x KR, K-major: a complex R stores
// (re, im) pairs along K (KR = 2K), a complex Q is expanded to two real rows
// per column, (re, -im) and (im, re), so that one real GEMM forms the
// complex product (4M).  Each plane is cut into 16 KB tiles of 128 rows x
// one 128-byte swizzled row of K (the shared-memory image the MMA reads),
// stored row tile by row tile and, within one, k-block by k-block, so that
// one k-block of one operand is a single contiguous bulk copy.  Split
// precisions store a hi plane then a lo plane.  With a K split (split > 1)
// the FP32 partial products [split][batch][M][N] follow the packed planes.
//
// Planar layout (tc_planar: complex nodes in a split precision with at least
// 128 complex rows and columns): neither operand is interleaved or expanded.
// R and Q each hold four planes -- Re hi, Re lo, Im hi, Im lo -- of
// [batch x rows] x K complex entries, cut into 8 KB tiles of 128 rows x one
// 64-byte swizzled row of K; the GEMM forms Re C = Re R Re Q - Im R Im Q and
// Im C = Re R Im Q + Im R Re Q as real products (the minus sign by the MMA's
// negate-A bit) into two accumulators.  Per unit of work this moves two
// thirds of the 4M layout's operand bytes, and the smaller stages leave room
// for a deeper pipeline.
struct TcGeom {
    int64_t rows_r;    // rows of R per batch entry
    int64_t cols_q;    // real rows of Q per batch entry in the packed layout: the
                       // node's real accumulator columns, padded up to one 128-row tile
    int64_t cols_valid;  // the node's real accumulator columns (<= cols_q)
    int q_pad_lg;      // log2(cols_q / cols_valid): packed Q rows beyond cols_valid are never written
    int64_t kr;        // packed row length (elements) before padding
    int ke;            // elements per 128-byte row (32 TF32, 64 BF16 / FP16)
    int64_t nkb;       // k-blocks (KR padded up to a multiple of ke)
    int esz;           // bytes per packed element (4 TF32, 2 BF16 / FP16)
    int parts;         // 1, or 2 for hi + lo
    int64_t plane_r;   // bytes of one R plane
    int64_t plane_q;   // bytes of one Q plane
    int64_t region_r;  // bytes of all R planes, 1 KB aligned (Q starts here)
    int64_t part_off;  // bytes: start of the split-K partials
    int64_t total;     // bytes per instance, 1 KB aligned
    int bn;            // GEMM tile columns: 256 where the columns allow, else 128
                       // (planar: 128 complex columns)
    int row_bytes;     // bytes of one K row of a tile: 128, or 64 (planar)
    int planar;        // planar complex layout
};

// Tile plan of one operand pack (tensor-core path), computed on the host:
// a tile is 2^t entries (t <= 10), enumerated in source order by the
// src_add offsets and in packed order by dst_pos (byte position in the
// packed planes) and idx_add (stage index); the u remaining bits step
// between tiles.  The byte position of an entry in the packed planes is the
// XOR of one constant per set bit of its packed index (K bits, then row
// bits, then batch bits): every size is a power of two, so tiles and rows
// are bit fields and the swizzle XORs row bits into chunk bits.  pos_row1:
// the position XOR from a complex column's first expanded row to its second
// (4M layout of Q).
struct PackPlan {
    int t, u;
    int64_t src_add[10];
    int64_t dst_pos[10];
    int32_t idx_add[10];
    int64_t rest_src[kMaxBits];  // an operand has at most 2^40 entries
    int64_t rest_pos[kMaxBits];
    int64_t pos_row1;
};

// Tile plan of an inner-product node (k_dot), computed on the host: a tile
// is 2^t K entries; entry e in A's order is at A offset sum of a_add and
// K-order index sum of ca_add over its set bits (likewise for B); the u
// remaining K bits step between tiles.
struct DotPlan {
    int t, u;
    int64_t a_add[10], b_add[10];
    int32_t ca_add[10], cb_add[10];
    int64_t rest_a[kMaxBits], rest_b[kMaxBits];
};

// Tensor-core precision of a mode (tn_mode values): 0 TF32 single product
// (4M), 1 TF32 hi+lo, 2 BF16 hi+lo, 3 TF32 single product (3M), 4 FP16
// hi+lo (operands scaled by 2^kF16Shift).
__host__ __device__ inline int tc_prec_of_mode(int mode) {
    return mode == 4 ? 4 : (mode == 3 ? 2 : (mode == 2 ? 1 : (mode == 1 ? 3 : 0)));
}

// FP16 operands: after the renormalisation (largest magnitude in [1/2, 1))
// the pack scales by 2^kF16Shift, so the largest packed magnitude is below
// 2^15 (FP16's largest finite value is 65504); the GEMM epilogue removes
// 2^(2 kF16Shift) with the rest of the residual scale.
constexpr int kF16Shift = 15;

// Bytes per packed element: 2 for the 16-bit formats, 4 for TF32.
__host__ __device__ inline int tc_esz_of_prec(int prec) { return (prec == 2 || prec == 4) ? 2 : 4; }

// 3M needs a complex node with >= 128 complex columns; otherwise the node
// runs the single-product 4M form.
__host__ __device__ inline int tc_prec_of_node(const TileArgs& a, bool cplx, int prec) {
    if (prec == 3 && (!cplx || a.nm < 7 || a.nn < 7)) return 0;
    return prec;
}

// With prec 3 (3M), R and Q are not interleaved or expanded: both hold three
// real planes [rows] x K -- Re, Im and Re + Im -- and the GEMM forms
// T1 = Re A Re B, T2 = Im A Im B, T3 = (Re A + Im A)(Re B + Im B), so that
// Re C = T1 - T2 and Im C = T3 - T1 - T2.
__host__ __device__ inline TcGeom tc_geom(const TileArgs& a, bool cplx, int prec) {
    TcGeom g;
    prec = tc_prec_of_node(a, cplx, prec);
    g.planar = a.tc_planar ? 1 : 0;
    const int c = cplx && prec != 3 && !g.planar ? 2 : 1;
    g.rows_r = int64_t(1) << (a.tc_swap ? a.nn : a.nm);
    g.cols_valid = (int64_t(1) << (a.tc_swap ? a.nm : a.nn)) * c;
    // narrow complex nodes (64 real columns) fill half of one 128-row Q tile; the
    // GEMM computes the whole tile and the epilogue keeps the valid columns
    g.q_pad_lg = 0;
    while ((g.cols_valid << g.q_pad_lg) < 128) ++g.q_pad_lg;
    g.cols_q = g.cols_valid << g.q_pad_lg;
    g.kr = (int64_t(1) << a.nk) * c;
    g.esz = tc_esz_of_prec(prec);
    g.row_bytes = g.planar ? 64 : 128;
    g.ke = g.row_bytes / g.esz;
    g.nkb = (g.kr + g.ke - 1) / g.ke;
    g.parts = g.planar ? 4 : (prec == 0 ? 1 : (prec == 3 ? 3 : 2));
    g.plane_r = a.nbatch * g.rows_r * g.nkb * g.row_bytes;
    g.plane_q = a.nbatch * g.cols_q * g.nkb * g.row_bytes;
    g.region_r = (g.parts * g.plane_r + 1023) / 1024 * 1024;
    g.part_off = g.region_r + (g.parts * g.plane_q + 1023) / 1024 * 1024;
    const int64_t parts_bytes =
        a.split > 1 ? (int64_t)a.split * a.nbatch * (int64_t(1) << (a.nm + a.nn)) * 4 * (cplx ? 2 : 1) : 0;
    g.total = g.part_off + (parts_bytes + 1023) / 1024 * 1024;
    g.bn = g.planar ? 128 : ((prec != 3 && g.cols_q % 256 == 0 && !a.tc_bn128) ? 256 : 128);
    return g;
}

// One CTA of a wave launch: outputs [o_begin, o_begin + o_count) of node;
// o_count < 0: a 64 x 64 tile item (o_begin = batch entry x tiles + tile).
struct WaveItem {
    int node;
    int pad;
    int64_t o_begin;
    int64_t o_count;
};

// Per-slice FP64 accumulation of the root tensor into the output
// (Sec. 4.7.1: the sliced contractions are summed), with exponent
// alignment.  od_*: digits of the output in the user's open-label order,
// fastest first, with strides into the root tensor.
struct AccumArgs {
    int32_t n_inst;       // roots folded per launch (slice-parallel), in order
    int32_t pad;
    int64_t r_is;         // element stride between the instances' roots
    int32_t s_is;         // slot stride between the instances
    int32_t pad2;
    const void* R;
    int64_t n_out;
    int n_od;
    int32_t od_dim[kMaxDigits];
    int64_t od_s[kMaxDigits];
    const unsigned* max_r;
    const int64_t* exp_r;
    double* acc;
    Control* ctl;
    int32_t advance;  // one-block launches: slices to advance ctl->slice by (set by the launcher)
    int32_t pad3;
};

// Reverse sweep: add a leaf's adjoint (times 2^exp) into its gradient
// accumulator at the slice offset; labels absent from the adjoint
// (summed in one tensor only) broadcast.  Digits fastest first.
struct LeafGradArgs {
    void* grad;
    const void* adj;
    const int64_t* exp_adj;
    int64_t grad_is, adj_is;  // elements between instances (grid z)
    int64_t exp_is;           // scale slots between instances
    int64_t n;
    int n_d;
    int32_t dim[kMaxDigits];
    int64_t gstride[kMaxDigits];
    int64_t astride[kMaxDigits];
    SliceDigits sl;
    const Control* ctl;
};

// Reverse sweep, per call: copies between the caller's tensors and the
// library's images of them (the leaves in, the leaf gradients out), one
// entry per tensor.
struct CopyEntry {
    const float* src;
    float* dst;
    int64_t nfloat;
    int64_t src_is;  // floats between the n_sum source copies
    int32_t n_sum;   // dst (+)= sum over i < n_sum of src[i * src_is + j], i ascending
    int32_t add;     // dst += ... instead of dst = ...
};

// Root adjoint of the reverse sweep: FP64 adjoint in the user's open-label
// order -> float mantissas in the root layout (perm[o] = root offset of
// output o), renormalised by its largest |component|; the exponent (plus
// exp_host and, when not NULL, *exp_dev) and the max go to the root's
// scale slots.
struct RootAdjArgs {
    const double* adj;
    const int64_t* exp_dev;
    int64_t exp_host;
    const int64_t* perm;
    int64_t n_out;
    int32_t cplx;
    int32_t pad;
    float* dst;
    unsigned* max_slot;
    int64_t* exp_slot;
    // instances (one block each): adjoint i at adj + i * n_out * (1|2),
    // exponent exp_dev[i], root dst + i * dst_is floats, slots + i * slot_is
    int64_t dst_is;
    int64_t slot_is;
};

// Batched networks: where each network's root lives and where its result goes.
struct BatchRoot {
    const void* root;           // scalar root value (float2 or float); NULL: a
                                // sliced member that writes its own result
    const int64_t* exp;         // root exponent slot
    const unsigned* max;        // root max slot (0: the value is exactly zero)
    int is_c;
    int pad;
};

// Launchers (tn_kernels.cu).  is_c: complex64 data.
cudaError_t launch_batch_start(unsigned long long* t_start, cudaStream_t s);
// latency = now - *t_start (%globaltimer), written after a batch member's own launches
cudaError_t launch_batch_mark(const unsigned long long* t_start, unsigned long long* latency, cudaStream_t s);
cudaError_t launch_batch_finish(const BatchRoot* roots, int n, double* out, int64_t* out_exp,
                                const unsigned long long* t_start, const unsigned long long* t_done,
                                unsigned long long* latency, cudaStream_t s);
// Leaf adjoints of the current slice for every entry of the device table
// (max_n: the largest entry's n).
cudaError_t launch_leaf_grads(const LeafGradArgs* tab, int n_entries, int64_t max_n, int n_inst, bool is_c,
                              cudaStream_t s);
cudaError_t launch_copy_table(const CopyEntry* tab, int n_entries, int64_t max_nfloat, cudaStream_t s);
// p[i * stride + j] = 0 for i < n, j < count (per-instance scale slots).
cudaError_t launch_zero_strided(unsigned* p, int64_t count, int64_t stride, int n, cudaStream_t s);
cudaError_t launch_root_adjoint(const RootAdjArgs& a, int n_inst, cudaStream_t s);
// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// cached per device); 152, the GB300 count, when no device is visible (host-only
// planning, e.g. tn_plan_info on a machine without a GPU).  Grid sizes and
// K splits are sized in multiples of it.
int sm_count();
cudaError_t launch_generic(const GenericArgs& a, bool is_c, cudaStream_t s);
cudaError_t launch_tile(const TileArgs& a, bool is_c, cudaStream_t s);  // tn_tiled.cu
// Tensor-core node (tn_tc.cu): prec as tc_prec_of_mode.
// Packs both operands into a.P (TcGeom, one launch) and runs the bulk-copy-
// fed tcgen05 GEMM: two launches, plus a fixed-order reduction with a K split.
cudaError_t launch_tc(const TileArgs& a, int prec, bool is_c, cudaStream_t s);
inline int tc_launches(const TileArgs& a) { return a.split > 1 ? 3 : 2; }
// Small nodes of one or more tree levels in one launch (tn_tiled.cu).  deps
// (per node: child a, its chunk count, child b, its chunk count; -1 = none)
// makes it a dataflow over levels with completion counters done[node * G +
// instance] and the item counter head, all zero at launch.
cudaError_t launch_wave(const WaveItem* items, int n_items, const TileArgs* descs,
                        const void* const* leaf_ptrs, bool is_c, cudaStream_t s,
                        const int4* deps = nullptr, unsigned* done = nullptr, unsigned* head = nullptr,
                        int G = 1, bool tiles = false);
// Folds the slice group's roots into the FP64 accumulator, leaves the
// result's exponent after the last group, and advances the slice counter by
// `advance` (in the same launch when it is one block).
cudaError_t launch_accumulate(const AccumArgs& a, bool is_c, cudaStream_t s, int advance);
// Leaf maxima (as launch_leaf_max) and the call's control block and
// accumulator (as launch_begin_call) in one launch after one memset.
cudaError_t launch_call_begin(const float* const* ptrs, const int64_t* nfloat, unsigned* out, int n,
                              int64_t max_nfloat, Control* ctl, int64_t slice_begin, int64_t slice_end,
                              double* acc, int64_t n_acc, cudaStream_t s);
// Copies the accumulator (n doubles) and the final exponent to out / out_exp.
cudaError_t launch_result(const double* acc, int64_t n, const Control* ctl, double* out, int64_t* out_exp,
                          cudaStream_t s);
cudaError_t launch_begin_call(Control* ctl, int64_t slice_begin, int64_t slice_end, double* acc,
                              int64_t n_acc_doubles, cudaStream_t s);
cudaError_t launch_begin_slice(unsigned* maxabs, int n_nodes, cudaStream_t s);
cudaError_t launch_advance(Control* ctl, cudaStream_t s, int step = 1);
cudaError_t launch_leaf_max(const float* const* ptrs, const int64_t* nfloat, unsigned* out, int n,
                            cudaStream_t s, int64_t max_nfloat);

}  // namespace tn
