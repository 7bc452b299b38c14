// tn_plan.h -- host-side node plan and runtime of libtn.so (internal).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/tn.h"
#include "tn_internal.h"

namespace tn {

struct LeafDesc {
    std::vector<int> lab;         // dense label ids, tensor axis order
    std::vector<int64_t> stride;  // row-major element strides
    int64_t size = 1;
    const void* ptr = nullptr;    // user pointer (device or host)
    int mem = -1;
    void* staged = nullptr;       // library copy of a host leaf
    int64_t staged_bytes = 0;
};

struct NetDesc {
    tn_dtype dt = TN_C64;
    int n = 0;
    std::vector<int64_t> dims;  // per dense label
    std::vector<int64_t> ids;   // dense -> user id
    std::unordered_map<int64_t, int> id2d;
    std::vector<LeafDesc> leaves;
    std::vector<int> open;  // dense labels, output axis order
    // host leaves of one call go to the device as one copy: a page-locked
    // image of all of them, its device twin, and the event of the last copy
    void* stage_host = nullptr;
    void* stage_dev = nullptr;
    int64_t stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;
    bool stage_pending = false;
    bool is_complex() const { return dt == TN_C64; }
    size_t elem_bytes() const { return dt == TN_C64 ? 8 : 4; }
};

enum NodeKind { kGeneric = 0, kTiled = 1, kTensorCore = 2 };

struct Node {
    int id = 0;                  // tree id (n + k)
    int ca = 0, cb = 0;          // child tree ids in the A and B roles (-1: unit scalar)
    std::vector<int> lab;        // output labels, slowest first (row-major)
    std::vector<int64_t> stride;
    int64_t size = 1;
    int64_t ws_off = 0;          // element offset in the workspace
    std::vector<int> gb, gm, gn, gk, gsa, gsb;  // label groups
    int kind = kGeneric;
    double vc = 0;               // log2 of 2^vc, Eq. vertexcon
    TileArgs tile{};             // index bits, config and split (kTiled); pointers set at alloc
};

// One launch of the per-slice sequence: a wave (all small nodes of a tree
// level, k_wave) or a single node (tiled or generic kernel).
struct Step {
    int wave = 0;
    int flow = 0;                  // wave over several levels run as one dataflow
    int node = -1;                 // single-node step
    int item_begin = 0, item_count = 0;
    std::vector<int> nodes;        // nodes run by this step
};

// Wave items (k_wave: one CTA of 256 threads per item, every output summed
// over all 2^nk entries of K by that CTA).  A tiled node joins a wave when
// it is small: at most 2^16 outputs, 2^22 multiply-adds counted over all
// copies that share the launch, 2^14 summed entries per output.  Narrow
// mid-size nodes (a few thousand outputs, 2^21..2^22 multiply-adds) fill
// the GPU better as items than as a tiled launch, whose tiles they cover
// only in part; bigger launches belong to the tiled and tensor-core kernels.
inline bool wave_node(const Node& nd, int copies = 1) {
    return nd.kind == kTiled && nd.tile.cfg != kTileDot && nd.size <= (1 << 16) &&
           nd.vc + std::log2((double)copies) <= 22.0 && nd.tile.nk <= 14;
}
// Outputs per item: at most 2^10 multiply-adds (4 per thread, one batch of
// independent loads: on the dataflow's critical path an item's latency must
// not grow with K), 2^12 when several copies share the launch (there
// throughput counts), and at most 1024 outputs.
// Persistent plans: nodes with >= 32 rows and columns and >= 4096 outputs
// run as 64 x 64 tile items.
inline bool tile_item_node(const Node& nd) {
    return nd.kind == kTiled && nd.tile.nm >= 5 && nd.tile.nn >= 5 && nd.size >= 4096;
}
inline int64_t wave_chunk(const Node& nd, int copies = 1) {
    const int bits = copies > 1 ? 12 : 10;
    const int sh = nd.tile.nk >= bits ? 0 : bits - nd.tile.nk;
    int64_t c = int64_t(1) << sh;
    if (c > 1024) c = 1024;
    return nd.size < c ? nd.size : c;
}

struct GradState;  // reverse-sweep plan and device state (tn_grad.cpp)

struct Plan {
    tn_mode mode = TN_MODE_FP32;
    // persistent launch: every node (every slice of a call side by side) in
    // one dataflow launch -- wave items for the small or narrow nodes, 64 x 64
    // tile items over all of K for the others; FP32 on the CUDA cores
    bool persistent = false;
    bool tuned = false;             // kernels chosen by autotune_plan
    bool no_flow = false;           // one launch per wave level (env TN_NO_FLOW)
    std::vector<int> flow_deps;     // per node: child a, its chunks, child b, its chunks
    int* flow_deps_dev = nullptr;
    unsigned* flow_cnt_dev = nullptr;  // done[node * G + inst], then one head per step
    bool force_generic = false;  // every node on the generic kernel
    bool no_waves = false;       // one launch per node
    bool no_tensor_cores = false;  // reduced-precision modes on CUDA cores only
    int copies = 1;  // copies sharing every node launch: K splits fill the GPU with tiles x copies
    std::vector<int32_t> pairs;
    std::vector<int64_t> sliced_ids;
    std::vector<int> sliced;  // dense
    int64_t d_sliced = 1;
    std::vector<Node> nodes;
    // per tree vertex (leaves then nodes): labels and strides after slicing
    std::vector<std::vector<int>> vlab;
    std::vector<std::vector<int64_t>> vstride;
    std::vector<SliceDigits> leaf_sl;
    int64_t ws_elems = 0;
    double W = 0, C = 0;
    int64_t n_out = 1;
    // device state
    void* ws = nullptr;
    unsigned* maxabs = nullptr;
    int64_t* exps = nullptr;
    Control* ctl = nullptr;
    double* acc = nullptr;
    double* out_stage = nullptr;           // [accumulator | exponent] for host outputs
    unsigned* leafmax = nullptr;           // max |component| of each leaf
    const float** leaf_ptr_dev = nullptr;  // device copy of the leaf pointers
    int64_t* leaf_nfloat_dev = nullptr;
    std::vector<const void*> leaf_ptr_uploaded;
    std::vector<GenericArgs> gen;
    GradState* grad = nullptr;
    // instances (slice-parallel or independent copies)
    int alloc_inst = 1;                 // instances the device state holds
    int cfg_inst = -1, cfg_step = 1;    // layout currently in the arguments
    std::vector<int64_t> cfg_leaf_is;
    std::vector<int> inst_items_begin;  // per step: first wave item (all instances)
    BatchRoot* inst_roots_dev = nullptr;
    double* inst_out_dev = nullptr;
    int64_t* inst_exp_dev = nullptr;
    int graph_inst = -1, graph_step = -1;
    int inst_roots_n = 0;
    std::vector<int64_t> leaf_nfloat_uploaded;
    std::vector<Step> steps;
    std::vector<WaveItem> items;
    WaveItem* items_dev = nullptr;
    TileArgs* descs_dev = nullptr;
    void* split_buf = nullptr;      // K-split partials, shared by all split nodes
    int64_t split_bytes = 0;
    AccumArgs acc_args{};
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;         // per-slice sequence without timing hooks
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void*> graph_ptrs;
    int graph_prof_first = 0, graph_prof_count = 0;
    // the same sequence with timing hooks (kept beside the plain one, so
    // that calls with and without hooks do not recapture)
    cudaGraph_t graph_h = nullptr;
    cudaGraphExec_t gexec_h = nullptr;
    std::vector<const void*> graph_ptrs_h;
    int graph_prof_first_h = 0, graph_prof_count_h = 0;
    int graph_inst_h = -1, graph_step_h = -1;
    std::vector<cudaEvent_t> prof_placeholder;  // events captured into the graph
    std::vector<cudaGraphNode_t> prof_nodes;    // their record nodes, in order
};

tn_status build_plan(const NetDesc& d, Plan& p, std::string& err);
Node build_node(const NetDesc& d, const Plan& p, int id, int a, int b, const std::vector<int>& keep);
bool plan_tile_node(const NetDesc& d, const Plan& p, Node& nd, int64_t& split_elems);
bool make_tensor_core(const NetDesc& d, tn_mode mode, Node& nd, int64_t& split_elems, int copies = 1);
// Autotuner variant code of the tensor-core kernel (tile shapes use TileCfg).
constexpr int kVariantTC = 8;
// ... and of the tensor-core kernel with 128-column tiles (twice the tiles:
// a fuller grid for nodes with few).
constexpr int kVariantTC128 = 9;
// ... and of the tensor-core kernel on the planar complex layout (split
// precisions, >= 128 complex rows and columns).
constexpr int kVariantTCPlanar = 10;
// Times every candidate kernel of the nodes that run alone in a launch step
// and keeps the fastest in the plan (device state must be allocated).
tn_status autotune_plan(NetDesc& d, Plan& p, int reps, int32_t* choice, cudaStream_t s, std::string& err);
tn_status make_generic_args_node(const NetDesc& d, const Plan& p, const Node& nd, GenericArgs& g,
                                 std::string& err);
tn_status alloc_plan(NetDesc& d, Plan& p, void* unit, std::string& err);
tn_status run_plan(NetDesc& d, Plan& p, void* unit, int64_t begin, int64_t count,
                   const tn_options& o, void* out, int out_mem, int64_t* out_exp2,
                   cudaStream_t stream, std::string& err);
tn_status run_instances(NetDesc& d, Plan& p, void* unit, int n_inst, const int64_t* leaf_is,
                        double* out, int64_t* out_exp2, int out_mem, cudaStream_t stream,
                        std::string& err);
// adj: FP64 adjoint in host (adj_mem TN_MEM_HOST) or device memory; its
// exponent is adj_exp2 plus, for a device adjoint, *adj_exp2_dev (if set).
// n_inst instances: leaf v of instance i at its pointer + i *
// leaf_inst_stride[v] elements (NULL or 0: shared), adjoint i at adj + i *
// (output size), exponent adj_exp2 + adj_exp2_dev[i]; a shared leaf's
// gradient is the sum over the instances, a varying leaf's is per instance.
// kept_forward: the workspace holds the forward of the last
// run_grad_forward (same copies and leaves): only the sweep runs.
tn_status run_grad(NetDesc& d, Plan& p, void* unit, const double* adj, int adj_mem, int64_t adj_exp2,
                   const int64_t* adj_exp2_dev, void* const* grads, bool accumulate, bool kept_forward,
                   int n_inst, const int64_t* leaf_inst_stride, int64_t slice_begin, int64_t slice_count,
                   cudaStream_t stream, std::string& err);
// Forward of n_inst copies (unsliced scalar networks) in the sweep's state,
// every intermediate kept; values as tn_contract_instances.
tn_status run_grad_forward(NetDesc& d, Plan& p, void* unit, int n_inst, const int64_t* leaf_inst_stride,
                           double* out, int64_t* out_exp2, int out_mem, cudaStream_t stream, std::string& err);
void plan_info(const NetDesc& d, const Plan& p, double out[8]);
void free_device(Plan& p);  // releases device state; the host plan stays valid
void free_grad(Plan& p);
// Generic-kernel arguments of node k (index digits, slice digits); pointers
// and bookkeeping slots are left for the caller to fill.
tn_status make_generic_args(const NetDesc& d, const Plan& p, int k, GenericArgs& g, std::string& err);
// The contraction with all scratch in the library's fixed device array
// (tn_noalloc.cu); allocates no device memory.
tn_status run_noalloc(const NetDesc& d, const Plan& p, void* out, int out_mem, int64_t* out_exp2,
                      cudaStream_t stream, std::string& err);

}  // namespace tn
