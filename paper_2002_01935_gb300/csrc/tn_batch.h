// tn_batch.h -- merged plan of a batch of independent networks (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "tn_plan.h"

namespace tn {

struct BatchStep {
    int wave = 0;
    bool cplx = false;
    int item_begin = 0, item_count = 0;
    int net = -1, node = -1;  // single-node step
};

// A sliced network of the batch: not part of the merged forest; its slices
// run after the forest, on the same stream, through its own plan (device
// state owned by its handle), G slices side by side per launch.
struct SlicedMember {
    int index = -1;
    NetDesc* d = nullptr;
    Plan* p = nullptr;
    void* unit = nullptr;
    int G = 1;
};

struct BatchPlan {
    tn_mode mode = TN_MODE_FP32;
    std::vector<const NetDesc*> nets;
    std::vector<Plan*> plans;  // host plans, owned by the network handles
    std::vector<SlicedMember> sliced;  // members with d_sliced > 1
    std::vector<char> is_sliced;       // per network
    std::vector<std::vector<int>> level, small;
    std::vector<int64_t> ws_base;  // bytes
    std::vector<int> slot_base, leaf_base, desc_base;
    int64_t ws_bytes = 0, split_bytes = 0;
    int n_slots = 0, n_leaves = 0;
    int64_t max_leaf_floats = 0;
    std::vector<TileArgs> descs;
    std::vector<GenericArgs> gen;
    std::vector<BatchStep> steps;
    std::vector<WaveItem> items;
    // device
    void* ws = nullptr;
    void* split_buf = nullptr;
    unsigned* maxabs = nullptr;
    int64_t* exps = nullptr;
    Control* ctl = nullptr;
    unsigned* leafmax = nullptr;
    const float** leaf_ptr_dev = nullptr;
    int64_t* leaf_nfloat_dev = nullptr;
    unsigned long long* t_start = nullptr;
    unsigned long long* t_done = nullptr;
    unsigned long long* lat_dev = nullptr;
    double* out_dev = nullptr;
    int64_t* exp_dev = nullptr;
    BatchRoot* roots_dev = nullptr;
    TileArgs* descs_dev = nullptr;
    WaveItem* items_dev = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<const void*> graph_ptrs;
};

tn_status build_batch(BatchPlan& b, std::string& err);
tn_status alloc_batch(BatchPlan& b, std::string& err);
tn_status run_batch(BatchPlan& b, double* out, int64_t* out_exp2, uint64_t* latency_ns, int out_mem,
                    cudaStream_t stream, std::string& err);
void free_batch(BatchPlan& b);

}  // namespace tn
