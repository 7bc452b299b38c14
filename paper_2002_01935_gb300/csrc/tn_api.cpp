// tn_api.cpp -- C-ABI entry points and host-side node planning of libtn.so.
//
// Planning follows the problem statement of arXiv 2002.01935:
//   * tree encoding and node incidence: Sec. 2 (Eq. incidence), generalised
//     so a node keeps a label iff it is open or occurs in a leaf outside the
//     node's subtree (hyperedges, Sec. 3.5; open labels, Sec. 4.7.3);
//   * width and cost: Eqs. edgecon and vertexcon; FLOPs 8C / 2C (Sec. 2);
//   * slicing: Sec. 4.7.1 -- a sliced label is fixed per slice, which only
//     offsets the leaves that hold it, so no leaf is copied.
// Each node's labels are grouped into batch (in both operands and kept),
// K (in both, summed), M / N (in one operand, kept) and summed-only (in one
// operand, not kept); the node's output is laid out [batch][M][N], each
// group ordered so its fastest label is the operand's fastest, which keeps
// every kernel's global accesses coalesced without permutation passes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/tn.h"
#include "tn_internal.h"
#include "tn_batch.h"
#include "tn_plan.h"

namespace {

thread_local std::string g_err;

tn_status fail(tn_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define TN_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(e_ == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA,           \
                        std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

}  // namespace

using tn::Plan;
using tn::NetDesc;

struct tn_net {
    NetDesc d;
    std::vector<std::unique_ptr<Plan>> plans;
    void* unit = nullptr;  // device scalar 1 for single-tensor networks
};

extern "C" {

const char* tn_last_error(void) { return g_err.c_str(); }

const char* tn_version(void) { return "tn-gb300 0.1 (sm_103a)"; }

tn_status tn_create(tn_net** out, tn_dtype dt, int32_t n_tensors, const int32_t* ranks,
                    const int64_t* labels, int32_t n_labels, const int64_t* label_ids,
                    const int64_t* label_dims, int32_t n_open, const int64_t* open_labels) {
    if (!out) return fail(TN_EINVAL, "tn_create: out is NULL");
    *out = nullptr;
    if (dt != TN_R32 && dt != TN_C64) return fail(TN_EINVAL, "tn_create: bad dtype");
    if (n_tensors < 1) return fail(TN_EINVAL, "tn_create: n_tensors < 1");
    if (n_labels < 0 || n_open < 0) return fail(TN_EINVAL, "tn_create: negative count");
    if (!ranks || (n_labels > 0 && (!label_ids || !label_dims)) || (n_open > 0 && !open_labels))
        return fail(TN_EINVAL, "tn_create: NULL array");
    std::unique_ptr<tn_net> net(new (std::nothrow) tn_net);
    if (!net) return fail(TN_ENOMEM, "tn_create: out of host memory");
    NetDesc& d = net->d;
    d.dt = dt;
    d.n = n_tensors;
    for (int i = 0; i < n_labels; ++i) {
        if (label_dims[i] < 1) return fail(TN_EINVAL, "tn_create: label size < 1");
        if (d.id2d.count(label_ids[i])) return fail(TN_EINVAL, "tn_create: duplicate label id");
        d.id2d[label_ids[i]] = (int)d.dims.size();
        d.ids.push_back(label_ids[i]);
        d.dims.push_back(label_dims[i]);
    }
    const int L = (int)d.dims.size();
    std::vector<int> used(L, 0);
    int64_t off = 0;
    d.leaves.resize(n_tensors);
    for (int v = 0; v < n_tensors; ++v) {
        if (ranks[v] < 0) return fail(TN_EINVAL, "tn_create: negative rank");
        if (ranks[v] > 0 && !labels) return fail(TN_EINVAL, "tn_create: labels is NULL");
        auto& lf = d.leaves[v];
        for (int i = 0; i < ranks[v]; ++i) {
            auto it = d.id2d.find(labels[off + i]);
            if (it == d.id2d.end()) return fail(TN_EINVAL, "tn_create: unknown label in tensor");
            if (std::find(lf.lab.begin(), lf.lab.end(), it->second) != lf.lab.end())
                return fail(TN_EINVAL, "tn_create: label repeated within a tensor");
            lf.lab.push_back(it->second);
            used[it->second]++;
        }
        off += ranks[v];
        double lg = 0;
        for (int l : lf.lab) lg += std::log2((double)d.dims[l]);
        if (lg > tn::kMaxLog2Entries) return fail(TN_EUNSUPPORTED, "tn_create: a tensor has more than 2^40 entries");
        lf.size = 1;
        lf.stride.assign(lf.lab.size(), 1);
        for (int i = (int)lf.lab.size() - 1; i >= 0; --i) {
            lf.stride[i] = lf.size;
            lf.size *= d.dims[lf.lab[i]];
        }
    }
    for (int i = 0; i < n_open; ++i) {
        auto it = d.id2d.find(open_labels[i]);
        if (it == d.id2d.end()) return fail(TN_EINVAL, "tn_create: unknown open label");
        if (!used[it->second]) return fail(TN_EINVAL, "tn_create: open label in no tensor");
        if (std::find(d.open.begin(), d.open.end(), it->second) != d.open.end())
            return fail(TN_EINVAL, "tn_create: open label repeated");
        d.open.push_back(it->second);
    }
    for (int l = 0; l < L; ++l)
        if (!used[l]) return fail(TN_EINVAL, "tn_create: label used by no tensor");
    *out = net.release();
    return TN_OK;
}

tn_status tn_set_tensor(tn_net* net, int32_t v, const void* ptr, int32_t mem) {
    if (!net) return fail(TN_EINVAL, "tn_set_tensor: net is NULL");
    if (v < 0 || v >= net->d.n) return fail(TN_EINVAL, "tn_set_tensor: tensor index out of range");
    if (mem != TN_MEM_DEVICE && mem != TN_MEM_HOST) return fail(TN_EINVAL, "tn_set_tensor: bad mem");
    if (!ptr) return fail(TN_EINVAL, "tn_set_tensor: NULL pointer");
    net->d.leaves[v].ptr = ptr;
    net->d.leaves[v].mem = mem;
    return TN_OK;
}

// Plans are kept per (tree, slicing, mode, copies): copies > 1 is the plan of
// tn_contract_instances with that many copies per launch, whose kernel
// choices and K splits count the copies (and which the autotuner, timing
// single copies, leaves alone).
static tn_status get_plan(tn_net* net, const int32_t* pairs, int32_t n_sliced, const int64_t* sliced,
                          tn_mode mode, Plan** out, int copies = 1, bool persistent = false) {
    NetDesc& d = net->d;
    const int n = d.n;
    if (n > 1 && !pairs) return fail(TN_EINVAL, "tree_pairs is NULL");
    if (n_sliced < 0 || (n_sliced > 0 && !sliced)) return fail(TN_EINVAL, "bad sliced labels");
    if (mode < TN_MODE_FP32 || mode > TN_MODE_FP16_SPLIT) return fail(TN_EINVAL, "bad mode");
    std::vector<int32_t> pv(pairs, pairs + 2 * (size_t)(n - 1));
    std::vector<int64_t> sv(sliced, sliced + n_sliced);
    for (auto& p : net->plans)
        if (p->mode == mode && p->pairs == pv && p->sliced_ids == sv && p->copies == copies &&
            p->persistent == persistent) {
            *out = p.get();
            return TN_OK;
        }
    std::unique_ptr<Plan> p(new (std::nothrow) Plan);
    if (!p) return fail(TN_ENOMEM, "out of host memory");
    p->mode = mode;
    p->pairs = pv;
    p->sliced_ids = sv;
    p->copies = copies;
    p->persistent = persistent;
    std::string err;
    tn_status st = tn::build_plan(d, *p, err);
    if (st != TN_OK) return fail(st, err);
    net->plans.push_back(std::move(p));
    *out = net->plans.back().get();
    return TN_OK;
}

// Device state of a plan is created on its first run (host-only planning
// stays usable without a GPU, e.g. for tn_plan_info).
static tn_status ensure_device(tn_net* net, Plan* p) {
    if (p->ws) return TN_OK;
    if (net->d.n == 1 && !net->unit) {
        float one[2] = {1.f, 0.f};
        TN_CUDA(cudaMalloc(&net->unit, 16));
        TN_CUDA(cudaMemcpy(net->unit, one, sizeof(one), cudaMemcpyHostToDevice));
    }
    std::string err;
    tn_status st = tn::alloc_plan(net->d, *p, net->unit, err);
    if (st != TN_OK) {
        tn::free_device(*p);
        return fail(st, err);
    }
    return TN_OK;
}

// Device state for at least G instances (reallocated outside capture).
static tn_status ensure_instances(tn_net* net, Plan* p, int G, cudaStream_t stream) {
    if (p->ws && p->alloc_inst >= G) return TN_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(TN_EUNSUPPORTED, "a plan's first call with more instances must run outside capture");
    if (p->ws) {
        cudaDeviceSynchronize();
        tn::free_device(*p);
    }
    p->alloc_inst = std::max(G, p->alloc_inst);
    return ensure_device(net, p);
}

tn_status tn_contract_ex(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                         const int64_t* sliced_labels, tn_mode mode, const tn_options* opt, void* out,
                         int32_t out_mem, int64_t* out_exp2, void* stream) {
    if (!net) return fail(TN_EINVAL, "tn_contract: net is NULL");
    if (!out || !out_exp2) return fail(TN_EINVAL, "tn_contract: NULL output");
    if (out_mem != TN_MEM_DEVICE && out_mem != TN_MEM_HOST) return fail(TN_EINVAL, "bad out_mem");
    for (int v = 0; v < net->d.n; ++v)
        if (!net->d.leaves[v].ptr) return fail(TN_EINVAL, "tn_contract: tensor without data");
    tn_options o{};
    if (opt) o = *opt;
    if (o.persistent != 0 && o.persistent != 1) return fail(TN_EINVAL, "persistent must be 0 or 1");
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, n_sliced, sliced_labels, mode, &p, 1, o.persistent == 1);
    if (st != TN_OK) return st;
    int64_t begin = o.slice_begin, count = o.slice_count;
    if (count <= 0) {
        begin = 0;
        count = p->d_sliced;
    }
    // (count > 0 here: written so that no sum can overflow)
    if (begin < 0 || begin > p->d_sliced - count) return fail(TN_EINVAL, "slice range out of bounds");
    if (o.slice_batch < 0) return fail(TN_EINVAL, "negative slice_batch");
    int G = (int)std::max<int64_t>(1, std::min<int64_t>(o.slice_batch, count));
    if (o.persistent) {
        // every slice of the call side by side in the one launch, as far as
        // 8 GiB of workspace copies and 2^31 work items allow (else several)
        const int64_t ws = std::max<int64_t>(p->ws_elems * (int64_t)net->d.elem_bytes(), 1);
        const int64_t items = std::max<int64_t>((int64_t)p->items.size(), 1);
        int64_t g = std::min<int64_t>(count, (int64_t(8) << 30) / ws);
        g = std::min<int64_t>(g, ((int64_t(1) << 31) - 1) / items);
        g = std::min<int64_t>(g, 1 << 20);
        G = (int)std::max<int64_t>(1, g);
    }
    st = ensure_instances(net, p, G, (cudaStream_t)stream);
    if (st != TN_OK) return st;
    std::string err;
    st = tn::run_plan(net->d, *p, net->unit, begin, count, o, out, out_mem, out_exp2,
                      (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

tn_status tn_contract_instances(tn_net* net, const int32_t* tree_pairs, tn_mode mode, int32_t n_inst,
                                const int64_t* leaf_inst_stride, double* out, int64_t* out_exp2,
                                int32_t out_mem, void* stream) {
    if (!net) return fail(TN_EINVAL, "tn_contract_instances: net is NULL");
    if (!out || !out_exp2 || n_inst < 1) return fail(TN_EINVAL, "tn_contract_instances: bad arguments");
    if (out_mem != TN_MEM_DEVICE && out_mem != TN_MEM_HOST) return fail(TN_EINVAL, "bad out_mem");
    for (int v = 0; v < net->d.n; ++v) {
        if (!net->d.leaves[v].ptr) return fail(TN_EINVAL, "tn_contract_instances: tensor without data");
        if (net->d.leaves[v].mem != TN_MEM_DEVICE)
            return fail(TN_EUNSUPPORTED, "tn_contract_instances: leaves must be device pointers");
        if (leaf_inst_stride && leaf_inst_stride[v] < 0)
            return fail(TN_EINVAL, "tn_contract_instances: negative stride");
    }
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, 0, nullptr, mode, &p, n_inst);
    if (st != TN_OK) return st;
    st = ensure_instances(net, p, n_inst, (cudaStream_t)stream);
    if (st != TN_OK) return st;
    std::string err;
    st = tn::run_instances(net->d, *p, net->unit, n_inst, leaf_inst_stride, out, out_exp2, out_mem,
                           (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

tn_status tn_contract(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                      const int64_t* sliced_labels, tn_mode mode, void* out, int32_t out_mem,
                      int64_t* out_exp2, void* stream) {
    return tn_contract_ex(net, tree_pairs, n_sliced, sliced_labels, mode, nullptr, out, out_mem,
                          out_exp2, stream);
}

tn_status tn_autotune(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced, const int64_t* sliced_labels,
                      tn_mode mode, int32_t reps, int32_t* choice, void* stream) {
    if (!net) return fail(TN_EINVAL, "tn_autotune: net is NULL");
    for (int v = 0; v < net->d.n; ++v)
        if (!net->d.leaves[v].ptr) return fail(TN_EINVAL, "tn_autotune: tensor without data");
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, n_sliced, sliced_labels, mode, &p);
    if (st != TN_OK) return st;
    st = ensure_instances(net, p, 1, (cudaStream_t)stream);
    if (st != TN_OK) return st;
    std::string err;
    st = tn::autotune_plan(net->d, *p, reps, choice, (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

tn_status tn_contract_grad_ex(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                              const int64_t* sliced_labels, tn_mode mode, const double* out_adjoint,
                              int32_t adj_mem, int64_t adj_exp2, const int64_t* adj_exp2_dev,
                              void* const* leaf_grads, uint32_t flags, int64_t slice_begin,
                              int64_t slice_count, void* stream) {
    if (!net) return fail(TN_EINVAL, "tn_contract_grad: net is NULL");
    if (!out_adjoint || !leaf_grads) return fail(TN_EINVAL, "tn_contract_grad: NULL argument");
    if (adj_mem != TN_MEM_DEVICE && adj_mem != TN_MEM_HOST) return fail(TN_EINVAL, "bad adj_mem");
    if (adj_exp2_dev && adj_mem != TN_MEM_DEVICE)
        return fail(TN_EINVAL, "tn_contract_grad: adj_exp2_dev needs a device adjoint");
    if (flags & ~(uint32_t)TN_GRAD_ACCUMULATE) return fail(TN_EINVAL, "tn_contract_grad: unknown flags");
    for (int v = 0; v < net->d.n; ++v)
        if (!net->d.leaves[v].ptr) return fail(TN_EINVAL, "tn_contract_grad: tensor without data");
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, n_sliced, sliced_labels, mode, &p);
    if (st != TN_OK) return st;
    st = ensure_device(net, p);
    if (st != TN_OK) return st;
    std::string err;
    st = tn::run_grad(net->d, *p, net->unit, out_adjoint, adj_mem, adj_exp2, adj_exp2_dev, leaf_grads,
                      (flags & TN_GRAD_ACCUMULATE) != 0, false, 1, nullptr, slice_begin, slice_count,
                      (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

tn_status tn_contract_grad_instances(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                                     const int64_t* sliced_labels, tn_mode mode, int32_t n_inst,
                                     const int64_t* leaf_inst_stride, const double* out_adjoint,
                                     int32_t adj_mem, int64_t adj_exp2, const int64_t* adj_exp2_dev,
                                     void* const* leaf_grads, uint32_t flags, int64_t slice_begin,
                                     int64_t slice_count, void* stream) {
    if (!net) return fail(TN_EINVAL, "tn_contract_grad_instances: net is NULL");
    if (!out_adjoint || !leaf_grads) return fail(TN_EINVAL, "tn_contract_grad_instances: NULL argument");
    if (n_inst < 1) return fail(TN_EINVAL, "tn_contract_grad_instances: n_inst < 1");
    if (adj_mem != TN_MEM_DEVICE && adj_mem != TN_MEM_HOST) return fail(TN_EINVAL, "bad adj_mem");
    if (adj_exp2_dev && adj_mem != TN_MEM_DEVICE)
        return fail(TN_EINVAL, "tn_contract_grad_instances: adj_exp2_dev needs a device adjoint");
    if (flags & ~(uint32_t)(TN_GRAD_ACCUMULATE | TN_GRAD_KEPT_FORWARD))
        return fail(TN_EINVAL, "tn_contract_grad_instances: unknown flags");
    for (int v = 0; v < net->d.n; ++v)
        if (!net->d.leaves[v].ptr) return fail(TN_EINVAL, "tn_contract_grad_instances: tensor without data");
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, n_sliced, sliced_labels, mode, &p);
    if (st != TN_OK) return st;
    st = ensure_device(net, p);
    if (st != TN_OK) return st;
    std::string err;
    st = tn::run_grad(net->d, *p, net->unit, out_adjoint, adj_mem, adj_exp2, adj_exp2_dev, leaf_grads,
                      (flags & TN_GRAD_ACCUMULATE) != 0, (flags & TN_GRAD_KEPT_FORWARD) != 0, n_inst,
                      leaf_inst_stride, slice_begin, slice_count, (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

tn_status tn_contract_instances_keep(tn_net* net, const int32_t* tree_pairs, tn_mode mode, int32_t n_inst,
                                     const int64_t* leaf_inst_stride, double* out, int64_t* out_exp2,
                                     int32_t out_mem, void* stream) {
    if (!net) return fail(TN_EINVAL, "tn_contract_instances_keep: net is NULL");
    if (!out || !out_exp2 || n_inst < 1) return fail(TN_EINVAL, "tn_contract_instances_keep: bad arguments");
    if (out_mem != TN_MEM_DEVICE && out_mem != TN_MEM_HOST) return fail(TN_EINVAL, "bad out_mem");
    for (int v = 0; v < net->d.n; ++v)
        if (!net->d.leaves[v].ptr) return fail(TN_EINVAL, "tn_contract_instances_keep: tensor without data");
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, 0, nullptr, mode, &p);
    if (st != TN_OK) return st;
    st = ensure_device(net, p);
    if (st != TN_OK) return st;
    std::string err;
    st = tn::run_grad_forward(net->d, *p, net->unit, n_inst, leaf_inst_stride, out, out_exp2, out_mem,
                              (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

tn_status tn_contract_grad(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                           const int64_t* sliced_labels, tn_mode mode, const double* out_adjoint,
                           int64_t adj_exp2, void* const* leaf_grads, void* stream) {
    return tn_contract_grad_ex(net, tree_pairs, n_sliced, sliced_labels, mode, out_adjoint, TN_MEM_HOST,
                               adj_exp2, nullptr, leaf_grads, 0u, 0, 0, stream);
}

tn_status tn_contract_noalloc(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                              const int64_t* sliced_labels, void* out, int32_t out_mem,
                              int64_t* out_exp2, void* stream) {
    if (!net) return fail(TN_EINVAL, "tn_contract_noalloc: net is NULL");
    if (!out || !out_exp2) return fail(TN_EINVAL, "tn_contract_noalloc: NULL output");
    if (out_mem != TN_MEM_DEVICE && out_mem != TN_MEM_HOST) return fail(TN_EINVAL, "bad out_mem");
    for (int v = 0; v < net->d.n; ++v)
        if (!net->d.leaves[v].ptr) return fail(TN_EINVAL, "tn_contract_noalloc: tensor without data");
    Plan* p = nullptr;  // host-side plan only: no device state is created
    tn_status st = get_plan(net, tree_pairs, n_sliced, sliced_labels, TN_MODE_FP32, &p);
    if (st != TN_OK) return st;
    std::string err;
    st = tn::run_noalloc(net->d, *p, out, out_mem, out_exp2, (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

tn_status tn_plan_info(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                       const int64_t* sliced_labels, tn_mode mode, double out[8]) {
    if (!net || !out) return fail(TN_EINVAL, "tn_plan_info: NULL argument");
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, n_sliced, sliced_labels, mode, &p);
    if (st != TN_OK) return st;
    tn::plan_info(net->d, *p, out);
    return TN_OK;
}

tn_status tn_selftest_flow_timeout(void* stream) {
    // one dataflow item (a one-output node) whose child counter nothing
    // raises: every index below stays inside these small buffers
    cudaStream_t s = (cudaStream_t)stream;
    char* buf = nullptr;
    const size_t kBytes = 4096;
    TN_CUDA(cudaMalloc(&buf, kBytes));
    tn::Control* ctl = reinterpret_cast<tn::Control*>(buf);
    float* A = reinterpret_cast<float*>(buf + 256);
    float* B = A + 16;
    float* C = A + 32;
    unsigned* max_c = reinterpret_cast<unsigned*>(buf + 512);
    int64_t* exp_c = reinterpret_cast<int64_t*>(buf + 520);
    unsigned* done = reinterpret_cast<unsigned*>(buf + 576);  // done[0..3]
    unsigned* head = reinterpret_cast<unsigned*>(buf + 640);
    int4* deps = reinterpret_cast<int4*>(buf + 704);          // one entry
    tn::WaveItem* item = reinterpret_cast<tn::WaveItem*>(buf + 768);
    tn::TileArgs* desc = reinterpret_cast<tn::TileArgs*>(buf + 1024);
    if (sizeof(tn::TileArgs) > kBytes - 1024) {
        cudaFree(buf);
        return fail(TN_EINVAL, "selftest: descriptor larger than its buffer");
    }
    tn::Control hc{};
    hc.slice = 0;
    hc.slice_begin = 0;
    hc.slice_end = 1;
    tn::TileArgs t;
    std::memset(&t, 0, sizeof(t));
    t.A = A;
    t.B = B;
    t.C = C;
    t.nbatch = 1;
    t.cfg = tn::kTile64x64;
    t.split = 1;
    t.kchunk = 1;
    t.ctl = ctl;
    t.sc.max_c = max_c;
    t.sc.exp_c = exp_c;
    t.a_leaf = -1;
    t.b_leaf = -1;
    const int4 dep = make_int4(1, 1, -1, 0);  // waits for one chunk of node 1: not in the launch
    tn::WaveItem it{0, 0, 0, 1};
    cudaError_t e = cudaMemsetAsync(buf, 0, kBytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(desc, &t, sizeof(t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(deps, &dep, sizeof(dep), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(item, &it, sizeof(it), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = tn::launch_wave(item, 1, desc, nullptr, false, s, deps, done, head, 1);
    int32_t status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&status, &ctl->status, sizeof(status), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(TN_ECUDA, std::string("selftest: ") + cudaGetErrorString(e));
    if (status != TN_OK) return fail((tn_status)status, "selftest: a bounded dataflow wait gave up (as intended)");
    return TN_OK;
}

tn_status tn_plan_steps(tn_net* net, const int32_t* tree_pairs, int32_t n_sliced,
                        const int64_t* sliced_labels, tn_mode mode, int32_t cap, int32_t* n_steps,
                        int32_t* step_info, int32_t* step_nodes) {
    if (!net || !n_steps) return fail(TN_EINVAL, "tn_plan_steps: NULL argument");
    Plan* p = nullptr;
    tn_status st = get_plan(net, tree_pairs, n_sliced, sliced_labels, mode, &p);
    if (st != TN_OK) return st;
    *n_steps = (int32_t)p->steps.size();
    if (cap < *n_steps || !step_info) return TN_OK;
    int pos = 0;
    for (size_t s = 0; s < p->steps.size(); ++s) {
        const tn::Step& stp = p->steps[s];
        const tn::Node& first = p->nodes[stp.nodes[0]];
        step_info[5 * s + 0] = stp.wave;
        step_info[5 * s + 1] = first.kind;
        step_info[5 * s + 2] = stp.wave ? 0 : (first.kind == tn::kTiled ? first.tile.cfg : 0);
        step_info[5 * s + 3] = (int32_t)stp.nodes.size();
        // a split-K tiled node adds its fixed-order reduction launch
        step_info[5 * s + 4] = stp.wave ? 1
                               : first.kind == tn::kTensorCore ? tn::tc_launches(first.tile)
                               : 1 + (first.kind == tn::kTiled && first.tile.split > 1 ? 1 : 0);
        if (step_nodes)
            for (int k : stp.nodes) step_nodes[pos++] = k;
    }
    return TN_OK;
}

struct tn_batch {
    tn::BatchPlan b;
};

static tn_status batch_create(tn_batch** out, int32_t n_nets, tn_net* const* nets,
                              const int32_t* const* tree_pairs, const int32_t* n_sliced,
                              const int64_t* const* sliced_labels, tn_mode mode) {
    if (!out || n_nets < 1 || !nets || !tree_pairs) return fail(TN_EINVAL, "tn_batch_create: bad arguments");
    *out = nullptr;
    std::unique_ptr<tn_batch> b(new (std::nothrow) tn_batch);
    if (!b) return fail(TN_ENOMEM, "out of host memory");
    b->b.mode = mode;
    for (int i = 0; i < n_nets; ++i) {
        if (!nets[i]) return fail(TN_EINVAL, "tn_batch_create: NULL network");
        const int32_t ns = n_sliced ? n_sliced[i] : 0;
        if (ns < 0 || (ns > 0 && (!sliced_labels || !sliced_labels[i])))
            return fail(TN_EINVAL, "tn_batch_create_sliced: bad sliced labels");
        Plan* p = nullptr;
        tn_status st = get_plan(nets[i], tree_pairs[i], ns, ns ? sliced_labels[i] : nullptr, mode, &p);
        if (st != TN_OK) return st;
        b->b.nets.push_back(&nets[i]->d);
        b->b.plans.push_back(p);
        if (p->d_sliced > 1) {
            // device state for G slices side by side: as many as fit a 2 GiB
            // workspace budget, at most 8
            const int64_t ws = p->ws_elems * (int64_t)nets[i]->d.elem_bytes() + p->split_bytes;
            int G = 1;
            while (G < 8 && 2 * (int64_t)G <= p->d_sliced && 2 * (int64_t)G * ws <= (int64_t(2) << 30)) G *= 2;
            st = ensure_instances(nets[i], p, G, nullptr);
            if (st != TN_OK) return st;
            tn::SlicedMember m;
            m.index = i;
            m.d = &nets[i]->d;
            m.p = p;
            m.unit = nets[i]->unit;
            m.G = G;
            b->b.sliced.push_back(m);
        }
    }
    std::string err;
    tn_status st = tn::build_batch(b->b, err);
    if (st == TN_OK) st = tn::alloc_batch(b->b, err);
    if (st != TN_OK) {
        tn::free_batch(b->b);
        return fail(st, err);
    }
    *out = b.release();
    return TN_OK;
}

tn_status tn_batch_create(tn_batch** out, int32_t n_nets, tn_net* const* nets,
                          const int32_t* const* tree_pairs, tn_mode mode) {
    return batch_create(out, n_nets, nets, tree_pairs, nullptr, nullptr, mode);
}

tn_status tn_batch_create_sliced(tn_batch** out, int32_t n_nets, tn_net* const* nets,
                                 const int32_t* const* tree_pairs, const int32_t* n_sliced,
                                 const int64_t* const* sliced_labels, tn_mode mode) {
    if (!n_sliced) return fail(TN_EINVAL, "tn_batch_create_sliced: n_sliced is NULL");
    return batch_create(out, n_nets, nets, tree_pairs, n_sliced, sliced_labels, mode);
}

tn_status tn_batch_contract(tn_batch* batch, double* out, int64_t* out_exp2, uint64_t* latency_ns,
                            int32_t out_mem, void* stream) {
    if (!batch || !out || !out_exp2) return fail(TN_EINVAL, "tn_batch_contract: NULL argument");
    if (out_mem != TN_MEM_DEVICE && out_mem != TN_MEM_HOST) return fail(TN_EINVAL, "bad out_mem");
    std::string err;
    tn_status st = tn::run_batch(batch->b, out, out_exp2, latency_ns, out_mem, (cudaStream_t)stream, err);
    if (st != TN_OK) return fail(st, err);
    return TN_OK;
}

void tn_batch_destroy(tn_batch* batch) {
    if (!batch) return;
    cudaDeviceSynchronize();
    tn::free_batch(batch->b);
    delete batch;
}

void tn_destroy(tn_net* net) {
    if (!net) return;
    cudaDeviceSynchronize();
    for (auto& p : net->plans) tn::free_device(*p);
    for (auto& lf : net->d.leaves)
        if (lf.staged) cudaFree(lf.staged);
    tn::NetDesc& d = net->d;
    if (d.stage_host) cudaFreeHost(d.stage_host);
    if (d.stage_dev) cudaFree(d.stage_dev);
    if (d.stage_done) cudaEventDestroy(d.stage_done);
    if (net->unit) cudaFree(net->unit);
    delete net;
}

}  // extern "C"
