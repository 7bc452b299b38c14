// tn_grad.cpp -- reverse-mode derivative of a contraction with respect to
// every leaf (tn_contract_grad).
//
// The forward value is a composition of pairwise contractions C = A * B
// (Sec. 2 of arXiv 2002.01935).  Each is bilinear, so with the adjoint Cbar
// of C the adjoints of its operands are again pairwise contractions:
//   Abar[a] = sum over the labels of (C u B) not in A of Cbar[c] conj(B[b]),
// and Bbar likewise (holomorphic derivative, conjugated as torch.autograd
// expects).  Per slice the forward intermediates are recomputed and all kept
// (no workspace reuse), then the tree is swept from the root to the
// leaves; leaf adjoints are added into gradient accumulators at the slice's
// offset, so the result is summed over slices.  A leaf label that
// occurs in that tensor only (summed at its first contraction) gives an
// adjoint constant along it: the gather broadcasts.  Renormalisation
// exponents are tracked exactly as in the forward pass.
//
// Launch structure.  The forward recompute and the sweep form one list of
// nodes (forward nodes, then adjoint nodes root to leaves) scheduled like
// the forward pass: by dependency level, the small nodes of consecutive
// levels as one dataflow wave launch, the others one launch each; every
// adjoint node comes after every forward node, so the per-slice sequence
// is two CUDA graphs (forward, sweep).  Both read the leaves from a
// library-owned image (refreshed by one gather launch per call) and the
// sweep adds the leaf adjoints into library-owned accumulators (copied, or
// added, to the caller's buffers by one launch at the end), so neither
// graph holds a per-call pointer: they are captured once and replayed by
// every later call.  n copies of the network (shared or per-copy leaves)
// run in every launch; a caller that ran the forward of those copies in
// this state (run_grad_forward) can run the sweep alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tn_plan.h"

namespace tn {

struct GradState {
    Plan g;                      // vertex table: forward vertices then adjoints
    int NV = 0;                  // forward vertices (leaves and nodes)
    std::vector<Node> fwd;       // forward nodes (own workspace regions)
    std::vector<Node> bwd;       // adjoint nodes in execution order
    std::vector<int> bwd_target; // forward vertex whose adjoint each computes
    std::vector<int> fwd_order;  // forward nodes in launch order
    std::vector<int64_t> adj_off;  // workspace offset of each vertex's adjoint
    int64_t ws_elems = 0;
    int64_t split_bytes = 0;
    int n_slots = 0;
    // schedule over the combined node list: forward node k is k, adjoint
    // node j is nn + j (Step.node / Step.nodes / WaveItem.node use these)
    std::vector<Step> steps;
    std::vector<WaveItem> items;
    std::vector<int> flow_deps;  // per combined node: child a, chunks, child b, chunks
    bool any_flow = false;
    // gradient accumulators (floats): leaf v at acc_off[v], one such block
    // of acc_floats per instance
    std::vector<int64_t> acc_off;
    int64_t acc_floats = 0;
    int64_t max_leaf_floats = 0;
    int64_t max_grad_n = 0;
    // instance layout of the device state (n_inst = 0: not allocated).
    // Leaves either are shared by all instances or have one copy each
    // (varying); the leaf image holds leaf v at img_off[v], its instance
    // copies img_is[v] floats apart (0: shared).
    int n_inst = 0;
    std::vector<char> varying;
    std::vector<int64_t> img_off, img_is;
    int64_t img_floats = 0;
    std::vector<int> inst_item_begin;  // per step: first item of the instance-replicated list
    int plan_inst = 1;                 // copies the node kernels and K splits were planned for
    int n_fwd_steps = 0;               // steps [0, n_fwd_steps) hold the forward nodes
    bool kept = false;                 // the workspace holds the forward of the last keep call
    BatchRoot* roots_dev = nullptr;    // per copy: root value and its scale slots
    double* val_dev = nullptr;         // per copy: FP64 value (2 doubles) ...
    int64_t* val_exp_dev = nullptr;    // ... and exponent, for host outputs
    std::vector<int> level;            // dependency level of each combined node
    // device
    void* ws = nullptr;
    void* split_buf = nullptr;
    unsigned* maxabs = nullptr;
    int64_t* exps = nullptr;
    Control* ctl = nullptr;
    unsigned* leafmax = nullptr;
    float* leaf_img = nullptr;
    float* gacc = nullptr;
    const float** img_ptr_dev = nullptr;   // leaf image pointers (fixed)
    int64_t* leaf_nfloat_dev = nullptr;
    TileArgs* descs_dev = nullptr;
    WaveItem* items_dev = nullptr;
    int* flow_deps_dev = nullptr;
    unsigned* flow_cnt_dev = nullptr;      // done[combined node], then one head per step
    LeafGradArgs* lg_dev = nullptr;        // one entry per leaf
    CopyEntry* copy_dev = nullptr;         // per call: gather entries, then scatter entries
    double* adj_dev = nullptr;             // host adjoints are staged here
    int64_t* perm_dev = nullptr;           // root offset of each output
    std::vector<GenericArgs> gen_f, gen_b;
    std::vector<TileArgs> tile_f, tile_b;
    // the per-slice sequence as two captured graphs (built on the first
    // call): the forward steps, then the sweep
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph_f = nullptr, graph_b = nullptr;
    cudaGraphExec_t gexec_f = nullptr, gexec_b = nullptr;
};

static bool has_label(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

static tn_status build_grad(const NetDesc& d, const Plan& f, GradState& G, int copies, std::string& err) {
    const int n = d.n;
    const int nn = (int)f.nodes.size();
    G.g = Plan();
    G.g.mode = f.mode;
    G.g.copies = copies;
    G.plan_inst = copies;
    G.g.vlab = f.vlab;
    G.g.vstride = f.vstride;
    G.g.leaf_sl = f.leaf_sl;
    G.g.sliced = f.sliced;
    G.g.d_sliced = f.d_sliced;
    G.NV = (int)f.vlab.size();
    const int NV = G.NV;
    G.g.vlab.resize(2 * NV);
    G.g.vstride.resize(2 * NV);
    // forward nodes: every intermediate kept (offsets without reuse)
    int64_t off = 0;
    auto take = [&](int64_t sz) {
        int64_t o = off;
        off += (sz + 63) / 64 * 64;
        return o;
    };
    G.fwd = f.nodes;
    if (copies > 1) {
        // many copies per launch: the single-copy kernel choices (autotuned,
        // K splits sized for one copy) give way to the planner's rule with
        // the copies counted
        int64_t se = 0;
        for (Node& nd : G.fwd) {
            nd.kind = kGeneric;
            if (f.force_generic || !plan_tile_node(d, G.g, nd, se)) continue;
            if (!f.no_tensor_cores) make_tensor_core(d, f.mode, nd, se, copies);
        }
    }
    G.fwd_order.clear();
    for (const Step& st : f.steps)
        for (int k : st.nodes) G.fwd_order.push_back(k);
    for (auto& nd : G.fwd) nd.ws_off = take(nd.size);
    // adjoint of the root: the root's own layout
    const int root_v = n + nn - 1;
    G.adj_off.assign(NV, -1);
    G.g.vlab[NV + root_v] = f.vlab[root_v];
    G.g.vstride[NV + root_v] = f.vstride[root_v];
    G.adj_off[root_v] = take(f.nodes.back().size);
    // adjoint nodes, root to leaves
    G.bwd.clear();
    G.bwd_target.clear();
    int64_t split_elems = 0;
    for (int k = nn - 1; k >= 0; --k) {
        const Node& C = f.nodes[k];
        const int cv = n + k;
        for (int side = 0; side < 2; ++side) {
            const int child = side == 0 ? C.ca : C.cb;
            const int other = side == 0 ? C.cb : C.ca;
            if (child < 0) continue;
            std::vector<int> keep;
            const std::vector<int>& lc = G.g.vlab[NV + cv];
            static const std::vector<int> none;
            const std::vector<int>& lo = other >= 0 ? f.vlab[other] : none;
            for (int l : f.vlab[child])
                if (has_label(lc, l) || has_label(lo, l)) keep.push_back(l);
            Node nd = build_node(d, G.g, NV + child, NV + cv, other, keep);
            // the forward operand is read conjugated
            if (d.is_complex()) {
                nd.tile.conj_a = nd.ca == other && other >= 0;
                nd.tile.conj_b = nd.cb == other && other >= 0;
            }
            G.g.vlab[NV + child] = nd.lab;
            G.g.vstride[NV + child] = nd.stride;
            nd.kind = kGeneric;
            const int ca0 = nd.tile.conj_a, cb0 = nd.tile.conj_b;
            if (plan_tile_node(d, G.g, nd, split_elems) && !f.no_tensor_cores)
                make_tensor_core(d, f.mode, nd, split_elems, copies);
            nd.tile.conj_a = ca0;
            nd.tile.conj_b = cb0;
            nd.ws_off = take(nd.size);
            G.adj_off[child] = nd.ws_off;
            G.bwd.push_back(nd);
            G.bwd_target.push_back(child);
        }
    }
    // forward split-K buffers count too
    for (const auto& nd : G.fwd) {
        if (nd.kind == kTiled && nd.tile.split > 1)
            split_elems = std::max(split_elems, (int64_t)nd.tile.split * nd.tile.nbatch *
                                                    (int64_t(1) << (nd.tile.nm + nd.tile.nn)));
        if (nd.kind == kTensorCore) {
            const int prec = tc_prec_of_mode(f.mode);
            const int64_t eb = d.elem_bytes();
            split_elems = std::max(split_elems, (tc_geom(nd.tile, d.is_complex(), prec).total + eb - 1) / eb);
        }
    }
    G.split_bytes = (split_elems * (int64_t)d.elem_bytes() + 1023) / 1024 * 1024;
    G.ws_elems = std::max<int64_t>(off, 64);
    // scale slots: forward node k -> k; adjoint of vertex v -> nn + v (root last)
    G.n_slots = nn + NV;
    // ---- schedule of the combined list (forward nodes, then adjoints)
    const int nb = (int)G.bwd.size();
    const int ncomb = nn + nb;
    std::vector<int> adj_prod(NV, -1);  // adjoint node of each vertex
    for (int j = 0; j < nb; ++j) adj_prod[G.bwd_target[j]] = nn + j;
    auto producer = [&](int v) -> int {  // combined node that writes vertex v, -1 if none
        if (v < n) return -1;            // unit, leaf
        if (v < NV) return v - n;        // forward node
        return adj_prod[v - NV];         // adjoint (-1: the root's, set per call)
    };
    auto cnode = [&](int c) -> const Node& { return c < nn ? G.fwd[c] : G.bwd[c - nn]; };
    std::vector<int> order(G.fwd_order);
    for (int j = 0; j < nb; ++j) order.push_back(nn + j);
    // levels: the adjoint nodes come after every forward node (the forward
    // steps form one graph, the sweep another: a caller that just ran the
    // forward keeps its intermediates and runs the sweep alone)
    std::vector<int> level(ncomb, 0);
    int max_level = 0, fwd_levels = 0;
    for (int c : order) {
        const Node& nd = cnode(c);
        int l = c < nn ? 0 : fwd_levels;
        for (int v : {nd.ca, nd.cb}) {
            const int pr = producer(v);
            if (pr >= 0) l = std::max(l, level[pr]);
        }
        level[c] = l + 1;
        max_level = std::max(max_level, level[c]);
        if (c < nn) fwd_levels = max_level;
    }
    G.level = level;
    std::vector<std::vector<int>> at(max_level + 1);
    for (int c : order) at[level[c]].push_back(c);
    G.steps.clear();
    G.items.clear();
    for (int L = 1; L <= max_level; ++L) {
        Step w;
        w.wave = 1;
        w.item_begin = (int)G.items.size();
        std::vector<int> singles;
        for (int c : at[L]) {
            const Node& nd = cnode(c);
            const bool small = wave_node(nd, G.plan_inst) && !f.no_waves;
            if (!small) {
                singles.push_back(c);
                continue;
            }
            const int64_t chunk = wave_chunk(nd, G.plan_inst);
            for (int64_t o = 0; o < nd.size; o += chunk) {
                WaveItem it;
                it.node = c;
                it.pad = 0;
                it.o_begin = o;
                it.o_count = chunk;
                G.items.push_back(it);
            }
            w.nodes.push_back(c);
        }
        w.item_count = (int)G.items.size() - w.item_begin;
        if (w.item_count > 0) G.steps.push_back(w);
        for (int c : singles) {
            Step s;
            s.node = c;
            s.nodes.push_back(c);
            G.steps.push_back(s);
        }
    }
    if (!f.no_flow) {  // consecutive waves: one dataflow launch
        std::vector<Step> merged;
        for (Step& st : G.steps) {
            if (st.wave && !merged.empty() && merged.back().wave &&
                merged.back().item_begin + merged.back().item_count == st.item_begin &&
                (merged.back().nodes[0] < nn) == (st.nodes[0] < nn)) {  // same phase
                Step& m = merged.back();
                m.item_count += st.item_count;
                m.nodes.insert(m.nodes.end(), st.nodes.begin(), st.nodes.end());
                m.flow = 1;
            } else {
                merged.push_back(st);
            }
        }
        G.steps = merged;
    }
    G.n_fwd_steps = 0;
    while (G.n_fwd_steps < (int)G.steps.size() && G.steps[G.n_fwd_steps].nodes[0] < nn) ++G.n_fwd_steps;
    G.flow_deps.assign(4 * (size_t)std::max(ncomb, 1), -1);
    G.any_flow = false;
    for (const Step& st : G.steps) {
        if (!st.flow) continue;
        G.any_flow = true;
        std::vector<char> in_step(ncomb, 0);
        for (int c : st.nodes) in_step[c] = 1;
        for (int c : st.nodes) {
            const Node& nd = cnode(c);
            int slot = 0;
            for (int v : {nd.ca, nd.cb}) {
                const int pr = producer(v);
                if (pr >= 0 && in_step[pr]) {
                    const Node& ch = cnode(pr);
                    const int64_t chunk = wave_chunk(ch, G.plan_inst);
                    G.flow_deps[4 * c + 2 * slot] = pr;
                    G.flow_deps[4 * c + 2 * slot + 1] = (int)((ch.size + chunk - 1) / chunk);
                }
                ++slot;
            }
        }
    }
    // ---- gradient accumulator layout
    G.acc_off.assign(n, 0);
    G.acc_floats = 0;
    G.max_leaf_floats = 0;
    for (int v = 0; v < n; ++v) {
        const int64_t nf = d.leaves[v].size * (d.is_complex() ? 2 : 1);
        G.acc_off[v] = G.acc_floats;
        G.acc_floats += (nf + 63) / 64 * 64;  // 256-byte aligned leaves
        G.max_leaf_floats = std::max(G.max_leaf_floats, nf);
    }
    (void)err;
    return TN_OK;
}

// Device state of the sweep for n_inst instances whose leaves are shared or
// varying (one copy per instance).  Everything holds one region per
// instance: workspace, packed-operand / split buffer, scale slots, gradient
// accumulators, dataflow counters; the node arguments carry the instance
// strides (InstanceInfo) and wave items are replicated per instance.
static tn_status alloc_grad(const NetDesc& d, const Plan& f, GradState& G, void* unit, int n_inst,
                            const std::vector<char>& varying, std::string& err) {
    const size_t eb = d.elem_bytes();
    const int n = d.n;
    const int nn = (int)G.fwd.size();
    const int nb = (int)G.bwd.size();
    const int NV = G.NV;
    const bool cplx = d.is_complex();
    const int cf = cplx ? 2 : 1;
    const int64_t NI = n_inst;
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess) {
            err = std::string(what) + ": " + cudaGetErrorString(e);
            return false;
        }
        return true;
    };
#define AL(ptr, bytes, what) \
    if (!ck(cudaMalloc((void**)&(ptr), (size_t)(bytes)), what)) return TN_ENOMEM
#define UP(dst, src, bytes) \
    if (!ck(cudaMemcpy((void*)(dst), (const void*)(src), (size_t)(bytes), cudaMemcpyHostToDevice), "cudaMemcpy")) \
        return TN_ECUDA
    G.n_inst = n_inst;
    G.varying = varying;
    // leaf image layout
    G.img_off.assign(n, 0);
    G.img_is.assign(n, 0);
    G.img_floats = 0;
    for (int v = 0; v < n; ++v) {
        const int64_t pad = (d.leaves[v].size * cf + 63) / 64 * 64;
        G.img_off[v] = G.img_floats;
        G.img_is[v] = varying[v] ? pad : 0;
        G.img_floats += varying[v] ? pad * NI : pad;
    }
    AL(G.ws, (size_t)G.ws_elems * eb * NI, "gradient workspace");
    if (G.split_bytes) AL(G.split_buf, G.split_bytes * NI, "cudaMalloc");
    AL(G.maxabs, sizeof(unsigned) * G.n_slots * NI, "cudaMalloc");
    AL(G.exps, sizeof(int64_t) * G.n_slots * NI, "cudaMalloc");
    AL(G.ctl, sizeof(Control), "cudaMalloc");
    AL(G.leafmax, sizeof(unsigned) * n, "cudaMalloc");
    AL(G.leaf_img, sizeof(float) * std::max<int64_t>(G.img_floats, 64), "leaf image");
    AL(G.gacc, sizeof(float) * std::max<int64_t>(G.acc_floats * NI, 64), "gradient accumulators");
    AL(G.img_ptr_dev, sizeof(void*) * n, "cudaMalloc");
    AL(G.leaf_nfloat_dev, sizeof(int64_t) * n, "cudaMalloc");
    AL(G.lg_dev, sizeof(LeafGradArgs) * n, "cudaMalloc");
    AL(G.copy_dev, sizeof(CopyEntry) * 2 * n * NI, "cudaMalloc");
    const int64_t n_out = f.n_out;
    AL(G.adj_dev, sizeof(double) * n_out * cf * NI, "cudaMalloc");
    AL(G.perm_dev, sizeof(int64_t) * n_out, "cudaMalloc");
    const int ncomb = nn + nb;
    AL(G.flow_deps_dev, sizeof(int) * G.flow_deps.size(), "cudaMalloc");
    AL(G.flow_cnt_dev, sizeof(unsigned) * ((size_t)ncomb * NI + G.steps.size() + 1), "cudaMalloc");
    UP(G.flow_deps_dev, G.flow_deps.data(), sizeof(int) * G.flow_deps.size());
    // the padding between image entries stays zero (leaf maxima read it)
    if (!ck(cudaMemset(G.leaf_img, 0, sizeof(float) * std::max<int64_t>(G.img_floats, 64)), "cudaMemset"))
        return TN_ECUDA;
    {
        std::vector<const float*> ip(n);
        std::vector<int64_t> nf(n);
        for (int v = 0; v < n; ++v) {
            ip[v] = G.leaf_img + G.img_off[v];
            const int64_t one = d.leaves[v].size * cf;
            nf[v] = varying[v] ? G.img_is[v] * (NI - 1) + one : one;  // all copies
        }
        UP(G.img_ptr_dev, ip.data(), sizeof(void*) * n);
        UP(G.leaf_nfloat_dev, nf.data(), sizeof(int64_t) * n);
    }
    char* ws = (char*)G.ws;
    auto fwd_ptr = [&](int v) -> const void* {
        if (v < 0) return unit;
        if (v < n) return G.leaf_img + G.img_off[v];
        return ws + G.fwd[v - n].ws_off * eb;
    };
    auto slot_max = [&](int v) -> const unsigned* {
        if (v < 0) return nullptr;
        if (v < n) return G.leafmax + v;
        if (v < NV) return G.maxabs + (v - n);
        return G.maxabs + nn + (v - NV);
    };
    auto slot_exp = [&](int v) -> const int64_t* {
        if (v < n) return nullptr;
        if (v < NV) return G.exps + (v - n);
        return G.exps + nn + (v - NV);
    };
    // instance strides of an operand vertex (elements, slots)
    auto op_is = [&](int v, int64_t& is, int32_t& sis) {
        if (v < 0) {
            is = 0;
            sis = 0;
        } else if (v < n) {
            is = G.img_is[v] / cf;
            sis = 0;  // leaf maxima are over all copies
        } else {
            is = G.ws_elems;
            sis = G.n_slots;
        }
    };
    auto wire = [&](Node& nd, GenericArgs& g, TileArgs& t, const void* A, const void* B, void* C,
                    unsigned* max_c, int64_t* exp_c) -> tn_status {
        tn_status st = make_generic_args_node(d, G.g, nd, g, err);
        if (st != TN_OK) return st;
        g.A = A;
        g.B = B;
        g.C = C;
        g.ctl = G.ctl;
        g.sc.max_a = slot_max(nd.ca);
        g.sc.exp_a = slot_exp(nd.ca);
        g.sc.max_b = slot_max(nd.cb);
        g.sc.exp_b = slot_exp(nd.cb);
        g.sc.max_c = max_c;
        g.sc.exp_c = exp_c;
        g.conj_a = nd.tile.conj_a;
        g.conj_b = nd.tile.conj_b;
        InstanceInfo in;
        memset(&in, 0, sizeof(in));
        in.n_inst = n_inst;
        in.slice_step = 0;  // every instance works on the current slice
        in.c_is = G.ws_elems;
        in.sc_is = G.n_slots;
        in.p_is = G.split_bytes / (int64_t)eb;
        op_is(nd.ca, in.a_is, in.sa_is);
        op_is(nd.cb, in.b_is, in.sb_is);
        g.in = in;
        t = nd.tile;
        t.in = in;
        t.A = A;
        t.B = B;
        t.C = C;
        t.P = G.split_buf;
        t.sla = g.sla;
        t.slb = g.slb;
        t.ctl = G.ctl;
        t.sc = g.sc;
        // grid z = batch x K splits x instances is at most 65535
        if (nd.kind == kTiled || nd.kind == kTensorCore) {
            if (t.nbatch * NI > 65535) {
                err = "tn_contract_grad: too many instances for a node with " + std::to_string(t.nbatch) +
                      " batch entries";
                return TN_EUNSUPPORTED;
            }
            if (t.split > 1 && t.nbatch * (int64_t)t.split * NI > 65535) {
                if (nd.kind == kTensorCore) {
                    err = "tn_contract_grad: too many instances for a K-split tensor-core node";
                    return TN_EUNSUPPORTED;
                }
                int split = t.split;
                while (split > 1 && t.nbatch * (int64_t)split * NI > 65535) split /= 2;
                const int64_t K = int64_t(1) << t.nk;
                const int64_t gran = t.cfg == kTileDot ? 256 : (t.cfg == kTile4x1024 ? 4 : 16);
                const int64_t units = (K + gran - 1) / gran;
                t.split = split;
                t.kchunk = ((units + split - 1) / split) * gran;
            }
        } else if (NI > 65535) {
            err = "tn_contract_grad: too many instances";
            return TN_EUNSUPPORTED;
        }
        return TN_OK;
    };
    G.gen_f.assign(nn, GenericArgs{});
    G.tile_f.assign(nn, TileArgs{});
    for (int k = 0; k < nn; ++k) {
        Node& nd = G.fwd[k];
        tn_status st = wire(nd, G.gen_f[k], G.tile_f[k], fwd_ptr(nd.ca), fwd_ptr(nd.cb),
                            ws + nd.ws_off * eb, G.maxabs + k, G.exps + k);
        if (st != TN_OK) return st;
    }
    G.gen_b.assign(nb, GenericArgs{});
    G.tile_b.assign(nb, TileArgs{});
    for (int j = 0; j < nb; ++j) {
        Node& nd = G.bwd[j];
        auto operand = [&](int v) -> const void* {
            if (v >= NV) return ws + G.adj_off[v - NV] * eb;
            return fwd_ptr(v);
        };
        const int target = G.bwd_target[j];
        tn_status st = wire(nd, G.gen_b[j], G.tile_b[j], operand(nd.ca), operand(nd.cb),
                            ws + nd.ws_off * eb, G.maxabs + nn + target, G.exps + nn + target);
        if (st != TN_OK) return st;
    }
    G.inst_item_begin.assign(G.steps.size(), 0);
    if (!G.items.empty()) {
        std::vector<TileArgs> descs(ncomb);
        for (int k = 0; k < nn; ++k) descs[k] = G.tile_f[k];
        for (int j = 0; j < nb; ++j) descs[nn + j] = G.tile_b[j];
        // within each step: level by level, every copy's items of a level
        // before the next level, so that the copies' dependency chains
        // advance together (a node's children always come earlier)
        std::vector<WaveItem> items;
        items.reserve(G.items.size() * NI);
        for (size_t s = 0; s < G.steps.size(); ++s) {
            const Step& st = G.steps[s];
            G.inst_item_begin[s] = (int)items.size();
            if (!st.wave) continue;
            int j0 = 0;
            while (j0 < st.item_count) {
                const int L = G.level[G.items[st.item_begin + j0].node];
                int j1 = j0;
                while (j1 < st.item_count && G.level[G.items[st.item_begin + j1].node] == L) ++j1;
                for (int i = 0; i < n_inst; ++i)
                    for (int j = j0; j < j1; ++j) {
                        WaveItem it = G.items[st.item_begin + j];
                        it.pad = i;
                        items.push_back(it);
                    }
                j0 = j1;
            }
        }
        AL(G.descs_dev, sizeof(TileArgs) * ncomb, "cudaMalloc");
        AL(G.items_dev, sizeof(WaveItem) * std::max<size_t>(items.size(), 1), "cudaMalloc");
        UP(G.descs_dev, descs.data(), sizeof(TileArgs) * ncomb);
        UP(G.items_dev, items.data(), sizeof(WaveItem) * items.size());
    }
    // leaf gathers: adjoint of leaf v -> its accumulator
    std::vector<LeafGradArgs> lg(n);
    G.max_grad_n = 0;
    for (int v = 0; v < n; ++v) {
        LeafGradArgs& a = lg[v];
        memset(&a, 0, sizeof(a));
        const LeafDesc& lf = d.leaves[v];
        a.grad = G.gacc + G.acc_off[v];
        a.grad_is = G.acc_floats / cf;
        a.adj = ws + G.adj_off[v] * eb;
        a.adj_is = G.ws_elems;
        a.exp_adj = G.exps + nn + v;
        a.exp_is = G.n_slots;
        a.ctl = G.ctl;
        a.sl = f.leaf_sl[v];
        const std::vector<int>& al = G.g.vlab[NV + v];
        const std::vector<int64_t>& as = G.g.vstride[NV + v];
        a.n = 1;
        int nd_ = 0;
        for (int i = (int)lf.lab.size() - 1; i >= 0; --i) {
            const int l = lf.lab[i];
            if (std::find(f.sliced.begin(), f.sliced.end(), l) != f.sliced.end()) continue;
            if (nd_ >= kMaxDigits) {
                err = "leaf rank exceeds the gradient gather limit";
                return TN_EUNSUPPORTED;
            }
            a.dim[nd_] = (int32_t)d.dims[l];
            a.gstride[nd_] = lf.stride[i];
            int64_t s = 0;
            for (size_t j = 0; j < al.size(); ++j)
                if (al[j] == l) s = as[j];
            a.astride[nd_] = s;
            a.n *= d.dims[l];
            ++nd_;
        }
        a.n_d = nd_;
        G.max_grad_n = std::max(G.max_grad_n, a.n);
    }
    UP(G.lg_dev, lg.data(), sizeof(LeafGradArgs) * n);
    // root layout of each output (open labels in tn_create order, last fastest)
    {
        const Node& root = G.fwd.back();
        std::vector<int64_t> perm(n_out);
        for (int64_t o = 0; o < n_out; ++o) {
            int64_t rem = o, dst = 0;
            for (int i = (int)d.open.size() - 1; i >= 0; --i) {
                const int l = d.open[i];
                const int64_t v = rem % d.dims[l];
                rem /= d.dims[l];
                for (size_t j = 0; j < root.lab.size(); ++j)
                    if (root.lab[j] == l) dst += v * root.stride[j];
            }
            perm[o] = dst;
        }
        UP(G.perm_dev, perm.data(), sizeof(int64_t) * n_out);
    }
    // root value of every copy (scalar networks), for the keeping forward
    if (n_out == 1) {
        const Node& root = G.fwd.back();
        std::vector<BatchRoot> roots(n_inst);
        for (int i = 0; i < n_inst; ++i) {
            roots[i].root = ws + (root.ws_off + (int64_t)i * G.ws_elems) * eb;
            roots[i].exp = G.exps + (nn - 1) + (int64_t)i * G.n_slots;
            roots[i].max = G.maxabs + (nn - 1) + (int64_t)i * G.n_slots;
            roots[i].is_c = cplx ? 1 : 0;
            roots[i].pad = 0;
        }
        AL(G.roots_dev, sizeof(BatchRoot) * n_inst, "cudaMalloc");
        AL(G.val_dev, sizeof(double) * 2 * n_inst, "cudaMalloc");
        AL(G.val_exp_dev, sizeof(int64_t) * n_inst, "cudaMalloc");
        UP(G.roots_dev, roots.data(), sizeof(BatchRoot) * n_inst);
    }
#undef AL
#undef UP
    return TN_OK;
}

// Releases the device state (the host plan of the sweep stays).
static void free_grad_device(GradState& G) {
    for (void* q : {(void*)G.ws, G.split_buf, (void*)G.maxabs, (void*)G.exps, (void*)G.ctl,
                    (void*)G.leafmax, (void*)G.leaf_img, (void*)G.gacc, (void*)G.img_ptr_dev,
                    (void*)G.leaf_nfloat_dev, (void*)G.descs_dev, (void*)G.items_dev,
                    (void*)G.flow_deps_dev, (void*)G.flow_cnt_dev, (void*)G.lg_dev,
                    (void*)G.copy_dev, (void*)G.adj_dev, (void*)G.perm_dev})
        if (q) cudaFree(q);
    G.ws = G.split_buf = nullptr;
    G.maxabs = nullptr;
    G.exps = nullptr;
    G.ctl = nullptr;
    G.leafmax = nullptr;
    G.leaf_img = G.gacc = nullptr;
    G.img_ptr_dev = nullptr;
    G.leaf_nfloat_dev = nullptr;
    G.descs_dev = nullptr;
    G.items_dev = nullptr;
    G.flow_deps_dev = nullptr;
    G.flow_cnt_dev = nullptr;
    G.lg_dev = nullptr;
    G.copy_dev = nullptr;
    G.adj_dev = nullptr;
    G.perm_dev = nullptr;
    for (void* q : {(void*)G.roots_dev, (void*)G.val_dev, (void*)G.val_exp_dev})
        if (q) cudaFree(q);
    G.roots_dev = nullptr;
    G.val_dev = nullptr;
    G.val_exp_dev = nullptr;
    if (G.gexec_f) cudaGraphExecDestroy(G.gexec_f);
    if (G.gexec_b) cudaGraphExecDestroy(G.gexec_b);
    if (G.graph_f) cudaGraphDestroy(G.graph_f);
    if (G.graph_b) cudaGraphDestroy(G.graph_b);
    G.gexec_f = G.gexec_b = nullptr;
    G.graph_f = G.graph_b = nullptr;
    G.n_inst = 0;
    G.kept = false;
}

void free_grad(Plan& p) {
    GradState* G = p.grad;
    if (!G) return;
    free_grad_device(*G);
    if (G->cap_stream) cudaStreamDestroy(G->cap_stream);
    delete G;
    p.grad = nullptr;
}

static cudaError_t launch_node(const Node& nd, const GenericArgs& g, const TileArgs& t, tn_mode mode,
                               bool c, cudaStream_t s) {
    if (nd.kind == kTensorCore)
        return launch_tc(t, tc_prec_of_mode(mode), c, s);
    if (nd.kind == kTiled) return launch_tile(t, c, s);
    return launch_generic(g, c, s);
}

// The steps [k0, k1) of the schedule for every instance.
static cudaError_t enqueue_steps(const GradState& G, int k0, int k1, tn_mode mode, bool cplx, cudaStream_t s) {
    const int nn = (int)G.fwd.size();
    const int ncomb = nn + (int)G.bwd.size();
    const int NI = G.n_inst;
    const void* const* leaf_tab = reinterpret_cast<const void* const*>(G.img_ptr_dev);
    cudaError_t e = cudaSuccess;
    for (int k = k0; k < k1 && e == cudaSuccess; ++k) {
        const Step& st = G.steps[k];
        if (st.wave) {
            const WaveItem* it = G.items_dev + G.inst_item_begin[k];
            if (st.flow)
                e = launch_wave(it, st.item_count * NI, G.descs_dev, leaf_tab, cplx, s,
                                reinterpret_cast<const int4*>(G.flow_deps_dev), G.flow_cnt_dev,
                                G.flow_cnt_dev + (size_t)ncomb * NI + k, NI);
            else
                e = launch_wave(it, st.item_count * NI, G.descs_dev, leaf_tab, cplx, s);
        } else if (st.node < nn) {
            e = launch_node(G.fwd[st.node], G.gen_f[st.node], G.tile_f[st.node], mode, cplx, s);
        } else {
            const int j = st.node - nn;
            e = launch_node(G.bwd[j], G.gen_b[j], G.tile_b[j], mode, cplx, s);
        }
    }
    return e;
}

// Zero scale slots [j0, j1) of every instance.
static cudaError_t zero_slots(const GradState& G, int j0, int j1, cudaStream_t s) {
    if (j1 <= j0) return cudaSuccess;
    if (G.n_inst == 1) return cudaMemsetAsync(G.maxabs + j0, 0, sizeof(unsigned) * (j1 - j0), s);
    return launch_zero_strided(G.maxabs + j0, j1 - j0, G.n_slots, G.n_inst, s);
}

// Forward half of one slice: forward scale slots and dataflow counters
// cleared, the forward steps.
static cudaError_t enqueue_forward(const GradState& G, tn_mode mode, bool cplx, cudaStream_t s) {
    const int nn = (int)G.fwd.size();
    const size_t ncomb = (size_t)nn + G.bwd.size();
    const size_t NI = (size_t)G.n_inst;
    cudaError_t e = zero_slots(G, 0, nn, s);
    if (e == cudaSuccess && G.any_flow) e = cudaMemsetAsync(G.flow_cnt_dev, 0, sizeof(unsigned) * nn * NI, s);
    if (e == cudaSuccess && G.any_flow)
        e = cudaMemsetAsync(G.flow_cnt_dev + ncomb * NI, 0, sizeof(unsigned) * G.n_fwd_steps, s);
    if (e == cudaSuccess) e = enqueue_steps(G, 0, G.n_fwd_steps, mode, cplx, s);
    return e;
}

// Sweep half of one slice: adjoint scale slots (all but the root's, set
// per call) and counters cleared, the adjoint steps, the leaf gathers, and
// the slice counter advanced.
static cudaError_t enqueue_sweep(const GradState& G, tn_mode mode, bool cplx, cudaStream_t s) {
    const int nn = (int)G.fwd.size();
    const size_t ncomb = (size_t)nn + G.bwd.size();
    const size_t NI = (size_t)G.n_inst;
    cudaError_t e = zero_slots(G, nn, G.n_slots - 1, s);
    if (e == cudaSuccess && G.any_flow)
        e = cudaMemsetAsync(G.flow_cnt_dev + nn * NI, 0, sizeof(unsigned) * (ncomb - nn) * NI, s);
    if (e == cudaSuccess && G.any_flow)
        e = cudaMemsetAsync(G.flow_cnt_dev + ncomb * NI + G.n_fwd_steps, 0,
                            sizeof(unsigned) * (G.steps.size() - G.n_fwd_steps), s);
    if (e == cudaSuccess) e = enqueue_steps(G, G.n_fwd_steps, (int)G.steps.size(), mode, cplx, s);
    if (e == cudaSuccess)
        e = launch_leaf_grads(G.lg_dev, (int)G.acc_off.size(), G.max_grad_n, G.n_inst, cplx, s);
    if (e == cudaSuccess) e = launch_advance(G.ctl, s);
    return e;
}

static cudaError_t capture(GradState& G, bool fwd, tn_mode mode, bool cplx) {
    cudaGraph_t& g = fwd ? G.graph_f : G.graph_b;
    cudaGraphExec_t& x = fwd ? G.gexec_f : G.gexec_b;
    cudaError_t e = cudaSuccess;
    if (!G.cap_stream) e = cudaStreamCreateWithFlags(&G.cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(G.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const cudaError_t e1 = fwd ? enqueue_forward(G, mode, cplx, G.cap_stream) : enqueue_sweep(G, mode, cplx, G.cap_stream);
    const cudaError_t e2 = cudaStreamEndCapture(G.cap_stream, &g);
    if (e1 != cudaSuccess) return e1;
    if (e2 != cudaSuccess) return e2;
    return cudaGraphInstantiate(&x, g, 0);
}

#define CK(x)                                                          \
    do {                                                               \
        cudaError_t e_ = (x);                                          \
        if (e_ != cudaSuccess) {                                       \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);     \
            return e_ == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA; \
        }                                                              \
    } while (0)

// Checks the call, (re)builds the sweep's plan and device state for this
// copy count and shared/varying pattern, and captures the two graphs.
static tn_status prepare(NetDesc& d, Plan& p, void* unit, int n_inst, const int64_t* leaf_inst_stride,
                         cudaStream_t stream, std::vector<char>& varying, std::string& err) {
    const int n = d.n;
    if (n_inst < 1) {
        err = "tn_contract_grad: n_inst < 1";
        return TN_EINVAL;
    }
    for (int v = 0; v < n; ++v)
        if (d.leaves[v].mem != TN_MEM_DEVICE) {
            err = "tn_contract_grad: leaves must be device pointers";
            return TN_EUNSUPPORTED;
        }
    varying.assign(n, 0);
    if (n_inst > 1 && leaf_inst_stride)
        for (int v = 0; v < n; ++v) {
            if (leaf_inst_stride[v] < 0 || (leaf_inst_stride[v] > 0 && leaf_inst_stride[v] < d.leaves[v].size)) {
                err = "tn_contract_grad: leaf_inst_stride[" + std::to_string(v) +
                      "] must be 0 or at least the leaf's size (copies may not overlap)";
                return TN_EINVAL;
            }
            varying[v] = leaf_inst_stride[v] > 0;
        }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        err = "tn_contract_grad: not available under stream capture (it uploads per-call tables; "
              "its per-slice work is already a CUDA graph)";
        return TN_EUNSUPPORTED;
    }
    if (p.grad && p.grad->plan_inst != n_inst) {
        CK(cudaStreamSynchronize(stream));
        free_grad(p);  // kernels and K splits are planned per copy count
    }
    if (!p.grad) {
        GradState* G = new GradState;
        tn_status st = build_grad(d, p, *G, n_inst, err);
        if (st != TN_OK) {
            delete G;
            return st;
        }
        p.grad = G;
    }
    GradState& G = *p.grad;
    if (G.n_inst != n_inst || G.varying != varying) {
        // another instance layout: the device state and graphs are rebuilt
        CK(cudaStreamSynchronize(stream));
        free_grad_device(G);
        tn_status st = alloc_grad(d, p, G, unit, n_inst, varying, err);
        if (st != TN_OK) {
            free_grad_device(G);
            return st;
        }
    }
    const bool cplx = d.is_complex();
    if (!G.gexec_f) CK(capture(G, true, p.mode, cplx));
    if (!G.gexec_b) CK(capture(G, false, p.mode, cplx));
    return TN_OK;
}

// Gather entries of the per-call copy table: the caller's leaves (copy i of
// a varying leaf at + i * stride) into the leaf image.
static void gather_entries(const NetDesc& d, const GradState& G, int n_inst, const int64_t* leaf_inst_stride,
                           std::vector<CopyEntry>& tab) {
    const int cf = d.is_complex() ? 2 : 1;
    for (int v = 0; v < d.n; ++v) {
        const int64_t nf = d.leaves[v].size * cf;
        const float* src = static_cast<const float*>(d.leaves[v].ptr);
        float* dst = G.leaf_img + G.img_off[v];
        if (!G.varying[v]) {
            tab.push_back(CopyEntry{src, dst, nf, 0, 1, 0});
        } else {
            for (int i = 0; i < n_inst; ++i)
                tab.push_back(CopyEntry{src + (int64_t)i * leaf_inst_stride[v] * cf, dst + i * G.img_is[v], nf, 0,
                                        1, 0});
        }
    }
}

static int64_t image_max_floats(const NetDesc& d, const GradState& G, int n_inst) {
    const int cf = d.is_complex() ? 2 : 1;
    int64_t mx = 0;
    for (int v = 0; v < d.n; ++v)
        mx = std::max(mx, G.varying[v] ? G.img_is[v] * (n_inst - 1) + d.leaves[v].size * cf : d.leaves[v].size * cf);
    return mx;
}

tn_status run_grad_forward(NetDesc& d, Plan& p, void* unit, int n_inst, const int64_t* leaf_inst_stride,
                           double* out, int64_t* out_exp2, int out_mem, cudaStream_t stream, std::string& err) {
    if (p.d_sliced != 1 || p.n_out != 1) {
        err = "tn_contract_instances_keep: unsliced scalar networks only";
        return TN_EUNSUPPORTED;
    }
    std::vector<char> varying;
    tn_status st = prepare(d, p, unit, n_inst, leaf_inst_stride, stream, varying, err);
    if (st != TN_OK) return st;
    GradState& G = *p.grad;
    G.kept = false;
    std::vector<CopyEntry> tab;
    gather_entries(d, G, n_inst, leaf_inst_stride, tab);
    CK(cudaMemcpyAsync(G.copy_dev, tab.data(), sizeof(CopyEntry) * tab.size(), cudaMemcpyHostToDevice, stream));
    CK(launch_copy_table(G.copy_dev, (int)tab.size(), G.max_leaf_floats, stream));
    CK(launch_leaf_max(G.img_ptr_dev, G.leaf_nfloat_dev, G.leafmax, d.n, stream, image_max_floats(d, G, n_inst)));
    CK(launch_begin_call(G.ctl, 0, 1, nullptr, 0, stream));
    CK(cudaGraphLaunch(G.gexec_f, stream));
    const bool host = out_mem == TN_MEM_HOST;
    CK(launch_batch_finish(G.roots_dev, n_inst, host ? G.val_dev : out, host ? G.val_exp_dev : out_exp2, nullptr,
                           nullptr, nullptr, stream));
    if (host) {
        CK(cudaMemcpyAsync(out, G.val_dev, sizeof(double) * 2 * n_inst, cudaMemcpyDeviceToHost, stream));
        CK(cudaMemcpyAsync(out_exp2, G.val_exp_dev, sizeof(int64_t) * n_inst, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
    }
    G.kept = true;
    return TN_OK;
}

tn_status run_grad(NetDesc& d, Plan& p, void* unit, const double* adj, int adj_mem, int64_t adj_exp2,
                   const int64_t* adj_exp2_dev, void* const* grads, bool accumulate, bool kept_forward,
                   int n_inst, const int64_t* leaf_inst_stride, int64_t slice_begin, int64_t slice_count,
                   cudaStream_t stream, std::string& err) {
    const int n = d.n;
    if (slice_count <= 0) {
        slice_begin = 0;
        slice_count = p.d_sliced;
    }
    if (slice_begin < 0 || slice_begin > p.d_sliced - slice_count) {  // no overflowing sum
        err = "tn_contract_grad: slice range out of bounds";
        return TN_EINVAL;
    }
    const bool cplx = d.is_complex();
    const int cf = cplx ? 2 : 1;
    if (kept_forward && (!p.grad || !p.grad->kept || p.grad->n_inst != n_inst)) {
        err = "tn_contract_grad: TN_GRAD_KEPT_FORWARD without a preceding tn_contract_instances_keep "
              "of this tree, mode and copy count";
        return TN_EINVAL;
    }
    std::vector<char> varying;
    tn_status st = prepare(d, p, unit, n_inst, leaf_inst_stride, stream, varying, err);
    if (st != TN_OK) return st;
    GradState& G = *p.grad;
    if (kept_forward && (G.varying != varying || !G.kept)) {
        err = "tn_contract_grad: TN_GRAD_KEPT_FORWARD with other leaf strides than the kept forward";
        return TN_EINVAL;
    }
    const int nn = (int)G.fwd.size();
    const int root_v = n + nn - 1;
    const size_t eb = d.elem_bytes();
    // per-call table: the leaves into the image (unless kept), then the
    // gradients out
    std::vector<CopyEntry> tab;
    tab.reserve((size_t)2 * n * n_inst);
    if (!kept_forward) gather_entries(d, G, n_inst, leaf_inst_stride, tab);
    const int n_gather = (int)tab.size();
    for (int v = 0; v < n; ++v) {
        if (!grads[v]) continue;
        const int64_t nf = d.leaves[v].size * cf;
        float* dst = static_cast<float*>(grads[v]);
        const float* src = G.gacc + G.acc_off[v];
        if (!varying[v]) {
            tab.push_back(CopyEntry{src, dst, nf, G.acc_floats, n_inst, accumulate ? 1 : 0});
        } else {
            for (int i = 0; i < n_inst; ++i)
                tab.push_back(CopyEntry{src + i * G.acc_floats, dst + (int64_t)i * leaf_inst_stride[v] * cf, nf, 0, 1,
                                        accumulate ? 1 : 0});
        }
    }
    const int n_scatter = (int)tab.size() - n_gather;
    // pageable source: the copy is staged before the call returns
    if (!tab.empty())
        CK(cudaMemcpyAsync(G.copy_dev, tab.data(), sizeof(CopyEntry) * tab.size(), cudaMemcpyHostToDevice,
                           stream));
    if (!kept_forward) {
        CK(launch_copy_table(G.copy_dev, n_gather, G.max_leaf_floats, stream));
        CK(launch_leaf_max(G.img_ptr_dev, G.leaf_nfloat_dev, G.leafmax, n, stream, image_max_floats(d, G, n_inst)));
    }
    // root adjoints
    const double* adj_src = adj;
    if (adj_mem == TN_MEM_HOST) {
        CK(cudaMemcpyAsync(G.adj_dev, adj, sizeof(double) * p.n_out * cf * n_inst, cudaMemcpyHostToDevice,
                           stream));
        adj_src = G.adj_dev;
    }
    RootAdjArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.adj = adj_src;
    ra.exp_dev = adj_mem == TN_MEM_HOST ? nullptr : adj_exp2_dev;
    ra.exp_host = adj_exp2;
    ra.perm = G.perm_dev;
    ra.n_out = p.n_out;
    ra.cplx = cplx ? 1 : 0;
    ra.dst = reinterpret_cast<float*>(static_cast<char*>(G.ws) + G.adj_off[root_v] * eb);
    ra.max_slot = G.maxabs + (G.n_slots - 1);
    ra.exp_slot = G.exps + (G.n_slots - 1);
    ra.dst_is = G.ws_elems * cf;
    ra.slot_is = G.n_slots;
    CK(launch_root_adjoint(ra, n_inst, stream));
    CK(cudaMemsetAsync(G.gacc, 0, sizeof(float) * G.acc_floats * n_inst, stream));
    CK(launch_begin_call(G.ctl, slice_begin, slice_begin + slice_count, nullptr, 0, stream));
    if (kept_forward) {
        CK(cudaGraphLaunch(G.gexec_b, stream));
    } else {
        G.kept = false;  // the workspace is rewritten slice by slice
        for (int64_t s = 0; s < slice_count; ++s) {
            CK(cudaGraphLaunch(G.gexec_f, stream));
            CK(cudaGraphLaunch(G.gexec_b, stream));
        }
    }
    if (n_scatter > 0) CK(launch_copy_table(G.copy_dev + n_gather, n_scatter, G.max_leaf_floats, stream));
    return TN_OK;
}
#undef CK

}  // namespace tn
