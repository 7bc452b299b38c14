// tn_batch.cpp -- many independent networks in one captured launch sequence.
//
// Each network keeps its own contraction tree and host plan (Sec. 2 of arXiv
// 2002.01935); the batch merges them into one forest: one workspace, one
// renormalisation slot array, one leaf table and device-resident node
// descriptors.  Execution goes by tree level across all networks: per level
// one wave launch per storage type runs every small node of every network,
// then the large nodes launch one by one.  A final kernel writes every
// network's (mantissa, exponent) and the time its root completed.  The
// whole sequence is captured once as a CUDA graph and replayed.  Sliced
// networks (Sec. 4.7.1: a tree sliced to a width cap) stay out of the forest:
// after the graph, each runs its own slice loop -- its per-slice graph
// replayed over its slices, several side by side, folded in FP64 -- on the
// same stream, and writes its value and completion latency into the batch's
// outputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "tn_batch.h"

namespace tn {

tn_status build_batch(BatchPlan& b, std::string& err) {
    const int N = (int)b.nets.size();
    b.ws_base.assign(N, 0);
    b.slot_base.assign(N, 0);
    b.leaf_base.assign(N, 0);
    b.desc_base.assign(N, 0);
    int64_t ws = 0;
    int slots = 0, leaves = 0, descs = 0;
    int64_t split_bytes = 0;
    int max_level = 0;
    b.level.assign(N, {});
    b.small.assign(N, {});
    b.is_sliced.assign(N, 0);
    for (const SlicedMember& m : b.sliced) b.is_sliced[m.index] = 1;
    for (int i = 0; i < N; ++i) {
        const NetDesc& d = *b.nets[i];
        const Plan& p = *b.plans[i];
        if (p.n_out != 1) {
            err = "tn_batch: every network must be scalar (no open labels)";
            return TN_EUNSUPPORTED;
        }
        if (p.d_sliced != 1 && !b.is_sliced[i]) {
            err = "tn_batch: a sliced tree must be given as a sliced member";
            return TN_EUNSUPPORTED;
        }
        if (b.is_sliced[i]) continue;  // runs its own slice loop after the forest
        b.ws_base[i] = ws;
        ws += (p.ws_elems * (int64_t)d.elem_bytes() + 255) / 256 * 256;
        b.slot_base[i] = slots;
        slots += (int)p.nodes.size();
        b.leaf_base[i] = leaves;
        leaves += d.n;
        b.desc_base[i] = descs;
        descs += (int)p.nodes.size();
        split_bytes = std::max(split_bytes, p.split_bytes);
        const int n = d.n;
        std::vector<int>& lv = b.level[i];
        lv.assign(p.nodes.size(), 0);
        for (size_t k = 0; k < p.nodes.size(); ++k) {
            const Node& nd = p.nodes[k];
            const int la = nd.ca >= n ? lv[nd.ca - n] : 0, lb = nd.cb >= n ? lv[nd.cb - n] : 0;
            lv[k] = 1 + std::max(la, lb);
            max_level = std::max(max_level, lv[k]);
        }
        b.small[i].assign(p.nodes.size(), 0);
        for (const Step& st : p.steps)
            if (st.wave)
                for (int k : st.nodes) b.small[i][k] = 1;
    }
    b.ws_bytes = std::max<int64_t>(ws, 256) + 256;  // + a unit scalar
    b.n_slots = slots;
    b.n_leaves = leaves;
    b.split_bytes = split_bytes;
    b.descs.assign(descs, TileArgs{});
    b.gen.assign(descs, GenericArgs{});
    // launch schedule: level by level across all networks
    b.steps.clear();
    b.items.clear();
    for (int L = 1; L <= max_level; ++L) {
        for (int cp = 0; cp < 2; ++cp) {
            BatchStep w;
            w.wave = 1;
            w.cplx = cp == 1;
            w.item_begin = (int)b.items.size();
            for (int i = 0; i < N; ++i) {
                if (b.is_sliced[i] || b.nets[i]->is_complex() != w.cplx) continue;
                const Plan& p = *b.plans[i];
                for (size_t k = 0; k < p.nodes.size(); ++k) {
                    if (b.level[i][k] != L || !b.small[i][k]) continue;
                    const int64_t size = p.nodes[k].size;
                    const int64_t chunk = wave_chunk(p.nodes[k], N);  // many networks: throughput
                    for (int64_t o = 0; o < size; o += chunk) {
                        WaveItem it;
                        it.node = b.desc_base[i] + (int)k;
                        it.pad = 0;
                        it.o_begin = o;
                        it.o_count = chunk;
                        b.items.push_back(it);
                    }
                }
            }
            w.item_count = (int)b.items.size() - w.item_begin;
            if (w.item_count) b.steps.push_back(w);
        }
        for (int i = 0; i < N; ++i) {
            if (b.is_sliced[i]) continue;
            const Plan& p = *b.plans[i];
            for (size_t k = 0; k < p.nodes.size(); ++k) {
                if (b.level[i][k] != L || b.small[i][k]) continue;
                BatchStep s;
                s.net = i;
                s.node = (int)k;
                s.cplx = b.nets[i]->is_complex();
                b.steps.push_back(s);
            }
        }
    }
    return TN_OK;
}

tn_status alloc_batch(BatchPlan& b, std::string& err) {
    const int N = (int)b.nets.size();
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess) {
            err = std::string(what) + ": " + cudaGetErrorString(e);
            return false;
        }
        return true;
    };
    if (!ck(cudaMalloc(&b.ws, b.ws_bytes), "batch workspace")) return TN_ENOMEM;
    if (b.split_bytes && !ck(cudaMalloc(&b.split_buf, b.split_bytes), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.maxabs, sizeof(unsigned) * std::max(b.n_slots, 1)), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.exps, sizeof(int64_t) * std::max(b.n_slots, 1)), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.ctl, sizeof(Control)), "cudaMalloc")) return TN_ENOMEM;
    const size_t nl = (size_t)std::max(b.n_leaves, 1);
    if (!ck(cudaMalloc(&b.leafmax, sizeof(unsigned) * nl), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc((void**)&b.leaf_ptr_dev, sizeof(void*) * nl), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.leaf_nfloat_dev, sizeof(int64_t) * nl), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.t_start, sizeof(unsigned long long)), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.t_done, sizeof(unsigned long long) * N), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.lat_dev, sizeof(unsigned long long) * N), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.out_dev, sizeof(double) * 2 * N), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.exp_dev, sizeof(int64_t) * N), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&b.roots_dev, sizeof(BatchRoot) * N), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking), "stream")) return TN_ECUDA;
    char* ws = (char*)b.ws;
    void* unit = ws + b.ws_bytes - 256;
    const float one[2] = {1.f, 0.f};
    if (!ck(cudaMemcpy(unit, one, sizeof(one), cudaMemcpyHostToDevice), "cudaMemcpy")) return TN_ECUDA;
    std::vector<int64_t> nf(b.n_leaves);
    std::vector<BatchRoot> roots(N);
    for (int i = 0; i < N; ++i) {
        if (b.is_sliced[i]) {
            memset(&roots[i], 0, sizeof(roots[i]));  // root NULL: written by its slice loop
            continue;
        }
        const NetDesc& d = *b.nets[i];
        const Plan& p = *b.plans[i];
        const int n = d.n;
        const size_t eb = d.elem_bytes();
        char* base = ws + b.ws_base[i];
        for (int v = 0; v < n; ++v) nf[b.leaf_base[i] + v] = d.leaves[v].size * (d.is_complex() ? 2 : 1);
        for (size_t k = 0; k < p.nodes.size(); ++k) {
            const Node& nd = p.nodes[k];
            const int di = b.desc_base[i] + (int)k;
            GenericArgs& g = b.gen[di];
            tn_status st = make_generic_args(d, p, (int)k, g, err);
            if (st != TN_OK) return st;
            auto ptr = [&](int c) -> const void* {
                if (c < 0) return unit;
                if (c < n) return nullptr;  // leaf: from the leaf table / patched per capture
                return base + p.nodes[c - n].ws_off * eb;
            };
            auto smax = [&](int c) -> const unsigned* {
                if (c < 0) return nullptr;
                if (c < n) return b.leafmax + b.leaf_base[i] + c;
                return b.maxabs + b.slot_base[i] + (c - n);
            };
            auto sexp = [&](int c) -> const int64_t* {
                if (c < n) return nullptr;
                return b.exps + b.slot_base[i] + (c - n);
            };
            g.A = ptr(nd.ca);
            g.B = ptr(nd.cb);
            g.C = base + nd.ws_off * eb;
            g.ctl = b.ctl;
            g.sc.max_a = smax(nd.ca);
            g.sc.exp_a = sexp(nd.ca);
            g.sc.max_b = smax(nd.cb);
            g.sc.exp_b = sexp(nd.cb);
            g.sc.max_c = b.maxabs + b.slot_base[i] + k;
            g.sc.exp_c = b.exps + b.slot_base[i] + k;
            const bool root = k + 1 == p.nodes.size();
            g.t_done = root ? b.t_done + i : nullptr;
            TileArgs& t = b.descs[di];
            t = nd.tile;
            memset(&t.in, 0, sizeof(t.in));  // single instance
            t.A = g.A;
            t.B = g.B;
            t.C = g.C;
            t.P = b.split_buf;
            t.sla = g.sla;
            t.slb = g.slb;
            t.ctl = b.ctl;
            t.sc = g.sc;
            t.a_leaf = nd.ca >= 0 && nd.ca < n ? b.leaf_base[i] + nd.ca : -1;
            t.b_leaf = nd.cb >= 0 && nd.cb < n ? b.leaf_base[i] + nd.cb : -1;
            t.t_done = g.t_done;
            if (root) {
                roots[i].root = g.C;
                roots[i].exp = g.sc.exp_c;
                roots[i].max = g.sc.max_c;
                roots[i].is_c = d.is_complex();
                roots[i].pad = 0;
            }
        }
    }
    b.max_leaf_floats = 0;
    for (int64_t x : nf) b.max_leaf_floats = std::max(b.max_leaf_floats, x);
    if (!ck(cudaMemcpy(b.leaf_nfloat_dev, nf.data(), sizeof(int64_t) * b.n_leaves, cudaMemcpyHostToDevice),
            "cudaMemcpy"))
        return TN_ECUDA;
    if (!ck(cudaMemcpy(b.roots_dev, roots.data(), sizeof(BatchRoot) * N, cudaMemcpyHostToDevice), "cudaMemcpy"))
        return TN_ECUDA;
    if (!ck(cudaMalloc(&b.descs_dev, sizeof(TileArgs) * std::max<size_t>(b.descs.size(), 1)), "cudaMalloc"))
        return TN_ENOMEM;
    if (!ck(cudaMemcpy(b.descs_dev, b.descs.data(), sizeof(TileArgs) * b.descs.size(), cudaMemcpyHostToDevice),
            "cudaMemcpy"))
        return TN_ECUDA;
    if (!b.items.empty()) {
        if (!ck(cudaMalloc(&b.items_dev, sizeof(WaveItem) * b.items.size()), "cudaMalloc")) return TN_ENOMEM;
        if (!ck(cudaMemcpy(b.items_dev, b.items.data(), sizeof(WaveItem) * b.items.size(),
                           cudaMemcpyHostToDevice),
                "cudaMemcpy"))
            return TN_ECUDA;
    }
    return TN_OK;
}

static cudaError_t enqueue_batch(BatchPlan& b, cudaStream_t s) {
    const int N = (int)b.nets.size();
    cudaError_t e = cudaMemsetAsync(b.maxabs, 0, sizeof(unsigned) * std::max(b.n_slots, 1), s);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b.t_done, 0, sizeof(unsigned long long) * N, s)) != cudaSuccess) return e;
    if ((e = launch_batch_start(b.t_start, s)) != cudaSuccess) return e;
    if ((e = launch_leaf_max(b.leaf_ptr_dev, b.leaf_nfloat_dev, b.leafmax, b.n_leaves, s, b.max_leaf_floats)) !=
        cudaSuccess)
        return e;
    if ((e = launch_begin_call(b.ctl, 0, 1, nullptr, 0, s)) != cudaSuccess) return e;
    for (const BatchStep& st : b.steps) {
        if (st.wave) {
            e = launch_wave(b.items_dev + st.item_begin, st.item_count, b.descs_dev,
                            reinterpret_cast<const void* const*>(b.leaf_ptr_dev), st.cplx, s);
        } else {
            const Plan& p = *b.plans[st.net];
            const Node& nd = p.nodes[st.node];
            const int di = b.desc_base[st.net] + st.node;
            if (nd.kind == kTensorCore)
                e = launch_tc(b.descs[di], tc_prec_of_mode(b.mode),
                              st.cplx, s);
            else if (nd.kind == kTiled)
                e = launch_tile(b.descs[di], st.cplx, s);
            else
                e = launch_generic(b.gen[di], st.cplx, s);
        }
        if (e != cudaSuccess) return e;
    }
    return launch_batch_finish(b.roots_dev, N, b.out_dev, b.exp_dev, b.t_start, b.t_done, b.lat_dev, s);
}

tn_status run_batch(BatchPlan& b, double* out, int64_t* out_exp2, uint64_t* latency_ns, int out_mem,
                    cudaStream_t stream, std::string& err) {
    const int N = (int)b.nets.size();
#define CK(x)                                                          \
    do {                                                               \
        cudaError_t e_ = (x);                                          \
        if (e_ != cudaSuccess) {                                       \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);     \
            return e_ == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA; \
        }                                                              \
    } while (0)
    std::vector<const void*> lp(b.n_leaves);
    for (int i = 0; i < N; ++i) {
        const NetDesc& d = *b.nets[i];
        for (int v = 0; v < d.n; ++v) {
            if (d.leaves[v].mem != TN_MEM_DEVICE || !d.leaves[v].ptr) {
                err = "tn_batch: every leaf must be a device pointer";
                return TN_EINVAL;
            }
            if (!b.is_sliced[i]) lp[b.leaf_base[i] + v] = d.leaves[v].ptr;
        }
    }
    if (!b.gexec || lp != b.graph_ptrs) {
        // leaf pointers go into the table (waves) and the single-node arguments
        CK(cudaMemcpyAsync(b.leaf_ptr_dev, lp.data(), sizeof(void*) * b.n_leaves, cudaMemcpyHostToDevice,
                           stream));
        CK(cudaStreamSynchronize(stream));
        for (int i = 0; i < N; ++i) {
            if (b.is_sliced[i]) continue;
            const Plan& p = *b.plans[i];
            const int n = b.nets[i]->n;
            for (size_t k = 0; k < p.nodes.size(); ++k) {
                const Node& nd = p.nodes[k];
                const int di = b.desc_base[i] + (int)k;
                if (nd.ca >= 0 && nd.ca < n) b.descs[di].A = b.gen[di].A = lp[b.leaf_base[i] + nd.ca];
                if (nd.cb >= 0 && nd.cb < n) b.descs[di].B = b.gen[di].B = lp[b.leaf_base[i] + nd.cb];
            }
        }
        if (b.gexec) CK(cudaGraphExecDestroy(b.gexec));
        b.gexec = nullptr;
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(b.cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_batch(b, b.cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(b.cap_stream, &g);
        CK(e);
        CK(e2);
        e = cudaGraphInstantiate(&b.gexec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        b.graph_ptrs = lp;
    }
    CK(cudaGraphLaunch(b.gexec, stream));
    // the sliced members, one after another: all their slices (G side by
    // side per launch, FP64 fold in slice order), value and exponent into
    // the batch's outputs, then their completion latency
    for (const SlicedMember& m : b.sliced) {
        tn_options o;
        memset(&o, 0, sizeof(o));
        o.slice_batch = m.G;
        tn_status st = run_plan(*m.d, *m.p, m.unit, 0, m.p->d_sliced, o, b.out_dev + 2 * m.index,
                                TN_MEM_DEVICE, b.exp_dev + m.index, stream, err);
        if (st != TN_OK) return st;
        CK(launch_batch_mark(b.t_start, b.lat_dev + m.index, stream));
    }
    cudaMemcpyKind kind = out_mem == TN_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(out, b.out_dev, sizeof(double) * 2 * N, kind, stream));
    CK(cudaMemcpyAsync(out_exp2, b.exp_dev, sizeof(int64_t) * N, kind, stream));
    if (latency_ns) CK(cudaMemcpyAsync(latency_ns, b.lat_dev, sizeof(uint64_t) * N, kind, stream));
    if (out_mem == TN_MEM_HOST) CK(cudaStreamSynchronize(stream));
#undef CK
    return TN_OK;
}

void free_batch(BatchPlan& b) {
    if (b.gexec) cudaGraphExecDestroy(b.gexec);
    if (b.cap_stream) cudaStreamDestroy(b.cap_stream);
    void* ptrs[] = {b.ws, b.split_buf, b.maxabs, b.exps, b.ctl, b.leafmax, (void*)b.leaf_ptr_dev,
                    b.leaf_nfloat_dev, b.t_start, b.t_done, b.lat_dev, b.out_dev, b.exp_dev,
                    b.roots_dev, b.descs_dev, b.items_dev};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    b = BatchPlan();
}

}  // namespace tn
