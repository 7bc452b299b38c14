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
// leaves; leaf adjoints are added into the caller's gradient buffers at the
// slice's offset, so the result is summed over slices.  A leaf label that
// occurs in that tensor only (summed at its first contraction) gives an
// adjoint constant along it: the gather broadcasts.  Renormalisation
// exponents are tracked exactly as in the forward pass.
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
    // device
    void* ws = nullptr;
    void* split_buf = nullptr;
    unsigned* maxabs = nullptr;
    int64_t* exps = nullptr;
    Control* ctl = nullptr;
    unsigned* leafmax = nullptr;
    const float** leaf_ptr_dev = nullptr;
    int64_t* leaf_nfloat_dev = nullptr;
    std::vector<GenericArgs> gen_f, gen_b;
    std::vector<TileArgs> tile_f, tile_b;
};

static bool has_label(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

static tn_status build_grad(const NetDesc& d, const Plan& f, GradState& G, std::string& err) {
    const int n = d.n;
    const int nn = (int)f.nodes.size();
    G.g = Plan();
    G.g.mode = f.mode;
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
                make_tensor_core(d, f.mode, nd, split_elems);
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
    (void)err;
    return TN_OK;
}

static tn_status alloc_grad(const NetDesc& d, GradState& G, void* unit, std::string& err) {
    const size_t eb = d.elem_bytes();
    const int n = d.n;
    const int nn = (int)G.fwd.size();
    const int NV = G.NV;
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess) {
            err = std::string(what) + ": " + cudaGetErrorString(e);
            return false;
        }
        return true;
    };
    if (!ck(cudaMalloc(&G.ws, (size_t)G.ws_elems * eb), "gradient workspace")) return TN_ENOMEM;
    if (G.split_bytes && !ck(cudaMalloc(&G.split_buf, G.split_bytes), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&G.maxabs, sizeof(unsigned) * G.n_slots), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&G.exps, sizeof(int64_t) * G.n_slots), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&G.ctl, sizeof(Control)), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&G.leafmax, sizeof(unsigned) * n), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc((void**)&G.leaf_ptr_dev, sizeof(void*) * n), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&G.leaf_nfloat_dev, sizeof(int64_t) * n), "cudaMalloc")) return TN_ENOMEM;
    std::vector<int64_t> nf(n);
    for (int v = 0; v < n; ++v) nf[v] = d.leaves[v].size * (d.is_complex() ? 2 : 1);
    if (!ck(cudaMemcpy(G.leaf_nfloat_dev, nf.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice),
            "cudaMemcpy"))
        return TN_ECUDA;
    char* ws = (char*)G.ws;
    auto fwd_ptr = [&](int v) -> const void* {
        if (v < 0) return unit;
        if (v < n) return nullptr;  // leaf: patched per call
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
        t = nd.tile;
        memset(&t.in, 0, sizeof(t.in));  // single instance
        t.A = A;
        t.B = B;
        t.C = C;
        t.P = G.split_buf;
        t.sla = g.sla;
        t.slb = g.slb;
        t.ctl = G.ctl;
        t.sc = g.sc;
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
    G.gen_b.assign(G.bwd.size(), GenericArgs{});
    G.tile_b.assign(G.bwd.size(), TileArgs{});
    for (size_t j = 0; j < G.bwd.size(); ++j) {
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
    return TN_OK;
}

void free_grad(Plan& p) {
    GradState* G = p.grad;
    if (!G) return;
    cudaFree(G->ws);
    if (G->split_buf) cudaFree(G->split_buf);
    cudaFree(G->maxabs);
    cudaFree(G->exps);
    cudaFree(G->ctl);
    cudaFree(G->leafmax);
    cudaFree(G->leaf_ptr_dev);
    cudaFree(G->leaf_nfloat_dev);
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

tn_status run_grad(NetDesc& d, Plan& p, void* unit, const double* adj, int64_t adj_exp2,
                   void* const* grads, cudaStream_t stream, std::string& err) {
    const int n = d.n;
    const bool cplx = d.is_complex();
    const size_t eb = d.elem_bytes();
#define CK(x)                                                          \
    do {                                                               \
        cudaError_t e_ = (x);                                          \
        if (e_ != cudaSuccess) {                                       \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);     \
            return e_ == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA; \
        }                                                              \
    } while (0)
    for (int v = 0; v < n; ++v)
        if (d.leaves[v].mem != TN_MEM_DEVICE) {
            err = "tn_contract_grad: leaves must be device pointers";
            return TN_EUNSUPPORTED;
        }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &cap));
    if (!p.grad) {
        if (cap != cudaStreamCaptureStatusNone) {
            err = "tn_contract_grad: the first call for a tree must run outside stream capture";
            return TN_EUNSUPPORTED;
        }
        GradState* G = new GradState;
        tn_status st = build_grad(d, p, *G, err);
        if (st == TN_OK) st = alloc_grad(d, *G, unit, err);
        if (st != TN_OK) {
            p.grad = G;
            free_grad(p);
            return st;
        }
        p.grad = G;
    }
    GradState& G = *p.grad;
    const int nn = (int)G.fwd.size();
    const int NV = G.NV;
    const int root_v = n + nn - 1;
    // leaf pointers into the forward arguments
    std::vector<const void*> lp(n);
    for (int v = 0; v < n; ++v) lp[v] = d.leaves[v].ptr;
    for (int k = 0; k < nn; ++k) {
        const Node& nd = G.fwd[k];
        if (nd.ca >= 0 && nd.ca < n) G.gen_f[k].A = G.tile_f[k].A = lp[nd.ca];
        if (nd.cb >= 0 && nd.cb < n) G.gen_f[k].B = G.tile_f[k].B = lp[nd.cb];
    }
    for (size_t j = 0; j < G.bwd.size(); ++j) {
        const Node& nd = G.bwd[j];
        if (nd.ca >= 0 && nd.ca < n) G.gen_b[j].A = G.tile_b[j].A = lp[nd.ca];
        if (nd.cb >= 0 && nd.cb < n) G.gen_b[j].B = G.tile_b[j].B = lp[nd.cb];
    }
    CK(cudaMemcpyAsync(G.leaf_ptr_dev, lp.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, stream));
    int64_t mx_leaf = 0;
    for (int v = 0; v < n; ++v) mx_leaf = std::max(mx_leaf, d.leaves[v].size * (d.is_complex() ? 2 : 1));
    CK(launch_leaf_max(G.leaf_ptr_dev, G.leaf_nfloat_dev, G.leafmax, n, stream, mx_leaf));
    // root adjoint: caller's FP64 array (open labels in tn_create order) ->
    // root layout, normalised to a power-of-two scaled float tensor
    const Node& root = G.fwd.back();
    const int64_t n_out = p.n_out;
    std::vector<double> perm((size_t)n_out * (cplx ? 2 : 1), 0.0);
    double amax = 0;
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t rem = o, dst = 0;
        for (int i = (int)d.open.size() - 1; i >= 0; --i) {
            const int l = d.open[i];
            const int64_t v = rem % d.dims[l];
            rem /= d.dims[l];
            for (size_t j = 0; j < root.lab.size(); ++j)
                if (root.lab[j] == l) dst += v * root.stride[j];
        }
        for (int c = 0; c < (cplx ? 2 : 1); ++c) {
            const double x = adj[o * (cplx ? 2 : 1) + c];
            perm[dst * (cplx ? 2 : 1) + c] = x;
            amax = std::max(amax, std::fabs(x));
        }
    }
    int eadj = 0;
    if (amax > 0) std::frexp(amax, &eadj);
    std::vector<float> rootadj(perm.size());
    for (size_t i = 0; i < perm.size(); ++i) rootadj[i] = (float)std::ldexp(perm[i], -eadj);
    const float rmax = amax > 0 ? (float)std::ldexp(amax, -eadj) : 0.f;
    unsigned rmax_bits;
    std::memcpy(&rmax_bits, &rmax, 4);
    const int64_t rexp = (int64_t)eadj + adj_exp2;
    char* ws = (char*)G.ws;
    CK(cudaMemcpyAsync(ws + G.adj_off[root_v] * eb, rootadj.data(), rootadj.size() * sizeof(float),
                       cudaMemcpyHostToDevice, stream));
    const int root_slot = nn + root_v;
    CK(cudaMemcpyAsync(G.maxabs + root_slot, &rmax_bits, sizeof(unsigned), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(G.exps + root_slot, &rexp, sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    // zero the outputs, then every slice: forward, reverse sweep, leaf gather
    for (int v = 0; v < n; ++v)
        if (grads[v]) CK(cudaMemsetAsync(grads[v], 0, d.leaves[v].size * eb, stream));
    CK(launch_begin_call(G.ctl, 0, p.d_sliced, nullptr, 0, stream));
    std::vector<LeafGradArgs> lg(n);
    for (int v = 0; v < n; ++v) {
        LeafGradArgs& a = lg[v];
        memset(&a, 0, sizeof(a));
        if (!grads[v]) continue;
        const LeafDesc& lf = d.leaves[v];
        a.grad = grads[v];
        a.adj = ws + G.adj_off[v] * eb;
        a.exp_adj = G.exps + nn + v;
        a.ctl = G.ctl;
        a.sl = p.leaf_sl[v];
        const std::vector<int>& al = G.g.vlab[NV + v];
        const std::vector<int64_t>& as = G.g.vstride[NV + v];
        a.n = 1;
        int nd_ = 0;
        for (int i = (int)lf.lab.size() - 1; i >= 0; --i) {
            const int l = lf.lab[i];
            if (std::find(p.sliced.begin(), p.sliced.end(), l) != p.sliced.end()) continue;
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
    }
    for (int64_t s = 0; s < p.d_sliced; ++s) {
        CK(cudaMemsetAsync(G.maxabs, 0, sizeof(unsigned) * (G.n_slots - 1), stream));
        for (int k : G.fwd_order)
            CK(launch_node(G.fwd[k], G.gen_f[k], G.tile_f[k], p.mode, cplx, stream));
        for (size_t j = 0; j < G.bwd.size(); ++j)
            CK(launch_node(G.bwd[j], G.gen_b[j], G.tile_b[j], p.mode, cplx, stream));
        for (int v = 0; v < n; ++v)
            if (grads[v]) CK(launch_leaf_grad(lg[v], cplx, stream));
        CK(launch_advance(G.ctl, stream));
    }
#undef CK
    return TN_OK;
}

}  // namespace tn
