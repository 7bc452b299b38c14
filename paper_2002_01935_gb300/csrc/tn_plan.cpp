// tn_plan.cpp -- node planning, workspace liveness and the per-call runtime
// of libtn.so.  See tn_api.cpp for the overview.
#include "tn_plan.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <map>

namespace tn {

namespace {

struct SubCount {
    std::vector<std::pair<int, int>> c;  // (label, leaves of the subtree holding it)
    int get(int l) const {
        for (auto& x : c)
            if (x.first == l) return x.second;
        return 0;
    }
};

int64_t stride_in(const std::vector<int>& lab, const std::vector<int64_t>& st, int l) {
    for (size_t i = 0; i < lab.size(); ++i)
        if (lab[i] == l) return st[i];
    return 0;
}

bool has(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

// Best-fit workspace allocator over element offsets (liveness planning).
struct Arena {
    std::map<int64_t, int64_t> free_;  // offset -> length
    int64_t end = 0;
    static int64_t round(int64_t n) { return (n + 63) / 64 * 64; }
    int64_t alloc(int64_t n) {
        n = round(n);
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n && (best == free_.end() || it->second < best->second)) best = it;
        if (best != free_.end()) {
            int64_t off = best->first, len = best->second;
            free_.erase(best);
            if (len > n) free_[off + n] = len - n;
            return off;
        }
        // extend, merging a free tail block
        if (!free_.empty()) {
            auto last = std::prev(free_.end());
            if (last->first + last->second == end) {
                int64_t off = last->first;
                free_.erase(last);
                end = off + n;
                return off;
            }
        }
        int64_t off = end;
        end += n;
        return off;
    }
    void release(int64_t off, int64_t n) {
        n = round(n);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

bool pow2(int64_t x) { return x >= 1 && (x & (x - 1)) == 0; }
int ilog2(int64_t x) {
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
}

// Tiled-kernel plan of a node whose labels and strides are all powers of
// two: index bits per group, K order, load directions, tile shape and K
// split.  Returns false (generic kernel) when a limit is exceeded.
bool plan_tile(const NetDesc& d, const Plan& p, Node& nd, int64_t& split_elems, int force_cfg = 0) {
    static const std::vector<int> none;
    static const std::vector<int64_t> nones;
    const std::vector<int>& la = nd.ca >= 0 ? p.vlab[nd.ca] : none;
    const std::vector<int>& lb = nd.cb >= 0 ? p.vlab[nd.cb] : none;
    const std::vector<int64_t>& sa = nd.ca >= 0 ? p.vstride[nd.ca] : nones;
    const std::vector<int64_t>& sb = nd.cb >= 0 ? p.vstride[nd.cb] : nones;
    for (size_t i = 0; i < la.size(); ++i)
        if (!pow2(d.dims[la[i]]) || !pow2(sa[i])) return false;
    for (size_t i = 0; i < lb.size(); ++i)
        if (!pow2(d.dims[lb[i]]) || !pow2(sb[i])) return false;
    TileArgs t;
    memset(&t, 0, sizeof(t));
    auto push = [&](uint8_t* arr, int& nbits, int l, int64_t stride) -> bool {
        const int j = ilog2(d.dims[l]);
        for (int r = 0; r < j; ++r) {
            if (nbits >= kMaxBits) return false;
            arr[nbits++] = stride ? (uint8_t)(ilog2(stride) + r) : kNoBit;
        }
        return true;
    };
    // batch, M, N: fastest label first (the lists are slowest first)
    int nb2 = 0;
    for (auto it = nd.gb.rbegin(); it != nd.gb.rend(); ++it) {
        int tmp = t.nb;
        if (!push(t.a_b, t.nb, *it, stride_in(la, sa, *it))) return false;
        if (!push(t.b_b, tmp, *it, stride_in(lb, sb, *it))) return false;
        nb2 = tmp;
    }
    (void)nb2;
    for (auto it = nd.gm.rbegin(); it != nd.gm.rend(); ++it)
        if (!push(t.a_m, t.nm, *it, stride_in(la, sa, *it))) return false;
    for (auto it = nd.gn.rbegin(); it != nd.gn.rend(); ++it)
        if (!push(t.b_n, t.nn, *it, stride_in(lb, sb, *it))) return false;
    // K (shared and summed-only labels): order by the stride of the operand
    // whose fastest label is a K label, so its loads stay contiguous
    std::vector<int> ks = nd.gk;
    ks.insert(ks.end(), nd.gsa.begin(), nd.gsa.end());
    ks.insert(ks.end(), nd.gsb.begin(), nd.gsb.end());
    auto fastest = [&](const std::vector<int>& lab, const std::vector<int64_t>& st) {
        int best = -1;
        int64_t bs = INT64_MAX;
        for (size_t i = 0; i < lab.size(); ++i)
            if (d.dims[lab[i]] > 1 && st[i] < bs) {
                bs = st[i];
                best = lab[i];
            }
        return best;
    };
    const int fa = fastest(la, sa), fb = fastest(lb, sb);
    const bool fa_k = fa >= 0 && has(ks, fa), fb_k = fb >= 0 && has(ks, fb);
    // K follows the strides of the operand that needs it for contiguous
    // loads; when both or neither do, the larger operand wins
    int64_t size_a = 1, size_b = 1;
    for (int l : la) size_a *= d.dims[l];
    for (int l : lb) size_b *= d.dims[l];
    const bool by_a = (fa_k && !fb_k) || (fa_k == fb_k && size_a > size_b);
    const int64_t big = INT64_MAX / 4;
    std::sort(ks.begin(), ks.end(), [&](int x, int y) {
        int64_t sx = by_a ? stride_in(la, sa, x) : stride_in(lb, sb, x);
        int64_t sy = by_a ? stride_in(la, sa, y) : stride_in(lb, sb, y);
        if (!sx) sx = big;
        if (!sy) sy = big;
        return sx < sy;
    });
    for (int l : ks) {
        int tmp = t.nk;
        if (!push(t.a_k, t.nk, l, stride_in(la, sa, l))) return false;
        if (!push(t.b_k, tmp, l, stride_in(lb, sb, l))) return false;
    }
    if (t.nb > 16 || t.nm > 31 || t.nn > 31 || t.nk > 40 || t.nm + t.nn > 40) return false;
    // the kernels keep per-thread operand offsets in 32 bits
    for (const std::vector<int>* lab : {&la, &lb}) {
        int64_t sz = 1;
        for (int l : *lab) sz *= d.dims[l];
        if (sz >= (int64_t(1) << 31)) return false;
    }
    t.nbatch = int64_t(1) << t.nb;
    t.a_mfast = fa >= 0 && has(nd.gm, fa);
    t.b_nfast = fb >= 0 && has(nd.gn, fb);
    const int64_t M = int64_t(1) << t.nm, N = int64_t(1) << t.nn, K = int64_t(1) << t.nk;
    int TM = 64, TN = 64, TK = 16;
    const bool dot = M * N <= 64 && K >= 512;
    if (force_cfg >= kTile64x64 && force_cfg <= kTile128x64 && force_cfg != kTileDot && !dot) {
        // a shape forced by the autotuner (any shape is valid: tiles clip)
        static const int shapes[7][3] = {{0, 0, 0},    {64, 64, 16},   {16, 256, 16}, {4, 1024, 4},
                                         {256, 16, 16}, {0, 0, 0},      {128, 64, 16}};
        t.cfg = force_cfg;
        TM = shapes[force_cfg][0];
        TN = shapes[force_cfg][1];
        TK = shapes[force_cfg][2];
    } else if (dot) {
        t.cfg = kTileDot;
        TM = (int)M;
        TN = (int)N;
    } else if (t.nm <= 2 && t.nn >= 10) {
        t.cfg = kTile4x1024;
        TM = 4;
        TN = 1024;
        TK = 4;
    } else if (t.nm <= 5 && t.nn >= 8) {  // 64-row tiles would run half empty at M = 32
        t.cfg = kTile16x256;
        TM = 16;
        TN = 256;
    } else if (t.nn <= 5 && t.nm >= 8) {
        t.cfg = kTile256x16;
        TM = 256;
        TN = 16;
    } else {
        t.cfg = kTile64x64;
    }
    t.split = 1;
    t.kchunk = K;
    if (t.cfg != kTileDot) {
        const int64_t tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN) * t.nbatch;
        const int64_t ktiles = (K + TK - 1) / TK;
        int split = 1;
        while (tiles * p.copies * split < 2 * sm_count() && split * 16 <= ktiles && split < 64 &&
               t.nbatch * split * 2 <= 65535)
            split *= 2;
        t.split = split;
        t.kchunk = ((ktiles + split - 1) / split) * TK;
        if (split > 1) split_elems = std::max(split_elems, (int64_t)split * t.nbatch * M * N);
    } else {
        if (t.nbatch > 65535) return false;
        const int64_t outs = M * N * t.nbatch;
        int split = 1;
        // one K tile (1024 entries) or more per part; at least eight parts per
        // SM in all (several CTAs per SM keep enough loads in flight for HBM)
        while (outs * p.copies * split < 8 * (int64_t)sm_count() && (K / (split * 2)) >= 1024 &&
               split < 4096 && (int64_t)split * 2 * p.copies <= 65535)
            split *= 2;
        t.split = split;
        t.kchunk = ((K / split + 255) / 256) * 256;
        if (split > 1) split_elems = std::max(split_elems, (int64_t)split * outs);
    }
    t.a_leaf = nd.ca >= 0 && nd.ca < d.n ? nd.ca : -1;
    t.b_leaf = nd.cb >= 0 && nd.cb < d.n ? nd.cb : -1;
    nd.tile = t;
    nd.kind = kTiled;
    return true;
}

}  // namespace

// A node contracting vertices a and b (tree ids, -1 = the unit scalar) into
// the labels in keep: label groups and the [batch][M][N] output layout.
// The larger operand takes the B role (its labels are the fastest).
Node build_node(const NetDesc& d, const Plan& p, int id, int a, int b, const std::vector<int>& keep) {
    auto log2size = [&](const std::vector<int>& lab) {
        double s = 0;
        for (int l : lab) s += std::log2((double)d.dims[l]);
        return s;
    };
    // a, b: tree ids or -1 (unit scalar: no labels)
    static const std::vector<int> none;
    static const std::vector<int64_t> nones;
    const std::vector<int>& la = a >= 0 ? p.vlab[a] : none;
    const std::vector<int>& lb = b >= 0 ? p.vlab[b] : none;
    const std::vector<int64_t>& sa = a >= 0 ? p.vstride[a] : nones;
    const std::vector<int64_t>& sb = b >= 0 ? p.vstride[b] : nones;
    int64_t size_a = 1, size_b = 1;
    for (int l : la) size_a *= d.dims[l];
    for (int l : lb) size_b *= d.dims[l];
    // role: the larger operand takes the B (inner, fastest output) role
    bool swap = size_a > size_b;
    Node nd;
    nd.id = id;
    nd.ca = swap ? b : a;
    nd.cb = swap ? a : b;
    const std::vector<int>& A = swap ? lb : la;
    const std::vector<int>& B = swap ? la : lb;
    const std::vector<int64_t>& SA = swap ? sb : sa;
    const std::vector<int64_t>& SB = swap ? sa : sb;
    for (int l : A) {
        bool inb = has(B, l), kept = has(keep, l);
        if (inb && kept) nd.gb.push_back(l);
        else if (inb) nd.gk.push_back(l);
        else if (kept) nd.gm.push_back(l);
        else nd.gsa.push_back(l);
    }
    for (int l : B) {
        if (has(A, l)) continue;
        if (has(keep, l)) nd.gn.push_back(l);
        else nd.gsb.push_back(l);
    }
    auto by_desc = [&](const std::vector<int64_t>& S, const std::vector<int>& lab) {
        return [&](int x, int y) { return stride_in(lab, S, x) > stride_in(lab, S, y); };
    };
    std::sort(nd.gb.begin(), nd.gb.end(), by_desc(SA, A));
    std::sort(nd.gm.begin(), nd.gm.end(), by_desc(SA, A));
    std::sort(nd.gn.begin(), nd.gn.end(), by_desc(SB, B));
    std::sort(nd.gk.begin(), nd.gk.end(), by_desc(SB, B));
    nd.lab = nd.gb;
    nd.lab.insert(nd.lab.end(), nd.gm.begin(), nd.gm.end());
    nd.lab.insert(nd.lab.end(), nd.gn.begin(), nd.gn.end());
    nd.stride.assign(nd.lab.size(), 1);
    nd.size = 1;
    for (int i = (int)nd.lab.size() - 1; i >= 0; --i) {
        nd.stride[i] = nd.size;
        nd.size *= d.dims[nd.lab[i]];
    }
    std::vector<int> uni = A;
    for (int l : B)
        if (!has(uni, l)) uni.push_back(l);
    nd.vc = log2size(uni);
    return nd;
}

// Work items of a node in the persistent launch (per instance).
static int64_t persistent_items(const Node& nd) {
    if (nd.tile.cfg == kTile64x64 && tile_item_node(nd)) {
        const int64_t M = int64_t(1) << nd.tile.nm, N = int64_t(1) << nd.tile.nn;
        return ((M + 63) / 64) * ((N + 63) / 64) * nd.tile.nbatch;
    }
    const int64_t chunk = wave_chunk(nd, 2);
    return (nd.size + chunk - 1) / chunk;
}

tn_status build_plan(const NetDesc& d, Plan& p, std::string& err) {
    const int n = d.n;
    // diagnostics: TN_FORCE_GENERIC=1 runs every node on the generic kernel,
    // TN_NO_WAVES=1 launches every node separately, TN_NO_FLOW=1 one launch
    // per wave level
    if (const char* e = getenv("TN_FORCE_GENERIC")) p.force_generic = e[0] == '1';
    if (const char* e = getenv("TN_NO_WAVES")) p.no_waves = e[0] == '1';
    if (const char* e = getenv("TN_NO_FLOW")) p.no_flow = e[0] == '1';
    if (const char* e = getenv("TN_NO_TENSOR_CORES")) p.no_tensor_cores = e[0] == '1';
    const int L = (int)d.dims.size();
    // ---- tree validation (Sec. 2: leaves first, children before parents)
    if ((int64_t)p.pairs.size() != 2 * (int64_t)(n - 1)) {
        err = "tree must have n_tensors-1 pairs";
        return TN_EINVAL;
    }
    std::vector<char> used(2 * n, 0);
    for (int k = 0; k < n - 1; ++k) {
        int me = n + k;
        for (int j = 0; j < 2; ++j) {
            int c = p.pairs[2 * k + j];
            if (c < 0 || c >= me) {
                err = "tree child id out of range";
                return TN_EINVAL;
            }
            if (used[c]) {
                err = "tree id used twice";
                return TN_EINVAL;
            }
            used[c] = 1;
        }
    }
    // ---- sliced labels (Sec. 4.7.1)
    std::vector<char> is_open(L, 0), is_sl(L, 0);
    for (int l : d.open) is_open[l] = 1;
    p.sliced.clear();
    p.d_sliced = 1;
    for (int64_t id : p.sliced_ids) {
        auto it = d.id2d.find(id);
        if (it == d.id2d.end()) {
            err = "unknown sliced label";
            return TN_EINVAL;
        }
        int l = it->second;
        if (is_open[l]) {
            err = "sliced label is open";
            return TN_EINVAL;
        }
        if (is_sl[l]) {
            err = "sliced label repeated";
            return TN_EINVAL;
        }
        is_sl[l] = 1;
        p.sliced.push_back(l);
        if (p.d_sliced > (INT64_MAX / 4) / d.dims[l]) {
            err = "too many slices";
            return TN_EUNSUPPORTED;
        }
        p.d_sliced *= d.dims[l];
    }
    const int ns = (int)p.sliced.size();
    std::vector<int64_t> sdiv(ns, 1);
    for (int j = ns - 2; j >= 0; --j) sdiv[j] = sdiv[j + 1] * d.dims[p.sliced[j + 1]];

    // ---- per-vertex labels after slicing
    const int NV = 2 * n - 1;
    p.vlab.assign(NV, {});
    p.vstride.assign(NV, {});
    p.leaf_sl.assign(n, SliceDigits{});
    std::vector<int> total(L, 0);
    std::vector<SubCount> sub(NV);
    for (int v = 0; v < n; ++v) {
        const LeafDesc& lf = d.leaves[v];
        SliceDigits& sd = p.leaf_sl[v];
        sd.n = 0;
        for (size_t i = 0; i < lf.lab.size(); ++i) {
            int l = lf.lab[i];
            if (is_sl[l]) {
                if (sd.n >= kMaxSliceDigits) {
                    err = "too many sliced labels in one tensor";
                    return TN_EUNSUPPORTED;
                }
                int j = (int)(std::find(p.sliced.begin(), p.sliced.end(), l) - p.sliced.begin());
                sd.div[sd.n] = sdiv[j];
                sd.dim[sd.n] = d.dims[l];
                sd.stride[sd.n] = lf.stride[i];
                sd.n++;
                continue;
            }
            p.vlab[v].push_back(l);
            p.vstride[v].push_back(lf.stride[i]);
            total[l]++;
            sub[v].c.push_back({l, 1});
        }
    }
    // ---- nodes
    p.nodes.clear();
    double W = 0, C = 0;
    auto log2size = [&](const std::vector<int>& lab) {
        double s = 0;
        for (int l : lab) s += std::log2((double)d.dims[l]);
        return s;
    };
    for (int v = 0; v < n; ++v) W = std::max(W, log2size(p.vlab[v]));
    auto make_node = [&](int id, int a, int b, const std::vector<int>& keep) -> Node {
        return build_node(d, p, id, a, b, keep);
    };
    if (n == 1) {
        std::vector<int> keep = d.open;
        Node nd = make_node(n, 0, -1, keep);
        // the unit operand is smaller: make sure the leaf is an operand
        p.vlab.push_back(nd.lab);
        p.vstride.push_back(nd.stride);
        W = std::max(W, log2size(nd.lab));
        // one leaf has no contraction vertex, so C = 0 (Sec. 2); the node
        // only sums the leaf's own summed labels and orders the open axes
        p.nodes.push_back(nd);
    } else {
        for (int k = 0; k < n - 1; ++k) {
            int a = p.pairs[2 * k], b = p.pairs[2 * k + 1], me = n + k;
            std::vector<int> keep;
            SubCount sc;
            auto visit = [&](int c, int other) {
                for (auto& x : sub[c].c) {
                    int l = x.first;
                    if (c == b && sub[a].get(l)) continue;
                    int cnt = x.second + (c == a ? sub[b].get(l) : 0);
                    if (is_open[l] || cnt < total[l]) {
                        keep.push_back(l);
                        sc.c.push_back({l, cnt});
                    }
                }
                (void)other;
            };
            visit(a, b);
            visit(b, a);
            // sizes are formed in int64 below: refuse what could overflow them
            std::vector<int> uni = p.vlab[a];
            for (int l : p.vlab[b])
                if (std::find(uni.begin(), uni.end(), l) == uni.end()) uni.push_back(l);
            if (log2size(keep) > kMaxLog2Entries) {
                err = "an intermediate of the sliced tree has more than 2^40 entries";
                return TN_EUNSUPPORTED;
            }
            if (log2size(uni) > kMaxLog2Work) {
                err = "a node of the sliced tree needs more than 2^62 multiply-adds";
                return TN_EUNSUPPORTED;
            }
            sub[me] = sc;
            sub[a].c.clear();
            sub[b].c.clear();
            Node nd = make_node(me, a, b, keep);
            p.vlab[me] = nd.lab;
            p.vstride[me] = nd.stride;
            W = std::max(W, log2size(nd.lab));
            C += std::pow(2.0, nd.vc);
            p.nodes.push_back(nd);
        }
    }
    // root labels must be exactly the open labels
    const Node& root = p.nodes.back();
    if (root.lab.size() != d.open.size()) {
        err = "internal: root labels differ from the open labels";
        return TN_EINVAL;
    }
    p.W = W;
    p.C = C;
    // ---- kernel choice per node: large GEMM-shaped nodes go to the tensor
    // cores in the reduced-precision modes (M >= 128 rows, N >= 128 real
    // accumulator columns, K >= 16); everything else on CUDA cores
    int64_t split_elems = 0;
    for (size_t k = 0; k < p.nodes.size(); ++k) {
        Node& nd = p.nodes[k];
        nd.kind = kGeneric;
        if (p.force_generic || !plan_tile(d, p, nd, split_elems)) {
            if (p.persistent) {
                err = "the persistent launch needs power-of-two label sizes on every node";
                return TN_EUNSUPPORTED;
            }
            continue;
        }
        if (p.persistent) {
            // tile items: 64 x 64 tiles, all of K in one item (no K split)
            if (tile_item_node(nd)) {
                int64_t unused = 0;
                Node t = nd;
                if (plan_tile(d, p, t, unused, kTile64x64)) {
                    t.tile.split = 1;
                    t.tile.kchunk = int64_t(1) << t.tile.nk;
                    nd = t;
                }
            }
            continue;
        }
        if (!p.no_tensor_cores) make_tensor_core(d, p.mode, nd, split_elems, p.copies);
    }
    p.split_bytes = (split_elems * (int64_t)d.elem_bytes() + 1023) / 1024 * 1024;
    // ---- launch schedule: tree levels; per level one wave launch for the
    // small tiled nodes, then one launch per remaining node
    std::vector<int> level(2 * n, 0);
    int max_level = 0;
    for (size_t k = 0; k < p.nodes.size(); ++k) {
        const Node& nd = p.nodes[k];
        int la = nd.ca >= n ? level[nd.ca] : 0, lb = nd.cb >= n ? level[nd.cb] : 0;
        level[n + k] = 1 + std::max(la, lb);
        max_level = std::max(max_level, level[n + k]);
    }
    p.steps.clear();
    p.items.clear();
    if (p.persistent) {
        // one dataflow launch over the whole tree, level by level
        Step w;
        w.wave = 1;
        w.flow = 1;
        w.item_begin = 0;
        for (int L = 1; L <= max_level; ++L)
            for (size_t k = 0; k < p.nodes.size(); ++k) {
                if (level[n + k] != L) continue;
                const Node& nd = p.nodes[k];
                const int64_t cnt = persistent_items(nd);
                for (int64_t i = 0; i < cnt; ++i) {
                    WaveItem it;
                    it.node = (int)k;
                    it.pad = 0;
                    if (nd.tile.cfg == kTile64x64 && tile_item_node(nd)) {
                        it.o_begin = i;
                        it.o_count = -1;
                    } else {
                        const int64_t chunk = wave_chunk(nd, 2);
                        it.o_begin = i * chunk;
                        it.o_count = std::min(chunk, nd.size - i * chunk);
                    }
                    p.items.push_back(it);
                }
                w.nodes.push_back((int)k);
            }
        w.item_count = (int)p.items.size();
        if ((int64_t)p.items.size() > (int64_t(1) << 30)) {
            err = "the persistent launch would need more than 2^30 work items";
            return TN_EUNSUPPORTED;
        }
        p.steps.push_back(w);
    }
    for (int L = 1; L <= max_level && !p.persistent; ++L) {
        Step w;
        w.wave = 1;
        w.item_begin = (int)p.items.size();
        std::vector<int> singles;
        for (size_t k = 0; k < p.nodes.size(); ++k) {
            if (level[n + k] != L) continue;
            const Node& nd = p.nodes[k];
            const bool small = wave_node(nd, p.copies) && !p.no_waves;
            if (!small) {
                singles.push_back((int)k);
                continue;
            }
            const int64_t chunk = wave_chunk(nd, p.copies);
            for (int64_t o = 0; o < nd.size; o += chunk) {
                WaveItem it;
                it.node = (int)k;
                it.pad = 0;
                it.o_begin = o;
                it.o_count = chunk;
                p.items.push_back(it);
            }
            w.nodes.push_back((int)k);
        }
        w.item_count = (int)p.items.size() - w.item_begin;
        if (w.item_count > 0) p.steps.push_back(w);
        for (int k : singles) {
            Step s;
            s.node = k;
            s.nodes.push_back(k);
            p.steps.push_back(s);
        }
    }
    // ---- consecutive wave levels become one dataflow launch (their items
    // are contiguous); a node waits for its children in the same launch
    if (!p.no_flow && !p.persistent) {
        std::vector<Step> merged;
        for (Step& st : p.steps) {
            if (st.wave && !merged.empty() && merged.back().wave &&
                merged.back().item_begin + merged.back().item_count == st.item_begin) {
                Step& m = merged.back();
                m.item_count += st.item_count;
                m.nodes.insert(m.nodes.end(), st.nodes.begin(), st.nodes.end());
                m.flow = 1;
            } else {
                merged.push_back(st);
            }
        }
        p.steps = merged;
    }
    p.flow_deps.assign(4 * p.nodes.size(), -1);
    for (const Step& st : p.steps) {
        if (!st.flow) continue;
        std::vector<char> in_step(p.nodes.size(), 0);
        for (int k : st.nodes) in_step[k] = 1;
        for (int k : st.nodes) {
            const Node& nd = p.nodes[k];
            int slot = 0;
            for (int c : {nd.ca, nd.cb}) {
                if (c >= n && in_step[c - n]) {
                    const Node& ch = p.nodes[c - n];
                    const int64_t chunk = wave_chunk(ch, p.copies);
                    p.flow_deps[4 * k + 2 * slot] = c - n;
                    p.flow_deps[4 * k + 2 * slot + 1] =
                        p.persistent ? (int)persistent_items(ch) : (int)((ch.size + chunk - 1) / chunk);
                }
                ++slot;
            }
        }
    }
    // ---- workspace liveness in execution order: a step's outputs are all
    // allocated before any of its operands is released (they run at once)
    Arena ar;
    for (const Step& st : p.steps) {
        for (int k : st.nodes) p.nodes[k].ws_off = ar.alloc(p.nodes[k].size);
        for (int k : st.nodes)
            for (int c : {p.nodes[k].ca, p.nodes[k].cb})
                if (c >= n) {
                    const Node& ch = p.nodes[c - n];
                    ar.release(ch.ws_off, ch.size);
                }
    }
    p.ws_elems = std::max<int64_t>(ar.end, 64);
    p.n_out = 1;
    for (int l : d.open) p.n_out *= d.dims[l];
    return TN_OK;
}

static tn_status fill_generic(const NetDesc& d, const Plan& p, const Node& nd, GenericArgs& g,
                              std::string& err) {
    memset(&g, 0, sizeof(g));
    const int n = d.n;
    static const std::vector<int> none;
    static const std::vector<int64_t> nones;
    const std::vector<int>& la = nd.ca >= 0 ? p.vlab[nd.ca] : none;
    const std::vector<int>& lb = nd.cb >= 0 ? p.vlab[nd.cb] : none;
    const std::vector<int64_t>& sa = nd.ca >= 0 ? p.vstride[nd.ca] : nones;
    const std::vector<int64_t>& sb = nd.cb >= 0 ? p.vstride[nd.cb] : nones;
    if ((int)nd.lab.size() > kMaxDigits) {
        err = "node rank exceeds the generic kernel limit";
        return TN_EUNSUPPORTED;
    }
    g.n_out = nd.size;
    g.n_od = (int)nd.lab.size();
    for (int i = 0; i < g.n_od; ++i) {
        int l = nd.lab[nd.lab.size() - 1 - i];
        g.od_dim[i] = (int32_t)d.dims[l];
        g.od_sa[i] = stride_in(la, sa, l);
        g.od_sb[i] = stride_in(lb, sb, l);
    }
    std::vector<int> ks = nd.gk;
    ks.insert(ks.end(), nd.gsa.begin(), nd.gsa.end());
    ks.insert(ks.end(), nd.gsb.begin(), nd.gsb.end());
    std::sort(ks.begin(), ks.end(), [&](int x, int y) {
        return stride_in(lb, sb, x) + stride_in(la, sa, x) < stride_in(lb, sb, y) + stride_in(la, sa, y);
    });
    if ((int)ks.size() > kMaxDigits) {
        err = "too many summed labels in one node";
        return TN_EUNSUPPORTED;
    }
    g.n_kd = (int)ks.size();
    g.n_sum = 1;
    for (int i = 0; i < g.n_kd; ++i) {
        int l = ks[i];
        g.kd_dim[i] = (int32_t)d.dims[l];
        g.kd_sa[i] = stride_in(la, sa, l);
        g.kd_sb[i] = stride_in(lb, sb, l);
        g.n_sum *= d.dims[l];
    }
    if (nd.ca >= 0 && nd.ca < n) g.sla = p.leaf_sl[nd.ca];
    if (nd.cb >= 0 && nd.cb < n) g.slb = p.leaf_sl[nd.cb];
    return TN_OK;
}

tn_status alloc_plan(NetDesc& d, Plan& p, void* unit, std::string& err) {
    const size_t eb = d.elem_bytes();
    const int nn = (int)p.nodes.size();
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess) {
            err = std::string(what) + ": " + cudaGetErrorString(e);
            return false;
        }
        return true;
    };
    const int G = std::max(p.alloc_inst, 1);
    if (!ck(cudaMalloc(&p.ws, (size_t)p.ws_elems * eb * G), "workspace allocation")) return TN_ENOMEM;
    // node maxima of every instance, then the dataflow counters (done per
    // node and instance, one item head per step): one region, cleared by one
    // memset per slice
    const size_t flow_cnt = (size_t)nn * G + p.steps.size() + 1;
    if (!ck(cudaMalloc(&p.maxabs, sizeof(unsigned) * ((size_t)nn * G + flow_cnt)), "cudaMalloc"))
        return TN_ENOMEM;
    p.flow_cnt_dev = p.maxabs + (size_t)nn * G;
    if (!ck(cudaMalloc(&p.exps, sizeof(int64_t) * nn * G), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&p.inst_roots_dev, sizeof(BatchRoot) * G), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&p.inst_out_dev, sizeof(double) * 2 * G), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&p.inst_exp_dev, sizeof(int64_t) * G), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&p.ctl, sizeof(Control)), "cudaMalloc")) return TN_ENOMEM;
    size_t acc_doubles = (size_t)p.n_out * (d.is_complex() ? 2 : 1);
    if (!ck(cudaMalloc(&p.acc, sizeof(double) * acc_doubles), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&p.out_stage, sizeof(double) * (acc_doubles + 1)), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking), "stream")) return TN_ECUDA;
    if (!ck(cudaMalloc(&p.leafmax, sizeof(unsigned) * d.n), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc((void**)&p.leaf_ptr_dev, sizeof(void*) * d.n), "cudaMalloc")) return TN_ENOMEM;
    if (!ck(cudaMalloc(&p.leaf_nfloat_dev, sizeof(int64_t) * d.n), "cudaMalloc")) return TN_ENOMEM;
    {
        std::vector<int64_t> nf(d.n);
        for (int v = 0; v < d.n; ++v) nf[v] = d.leaves[v].size * (d.is_complex() ? 2 : 1);
        if (!ck(cudaMemcpy(p.leaf_nfloat_dev, nf.data(), sizeof(int64_t) * d.n,
                           cudaMemcpyHostToDevice), "cudaMemcpy"))
            return TN_ECUDA;
        p.leaf_nfloat_uploaded = nf;
    }
    if (p.split_bytes > 0 && !ck(cudaMalloc(&p.split_buf, p.split_bytes * G), "split-K buffer"))
        return TN_ENOMEM;
    // node launch arguments; leaf pointers are patched per call
    p.gen.resize(nn);
    const int n = d.n;
    for (int k = 0; k < nn; ++k) {
        const Node& nd = p.nodes[k];
        GenericArgs& g = p.gen[k];
        tn_status st = fill_generic(d, p, nd, g, err);
        if (st != TN_OK) return st;
        char* ws = (char*)p.ws;
        g.C = ws + nd.ws_off * eb;
        g.A = nd.ca >= n ? (const void*)(ws + p.nodes[nd.ca - n].ws_off * eb) : nullptr;
        g.B = nd.cb >= n ? (const void*)(ws + p.nodes[nd.cb - n].ws_off * eb) : nullptr;
        if (nd.ca < 0) g.A = unit;
        if (nd.cb < 0) g.B = unit;
        g.ctl = p.ctl;
        // leaves: renormalised by their own max, stored exponent 0
        g.sc.max_a = nd.ca >= n ? p.maxabs + (nd.ca - n) : (nd.ca >= 0 ? p.leafmax + nd.ca : nullptr);
        g.sc.exp_a = nd.ca >= n ? p.exps + (nd.ca - n) : nullptr;
        g.sc.max_b = nd.cb >= n ? p.maxabs + (nd.cb - n) : (nd.cb >= 0 ? p.leafmax + nd.cb : nullptr);
        g.sc.exp_b = nd.cb >= n ? p.exps + (nd.cb - n) : nullptr;
        g.sc.max_c = p.maxabs + k;
        g.sc.exp_c = p.exps + k;
        Node& ndm = p.nodes[k];
        if (ndm.kind == kTiled || ndm.kind == kTensorCore) {
            TileArgs& t = ndm.tile;
            t.A = g.A;
            t.B = g.B;
            t.C = g.C;
            t.P = p.split_buf;
            t.sla = g.sla;
            t.slb = g.slb;
            t.ctl = g.ctl;
            t.sc = g.sc;
        }
    }
    {
        // dataflow waves: dependencies, and completion / item counters
        if (!ck(cudaMalloc(&p.flow_deps_dev, sizeof(int) * 4 * std::max(nn, 1)), "cudaMalloc")) return TN_ENOMEM;
        if (!ck(cudaMemcpy(p.flow_deps_dev, p.flow_deps.data(), sizeof(int) * p.flow_deps.size(),
                           cudaMemcpyHostToDevice), "cudaMemcpy"))
            return TN_ECUDA;
    }
    if (!p.items.empty()) {
        std::vector<TileArgs> descs(nn);
        for (int k = 0; k < nn; ++k) descs[k] = p.nodes[k].tile;
        if (!ck(cudaMalloc(&p.descs_dev, sizeof(TileArgs) * nn), "cudaMalloc")) return TN_ENOMEM;
        if (!ck(cudaMalloc(&p.items_dev, sizeof(WaveItem) * p.items.size() * G), "cudaMalloc"))
            return TN_ENOMEM;
        if (!ck(cudaMemcpy(p.descs_dev, descs.data(), sizeof(TileArgs) * nn, cudaMemcpyHostToDevice),
                "cudaMemcpy"))
            return TN_ECUDA;
        if (!ck(cudaMemcpy(p.items_dev, p.items.data(), sizeof(WaveItem) * p.items.size(),
                           cudaMemcpyHostToDevice),
                "cudaMemcpy"))
            return TN_ECUDA;
    }
    // root accumulation: user open-label order -> root layout
    const Node& root = p.nodes.back();
    AccumArgs& a = p.acc_args;
    memset(&a, 0, sizeof(a));
    a.R = (char*)p.ws + root.ws_off * eb;
    a.n_out = p.n_out;
    a.n_od = (int)d.open.size();
    if (a.n_od > kMaxDigits) {
        err = "too many open labels";
        return TN_EUNSUPPORTED;
    }
    for (int i = 0; i < a.n_od; ++i) {
        int l = d.open[d.open.size() - 1 - i];
        a.od_dim[i] = (int32_t)d.dims[l];
        a.od_s[i] = stride_in(root.lab, root.stride, l);
    }
    a.max_r = p.maxabs + (nn - 1);
    a.exp_r = p.exps + (nn - 1);
    a.acc = p.acc;
    a.ctl = p.ctl;
    a.n_inst = 1;
    a.r_is = p.ws_elems;
    a.s_is = nn;
    p.cfg_inst = -1;  // instance layout not yet written to the arguments
    return TN_OK;
}

// Write the instance layout (G instances; step 1: instance i = slice s+i,
// step 0: independent copies whose leaf v sits leaf_is[v] elements apart)
// into every node's launch arguments, the wave items and the accumulator.
static tn_status configure_instances(const NetDesc& d, Plan& p, int G, int step,
                                     const std::vector<int64_t>& leaf_is, std::string& err) {
    if (p.cfg_inst == G && p.cfg_step == step && p.cfg_leaf_is == leaf_is) return TN_OK;
    const int n = d.n;
    const int nn = (int)p.nodes.size();
    const int64_t p_is = p.split_bytes / (int64_t)d.elem_bytes();
    for (int k = 0; k < nn; ++k) {
        Node& nd = p.nodes[k];
        InstanceInfo in;
        memset(&in, 0, sizeof(in));
        in.n_inst = G;
        in.slice_step = step;
        in.c_is = p.ws_elems;
        in.sc_is = nn;
        in.p_is = p_is;
        auto set = [&](int c, int64_t& is, int32_t& sis) {
            if (c >= n) {
                is = p.ws_elems;
                sis = nn;
            } else if (c >= 0) {
                is = leaf_is.empty() ? 0 : leaf_is[c];
                sis = 0;
            }
        };
        set(nd.ca, in.a_is, in.sa_is);
        set(nd.cb, in.b_is, in.sb_is);
        p.gen[k].in = in;
        nd.tile.in = in;
        // the launch grid's z extent (batch x K splits x instances) is at most
        // 65535: fewer K splits when many instances run side by side
        if (!p.persistent && (nd.kind == kTiled || nd.kind == kTensorCore)) {
            TileArgs& t = nd.tile;
            if (t.nbatch * (int64_t)G > 65535) {
                err = "too many instances for a node with " + std::to_string(t.nbatch) + " batch entries";
                return TN_EUNSUPPORTED;
            }
            if (t.split > 1 && t.nbatch * (int64_t)t.split * G > 65535) {
                int split = t.split;
                while (split > 1 && t.nbatch * (int64_t)split * G > 65535) split /= 2;
                const int64_t K = int64_t(1) << t.nk;
                const int64_t gran = t.cfg == kTileDot ? 256 : (t.cfg == kTile4x1024 ? 4 : 16);
                const int64_t units = (K + gran - 1) / gran;
                t.split = split;
                t.kchunk = ((units + split - 1) / split) * gran;
            }
        }
        if (!p.persistent && nd.kind == kGeneric && G > 65535) {
            err = "too many instances";
            return TN_EUNSUPPORTED;
        }
    }
    if (!p.items.empty()) {
        std::vector<TileArgs> descs(nn);
        for (int k = 0; k < nn; ++k) descs[k] = p.nodes[k].tile;
        std::vector<WaveItem> items;
        items.reserve(p.items.size() * G);
        // within each step: level by level, every instance's items of a
        // level before the next level (the instances' dependency chains
        // advance together; a node's children always come earlier)
        std::vector<int> level(nn, 0);
        for (int k = 0; k < nn; ++k) {
            const Node& nd = p.nodes[k];
            const int la = nd.ca >= n ? level[nd.ca - n] : 0, lb = nd.cb >= n ? level[nd.cb - n] : 0;
            level[k] = 1 + std::max(la, lb);
        }
        p.inst_items_begin.assign(p.steps.size(), 0);
        for (size_t s = 0; s < p.steps.size(); ++s) {
            const Step& st = p.steps[s];
            p.inst_items_begin[s] = (int)items.size();
            if (!st.wave) continue;
            int j0 = 0;
            while (j0 < st.item_count) {
                const int L = level[p.items[st.item_begin + j0].node];
                int j1 = j0;
                while (j1 < st.item_count && level[p.items[st.item_begin + j1].node] == L) ++j1;
                for (int i = 0; i < G; ++i)
                    for (int j = j0; j < j1; ++j) {
                        WaveItem it = p.items[st.item_begin + j];
                        it.pad = i;
                        items.push_back(it);
                    }
                j0 = j1;
            }
        }
        cudaError_t e = cudaMemcpy(p.descs_dev, descs.data(), sizeof(TileArgs) * nn, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p.items_dev, items.data(), sizeof(WaveItem) * items.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            err = std::string("instance layout upload: ") + cudaGetErrorString(e);
            return TN_ECUDA;
        }
    }
    p.acc_args.n_inst = step == 1 ? G : 1;
    p.cfg_inst = G;
    p.cfg_step = step;
    p.cfg_leaf_is = leaf_is;
    return TN_OK;
}

// One launch group: reset the node maxima of all instances, run every node
// (each launch covers all instances), then either fold the instances' roots
// (consecutive slices) into the FP64 accumulator and advance the slice
// counter, or write each independent instance's root to its output.
// ev: optional timing events around launch steps [pf, pf + pc).
static cudaError_t enqueue_slice(const NetDesc& d, Plan& p, cudaStream_t s, const cudaEvent_t* ev,
                                 int pf, int pc) {
    const int G = std::max(p.cfg_inst, 1);
    const int nn = (int)p.nodes.size();
    bool any_flow = false;
    for (const Step& st : p.steps) any_flow |= st.flow != 0;
    // the node maxima and (dataflow) the counters that follow them
    const size_t n_zero = any_flow ? (size_t)(p.flow_cnt_dev - p.maxabs) + (size_t)nn * G + p.steps.size()
                                   : (size_t)nn * G;
    cudaError_t e = cudaMemsetAsync(p.maxabs, 0, sizeof(unsigned) * n_zero, s);
    if (e != cudaSuccess) return e;
    const bool c = d.is_complex();
    for (int k = 0; k < (int)p.steps.size(); ++k) {
        // External records become event-record nodes under stream capture.
        if (ev && k >= pf && k < pf + pc &&
            (e = cudaEventRecordWithFlags(ev[k - pf], s, cudaEventRecordExternal)) != cudaSuccess)
            return e;
        const Step& st = p.steps[k];
        if (st.wave) {
            if (st.flow)
                e = launch_wave(p.items_dev + p.inst_items_begin[k], st.item_count * G, p.descs_dev,
                                reinterpret_cast<const void* const*>(p.leaf_ptr_dev), c, s,
                                reinterpret_cast<const int4*>(p.flow_deps_dev), p.flow_cnt_dev,
                                p.flow_cnt_dev + (size_t)nn * G + k, G, p.persistent);
            else
                e = launch_wave(p.items_dev + p.inst_items_begin[k], st.item_count * G, p.descs_dev,
                                reinterpret_cast<const void* const*>(p.leaf_ptr_dev), c, s);
        } else {
            const Node& nd = p.nodes[st.node];
            if (nd.kind == kTensorCore)
                e = launch_tc(nd.tile, tc_prec_of_mode(p.mode),
                              c, s);
            else if (nd.kind == kTiled)
                e = launch_tile(nd.tile, c, s);
            else
                e = launch_generic(p.gen[st.node], c, s);
        }
        if (e != cudaSuccess) return e;
        if (ev && k == pf + pc - 1 &&
            (e = cudaEventRecordWithFlags(ev[pc], s, cudaEventRecordExternal)) != cudaSuccess)
            return e;
    }
    if (p.cfg_step == 0)
        return launch_batch_finish(p.inst_roots_dev, G, p.inst_out_dev, p.inst_exp_dev, nullptr, nullptr,
                                   nullptr, s);
    return launch_accumulate(p.acc_args, c, s, G);
}

#define CK(x)                                                     \
    do {                                                          \
        cudaError_t e_ = (x);                                     \
        if (e_ != cudaSuccess) {                                  \
            err = std::string(#x) + ": " + cudaGetErrorString(e_); \
            return e_ == cudaErrorMemoryAllocation ? TN_ENOMEM : TN_ECUDA; \
        }                                                         \
    } while (0)

// Leaf pointers of this call (host leaves are staged into library memory),
// patched into the node arguments and the device leaf table.
static tn_status prepare_leaves(NetDesc& d, Plan& p, bool capturing, std::vector<const void*>& lp,
                                cudaStream_t stream, std::string& err) {
    const int n = d.n;
    const size_t eb = d.elem_bytes();
    lp.assign(n, nullptr);
    // several host leaves outside capture: one page-locked image, one copy
    int n_host = 0;
    int64_t total = 0;
    for (int v = 0; v < n; ++v)
        if (d.leaves[v].mem == TN_MEM_HOST) {
            ++n_host;
            total += (d.leaves[v].size * (int64_t)eb + 15) / 16 * 16;
        }
    if (!capturing && n_host > 1) {
        if (d.stage_bytes < total) {
            if (d.stage_pending) CK(cudaEventSynchronize(d.stage_done));
            d.stage_pending = false;
            if (d.stage_host) CK(cudaFreeHost(d.stage_host));
            if (d.stage_dev) CK(cudaFree(d.stage_dev));
            d.stage_host = d.stage_dev = nullptr;
            d.stage_bytes = 0;
            CK(cudaMallocHost(&d.stage_host, total));
            CK(cudaMalloc(&d.stage_dev, total));
            d.stage_bytes = total;
            if (!d.stage_done) CK(cudaEventCreateWithFlags(&d.stage_done, cudaEventDisableTiming));
        }
        // the image may still be read by the previous call's copy
        if (d.stage_pending) CK(cudaEventSynchronize(d.stage_done));
        int64_t off = 0;
        for (int v = 0; v < n; ++v) {
            LeafDesc& lf = d.leaves[v];
            if (lf.mem == TN_MEM_HOST) {
                memcpy((char*)d.stage_host + off, lf.ptr, lf.size * eb);
                lp[v] = (char*)d.stage_dev + off;
                off += (lf.size * (int64_t)eb + 15) / 16 * 16;
            } else {
                lp[v] = lf.ptr;
            }
        }
        CK(cudaMemcpyAsync(d.stage_dev, d.stage_host, off, cudaMemcpyHostToDevice, stream));
        CK(cudaEventRecord(d.stage_done, stream));
        d.stage_pending = true;
    }
    for (int v = 0; v < n; ++v) {
        LeafDesc& lf = d.leaves[v];
        if (lf.mem == TN_MEM_HOST && lp[v]) continue;  // staged above
        if (lf.mem == TN_MEM_HOST) {
            int64_t bytes = std::max<int64_t>(lf.size * (int64_t)eb, 16);
            if (lf.staged_bytes < bytes) {
                if (capturing) {
                    err = "host leaves need a first call outside stream capture";
                    return TN_EUNSUPPORTED;
                }
                if (lf.staged) CK(cudaFree(lf.staged));
                lf.staged = nullptr;
                CK(cudaMalloc(&lf.staged, bytes));
                lf.staged_bytes = bytes;
            }
            CK(cudaMemcpyAsync(lf.staged, lf.ptr, lf.size * eb, cudaMemcpyHostToDevice, stream));
            lp[v] = lf.staged;
        } else {
            lp[v] = lf.ptr;
        }
    }
    for (size_t k = 0; k < p.nodes.size(); ++k) {
        Node& nd = p.nodes[k];
        if (nd.ca >= 0 && nd.ca < n) p.gen[k].A = nd.tile.A = lp[nd.ca];
        if (nd.cb >= 0 && nd.cb < n) p.gen[k].B = nd.tile.B = lp[nd.cb];
    }
    if (p.leaf_ptr_uploaded != lp) {
        // the pointer table changes only when leaves are re-attached
        CK(cudaMemcpyAsync(p.leaf_ptr_dev, lp.data(), sizeof(void*) * n, cudaMemcpyHostToDevice, stream));
        CK(cudaStreamSynchronize(stream));
        p.leaf_ptr_uploaded = lp;
    }
    return TN_OK;
}

// (Re)capture the per-group graph when the leaves, the timing hooks or the
// instance layout changed.
static tn_status ensure_graph(const NetDesc& d, Plan& p, const std::vector<const void*>& lp, int pf,
                              int pc, std::string& err) {
    const bool h = pc > 0;
    cudaGraph_t& graph = h ? p.graph_h : p.graph;
    cudaGraphExec_t& gexec = h ? p.gexec_h : p.gexec;
    std::vector<const void*>& gptrs = h ? p.graph_ptrs_h : p.graph_ptrs;
    int& gpf = h ? p.graph_prof_first_h : p.graph_prof_first;
    int& gpc = h ? p.graph_prof_count_h : p.graph_prof_count;
    int& ginst = h ? p.graph_inst_h : p.graph_inst;
    int& gstep = h ? p.graph_step_h : p.graph_step;
    if (gexec && gptrs == lp && gpf == pf && gpc == pc && ginst == p.cfg_inst && gstep == p.cfg_step)
        return TN_OK;
    if (gexec) CK(cudaGraphExecDestroy(gexec));
    if (graph) CK(cudaGraphDestroy(graph));
    gexec = nullptr;
    graph = nullptr;
    while ((int)p.prof_placeholder.size() < pc + 1) {
        cudaEvent_t ev;
        CK(cudaEventCreate(&ev));
        p.prof_placeholder.push_back(ev);
    }
    CK(cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_slice(d, p, p.cap_stream, pc ? p.prof_placeholder.data() : nullptr, pf, pc);
    cudaError_t e2 = cudaStreamEndCapture(p.cap_stream, &graph);
    CK(e);
    CK(e2);
    CK(cudaGraphInstantiate(&gexec, graph, 0));
    gptrs = lp;
    gpf = pf;
    gpc = pc;
    ginst = p.cfg_inst;
    gstep = p.cfg_step;
    if (!h) return TN_OK;
    p.prof_nodes.assign(pc + 1, nullptr);
    if (pc) {
        size_t nn = 0;
        CK(cudaGraphGetNodes(graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> all(nn);
        CK(cudaGraphGetNodes(graph, all.data(), &nn));
        for (auto g : all) {
            cudaGraphNodeType t;
            CK(cudaGraphNodeGetType(g, &t));
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(g, &ev));
            for (int i = 0; i <= pc; ++i)
                if (p.prof_placeholder[i] == ev) p.prof_nodes[i] = g;
        }
        for (auto g : p.prof_nodes)
            if (!g) {
                err = "internal: timing event node missing from the captured graph";
                return TN_ECUDA;
            }
    }
    return TN_OK;
}

static int64_t max_leaf_floats(const NetDesc& d) {
    int64_t m = 0;
    for (int v = 0; v < d.n; ++v) m = std::max(m, d.leaves[v].size * (d.is_complex() ? 2 : 1));
    return m;
}

static tn_status upload_leaf_sizes(const NetDesc& d, Plan& p, int G, const std::vector<int64_t>& leaf_is,
                                   std::string& err) {
    std::vector<int64_t> nf(d.n);
    for (int v = 0; v < d.n; ++v) {
        const int64_t is = leaf_is.empty() ? 0 : leaf_is[v];
        nf[v] = ((int64_t)(G - 1) * is + d.leaves[v].size) * (d.is_complex() ? 2 : 1);
    }
    if (nf == p.leaf_nfloat_uploaded) return TN_OK;
    CK(cudaMemcpy(p.leaf_nfloat_dev, nf.data(), sizeof(int64_t) * d.n, cudaMemcpyHostToDevice));
    p.leaf_nfloat_uploaded = nf;
    return TN_OK;
}

tn_status run_plan(NetDesc& d, Plan& p, void* unit, int64_t begin, int64_t count,
                   const tn_options& o, void* out, int out_mem, int64_t* out_exp2,
                   cudaStream_t stream, std::string& err) {
    (void)unit;
    const int n = d.n;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    // profiling hooks
    int pf = 0, pc = 0;
    const cudaEvent_t* uev = nullptr;
    if (o.prof_events && o.prof_count > 0) {
        pf = o.prof_first;
        pc = o.prof_count;
        if (pf < 0 || pf + pc > (int)p.steps.size()) {
            err = "profiling step range out of bounds";
            return TN_EINVAL;
        }
        uev = reinterpret_cast<const cudaEvent_t*>(o.prof_events);
    }
    // slices per launch group (instances); the device state was sized for it
    int G = o.slice_batch > 1 ? o.slice_batch : 1;
    if (G > count) G = (int)count;
    if (G > p.alloc_inst) {
        err = "internal: slice batch exceeds the allocated instances";
        return TN_ECUDA;
    }
    if (capturing && (p.cfg_inst != G || p.cfg_step != 1)) {
        err = "the first call with a new slice batch must run outside stream capture";
        return TN_EUNSUPPORTED;
    }
    tn_status st = configure_instances(d, p, G, 1, std::vector<int64_t>(), err);
    if (st != TN_OK) return st;
    if (!capturing) {
        st = upload_leaf_sizes(d, p, 1, std::vector<int64_t>(), err);
        if (st != TN_OK) return st;
    }
    std::vector<const void*> lp;
    st = prepare_leaves(d, p, capturing, lp, stream, err);
    if (st != TN_OK) return st;
    const int64_t n_acc = p.n_out * (d.is_complex() ? 2 : 1);
    CK(launch_call_begin(p.leaf_ptr_dev, p.leaf_nfloat_dev, p.leafmax, n, max_leaf_floats(d), p.ctl, begin,
                         begin + count, p.acc, n_acc, stream));
    const int64_t groups = (count + G - 1) / G;
    const bool use_graph = !o.no_graph && !capturing;
    if (use_graph) {
        st = ensure_graph(d, p, lp, pf, pc, err);
        if (st != TN_OK) return st;
        cudaGraphExec_t gx = pc ? p.gexec_h : p.gexec;
        for (int i = 0; i < pc + (pc ? 1 : 0); ++i)
            CK(cudaGraphExecEventRecordNodeSetEvent(gx, p.prof_nodes[i], uev[i]));
        for (int64_t s = 0; s < groups; ++s) CK(cudaGraphLaunch(gx, stream));
    } else {
        for (int64_t s = 0; s < groups; ++s) CK(enqueue_slice(d, p, stream, uev, pf, pc));
    }
    // the result: one launch to device outputs; to host outputs, one copy of
    // [accumulator | exponent] staged on the device
    if (out_mem == TN_MEM_HOST) {
        CK(launch_result(p.acc, n_acc, p.ctl, p.out_stage, reinterpret_cast<int64_t*>(p.out_stage + n_acc), stream));
        std::vector<double> host((size_t)n_acc + 1);
        CK(cudaMemcpyAsync(host.data(), p.out_stage, sizeof(double) * (n_acc + 1), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        std::memcpy(out, host.data(), sizeof(double) * n_acc);
        std::memcpy(out_exp2, host.data() + n_acc, sizeof(int64_t));
    } else {
        CK(launch_result(p.acc, n_acc, p.ctl, static_cast<double*>(out), out_exp2, stream));
    }
    return TN_OK;
}

tn_status run_instances(NetDesc& d, Plan& p, void* unit, int n_inst, const int64_t* leaf_is_arr,
                        double* out, int64_t* out_exp2, int out_mem, cudaStream_t stream,
                        std::string& err) {
    (void)unit;
    const int n = d.n;
    const int nn = (int)p.nodes.size();
    const size_t eb = d.elem_bytes();
    if (p.d_sliced != 1 || p.n_out != 1) {
        err = "tn_contract_instances: the network must be scalar and the tree unsliced";
        return TN_EUNSUPPORTED;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        err = "tn_contract_instances: not available during stream capture";
        return TN_EUNSUPPORTED;
    }
    const int G = n_inst;
    if (G > p.alloc_inst) {
        err = "internal: instances exceed the allocation";
        return TN_ECUDA;
    }
    std::vector<int64_t> leaf_is(n, 0);
    if (leaf_is_arr)
        for (int v = 0; v < n; ++v) leaf_is[v] = leaf_is_arr[v];
    tn_status st = configure_instances(d, p, G, 0, leaf_is, err);
    if (st != TN_OK) return st;
    st = upload_leaf_sizes(d, p, G, leaf_is, err);
    if (st != TN_OK) return st;
    if (p.inst_roots_n != G) {
        const Node& root = p.nodes.back();
        std::vector<BatchRoot> roots(G);
        for (int i = 0; i < G; ++i) {
            roots[i].root = (char*)p.ws + ((int64_t)i * p.ws_elems + root.ws_off) * eb;
            roots[i].exp = p.exps + (int64_t)i * nn + (nn - 1);
            roots[i].max = p.maxabs + (int64_t)i * nn + (nn - 1);
            roots[i].is_c = d.is_complex();
            roots[i].pad = 0;
        }
        CK(cudaMemcpy(p.inst_roots_dev, roots.data(), sizeof(BatchRoot) * G, cudaMemcpyHostToDevice));
        p.inst_roots_n = G;
    }
    std::vector<const void*> lp;
    st = prepare_leaves(d, p, false, lp, stream, err);
    if (st != TN_OK) return st;
    CK(launch_call_begin(p.leaf_ptr_dev, p.leaf_nfloat_dev, p.leafmax, n, max_leaf_floats(d), p.ctl, 0, 1, p.acc,
                         0, stream));
    st = ensure_graph(d, p, lp, 0, 0, err);
    if (st != TN_OK) return st;
    CK(cudaGraphLaunch(p.gexec, stream));
    cudaMemcpyKind kind = out_mem == TN_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(out, p.inst_out_dev, sizeof(double) * 2 * G, kind, stream));
    CK(cudaMemcpyAsync(out_exp2, p.inst_exp_dev, sizeof(int64_t) * G, kind, stream));
    if (out_mem == TN_MEM_HOST) CK(cudaStreamSynchronize(stream));
    return TN_OK;
}


tn_status make_generic_args_node(const NetDesc& d, const Plan& p, const Node& nd, GenericArgs& g,
                                 std::string& err) {
    return fill_generic(d, p, nd, g, err);
}

// Tensor-core choice for a tiled node in a reduced-precision mode: the
// GEMM tile needs >= 128 accumulator rows, >= 128 real accumulator columns
// (a complex node: >= 64, its 32 complex columns expand to 64 real ones that
// fill half of the 128-column tile, the rest is padding the epilogue drops)
// and K >= 16.  A complex node puts its larger
// operand in the row role (the column operand is expanded to two real rows
// per column).  The packed operands live in the shared P buffer, which
// grows to hold them.
bool make_tensor_core(const NetDesc& d, tn_mode mode, Node& nd, int64_t& split_elems, int copies) {
    TileArgs& t = nd.tile;
    if (mode == TN_MODE_FP32 || t.cfg == kTileDot || t.nk < 4 || t.nbatch > 65535) return false;
    const bool c = d.is_complex();
    int swap = 0;
    if (c) {
        if (std::max(t.nm, t.nn) < 7 || std::min(t.nm, t.nn) < 5) return false;
        swap = t.nn > t.nm ? 1 : 0;
    } else if (t.nm < 7 || t.nn < 7) {
        return false;
    }
    t.tc_swap = swap;
    t.split = 1;
    t.kchunk = int64_t(1) << t.nk;
    const int prec = tc_prec_of_mode(mode);
    // the planar layout (asked for by the autotuner's planar variant, or for
    // every eligible node by the diagnostic switch TN_PLANAR=1, read when a
    // plan is built) needs a complex node in a split precision with >= 128
    // complex rows and columns
    if (const char* e = getenv("TN_PLANAR"))
        if (e[0] == '1') t.tc_planar = 1;
    // 256-column GEMMs run on CTA pairs (pair MMA) where the row tiles pair
    // up; the diagnostic switch TN_NO_PAIR=1, read when a plan is built,
    // keeps the single-CTA GEMM
    t.tc_nopair = 0;
    if (const char* e = getenv("TN_NO_PAIR"))
        if (e[0] == '1') t.tc_nopair = 1;
    t.tc_planar = (t.tc_planar && c && (prec == 1 || prec == 2 || prec == 4) && t.nm >= 7 && t.nn >= 7 &&
                   !t.tc_bn128) ? 1 : 0;
    // K split: the grid should fill whole waves of the SMs (one CTA
    // each); split only while every part keeps >= 8 k-blocks
    {
        const TcGeom g0 = tc_geom(t, c, prec);
        const double tiles = (double)t.nbatch * (g0.rows_r / 128) * (g0.cols_q / g0.bn) * copies;
        double best = 0.0;
        for (int s = 1; s <= 16 && g0.nkb / s >= 8; s *= 2) {
            const double w = tiles * s / (double)sm_count();
            const double eff = w / std::ceil(w);
            if (eff > best + 0.03) {
                best = eff;
                t.split = s;
            }
        }
        if (t.nbatch * (int64_t)t.split > 65535) t.split = 1;
    }
    const int64_t eb = d.elem_bytes();
    split_elems = std::max(split_elems, (tc_geom(t, c, prec).total + eb - 1) / eb);
    nd.kind = kTensorCore;
    return true;
}

// ---- autotuner: the kernel of every node that runs alone in its launch
// step is chosen by timing each candidate on the device.
static cudaError_t launch_node(const NetDesc& d, const Plan& p, const Node& nd, cudaStream_t s) {
    if (nd.kind == kTensorCore)
        return launch_tc(nd.tile, tc_prec_of_mode(p.mode),
                         d.is_complex(), s);
    return launch_tile(nd.tile, d.is_complex(), s);
}

// Node k rebuilt as variant v (1..4: tile shape, kVariantTC: tensor core),
// keeping its device bindings; false if the variant does not apply.
static bool make_variant(const NetDesc& d, const Plan& p, int k, int v, Node& out, int64_t& split_elems,
                         int split_mult = 1) {
    const Node& nd = p.nodes[k];
    Node t = nd;
    const bool tcv = v == kVariantTC || v == kVariantTC128 || v == kVariantTCPlanar;
    if (!plan_tile(d, p, t, split_elems, tcv ? 0 : v)) return false;
    if (v == kVariantTC128) t.tile.tc_bn128 = 1;
    if (v == kVariantTCPlanar) t.tile.tc_planar = 1;
    if (t.tile.cfg == kTileDot) return false;
    t.kind = kTiled;
    if (tcv && !make_tensor_core(d, p.mode, t, split_elems)) return false;
    if (!tcv && split_mult > 1) {
        // finer K split: more blocks for short grids over long K (>= 2 K tiles each)
        TileArgs& a = t.tile;
        const int TK = a.cfg == kTile4x1024 ? 4 : 16;
        const int64_t K = int64_t(1) << a.nk, ktiles = (K + TK - 1) / TK;
        const int split = a.split * split_mult;
        if (split > 256 || ktiles / split < 2 || a.nbatch * (int64_t)split > 65535) return false;
        a.split = split;
        a.kchunk = ((ktiles + split - 1) / split) * TK;
        split_elems = std::max(split_elems, (int64_t)split * a.nbatch * (int64_t(1) << (a.nm + a.nn)));
    }
    TileArgs& a = t.tile;
    const TileArgs& o = nd.tile;
    a.A = o.A;
    a.B = o.B;
    a.C = o.C;
    a.P = o.P;
    a.sla = o.sla;
    a.slb = o.slb;
    a.ctl = o.ctl;
    a.sc = o.sc;
    a.conj_a = o.conj_a;
    a.conj_b = o.conj_b;
    a.t_done = o.t_done;
    a.in = o.in;
    out = t;
    return true;
}

tn_status autotune_plan(NetDesc& d, Plan& p, int reps, int32_t* choice, cudaStream_t s, std::string& err) {
    const int nn = (int)p.nodes.size();
    if (choice)
        for (int k = 0; k < nn; ++k) choice[k] = 0;
    if (reps < 1) reps = 1;
    // nodes that run alone in their step, on a tiled or tensor-core kernel
    std::vector<int> tune;
    for (const Step& st : p.steps)
        if (!st.wave) {
            const Node& nd = p.nodes[st.node];
            if ((nd.kind == kTiled && nd.tile.cfg != kTileDot) || nd.kind == kTensorCore) tune.push_back(st.node);
        }
    if (tune.empty()) return TN_OK;
    // bind this call's leaves (their values do not matter for timing)
    tn_status st = configure_instances(d, p, 1, 1, std::vector<int64_t>(), err);
    if (st != TN_OK) return st;
    st = upload_leaf_sizes(d, p, 1, std::vector<int64_t>(), err);
    if (st != TN_OK) return st;
    std::vector<const void*> lp;
    st = prepare_leaves(d, p, false, lp, s, err);
    if (st != TN_OK) return st;
    CK(launch_leaf_max(p.leaf_ptr_dev, p.leaf_nfloat_dev, p.leafmax, d.n, s, max_leaf_floats(d)));
    // candidates and the shared P buffer they need
    std::vector<std::vector<std::pair<int, Node>>> cand(nn);
    int64_t split_elems = 0;
    for (int k : tune) {
        const Node& nd = p.nodes[k];
        const int vc = nd.tile.nm + nd.tile.nn + nd.tile.nk + nd.tile.nb;  // log2 of the products
        Node tc;
        const bool has_tc = !p.no_tensor_cores && make_variant(d, p, k, kVariantTC, tc, split_elems);
        if (has_tc) {
            cand[k].push_back({kVariantTC, tc});
            if (tc.tile.split > 1) {  // the same GEMM without its K split (no reduction launch)
                Node t1 = tc;
                t1.tile.split = 1;
                cand[k].push_back({kVariantTC, t1});
            }
            // the planar layout (complex nodes in a split precision)
            Node tpl;
            if (make_variant(d, p, k, kVariantTCPlanar, tpl, split_elems) && tpl.tile.tc_planar) {
                cand[k].push_back({kVariantTCPlanar, tpl});
                if (tpl.tile.split > 1) {
                    Node t1 = tpl;
                    t1.tile.split = 1;
                    cand[k].push_back({kVariantTCPlanar, t1});
                }
            }
            // 128-column tiles where 256 were chosen: twice the CTAs
            Node tn;
            const TcGeom g_tc = tc_geom(tc.tile, d.is_complex(), tc_prec_of_mode(p.mode));
            if (g_tc.bn == 256 &&
                make_variant(d, p, k, kVariantTC128, tn, split_elems)) {
                cand[k].push_back({kVariantTC128, tn});
                if (tn.tile.split > 1) {
                    Node t1 = tn;
                    t1.tile.split = 1;
                    cand[k].push_back({kVariantTC128, t1});
                }
            }
        }
        // CUDA-core shapes, unless the node is so large that they cannot win
        if (!has_tc || vc < 32)
            for (int v : {int(kTile64x64), int(kTile16x256), int(kTile4x1024), int(kTile256x16), int(kTile128x64)})
                for (int mult : {1, 4}) {
                    Node t;
                    if (make_variant(d, p, k, v, t, split_elems, mult)) cand[k].push_back({v, t});
                }
    }
    const int64_t need = (split_elems * (int64_t)d.elem_bytes() + 1023) / 1024 * 1024;
    const int G = std::max(p.alloc_inst, 1);
    if (need > p.split_bytes) {
        CK(cudaStreamSynchronize(s));
        if (p.split_buf) CK(cudaFree(p.split_buf));
        p.split_buf = nullptr;
        CK(cudaMalloc(&p.split_buf, need * G));
        p.split_bytes = need;
        for (auto& nd : p.nodes) nd.tile.P = p.split_buf;
        for (auto& cs : cand)
            for (auto& c : cs) c.second.tile.P = p.split_buf;
    }
    // a valid control block (slice 0 of the range) for the single-node launches
    CK(launch_begin_call(p.ctl, 0, p.d_sliced, p.acc, 0, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int k : tune) {
        float best = 1e30f;
        int best_v = 0;
        Node best_node = p.nodes[k];
        for (auto& c : cand[k]) {
            c.second.tile.in = p.nodes[k].tile.in;
            cudaError_t e = launch_node(d, p, c.second, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_node(d, p, c.second, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                err = std::string("autotune: ") + cudaGetErrorString(e);
                return TN_ECUDA;
            }
            // the planner's choice stays unless another is clearly faster
            const bool planned = c.second.kind == p.nodes[k].kind &&
                                 (c.second.kind == kTensorCore || c.second.tile.cfg == p.nodes[k].tile.cfg);
            const float eff = planned ? ms * 0.95f : ms;
            if (eff < best) {
                best = eff;
                best_v = c.first;
                best_node = c.second;
            }
        }
        p.nodes[k] = best_node;
        if (choice) choice[k] = best_v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the control block must not look like a finished call; the next call
    // rebuilds the instance configuration and the captured graph
    CK(cudaStreamSynchronize(s));
    Control zero{};
    CK(cudaMemcpy(p.ctl, &zero, sizeof(Control), cudaMemcpyHostToDevice));
    if (p.descs_dev) {
        std::vector<TileArgs> descs(nn);
        for (int k = 0; k < nn; ++k) descs[k] = p.nodes[k].tile;
        CK(cudaMemcpy(p.descs_dev, descs.data(), sizeof(TileArgs) * nn, cudaMemcpyHostToDevice));
    }
    p.cfg_inst = -1;
    p.graph_ptrs.clear();
    p.graph_ptrs_h.clear();
    p.tuned = true;
    return TN_OK;
}

#undef CK

bool plan_tile_node(const NetDesc& d, const Plan& p, Node& nd, int64_t& split_elems) {
    return plan_tile(d, p, nd, split_elems);
}

tn_status make_generic_args(const NetDesc& d, const Plan& p, int k, GenericArgs& g, std::string& err) {
    return fill_generic(d, p, p.nodes[k], g, err);
}

void plan_info(const NetDesc& d, const Plan& p, double out[8]) {
    out[0] = p.W;
    out[1] = p.C;
    out[2] = (double)p.d_sliced;
    out[3] = (d.is_complex() ? 8.0 : 2.0) * p.C * (double)p.d_sliced;
    out[4] = (double)p.ws_elems * (double)d.elem_bytes();
    int cnt[3] = {0, 0, 0};
    for (auto& nd : p.nodes) cnt[nd.kind]++;
    out[5] = cnt[kTiled];
    out[6] = cnt[kTensorCore];
    out[7] = cnt[kGeneric];
}

void free_device(Plan& p) {
    free_grad(p);
    if (p.gexec) cudaGraphExecDestroy(p.gexec);
    if (p.graph) cudaGraphDestroy(p.graph);
    if (p.gexec_h) cudaGraphExecDestroy(p.gexec_h);
    if (p.graph_h) cudaGraphDestroy(p.graph_h);
    p.gexec_h = nullptr;
    p.graph_h = nullptr;
    p.graph_ptrs_h.clear();
    p.graph_inst_h = p.graph_step_h = -1;
    for (auto ev : p.prof_placeholder) cudaEventDestroy(ev);
    p.prof_placeholder.clear();
    p.prof_nodes.clear();
    p.graph = nullptr;
    if (p.cap_stream) cudaStreamDestroy(p.cap_stream);
    if (p.ws) cudaFree(p.ws);
    if (p.maxabs) cudaFree(p.maxabs);
    if (p.exps) cudaFree(p.exps);
    if (p.ctl) cudaFree(p.ctl);
    if (p.acc) cudaFree(p.acc);
    if (p.out_stage) cudaFree(p.out_stage);
    p.out_stage = nullptr;
    if (p.leafmax) cudaFree(p.leafmax);
    if (p.split_buf) cudaFree(p.split_buf);
    p.split_buf = nullptr;
    if (p.descs_dev) cudaFree(p.descs_dev);
    if (p.items_dev) cudaFree(p.items_dev);
    if (p.flow_deps_dev) cudaFree(p.flow_deps_dev);
    p.flow_deps_dev = nullptr;
    p.flow_cnt_dev = nullptr;
    if (p.inst_roots_dev) cudaFree(p.inst_roots_dev);
    if (p.inst_out_dev) cudaFree(p.inst_out_dev);
    if (p.inst_exp_dev) cudaFree(p.inst_exp_dev);
    p.inst_roots_dev = nullptr;
    p.inst_out_dev = nullptr;
    p.inst_exp_dev = nullptr;
    p.cfg_inst = -1;
    p.inst_roots_n = 0;
    p.graph_inst = -1;
    p.graph_step = -1;
    p.leaf_nfloat_uploaded.clear();
    p.descs_dev = nullptr;
    p.items_dev = nullptr;
    if (p.leaf_ptr_dev) cudaFree(p.leaf_ptr_dev);
    if (p.leaf_nfloat_dev) cudaFree(p.leaf_nfloat_dev);
    p.leafmax = nullptr;
    p.leaf_ptr_dev = nullptr;
    p.leaf_nfloat_dev = nullptr;
    p.leaf_ptr_uploaded.clear();
    p.gexec = nullptr;
    p.cap_stream = nullptr;
    p.ws = nullptr;
    p.maxabs = nullptr;
    p.exps = nullptr;
    p.ctl = nullptr;
    p.acc = nullptr;
    p.graph_ptrs.clear();
}

}  // namespace tn
