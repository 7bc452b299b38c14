// tn_noalloc.cu -- the contraction call for callers that cannot allocate
// device memory.
//
// tn_contract keeps a per-plan workspace that it obtains with cudaMalloc the
// first time a tree is run.  Some callers cannot allow that: hosts that must
// not allocate device memory after start-up (fixed memory budgets, real-time
// loops whose latency an allocation would break), and processes whose device
// memory is owned by another allocator's pool (a framework's caching
// allocator, which cudaMalloc calls behind its back would starve).  For them
// this file
// offers the same contraction with every piece of scratch -- workspace for
// the intermediate tensors, node maxima and exponents, leaf maxima, the
// control block and the FP64 accumulator -- carved out of one fixed array
// that is part of the library image.  The caller still passes the leaves
// (device memory) and the outputs.
//
// The array costs kNoAllocScratchBytes of device memory on every GPU that
// loads the library, for as long as the process lives.  Calls share it and
// it keeps the last call's contents; everything a call relies on starting at
// zero is cleared by the call itself.  Calls whose GPU work overlaps (on
// different streams, or from several threads) race on the array.  The small
// per-call tables (leaf pointers and sizes, the unit scalar) travel as kernel
// parameters, so a call reads no host memory after it has returned.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "tn_internal.h"
#include "tn_plan.h"

namespace tn {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// In host code g_noalloc_scratch names a host-side shadow, not device
// memory; the device address is looked up once per device, with that
// device current.
bool scratch_address(void** out, std::string& err) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return false;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        err = "device index out of range for the no-allocation scratch table";
        return false;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                  cudaGetErrorString(e);
            return false;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return true;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// One chunk of the leaf tables, passed by value as a kernel parameter.
constexpr int kTableChunk = 128;
struct LeafTableChunk {
    int32_t first, count;
    const void* ptr[kTableChunk];
    int64_t nfloat[kTableChunk];
};

__global__ void k_noalloc_tables(const __grid_constant__ LeafTableChunk c, const float** lptr,
                                 int64_t* lnf, float* unit) {
    const int i = threadIdx.x;
    if (i < c.count) {
        lptr[c.first + i] = static_cast<const float*>(c.ptr[i]);
        lnf[c.first + i] = c.nfloat[i];
    }
    // the scalar 1 that stands in for a missing operand
    if (c.first == 0 && i < 4) unit[i] = i == 0 ? 1.f : 0.f;
}

}  // namespace

tn_status run_noalloc(const NetDesc& d, const Plan& p, void* out, int out_mem, int64_t* out_exp2,
                      cudaStream_t stream, std::string& err) {
    const int n = d.n;
    const int nn = (int)p.nodes.size();
    const size_t eb = d.elem_bytes();
    const bool cplx = d.is_complex();
    if (out_mem == TN_MEM_HOST) {
        // a host result is waited for; a capturing stream cannot be waited on
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing(stream, &cs);
        if (ce != cudaSuccess) {
            err = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce);
            return TN_ECUDA;
        }
        if (cs != cudaStreamCaptureStatusNone) {
            err = "tn_contract_noalloc: host outputs need a stream synchronisation, which a "
                  "capturing stream does not allow; pass device outputs";
            return TN_EUNSUPPORTED;
        }
    }
    for (int v = 0; v < n; ++v)
        if (d.leaves[v].mem != TN_MEM_DEVICE) {
            err = "tn_contract_noalloc: leaves must be device pointers (staging a host leaf "
                  "would need device memory)";
            return TN_EUNSUPPORTED;
        }
    // scratch layout (256-byte aligned sections)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_ctl = take(sizeof(Control));
    const size_t o_unit = take(16);
    const size_t o_max = take(sizeof(unsigned) * nn);
    const size_t o_exp = take(sizeof(int64_t) * nn);
    const size_t o_lmax = take(sizeof(unsigned) * n);
    const size_t o_lptr = take(sizeof(void*) * n);
    const size_t o_lnf = take(sizeof(int64_t) * n);
    const size_t acc_doubles = (size_t)p.n_out * (cplx ? 2 : 1);
    const size_t o_acc = take(sizeof(double) * acc_doubles);
    const size_t o_ws = take((size_t)p.ws_elems * eb);
    if (off > kNoAllocScratchBytes) {
        err = "tn_contract_noalloc: this tree needs " + std::to_string(off) +
              " bytes of scratch; the no-allocation scratch holds " +
              std::to_string(kNoAllocScratchBytes) + " bytes (8 MiB): use tn_contract";
        return TN_EUNSUPPORTED;
    }
    void* base = nullptr;
    if (!scratch_address(&base, err)) return TN_ECUDA;
    char* S = static_cast<char*>(base);
    Control* ctl = reinterpret_cast<Control*>(S + o_ctl);
    void* unit = S + o_unit;
    unsigned* maxabs = reinterpret_cast<unsigned*>(S + o_max);
    int64_t* exps = reinterpret_cast<int64_t*>(S + o_exp);
    unsigned* leafmax = reinterpret_cast<unsigned*>(S + o_lmax);
    const float** lptr = reinterpret_cast<const float**>(S + o_lptr);
    int64_t* lnf = reinterpret_cast<int64_t*>(S + o_lnf);
    double* acc = reinterpret_cast<double*>(S + o_acc);
    char* ws = S + o_ws;

#define CK(x)                                                          \
    do {                                                               \
        cudaError_t e_ = (x);                                          \
        if (e_ != cudaSuccess) {                                       \
            err = std::string(#x) + ": " + cudaGetErrorString(e_);     \
            return TN_ECUDA;                                           \
        }                                                              \
    } while (0)

    // the leaf pointer and size tables and the unit scalar, written by
    // kernels that take them as parameters (no host memory is read later)
    for (int first = 0; first < n || first == 0; first += kTableChunk) {
        LeafTableChunk c;
        memset(&c, 0, sizeof(c));
        c.first = first;
        c.count = std::min(kTableChunk, n - first);
        for (int i = 0; i < c.count; ++i) {
            c.ptr[i] = d.leaves[first + i].ptr;
            c.nfloat[i] = d.leaves[first + i].size * (cplx ? 2 : 1);
        }
        k_noalloc_tables<<<1, kTableChunk, 0, stream>>>(c, lptr, lnf, static_cast<float*>(unit));
        CK(cudaGetLastError());
        if (n == 0) break;
    }

    // node arguments, pointing into the scratch
    std::vector<GenericArgs> gen(nn);
    for (int k = 0; k < nn; ++k) {
        const Node& nd = p.nodes[k];
        GenericArgs& g = gen[k];
        tn_status st = make_generic_args(d, p, k, g, err);
        if (st != TN_OK) return st;
        auto operand = [&](int c) -> const void* {
            if (c < 0) return unit;
            if (c < n) return d.leaves[c].ptr;
            return ws + p.nodes[c - n].ws_off * eb;
        };
        g.A = operand(nd.ca);
        g.B = operand(nd.cb);
        g.C = ws + nd.ws_off * eb;
        g.ctl = ctl;
        g.sc.max_a = nd.ca >= n ? maxabs + (nd.ca - n) : (nd.ca >= 0 ? leafmax + nd.ca : nullptr);
        g.sc.exp_a = nd.ca >= n ? exps + (nd.ca - n) : nullptr;
        g.sc.max_b = nd.cb >= n ? maxabs + (nd.cb - n) : (nd.cb >= 0 ? leafmax + nd.cb : nullptr);
        g.sc.exp_b = nd.cb >= n ? exps + (nd.cb - n) : nullptr;
        g.sc.max_c = maxabs + k;
        g.sc.exp_c = exps + k;
    }
    const Node& root = p.nodes.back();
    AccumArgs a;
    memset(&a, 0, sizeof(a));
    a.R = ws + root.ws_off * eb;
    a.n_out = p.n_out;
    a.n_od = (int)d.open.size();
    if (a.n_od > kMaxDigits) {
        err = "too many open labels";
        return TN_EUNSUPPORTED;
    }
    for (int i = 0; i < a.n_od; ++i) {
        int l = d.open[d.open.size() - 1 - i];
        a.od_dim[i] = (int32_t)d.dims[l];
        int64_t s = 0;
        for (size_t j = 0; j < root.lab.size(); ++j)
            if (root.lab[j] == l) s = root.stride[j];
        a.od_s[i] = s;
    }
    a.max_r = maxabs + (nn - 1);
    a.exp_r = exps + (nn - 1);
    a.acc = acc;
    a.ctl = ctl;

    // the call: leaf maxima, control block and accumulator cleared, then
    // every slice in order, then the result
    int64_t mx_leaf = 0;
    for (int v = 0; v < n; ++v) mx_leaf = std::max(mx_leaf, d.leaves[v].size * (d.is_complex() ? 2 : 1));
    CK(launch_call_begin(lptr, lnf, leafmax, n, mx_leaf, ctl, 0, p.d_sliced, acc, (int64_t)acc_doubles, stream));
    for (int64_t s = 0; s < p.d_sliced; ++s) {
        CK(launch_begin_slice(maxabs, nn, stream));
        // the workspace offsets assume the plan's step order
        for (const Step& st : p.steps)
            for (int k : st.nodes) CK(launch_generic(gen[k], cplx, stream));
        CK(launch_accumulate(a, cplx, stream, 1));
    }
    cudaMemcpyKind kind = out_mem == TN_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(out, acc, sizeof(double) * acc_doubles, kind, stream));
    CK(cudaMemcpyAsync(out_exp2, &ctl->final_exp, sizeof(int64_t), kind, stream));
    if (out_mem == TN_MEM_HOST) CK(cudaStreamSynchronize(stream));
#undef CK
    return TN_OK;
}

}  // namespace tn
