// tn_tiled.cu -- tiled node kernels for power-of-two label sizes (FP32 on
// CUDA cores).
//
// A tree node contracts A and B over the shared labels (Sec. 2 of arXiv
// 2002.01935).  With every label size a power of two, each group of labels
// (batch, M, N, K) is a set of index bits and an operand offset is a
// scatter of those bits to the operand's strides.  The node output is laid
// out [batch][M][N], i.e. a row-major M x N matrix per batch index, so a
// node is a batched GEMM whose operands are read through bit scatters:
//   C[b, m, n] = sum_k A[sA(b) + sA(m) + sA(k)] * B[sB(b) + sB(k) + sB(n)].
// The index permutation of a classic transpose-transpose-GEMM scheme is
// folded into the operand loads: each CTA builds tile-local offset tables
// once, and the planner orders every group's bits by operand stride so
// that tiles cover the operands' contiguous bits (coalesced loads).
//
// Renormalisation (Sec. 4.2): operands are multiplied by 2^-e at load,
// e = frexp exponent of their max |component|, which is exact; the output
// max goes to the node's slot for its consumer.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstring>
#include <stdint.h>

#include "../../include/tn.h"
#include "tn_internal.h"

namespace tn {

namespace {

template <bool CPLX>
struct VT;
template <>
struct VT<true> {
    using T = float2;
};
template <>
struct VT<false> {
    using T = float;
};

__device__ __forceinline__ int64_t scatter_bits(uint64_t x, const uint8_t* sh, int nbits) {
    int64_t o = 0;
    for (int i = 0; i < nbits; ++i)
        if (((x >> i) & 1ull) && sh[i] != kNoBit) o += (int64_t)1 << sh[i];
    return o;
}

// Scale slots are read through L2 (ld.global.cg): inside a dataflow launch
// other CTAs write them, and a line an earlier item left in this SM's L1
// could be stale.
__device__ __forceinline__ int exp_of(const unsigned* slot) {
    if (slot == nullptr) return 0;
    float m = __uint_as_float(__ldcg(slot));
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m, &e);
    return e;
}

__device__ __forceinline__ int64_t slice_off(const SliceDigits& d, int64_t slice) {
    int64_t off = 0;
    for (int i = 0; i < d.n; ++i) off += ((slice / d.div[i]) % d.dim[i]) * d.stride[i];
    return off;
}

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// scaled load value, complex-conjugated when cj != 0 (a sign flip of Im)
__device__ __forceinline__ float2 cmul(float2 x, float f, int cj) {
    return make_float2(x.x * f, cj ? -x.y * f : x.y * f);
}
__device__ __forceinline__ float cmul(float x, float f, int) { return x * f; }
__device__ __forceinline__ float absmax(float2 x) { return fmaxf(fabsf(x.x), fabsf(x.y)); }
__device__ __forceinline__ float absmax(float x) { return fabsf(x); }
__device__ __forceinline__ void fma_acc(float2& c, float2 a, float2 b) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
}
__device__ __forceinline__ void fma_acc(float& c, float a, float b) { c = fmaf(a, b, c); }
template <typename T>
__device__ __forceinline__ T zero();
template <>
__device__ __forceinline__ float2 zero<float2>() {
    return make_float2(0.f, 0.f);
}
template <>
__device__ __forceinline__ float zero<float>() {
    return 0.f;
}
__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float add(float a, float b) { return a + b; }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void block_max(float v, unsigned* slot) {
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0 && v > 0.f) atomicMax(slot, __float_as_uint(v));
    }
}

// Operand scales 2^-e (clamped so the float factor stays finite) and the
// residual exponent applied to the result.
struct Scales {
    float fa, fb;
    int resid;
};

// One instance's view of a node: operand/result pointers, scale slots and
// slice id, all offset by the instance index.
struct View {
    const void* A;
    const void* B;
    void* C;
    void* P;
    ScaleIO sc;
    int64_t slice;
    bool live;
};

__device__ __forceinline__ View inst_view(const TileArgs& a, int inst, int esz) {
    const InstanceInfo& in = a.in;
    View v;
    v.A = (const char*)a.A + (int64_t)inst * in.a_is * esz;
    v.B = (const char*)a.B + (int64_t)inst * in.b_is * esz;
    v.C = (char*)a.C + (int64_t)inst * in.c_is * esz;
    v.P = (char*)a.P + (int64_t)inst * in.p_is * esz;
    v.sc = a.sc;
    if (v.sc.max_a) v.sc.max_a += (int64_t)inst * in.sa_is;
    if (v.sc.exp_a) v.sc.exp_a += (int64_t)inst * in.sa_is;
    if (v.sc.max_b) v.sc.max_b += (int64_t)inst * in.sb_is;
    if (v.sc.exp_b) v.sc.exp_b += (int64_t)inst * in.sb_is;
    if (v.sc.max_c) v.sc.max_c += (int64_t)inst * in.sc_is;
    if (v.sc.exp_c) v.sc.exp_c += (int64_t)inst * in.sc_is;
    v.slice = a.ctl->slice + (int64_t)inst * in.slice_step;
    v.live = v.slice < a.ctl->slice_end;
    return v;
}

__device__ __forceinline__ Scales node_scales(const ScaleIO& sio, bool write_exp) {
    const int eA = exp_of(sio.max_a), eB = exp_of(sio.max_b);
    const int cA = max(-120, min(120, eA)), cB = max(-120, min(120, eB));
    if (write_exp && sio.exp_c)
        *sio.exp_c = (sio.exp_a ? __ldcg(sio.exp_a) : 0) + (sio.exp_b ? __ldcg(sio.exp_b) : 0) + eA + eB;
    Scales s;
    s.fa = ldexpf(1.f, -cA);
    s.fb = ldexpf(1.f, -cB);
    s.resid = (eA - cA) + (eB - cB);
    return s;
}

// node_scales from values already read: the children's max bits and
// exponents (0 where absent); exp_c (may be null) receives the node's
// exponent.
__device__ __forceinline__ Scales scales_from(unsigned ma, unsigned mb, int64_t ea, int64_t eb, int64_t* exp_c) {
    auto ex = [](unsigned bits) {
        const float m = __uint_as_float(bits);
        if (!(m > 0.f)) return 0;
        int e;
        frexpf(m, &e);
        return e;
    };
    const int eA = ex(ma), eB = ex(mb);
    const int cA = max(-120, min(120, eA)), cB = max(-120, min(120, eB));
    if (exp_c) *exp_c = ea + eb + eA + eB;
    Scales s;
    s.fa = ldexpf(1.f, -cA);
    s.fb = ldexpf(1.f, -cB);
    s.resid = (eA - cA) + (eB - cB);
    return s;
}

}  // namespace

template <bool CPLX>
__device__ __forceinline__ typename VT<CPLX>::T ld_cg(const typename VT<CPLX>::T* p) {
    if constexpr (CPLX) return __ldcg(reinterpret_cast<const float2*>(p));
    else return __ldcg(reinterpret_cast<const float*>(p));
}

// --------------------------------------------------------------------------
// Register-blocked tile: TM x TN outputs of one batch index and one K split;
// TK-deep steps through shared memory.  This body serves the tile items of
// the persistent dataflow launch (CG: operands read through L2 only -- they
// may have been written earlier in the same launch by other CTAs); the tile
// kernel below is the same computation.  A and B are the instance's operand
// bases; the epilogue writes C (or the K part's partial) and the maximum.
// --------------------------------------------------------------------------
template <bool CPLX, int TM, int TN, int TK, int RM, int RN, bool CG>
__device__ __forceinline__ void tile_body(const TileArgs& a, int64_t tile_x, int split_id, int64_t b,
                                          const View& vw, const typename VT<CPLX>::T* A,
                                          const typename VT<CPLX>::T* B, const Scales& sc) {
    using T = typename VT<CPLX>::T;
    constexpr int TX = TN / RN, TY = TM / RM, NT = TX * TY;
    constexpr int PB = CPLX ? 2 : 4;  // keeps sB rows 16-byte aligned
    __shared__ T sA[TK][TM + 1];
    __shared__ __align__(16) T sB[TK][TN + PB];
    __shared__ int64_t rowA[TM], colB[TN], kA[TK], kB[TK];
    auto ldx = [](const T* p) -> T {
        if constexpr (CG) return ld_cg<CPLX>(p);
        else return *p;
    };

    const int tid = threadIdx.x;
    const int64_t M = 1ll << a.nm, N = 1ll << a.nn, K = 1ll << a.nk;
    const int64_t tiles_n = (N + TN - 1) / TN;
    const int64_t m0 = (tile_x / tiles_n) * TM;
    const int64_t n0 = (tile_x % tiles_n) * TN;
    const int64_t slice = vw.slice;
    const int64_t baseA =
        slice_off(a.sla, slice) + scatter_bits(b, a.a_b, a.nb) + scatter_bits(m0, a.a_m, a.nm);
    const int64_t baseB =
        slice_off(a.slb, slice) + scatter_bits(b, a.b_b, a.nb) + scatter_bits(n0, a.b_n, a.nn);
    for (int i = tid; i < TM; i += NT) rowA[i] = scatter_bits(i, a.a_m, a.nm);
    for (int j = tid; j < TN; j += NT) colB[j] = scatter_bits(j, a.b_n, a.nn);
    for (int t = tid; t < TK; t += NT) {
        kA[t] = scatter_bits(t, a.a_k, a.nk);
        kB[t] = scatter_bits(t, a.b_k, a.nk);
    }
    __syncthreads();
    const int mlim = (int)min64(M - m0, TM);
    const int nlim = (int)min64(N - n0, TN);
    const int64_t kbeg = (int64_t)split_id * a.kchunk;
    const int64_t kend = min64(K, kbeg + a.kchunk);
    const int tx = tid % TX, ty = tid / TX;

    T acc[RM][RN];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < RN; ++c) acc[r][c] = zero<T>();

    // global -> registers for one K step (all loads issued back to back).
    // The operand offsets of the K step's base k0 are kept incrementally:
    // k0 advances by TK, so only the bits of its carry chain change.
    constexpr int LA = (TM * TK + NT - 1) / NT, LB = (TN * TK + NT - 1) / NT;
    constexpr int LG_TK = TK == 16 ? 4 : (TK == 8 ? 3 : (TK == 4 ? 2 : 0));
    static_assert((1 << LG_TK) == TK, "TK must be a power of two");
    T ra[LA], rb[LB];
    int64_t cur_k = kbeg;
    int64_t kaA = scatter_bits(kbeg, a.a_k, a.nk), kaB = scatter_bits(kbeg, a.b_k, a.nk);
    auto step_k = [&]() {  // cur_k += TK, offsets follow
        int i = LG_TK;
        while (i < a.nk && ((cur_k >> i) & 1)) {
            if (a.a_k[i] != kNoBit) kaA -= int64_t(1) << a.a_k[i];
            if (a.b_k[i] != kNoBit) kaB -= int64_t(1) << a.b_k[i];
            ++i;
        }
        if (i < a.nk) {
            if (a.a_k[i] != kNoBit) kaA += int64_t(1) << a.a_k[i];
            if (a.b_k[i] != kNoBit) kaB += int64_t(1) << a.b_k[i];
        }
        cur_k += TK;
    };
    auto gload = [&](int64_t k0) {
        const int klim = (int)min64(kend - k0, TK);
#pragma unroll
        for (int q = 0; q < LA; ++q) {
            const int e = tid + q * NT;
            const int i = a.a_mfast ? e % TM : e / TK;
            const int t = a.a_mfast ? e / TM : e % TK;
            const bool in = e < TM * TK && i < mlim && t < klim;
            ra[q] = in ? cmul(ldx(A + baseA + rowA[i] + kaA + kA[t]), sc.fa, a.conj_a) : zero<T>();
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const int e = tid + q * NT;
            const int j = a.b_nfast ? e % TN : e / TK;
            const int t = a.b_nfast ? e / TN : e % TK;
            const bool in = e < TN * TK && j < nlim && t < klim;
            rb[q] = in ? cmul(ldx(B + baseB + colB[j] + kaB + kB[t]), sc.fb, a.conj_b) : zero<T>();
        }
    };
    if (kbeg < kend) gload(kbeg);
    for (int64_t k0 = kbeg; k0 < kend; k0 += TK) {
        // kaA/kaB describe k0 here; gload of k0 + TK needs them advanced
#pragma unroll
        for (int q = 0; q < LA; ++q) {
            const int e = tid + q * NT;
            if (e < TM * TK) {
                const int i = a.a_mfast ? e % TM : e / TK;
                const int t = a.a_mfast ? e / TM : e % TK;
                sA[t][i] = ra[q];
            }
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const int e = tid + q * NT;
            if (e < TN * TK) {
                const int j = a.b_nfast ? e % TN : e / TK;
                const int t = a.b_nfast ? e / TN : e % TK;
                sB[t][j] = rb[q];
            }
        }
        __syncthreads();
        if (k0 + TK < kend) {
            step_k();
            gload(k0 + TK);  // next step's loads overlap this step's FMAs
        }
#pragma unroll 4
        for (int t = 0; t < TK; ++t) {
            T af[RM], bf[RN];
#pragma unroll
            for (int r = 0; r < RM; ++r) af[r] = sA[t][ty * RM + r];
#pragma unroll
            for (int c = 0; c < RN; ++c) bf[c] = sB[t][tx + c * TX];  // conflict-free
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < RN; ++c) fma_acc(acc[r][c], af[r], bf[c]);
        }
        __syncthreads();
    }

    // epilogue: direct output (one split) or a partial for the reduce pass
    float lmax = 0.f;
    T* out = reinterpret_cast<T*>(a.split > 1 ? vw.P : vw.C);
    const int64_t plane = (a.split > 1 ? (int64_t)split_id * ((int64_t)a.nbatch) : 0) + b;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        const int i = ty * RM + r;
        if (i >= mlim) continue;
        const int64_t rowoff = (plane * M + m0 + i) * N + n0;
#pragma unroll
        for (int c = 0; c < RN; ++c) {
            const int j = tx + c * TX;
            if (j >= nlim) continue;
            T v = acc[r][c];
            if (a.split == 1) {
                if (sc.resid) {
                    if constexpr (CPLX) {
                        v.x = ldexpf(v.x, -sc.resid);
                        v.y = ldexpf(v.y, -sc.resid);
                    } else {
                        v = ldexpf(v, -sc.resid);
                    }
                }
                lmax = fmaxf(lmax, absmax(v));
            }
            out[rowoff + j] = v;
        }
    }
    if (a.split == 1) {
        block_max(lmax, vw.sc.max_c);
        if (a.t_done && threadIdx.x == 0) atomicMax(a.t_done, global_ns());
    }
}

// --------------------------------------------------------------------------
// The tile kernel: one CTA = TM x TN outputs of one batch index and one K
// split (the same computation as tile_body above, written out for the
// kernel: the shared body costs the kernel registers, hence occupancy).
// --------------------------------------------------------------------------
template <bool CPLX, int TM, int TN, int TK, int RM, int RN>
__global__ void __launch_bounds__((TM / RM) * (TN / RN))
    k_tile(const __grid_constant__ TileArgs a) {
    using T = typename VT<CPLX>::T;
    constexpr int TX = TN / RN, TY = TM / RM, NT = TX * TY;
    constexpr int PB = CPLX ? 2 : 4;  // keeps sB rows 16-byte aligned
    __shared__ T sA[TK][TM + 1];
    __shared__ __align__(16) T sB[TK][TN + PB];
    __shared__ int64_t rowA[TM], colB[TN], kA[TK], kB[TK];

    const int tid = threadIdx.x;
    const int64_t M = 1ll << a.nm, N = 1ll << a.nn, K = 1ll << a.nk;
    const int64_t tiles_n = (N + TN - 1) / TN;
    const int64_t m0 = ((int64_t)blockIdx.x / tiles_n) * TM;
    const int64_t n0 = ((int64_t)blockIdx.x % tiles_n) * TN;
    const int per_inst = (int)(a.nbatch * a.split);
    const int inst = blockIdx.z / per_inst;
    const int zz = blockIdx.z % per_inst;
    const int split_id = zz % a.split;
    const int64_t b = zz / a.split;
    const View vw = inst_view(a, inst, (int)sizeof(T));
    if (!vw.live) return;
    const Scales sc = node_scales(vw.sc, blockIdx.x == 0 && zz == 0 && tid == 0);
    const int64_t slice = vw.slice;
    const int64_t baseA =
        slice_off(a.sla, slice) + scatter_bits(b, a.a_b, a.nb) + scatter_bits(m0, a.a_m, a.nm);
    const int64_t baseB =
        slice_off(a.slb, slice) + scatter_bits(b, a.b_b, a.nb) + scatter_bits(n0, a.b_n, a.nn);
    for (int i = tid; i < TM; i += NT) rowA[i] = scatter_bits(i, a.a_m, a.nm);
    for (int j = tid; j < TN; j += NT) colB[j] = scatter_bits(j, a.b_n, a.nn);
    for (int t = tid; t < TK; t += NT) {
        kA[t] = scatter_bits(t, a.a_k, a.nk);
        kB[t] = scatter_bits(t, a.b_k, a.nk);
    }
    __syncthreads();
    const int mlim = (int)min64(M - m0, TM);
    const int nlim = (int)min64(N - n0, TN);
    const int64_t kbeg = (int64_t)split_id * a.kchunk;
    const int64_t kend = min64(K, kbeg + a.kchunk);
    const T* A = reinterpret_cast<const T*>(vw.A);
    const T* B = reinterpret_cast<const T*>(vw.B);
    const int tx = tid % TX, ty = tid / TX;

    T acc[RM][RN];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < RN; ++c) acc[r][c] = zero<T>();

    // global -> registers for one K step (all loads issued back to back).
    // The operand offsets of the K step's base k0 are kept incrementally:
    // k0 advances by TK, so only the bits of its carry chain change.
    constexpr int LA = (TM * TK + NT - 1) / NT, LB = (TN * TK + NT - 1) / NT;
    constexpr int LG_TK = TK == 16 ? 4 : (TK == 8 ? 3 : (TK == 4 ? 2 : 0));
    static_assert((1 << LG_TK) == TK, "TK must be a power of two");
    T ra[LA], rb[LB];
    int64_t cur_k = kbeg;
    int64_t kaA = scatter_bits(kbeg, a.a_k, a.nk), kaB = scatter_bits(kbeg, a.b_k, a.nk);
    auto step_k = [&]() {  // cur_k += TK, offsets follow
        int i = LG_TK;
        while (i < a.nk && ((cur_k >> i) & 1)) {
            if (a.a_k[i] != kNoBit) kaA -= int64_t(1) << a.a_k[i];
            if (a.b_k[i] != kNoBit) kaB -= int64_t(1) << a.b_k[i];
            ++i;
        }
        if (i < a.nk) {
            if (a.a_k[i] != kNoBit) kaA += int64_t(1) << a.a_k[i];
            if (a.b_k[i] != kNoBit) kaB += int64_t(1) << a.b_k[i];
        }
        cur_k += TK;
    };
    auto gload = [&](int64_t k0) {
        const int klim = (int)min64(kend - k0, TK);
#pragma unroll
        for (int q = 0; q < LA; ++q) {
            const int e = tid + q * NT;
            const int i = a.a_mfast ? e % TM : e / TK;
            const int t = a.a_mfast ? e / TM : e % TK;
            const bool in = e < TM * TK && i < mlim && t < klim;
            ra[q] = in ? cmul(A[baseA + rowA[i] + kaA + kA[t]], sc.fa, a.conj_a) : zero<T>();
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const int e = tid + q * NT;
            const int j = a.b_nfast ? e % TN : e / TK;
            const int t = a.b_nfast ? e / TN : e % TK;
            const bool in = e < TN * TK && j < nlim && t < klim;
            rb[q] = in ? cmul(B[baseB + colB[j] + kaB + kB[t]], sc.fb, a.conj_b) : zero<T>();
        }
    };
    if (kbeg < kend) gload(kbeg);
    for (int64_t k0 = kbeg; k0 < kend; k0 += TK) {
        // kaA/kaB describe k0 here; gload of k0 + TK needs them advanced
#pragma unroll
        for (int q = 0; q < LA; ++q) {
            const int e = tid + q * NT;
            if (e < TM * TK) {
                const int i = a.a_mfast ? e % TM : e / TK;
                const int t = a.a_mfast ? e / TM : e % TK;
                sA[t][i] = ra[q];
            }
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const int e = tid + q * NT;
            if (e < TN * TK) {
                const int j = a.b_nfast ? e % TN : e / TK;
                const int t = a.b_nfast ? e / TN : e % TK;
                sB[t][j] = rb[q];
            }
        }
        __syncthreads();
        if (k0 + TK < kend) {
            step_k();
            gload(k0 + TK);  // next step's loads overlap this step's FMAs
        }
#pragma unroll 4
        for (int t = 0; t < TK; ++t) {
            T af[RM], bf[RN];
#pragma unroll
            for (int r = 0; r < RM; ++r) af[r] = sA[t][ty * RM + r];
#pragma unroll
            for (int c = 0; c < RN; ++c) bf[c] = sB[t][tx + c * TX];  // conflict-free
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < RN; ++c) fma_acc(acc[r][c], af[r], bf[c]);
        }
        __syncthreads();
    }

    // epilogue: direct output (one split) or a partial for the reduce pass
    float lmax = 0.f;
    T* out = reinterpret_cast<T*>(a.split > 1 ? vw.P : vw.C);
    const int64_t plane = (a.split > 1 ? (int64_t)split_id * ((int64_t)a.nbatch) : 0) + b;
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        const int i = ty * RM + r;
        if (i >= mlim) continue;
        const int64_t rowoff = (plane * M + m0 + i) * N + n0;
#pragma unroll
        for (int c = 0; c < RN; ++c) {
            const int j = tx + c * TX;
            if (j >= nlim) continue;
            T v = acc[r][c];
            if (a.split == 1) {
                if (sc.resid) {
                    if constexpr (CPLX) {
                        v.x = ldexpf(v.x, -sc.resid);
                        v.y = ldexpf(v.y, -sc.resid);
                    } else {
                        v = ldexpf(v, -sc.resid);
                    }
                }
                lmax = fmaxf(lmax, absmax(v));
            }
            out[rowoff + j] = v;
        }
    }
    if (a.split == 1) {
        block_max(lmax, vw.sc.max_c);
        if (a.t_done && threadIdx.x == 0) atomicMax(a.t_done, global_ns());
    }
}

// Sums the K-split partials of a node in a fixed order and applies its
// epilogue.  G threads share one output (G = 1 when the outputs alone fill
// the GPU): thread g sums splits [g*split/G, (g+1)*split/G) in eight
// independent chains, then the G sums are added in g order.
template <bool CPLX>
__global__ void __launch_bounds__(256) k_split_reduce(const __grid_constant__ TileArgs a, int G) {
    using T = typename VT<CPLX>::T;
    __shared__ T red[256];
    const int64_t plane_sz = (int64_t)a.nbatch << (a.nm + a.nn);
    const View vw = inst_view(a, blockIdx.y, (int)sizeof(T));
    if (!vw.live) return;
    const Scales sc = node_scales(vw.sc, blockIdx.x == 0 && threadIdx.x == 0);
    const T* P = reinterpret_cast<const T*>(vw.P);
    T* C = reinterpret_cast<T*>(vw.C);
    const int tid = threadIdx.x, g = tid % G, per_blk = 256 / G;
    const int s0 = (int)((int64_t)a.split * g / G), s1 = (int)((int64_t)a.split * (g + 1) / G);
    float lmax = 0.f;
    for (int64_t ob = (int64_t)blockIdx.x * per_blk; ob < plane_sz; ob += (int64_t)gridDim.x * per_blk) {
        const int64_t o = ob + tid / G;
        T v = zero<T>();
        if (o < plane_sz) {
            T part[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) part[q] = zero<T>();
            int sp = s0;
            for (; sp + 8 <= s1; sp += 8)
#pragma unroll
                for (int q = 0; q < 8; ++q) part[q] = add(part[q], P[(int64_t)(sp + q) * plane_sz + o]);
            for (int q = 0; sp < s1; ++sp, ++q) part[q] = add(part[q], P[(int64_t)sp * plane_sz + o]);
            v = add(add(add(part[0], part[1]), add(part[2], part[3])),
                    add(add(part[4], part[5]), add(part[6], part[7])));
        }
        if (G > 1) {  // uniform over the block: every thread runs the same iterations
            red[tid] = v;
            __syncthreads();
            if (g == 0)
                for (int q = 1; q < G; ++q) v = add(v, red[tid + q]);
            __syncthreads();
        }
        if (g != 0 || o >= plane_sz) continue;
        if (sc.resid) {
            if constexpr (CPLX) {
                v.x = ldexpf(v.x, -sc.resid);
                v.y = ldexpf(v.y, -sc.resid);
            } else {
                v = ldexpf(v, -sc.resid);
            }
        }
        lmax = fmaxf(lmax, absmax(v));
        C[o] = v;
    }
    block_max(lmax, vw.sc.max_c);
    if (a.t_done && threadIdx.x == 0) atomicMax(a.t_done, global_ns());
}

// Tiny output, long K: grid (outputs, batch, K splits); each CTA reduces its
// K range in a fixed order; with several splits the partials go to P and
// k_split_reduce sums them in split order (deterministic).
// Inner-product node (few outputs, long K): out[b,m,n] = sum_k A[.., k] B[.., k].
// The K range is cut into tiles of up to 2^(2 kDotLow) entries holding the
// kDotLow lowest strides of A, the kDotLow lowest of B and the next K bits;
// every tile is read twice in the operands' own orders (consecutive threads,
// consecutive addresses) by asynchronous copies straight into shared memory,
// where each entry lands at its K position, and multiplied there.  A ring of
// kDotStages tiles keeps two tiles of copies in flight per CTA while a third
// is multiplied; the tile base offsets follow the tile index by its carry
// chain.  blockIdx.x: output, y: batch entry, z: K part x instance.
constexpr int kDotLow = 5;
constexpr int kDotTile = 1 << (2 * kDotLow);
constexpr int kDotPad = kDotTile + kDotTile / 32;  // one padding entry per 32: no bank conflicts
constexpr int kDotStages = 3;

template <bool CPLX>
constexpr size_t dot_smem_bytes() {
    using T = typename VT<CPLX>::T;
    return (size_t)kDotStages * 2 * kDotPad * sizeof(T) + 2 * kDotTile * sizeof(int32_t) +
           2 * kDotTile * sizeof(uint16_t);
}

// asynchronous global -> shared copy of one 4- or 8-byte element
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* dst, const void* src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <bool CPLX>
__global__ void __launch_bounds__(256) k_dot(const __grid_constant__ TileArgs a, const __grid_constant__ DotPlan dp) {
    using T = typename VT<CPLX>::T;
    extern __shared__ __align__(16) unsigned char dot_smem[];
    T* const stg = reinterpret_cast<T*>(dot_smem);  // [stage][A, B][kDotPad]
    int32_t* const offA = reinterpret_cast<int32_t*>(dot_smem + (size_t)kDotStages * 2 * kDotPad * sizeof(T));
    int32_t* const offB = offA + kDotTile;
    uint16_t* const canA = reinterpret_cast<uint16_t*>(offB + kDotTile);
    uint16_t* const canB = canA + kDotTile;
    __shared__ T red[256];
    const int64_t N = 1ll << a.nn, M = 1ll << a.nm;
    const int64_t m = (int64_t)blockIdx.x / N, n = (int64_t)blockIdx.x % N;
    const int64_t b = blockIdx.y;
    const int sp = blockIdx.z % a.split;
    const View vw = inst_view(a, blockIdx.z / a.split, (int)sizeof(T));
    if (!vw.live) return;
    const Scales sc = node_scales(vw.sc, blockIdx.x == 0 && blockIdx.y == 0 && sp == 0 && threadIdx.x == 0);
    const int t = dp.t, u = dp.u, tsz = 1 << t;
    for (int e = threadIdx.x; e < tsz; e += blockDim.x) {
        int64_t xa = 0, xb = 0;
        int ca = 0, cb = 0;
        for (int w = 0; w < t; ++w)
            if ((e >> w) & 1) {
                xa += dp.a_add[w];
                xb += dp.b_add[w];
                ca += dp.ca_add[w];
                cb += dp.cb_add[w];
            }
        offA[e] = (int32_t)xa;  // within one operand: the planner keeps tiled operands below 2^31 entries
        offB[e] = (int32_t)xb;
        canA[e] = (uint16_t)(ca + (ca >> 5));
        canB[e] = (uint16_t)(cb + (cb >> 5));
    }
    __syncthreads();
    const int64_t slice = vw.slice;
    const int64_t baseA =
        slice_off(a.sla, slice) + scatter_bits(b, a.a_b, a.nb) + scatter_bits(m, a.a_m, a.nm);
    const int64_t baseB =
        slice_off(a.slb, slice) + scatter_bits(b, a.b_b, a.nb) + scatter_bits(n, a.b_n, a.nn);
    const T* A = reinterpret_cast<const T*>(vw.A);
    const T* B = reinterpret_cast<const T*>(vw.B);
    const int64_t n_tiles = int64_t(1) << u;
    const int64_t per = (n_tiles + a.split - 1) / a.split;
    const int64_t t0 = (int64_t)sp * per, t1 = min64(n_tiles, t0 + per);
    // offsets of the next tile to copy; advanced tile by tile along the carry chain
    int64_t nt = t0, ba = baseA, bb = baseB;
    for (int j = 0; j < u; ++j)
        if ((t0 >> j) & 1) {
            ba += dp.rest_a[j];
            bb += dp.rest_b[j];
        }
    auto issue = [&](int stage) {
        if (nt < t1) {
            T* sA = stg + (size_t)stage * 2 * kDotPad;
            T* sB = sA + kDotPad;
#pragma unroll
            for (int r = 0; r < kDotTile / 256; ++r) {
                const int e = threadIdx.x + r * 256;
                if (e < tsz) {
                    cp_async_elem<sizeof(T)>(sA + canA[e], A + ba + offA[e]);
                    cp_async_elem<sizeof(T)>(sB + canB[e], B + bb + offB[e]);
                }
            }
            int j = 0;
            while (j < u && ((nt >> j) & 1)) {
                ba -= dp.rest_a[j];
                bb -= dp.rest_b[j];
                ++j;
            }
            if (j < u) {
                ba += dp.rest_a[j];
                bb += dp.rest_b[j];
            }
            ++nt;
        }
        cp_async_commit();  // one group per call, empty or not: the wait counts stay uniform
    };
#pragma unroll
    for (int q = 0; q < kDotStages - 1; ++q) issue(q);
    T acc0 = zero<T>(), acc1 = zero<T>();
    int stage = 0;
    for (int64_t tile = t0; tile < t1; ++tile) {
        issue((stage + kDotStages - 1) % kDotStages);
        cp_async_wait<kDotStages - 1>();  // this thread's copies of `tile` have landed
        __syncthreads();                  // ... and every other thread's
        const T* sA = stg + (size_t)stage * 2 * kDotPad;
        const T* sB = sA + kDotPad;
#pragma unroll
        for (int r = 0; r < kDotTile / 256; ++r) {
            const int i = threadIdx.x + r * 256;
            if (i < tsz) {
                const int ip = i + (i >> 5);
                if (r & 1) fma_acc(acc1, cmul(sA[ip], sc.fa, a.conj_a), cmul(sB[ip], sc.fb, a.conj_b));
                else fma_acc(acc0, cmul(sA[ip], sc.fa, a.conj_a), cmul(sB[ip], sc.fb, a.conj_b));
            }
        }
        __syncthreads();  // the stage is refilled by the next iteration's copies
        stage = (stage + 1) % kDotStages;
    }
    cp_async_wait<0>();
    // fixed-order block reduction
    red[threadIdx.x] = add(acc0, acc1);
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = add(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        T v = red[0];
        const int64_t o = (b * M + m) * N + n;
        if (a.split > 1) {
            reinterpret_cast<T*>(vw.P)[(int64_t)sp * (a.nbatch * M * N) + o] = v;
            return;
        }
        if (sc.resid) {
            if constexpr (CPLX) {
                v.x = ldexpf(v.x, -sc.resid);
                v.y = ldexpf(v.y, -sc.resid);
            } else {
                v = ldexpf(v, -sc.resid);
            }
        }
        reinterpret_cast<T*>(vw.C)[o] = v;
        float mx = absmax(v);
        if (mx > 0.f) atomicMax(vw.sc.max_c, __float_as_uint(mx));
        if (a.t_done) atomicMax(a.t_done, global_ns());
    }
}

// One launch for the small nodes of one or more consecutive tree levels.
// Each work item is a chunk of one node's outputs; descriptors live in
// device memory.  With fewer than 256 outputs in the chunk, g = 256/outputs
// threads share each output's K range and reduce it in a fixed order.
//
// Without dependencies (deps == nullptr) item i is CTA i.  With them, the
// launch covers several levels as one dataflow: persistent CTAs take items
// in order from a counter; before an item runs, the chunks of its children
// that belong to the same launch must have finished (per node and instance
// completion counters; a bounded wait that records TN_ETIMEOUT); after it,
// its own counter is raised.  Items only depend on earlier items, and every
// taken item belongs to a running CTA, so the waits always end.  Inputs that
// other CTAs of the launch produced are read through L2 (ld.global.cg).
// The persistent launch (every node of every slice of a call in one
// dataflow) adds tile items (o_count < 0): a 64 x 64 output tile of a large
// node computed by the tile kernel's body over all of K.
constexpr long long kFlowWaitCycles = 4000000000ll;  // ~2 s

// Completion counters: the producer's release add (after a CTA barrier, so
// it covers the whole CTA's writes) pairs with the consumer's acquire load.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <bool CPLX, bool TILES>
__global__ void __launch_bounds__(256)
    k_wave(const WaveItem* items, int n_items, const TileArgs* descs, const void* const* leaf_ptrs,
           const int4* deps, unsigned* done, unsigned* head, int G) {
    using T = typename VT<CPLX>::T;
    __shared__ TileArgs d;
    // K offsets: low 8 bits of the K index from kA / kB, the rest (at most
    // 6 more bits: wave nodes have nk <= 14) from kAh / kBh
    __shared__ int64_t kA[256], kB[256], kAh[64], kBh[64];
    __shared__ T red[256];
    __shared__ int cur;
    __shared__ int loaded;  // node whose descriptor and K tables are in shared memory
    const int tid = threadIdx.x;
    if (tid == 0) loaded = -1;
    for (int pass = 0;; ++pass) {
        // ---- take an item
        if (deps == nullptr) {
            if (pass > 0) break;
            if (tid == 0) cur = blockIdx.x;
        } else if (tid == 0) {
            cur = (int)atomicAdd(head, 1u);
        }
        __syncthreads();
        const int idx = cur;
        if (idx >= n_items) break;
        const WaveItem it = items[idx];
        // ---- everything that does not depend on the children first: the
        // descriptor and the K offset tables (kept from the previous item
        // when it was of the same node), the instance view
        const bool fresh = it.node != loaded;
        if (fresh) {
            const int4* src = reinterpret_cast<const int4*>(descs + it.node);
            int4* dst = reinterpret_cast<int4*>(&d);
            for (int i = tid; i < (int)(sizeof(TileArgs) / 16); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        if (tid == 0) loaded = it.node;  // every thread has read the old value
        const View vw = inst_view(d, it.pad, (int)sizeof(T));
        const int kt = d.nk < 8 ? (int)(1ll << d.nk) : 256;  // table covers k & 255
        const int kh = d.nk > 8 && d.nk <= 14 ? (int)(1ll << (d.nk - 8)) : 0;  // k >> 8
        if (fresh) {
            for (int t = tid; t < kt; t += 256) {
                kA[t] = scatter_bits(t, d.a_k, d.nk);
                kB[t] = scatter_bits(t, d.b_k, d.nk);
            }
            for (int h = tid; h < kh; h += 256) {
                kAh[h] = scatter_bits((int64_t)h << 8, d.a_k, d.nk);
                kBh[h] = scatter_bits((int64_t)h << 8, d.b_k, d.nk);
            }
        }
        // operand bases need only the descriptor and the leaf table
        const int64_t isz = (int64_t)sizeof(T);
        const T* A = nullptr;
        const T* B = nullptr;
        int64_t sA = 0, sB = 0;
        if (vw.live) {
            A = reinterpret_cast<const T*>(
                d.a_leaf >= 0 ? (const char*)leaf_ptrs[d.a_leaf] + (int64_t)it.pad * d.in.a_is * isz : vw.A);
            B = reinterpret_cast<const T*>(
                d.b_leaf >= 0 ? (const char*)leaf_ptrs[d.b_leaf] + (int64_t)it.pad * d.in.b_is * isz : vw.B);
            sA = slice_off(d.sla, vw.slice);
            sB = slice_off(d.slb, vw.slice);
        }
        // ---- then wait for children computed in this launch
        if (deps != nullptr && tid == 0) {
            const int4 dp = deps[it.node];
            const long long t0 = clock64();
            for (int side = 0; side < 2; ++side) {
                const int child = side ? dp.z : dp.x;
                const unsigned need = (unsigned)(side ? dp.w : dp.y);
                if (child < 0) continue;
                const unsigned* cnt = done + (int64_t)child * G + it.pad;
                while (ld_acquire_gpu(cnt) < need) {
                    if (clock64() - t0 > kFlowWaitCycles) {
                        atomicExch(const_cast<int32_t*>(&d.ctl->status), (int32_t)TN_ETIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                }
            }
        }
        __syncthreads();
        if (TILES && vw.live && it.o_count < 0) {
            // a tile item of the persistent launch: 64 x 64 outputs of one
            // batch entry (o_begin = batch entry x tiles + tile), all of K
            const unsigned rma = vw.sc.max_a ? __ldcg(vw.sc.max_a) : 0u;
            const unsigned rmb = vw.sc.max_b ? __ldcg(vw.sc.max_b) : 0u;
            const int64_t rea = vw.sc.exp_a ? __ldcg(vw.sc.exp_a) : 0;
            const int64_t reb = vw.sc.exp_b ? __ldcg(vw.sc.exp_b) : 0;
            const Scales sc = scales_from(rma, rmb, rea, reb, it.o_begin == 0 && tid == 0 ? vw.sc.exp_c : nullptr);
            const int64_t tiles = ((1ll << d.nm) + 63) / 64 * (((1ll << d.nn) + 63) / 64);
            if constexpr (TILES)
                tile_body<CPLX, 64, 64, 16, 4, 4, true>(d, it.o_begin % tiles, 0, it.o_begin / tiles, vw, A, B, sc);
        } else if (vw.live) {
            const int64_t K = 1ll << d.nk;
            const int64_t nmask = (1ll << d.nn) - 1, mmask = (1ll << d.nm) - 1;
            const int O = (int)it.o_count;
            const int g = O >= 256 ? 1 : 256 / O;
            auto k_off = [&](int64_t t, int64_t& ka, int64_t& kb2) {
                if (d.nk < 8) {
                    ka = kA[t];
                    kb2 = kB[t];
                } else if (kh > 0) {
                    ka = kA[t & 255] + kAh[t >> 8];
                    kb2 = kB[t & 255] + kBh[t >> 8];
                } else {
                    const int64_t hi = t & ~255ll;
                    ka = kA[t & 255] + (hi ? scatter_bits(hi, d.a_k, d.nk) : 0);
                    kb2 = kB[t & 255] + (hi ? scatter_bits(hi, d.b_k, d.nk) : 0);
                }
            };
            auto o_off = [&](int64_t o, int64_t& offA, int64_t& offB) {
                const int64_t n = o & nmask, m = (o >> d.nn) & mmask, b = o >> (d.nn + d.nm);
                offA = sA + scatter_bits(b, d.a_b, d.nb) + scatter_bits(m, d.a_m, d.nm);
                offB = sB + scatter_bits(b, d.b_b, d.nb) + scatter_bits(n, d.b_n, d.nn);
            };
            // the children's scale slots and this thread's first operand
            // pair are read together (one L2 round trip, not two)
            const unsigned rma = vw.sc.max_a ? __ldcg(vw.sc.max_a) : 0u;
            const unsigned rmb = vw.sc.max_b ? __ldcg(vw.sc.max_b) : 0u;
            const int64_t rea = vw.sc.exp_a ? __ldcg(vw.sc.exp_a) : 0;
            const int64_t reb = vw.sc.exp_b ? __ldcg(vw.sc.exp_b) : 0;
            bool first = tid / g < O && (int64_t)(tid % g) < K;
            T a0 = zero<T>(), b0 = zero<T>();
            if (first) {
                int64_t offA, offB, ka, kb2;
                o_off(it.o_begin + tid / g, offA, offB);
                k_off(tid % g, ka, kb2);
                a0 = ld_cg<CPLX>(A + offA + ka);
                b0 = ld_cg<CPLX>(B + offB + kb2);
            }
            const Scales sc = scales_from(rma, rmb, rea, reb, it.o_begin == 0 && tid == 0 ? vw.sc.exp_c : nullptr);
            float lmax = 0.f;
            T* C = reinterpret_cast<T*>(vw.C);
            for (int ol = tid / g; ol < O; ol += 256 / g) {
                const int64_t o = it.o_begin + ol;
                int64_t offA, offB;
                o_off(o, offA, offB);
                T acc = zero<T>();
#pragma unroll 4
                for (int64_t t = tid % g; t < K; t += g) {
                    T va, vb;
                    if (first) {
                        va = a0;
                        vb = b0;
                        first = false;
                    } else {
                        int64_t ka, kb2;
                        k_off(t, ka, kb2);
                        va = ld_cg<CPLX>(A + offA + ka);
                        vb = ld_cg<CPLX>(B + offB + kb2);
                    }
                    fma_acc(acc, cmul(va, sc.fa, d.conj_a), cmul(vb, sc.fb, d.conj_b));
                }
                if (g > 1) {
                    red[tid] = acc;
                    __syncthreads();
                    const int j = tid % g;
                    for (int s2 = g / 2; s2 > 0; s2 >>= 1) {
                        if (j < s2) red[tid] = add(red[tid], red[tid + s2]);
                        __syncthreads();
                    }
                    if (j != 0) continue;
                    acc = red[tid];
                }
                if (sc.resid) {
                    if constexpr (CPLX) {
                        acc.x = ldexpf(acc.x, -sc.resid);
                        acc.y = ldexpf(acc.y, -sc.resid);
                    } else {
                        acc = ldexpf(acc, -sc.resid);
                    }
                }
                lmax = fmaxf(lmax, absmax(acc));
                C[o] = acc;
            }
            block_max(lmax, vw.sc.max_c);
            if (d.t_done && tid == 0) atomicMax(d.t_done, global_ns());
        }
        // ---- publish: outputs, maximum and exponent before the counter
        __syncthreads();
        if (deps != nullptr && tid == 0) red_release_gpu_add(done + (int64_t)it.node * G + it.pad, 1u);
    }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

template <bool CPLX, int TM, int TN, int TK, int RM, int RN>
static cudaError_t launch_cfg(const TileArgs& a, cudaStream_t s) {
    const int64_t M = 1ll << a.nm, N = 1ll << a.nn;
    const int64_t tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
    const int ni = a.in.n_inst > 1 ? a.in.n_inst : 1;
    dim3 grid((unsigned)tiles, 1, (unsigned)(a.nbatch * a.split * ni));
    k_tile<CPLX, TM, TN, TK, RM, RN><<<grid, (TM / RM) * (TN / RN), 0, s>>>(a);
    return cudaGetLastError();
}

// Tile bits of an inner-product node: the kDotLow lowest strides of each
// operand, then the lowest K positions, up to 2 * kDotLow bits; each
// operand's order of them (ascending stride, absent bits last).
static DotPlan make_dot_plan(const TileArgs& a) {
    DotPlan dp;
    memset(&dp, 0, sizeof(dp));
    const int nk = a.nk;
    int by[2][64];
    for (int q = 0; q < 64; ++q) by[0][q] = by[1][q] = -1;
    bool in[kMaxBits] = {};
    for (int p = 0; p < nk; ++p) {
        if (a.a_k[p] < 64) by[0][a.a_k[p]] = p;
        if (a.b_k[p] < 64) by[1][a.b_k[p]] = p;
    }
    int cnt = 0;
    for (int side = 0; side < 2; ++side)
        for (int q = 0, r = 0; q < 64 && r < kDotLow; ++q)
            if (by[side][q] >= 0) {
                if (!in[by[side][q]]) ++cnt;
                in[by[side][q]] = true;
                ++r;
            }
    for (int p = 0; p < nk && cnt < 2 * kDotLow; ++p)
        if (!in[p]) {
            in[p] = true;
            ++cnt;
        }
    int tk[2 * kDotLow], pos[kMaxBits];
    int t = 0, u = 0;
    for (int p = 0; p < nk; ++p) {
        if (in[p]) {
            pos[p] = t;
            tk[t++] = p;
        } else {
            dp.rest_a[u] = a.a_k[p] != kNoBit ? int64_t(1) << a.a_k[p] : 0;
            dp.rest_b[u] = a.b_k[p] != kNoBit ? int64_t(1) << a.b_k[p] : 0;
            ++u;
        }
    }
    for (int side = 0; side < 2; ++side) {
        const uint8_t* sh = side ? a.b_k : a.a_k;
        int order[2 * kDotLow];
        int w = 0;
        for (int q = 0; q < 64; ++q)
            if (by[side][q] >= 0 && in[by[side][q]]) order[w++] = pos[by[side][q]];
        for (int j = 0; j < t; ++j)
            if (sh[tk[j]] >= 64) order[w++] = j;
        for (int i = 0; i < t; ++i) {
            const int p = tk[order[i]];
            const int64_t add = sh[p] != kNoBit ? int64_t(1) << sh[p] : 0;
            (side ? dp.b_add : dp.a_add)[i] = add;
            (side ? dp.cb_add : dp.ca_add)[i] = 1 << order[i];
        }
    }
    dp.t = t;
    dp.u = u;
    return dp;
}

template <bool CPLX>
static cudaError_t launch_tile_t(const TileArgs& a, cudaStream_t s) {
    cudaError_t e;
    switch (a.cfg) {
        case kTile64x64: e = launch_cfg<CPLX, 64, 64, 16, 4, 4>(a, s); break;
        case kTile16x256: e = launch_cfg<CPLX, 16, 256, 16, 4, 4>(a, s); break;
        case kTile4x1024: e = launch_cfg<CPLX, 4, 1024, 4, 4, 4>(a, s); break;
        case kTile256x16: e = launch_cfg<CPLX, 256, 16, 16, 4, 4>(a, s); break;
        case kTile128x64: e = launch_cfg<CPLX, 128, 64, 16, 8, 4>(a, s); break;
        case kTileDot: {
            const int64_t outs = 1ll << (a.nm + a.nn);
            const int ni = a.in.n_inst > 1 ? a.in.n_inst : 1;
            constexpr size_t smem = dot_smem_bytes<CPLX>();
            static bool configured = false;
            if (!configured) {
                e = cudaFuncSetAttribute(k_dot<CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                configured = true;
            }
            k_dot<CPLX><<<dim3((unsigned)outs, (unsigned)a.nbatch, (unsigned)(a.split * ni)), 256, smem, s>>>(
                a, make_dot_plan(a));
            e = cudaGetLastError();
            break;
        }
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || a.split == 1) return e;
    const int64_t n = (int64_t)a.nbatch << (a.nm + a.nn);
    const int ni = a.in.n_inst > 1 ? a.in.n_inst : 1;
    // threads per output: enough that outputs x G fill the GPU's threads;
    // chosen from one instance's outputs, so that every instance sums in the
    // same order however many run side by side (results independent of the
    // slice batch)
    int G = 1;
    while (G < 32 && G * 2 <= a.split && n * G < (int64_t)sm_count() * 256 * 4) G *= 2;
    int64_t blocks = (n + 256 / G - 1) / (256 / G);
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    k_split_reduce<CPLX><<<dim3((unsigned)blocks, (unsigned)ni), 256, 0, s>>>(a, G);
    return cudaGetLastError();
}

cudaError_t launch_tile(const TileArgs& a, bool is_c, cudaStream_t s) {
    return is_c ? launch_tile_t<true>(a, s) : launch_tile_t<false>(a, s);
}

cudaError_t launch_wave(const WaveItem* items, int n_items, const TileArgs* descs,
                        const void* const* leaf_ptrs, bool is_c, cudaStream_t s, const int4* deps,
                        unsigned* done, unsigned* head, int G, bool tiles) {
    if (n_items <= 0) return cudaSuccess;
    // dataflow: persistent CTAs (8 per SM for the plain waves), else one per item
    const int grid = deps ? std::min(n_items, sm_count() * 8) : n_items;
    if (tiles) {
        if (is_c)
            k_wave<true, true><<<grid, 256, 0, s>>>(items, n_items, descs, leaf_ptrs, deps, done, head, G);
        else
            k_wave<false, true><<<grid, 256, 0, s>>>(items, n_items, descs, leaf_ptrs, deps, done, head, G);
    } else if (is_c) {
        k_wave<true, false><<<grid, 256, 0, s>>>(items, n_items, descs, leaf_ptrs, deps, done, head, G);
    } else {
        k_wave<false, false><<<grid, 256, 0, s>>>(items, n_items, descs, leaf_ptrs, deps, done, head, G);
    }
    return cudaGetLastError();
}

}  // namespace tn
