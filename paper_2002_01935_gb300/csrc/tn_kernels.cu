// tn_kernels.cu -- generic node kernel, renormalisation helpers and the FP64
// cross-slice accumulation of libtn.so (sm_103a).
//
// Semantics (arXiv 2002.01935):
//   * a pairwise contraction takes the inner product over the shared
//     labels, an outer product if there are none (Sec. 2);
//   * after each contraction the tensor is renormalised by a power of two
//     and the exponent is carried along (Sec. 4.2, active renormalisation);
//     here the scale is applied when the consumer reads the tensor: the
//     stored tensor S and exponent E mean S * 2^E, and a consumer multiplies
//     S by 2^-e, e = frexp exponent of max |component| of S, which is exact;
//   * the sliced contractions are summed in FP64 with exponent alignment
//     (Sec. 4.7.1).
#include <cuda_runtime.h>
#include <stdint.h>

#include "tn_internal.h"

namespace tn {

__device__ __forceinline__ int exp_of_max(const unsigned* slot) {
    if (slot == nullptr) return 0;
    float m = __uint_as_float(*slot);
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m, &e);
    return e;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int64_t slice_offset(const SliceDigits& d, int64_t slice) {
    int64_t off = 0;
    for (int i = 0; i < d.n; ++i) off += ((slice / d.div[i]) % d.dim[i]) * d.stride[i];
    return off;
}

// Block-wide max of non-negative floats, folded into *slot with atomicMax
// on the float bit pattern (order-preserving for non-negative floats).
__device__ __forceinline__ void block_max_to(float v, unsigned* slot) {
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0 && v > 0.f) atomicMax(slot, __float_as_uint(v));
    }
}

template <bool CPLX>
__global__ void __launch_bounds__(256) k_generic(const __grid_constant__ GenericArgs a) {
    // instance blockIdx.y: offset pointers, scale slots and slice id
    const int inst = blockIdx.y;
    const InstanceInfo& in = a.in;
    const int64_t slice = a.ctl->slice + (int64_t)inst * in.slice_step;
    if (slice >= a.ctl->slice_end) return;
    const int esz = CPLX ? 8 : 4;
    const void* Ap = (const char*)a.A + (int64_t)inst * in.a_is * esz;
    const void* Bp = (const char*)a.B + (int64_t)inst * in.b_is * esz;
    void* Cp = (char*)a.C + (int64_t)inst * in.c_is * esz;
    ScaleIO sc = a.sc;
    if (sc.max_a) sc.max_a += (int64_t)inst * in.sa_is;
    if (sc.exp_a) sc.exp_a += (int64_t)inst * in.sa_is;
    if (sc.max_b) sc.max_b += (int64_t)inst * in.sb_is;
    if (sc.exp_b) sc.exp_b += (int64_t)inst * in.sb_is;
    sc.max_c += (int64_t)inst * in.sc_is;
    sc.exp_c += (int64_t)inst * in.sc_is;
    const int eA = exp_of_max(sc.max_a);
    const int eB = exp_of_max(sc.max_b);
    const int esum = eA + eB;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t s = (sc.exp_a ? *sc.exp_a : 0) + (sc.exp_b ? *sc.exp_b : 0) + esum;
        *sc.exp_c = s;
    }
    const int64_t baseA = slice_offset(a.sla, slice);
    const int64_t baseB = slice_offset(a.slb, slice);
    float lmax = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < a.n_out; o += stride) {
        int64_t ia = baseA, ib = baseB, rem = o;
        for (int i = 0; i < a.n_od; ++i) {
            int64_t d = a.od_dim[i];
            int64_t v = rem % d;
            rem /= d;
            ia += v * a.od_sa[i];
            ib += v * a.od_sb[i];
        }
        int cnt[kMaxDigits];
        for (int i = 0; i < a.n_kd; ++i) cnt[i] = 0;
        float re = 0.f, im = 0.f;
        for (int64_t k = 0; k < a.n_sum; ++k) {
            if (CPLX) {
                float2 x = reinterpret_cast<const float2*>(Ap)[ia];
                float2 y = reinterpret_cast<const float2*>(Bp)[ib];
                if (a.conj_a) x.y = -x.y;
                if (a.conj_b) y.y = -y.y;
                re = fmaf(x.x, y.x, re);
                re = fmaf(-x.y, y.y, re);
                im = fmaf(x.x, y.y, im);
                im = fmaf(x.y, y.x, im);
            } else {
                re = fmaf(reinterpret_cast<const float*>(Ap)[ia],
                          reinterpret_cast<const float*>(Bp)[ib], re);
            }
            for (int i = 0; i < a.n_kd; ++i) {
                ia += a.kd_sa[i];
                ib += a.kd_sb[i];
                if (++cnt[i] < a.kd_dim[i]) break;
                ia -= a.kd_sa[i] * a.kd_dim[i];
                ib -= a.kd_sb[i] * a.kd_dim[i];
                cnt[i] = 0;
            }
        }
        re = ldexpf(re, -esum);
        if (CPLX) {
            im = ldexpf(im, -esum);
            reinterpret_cast<float2*>(Cp)[o] = make_float2(re, im);
            lmax = fmaxf(lmax, fmaxf(fabsf(re), fabsf(im)));
        } else {
            reinterpret_cast<float*>(Cp)[o] = re;
            lmax = fmaxf(lmax, fabsf(re));
        }
    }
    block_max_to(lmax, sc.max_c);
    if (a.t_done && threadIdx.x == 0) atomicMax(a.t_done, global_ns());
}

int sm_count() {
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 152;
    }
    if (cache[dev] <= 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

cudaError_t launch_generic(const GenericArgs& a, bool is_c, cudaStream_t s) {
    int64_t blocks = (a.n_out + 255) / 256;
    if (blocks > sm_count() * 16) blocks = sm_count() * 16;
    if (blocks < 1) blocks = 1;
    const unsigned ni = a.in.n_inst > 1 ? (unsigned)a.in.n_inst : 1u;
    if (is_c)
        k_generic<true><<<dim3((unsigned)blocks, ni), 256, 0, s>>>(a);
    else
        k_generic<false><<<dim3((unsigned)blocks, ni), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// FP64 cross-slice accumulation (Sec. 4.7.1) with exponent alignment
// --------------------------------------------------------------------------

template <bool CPLX>
__global__ void __launch_bounds__(256) k_accumulate(const __grid_constant__ AccumArgs a) {
    // the n_inst roots of this launch are slices ctl->slice + i (i in order);
    // fold them with one common exponent, skipping zero and idle slices
    const int ni = a.n_inst > 1 ? a.n_inst : 1;
    const int64_t step = (a.ctl->slice - a.ctl->slice_begin) / ni;
    const int par = (int)(step & 1);
    const int64_t accE = a.ctl->acc_exp[par];
    const bool empty = accE == INT64_MIN;
    int64_t newE = accE;
    bool any = false;
    for (int i = 0; i < ni; ++i) {
        if (a.ctl->slice + i >= a.ctl->slice_end) break;
        const float rmax = __uint_as_float(a.max_r[(int64_t)i * a.s_is]);
        if (!(rmax > 0.f)) continue;
        const int64_t S = a.exp_r[(int64_t)i * a.s_is];
        newE = (empty && !any) ? S : (S > newE ? S : newE);
        any = true;
    }
    double fa = 1.0;
    if (any && !empty) {
        const int64_t da = accE - newE;
        fa = ldexp(1.0, (int)(da < -2000 ? -2000 : da));
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < a.n_out; o += stride) {
        if (!any) continue;
        int64_t src = 0, rem = o;
        for (int i = 0; i < a.n_od; ++i) {
            const int64_t d = a.od_dim[i];
            if ((d & (d - 1)) == 0) {  // power of two: mask and shift
                src += (rem & (d - 1)) * a.od_s[i];
                rem >>= __ffsll(d) - 1;
            } else {
                src += (rem % d) * a.od_s[i];
                rem /= d;
            }
        }
        double vr = 0.0, vi = 0.0;
        if (CPLX) {
            const double2 v = reinterpret_cast<double2*>(a.acc)[o];
            vr = v.x * fa;
            vi = v.y * fa;
        } else {
            vr = a.acc[o] * fa;
        }
        for (int i = 0; i < ni; ++i) {
            if (a.ctl->slice + i >= a.ctl->slice_end) break;
            const float rmax = __uint_as_float(a.max_r[(int64_t)i * a.s_is]);
            if (!(rmax > 0.f)) continue;
            const int64_t dr = a.exp_r[(int64_t)i * a.s_is] - newE;
            const double fr = ldexp(1.0, (int)(dr < -2000 ? -2000 : dr));
            const int64_t at = src + (int64_t)i * a.r_is;
            if (CPLX) {
                const float2 r = reinterpret_cast<const float2*>(a.R)[at];
                vr += (double)r.x * fr;
                vi += (double)r.y * fr;
            } else {
                vr += (double)reinterpret_cast<const float*>(a.R)[at] * fr;
            }
        }
        if (CPLX)
            reinterpret_cast<double2*>(a.acc)[o] = make_double2(vr, vi);
        else
            a.acc[o] = vr;
    }
    if (gridDim.x == 1 && a.advance) __syncthreads();  // every thread has read ctl->slice
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->acc_exp[par ^ 1] = newE;
        // the last group of the call leaves the result's exponent
        if (a.ctl->slice + ni >= a.ctl->slice_end) a.ctl->final_exp = newE == INT64_MIN ? 0 : newE;
        if (gridDim.x == 1 && a.advance) a.ctl->slice += a.advance;
    }
}

cudaError_t launch_accumulate(const AccumArgs& a0, bool is_c, cudaStream_t s, int advance) {
    int64_t blocks = (a0.n_out + 255) / 256;
    if (blocks > sm_count() * 8) blocks = sm_count() * 8;
    if (blocks < 1) blocks = 1;
    AccumArgs a = a0;
    a.advance = blocks == 1 ? advance : 0;  // one block advances the slice counter itself
    if (is_c)
        k_accumulate<true><<<(unsigned)blocks, 256, 0, s>>>(a);
    else
        k_accumulate<false><<<(unsigned)blocks, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && blocks > 1 && advance) e = launch_advance(a.ctl, s, advance);
    return e;
}

__global__ void k_begin_call(Control* ctl, int64_t slice_begin, int64_t slice_end, double* acc,
                             int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        ctl->slice = slice_begin;
        ctl->slice_begin = slice_begin;
        ctl->slice_end = slice_end;
        ctl->acc_exp[0] = INT64_MIN;
        ctl->acc_exp[1] = INT64_MIN;
        ctl->status = 0;
    }
    for (; i < n; i += (int64_t)gridDim.x * blockDim.x) acc[i] = 0.0;
}

cudaError_t launch_begin_call(Control* ctl, int64_t slice_begin, int64_t slice_end, double* acc,
                              int64_t n, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_begin_call<<<(unsigned)blocks, 256, 0, s>>>(ctl, slice_begin, slice_end, acc, n);
    return cudaGetLastError();
}

cudaError_t launch_begin_slice(unsigned* maxabs, int n_nodes, cudaStream_t s) {
    return cudaMemsetAsync(maxabs, 0, sizeof(unsigned) * (size_t)n_nodes, s);
}

__global__ void k_advance(Control* ctl, int step) { ctl->slice += step; }

cudaError_t launch_advance(Control* ctl, cudaStream_t s, int step) {
    k_advance<<<1, 1, 0, s>>>(ctl, step);
    return cudaGetLastError();
}

// Largest |component| of every leaf, so that leaves are renormalised like
// intermediates before their first contraction.  blockIdx.x: leaf,
// blockIdx.y: one of gridDim.y interleaved parts of it.
// Part blockIdx.y of leaf blockIdx.x: the largest |component| over its
// entries, combined over the parts by atomicMax on the float bits
// (non-negative floats order like unsigned), or stored directly when one
// block covers the leaf and `direct` allows it (no zeroing needed then).
__device__ __forceinline__ void leaf_max_part(const float* const* ptrs, const int64_t* nfloat, unsigned* out,
                                              int n, bool direct) {
    const int v = blockIdx.x;
    if (v >= n) return;
    const float* p = ptrs[v];
    const int64_t m = nfloat[v];
    const int64_t first = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if ((int64_t)blockIdx.y * blockDim.x >= m && blockIdx.y > 0) return;
    float lmax = 0.f;
    for (int64_t i = first; i < m; i += (int64_t)gridDim.y * blockDim.x) lmax = fmaxf(lmax, fabsf(p[i]));
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        lmax = threadIdx.x < nw ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        if (threadIdx.x == 0) {
            if (direct && gridDim.y == 1)
                out[v] = __float_as_uint(lmax);
            else
                atomicMax(&out[v], __float_as_uint(lmax));
        }
    }
}

__global__ void __launch_bounds__(256) k_leaf_max(const float* const* ptrs, const int64_t* nfloat,
                                                  unsigned* out, int n) {
    leaf_max_part(ptrs, nfloat, out, n, false);
}

// The start of a call: leaf maxima as k_leaf_max, and (block 0) the control
// block and the FP64 accumulator as k_begin_call.
__global__ void __launch_bounds__(256) k_call_begin(const float* const* ptrs, const int64_t* nfloat,
                                                    unsigned* out, int n, Control* ctl, int64_t slice_begin,
                                                    int64_t slice_end, double* acc, int64_t n_acc) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        ctl->slice = slice_begin;
        ctl->slice_begin = slice_begin;
        ctl->slice_end = slice_end;
        ctl->acc_exp[0] = INT64_MIN;
        ctl->acc_exp[1] = INT64_MIN;
        ctl->status = 0;
    }
    {
        const int64_t nblk = (int64_t)gridDim.x * gridDim.y, bid = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
        for (int64_t i = bid * blockDim.x + threadIdx.x; i < n_acc; i += nblk * blockDim.x) acc[i] = 0.0;
    }
    leaf_max_part(ptrs, nfloat, out, n, true);
}

cudaError_t launch_call_begin(const float* const* ptrs, const int64_t* nfloat, unsigned* out, int n,
                              int64_t max_nfloat, Control* ctl, int64_t slice_begin, int64_t slice_end,
                              double* acc, int64_t n_acc, cudaStream_t s) {
    int64_t parts = (max_nfloat + 32767) / 32768;
    parts = parts < 1 ? 1 : (parts > 256 ? 256 : parts);
    if (n > 0 && parts > 1) {  // several blocks per leaf combine by atomicMax from zero
        const cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned) * (size_t)n, s);
        if (e != cudaSuccess) return e;
    }
    const unsigned gx = (unsigned)(n > 0 ? n : 1);
    k_call_begin<<<dim3(gx, (unsigned)parts), 256, 0, s>>>(ptrs, nfloat, out, n, ctl, slice_begin, slice_end, acc,
                                                          n_acc);
    return cudaGetLastError();
}

// The call's result: the FP64 accumulator and the exponent, to the caller's
// device buffers (or a staging buffer for one host copy: exp after acc).
__global__ void k_result(const double* acc, int64_t n, const Control* ctl, double* out, int64_t* out_exp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = acc[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *out_exp = ctl->final_exp;
}

cudaError_t launch_result(const double* acc, int64_t n, const Control* ctl, double* out, int64_t* out_exp,
                          cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    blocks = blocks < 1 ? 1 : (blocks > sm_count() * 4 ? sm_count() * 4 : blocks);
    k_result<<<(unsigned)blocks, 256, 0, s>>>(acc, n, ctl, out, out_exp);
    return cudaGetLastError();
}

cudaError_t launch_leaf_max(const float* const* ptrs, const int64_t* nfloat, unsigned* out, int n,
                            cudaStream_t s, int64_t max_nfloat) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    int64_t parts = (max_nfloat + 32767) / 32768;
    parts = parts < 1 ? 1 : (parts > 256 ? 256 : parts);
    k_leaf_max<<<dim3((unsigned)n, (unsigned)parts), 256, 0, s>>>(ptrs, nfloat, out, n);
    return cudaGetLastError();
}

// Leaf adjoints of one slice, all leaves in one launch: blockIdx.y picks
// the table entry, blockIdx.x a chunk of its elements.
template <bool CPLX>
__global__ void __launch_bounds__(256) k_leaf_grads(const LeafGradArgs* tab, int n_entries) {
    __shared__ LeafGradArgs a;
    if ((int)blockIdx.y >= n_entries) return;
    {
        const int* src = reinterpret_cast<const int*>(tab + blockIdx.y);
        int* dst = reinterpret_cast<int*>(&a);
        for (int i = threadIdx.x; i < (int)(sizeof(LeafGradArgs) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if ((int64_t)blockIdx.x * blockDim.x >= a.n) return;
    const int64_t inst = blockIdx.z;
    const int64_t slice = a.ctl->slice;
    const int64_t base = slice_offset(a.sl, slice);
    int64_t e = a.exp_adj[inst * a.exp_is];
    const int ex = (int)(e < -400 ? -400 : (e > 400 ? 400 : e));
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < a.n; o += stride) {
        int64_t g = base, s = 0, rem = o;
        for (int i = 0; i < a.n_d; ++i) {
            const int64_t d = a.dim[i];
            const int64_t v = rem % d;
            rem /= d;
            g += v * a.gstride[i];
            s += v * a.astride[i];
        }
        s += inst * a.adj_is;
        g += inst * a.grad_is;
        if (CPLX) {
            const float2 x = reinterpret_cast<const float2*>(a.adj)[s];
            float2* G = reinterpret_cast<float2*>(a.grad);
            float2 y = G[g];
            y.x += ldexpf(x.x, ex);
            y.y += ldexpf(x.y, ex);
            G[g] = y;
        } else {
            reinterpret_cast<float*>(a.grad)[g] += ldexpf(reinterpret_cast<const float*>(a.adj)[s], ex);
        }
    }
}

cudaError_t launch_leaf_grads(const LeafGradArgs* tab, int n_entries, int64_t max_n, int n_inst, bool is_c,
                              cudaStream_t s) {
    if (n_entries <= 0) return cudaSuccess;
    int64_t blocks = (max_n + 255) / 256;
    blocks = blocks < 1 ? 1 : (blocks > sm_count() * 8 ? sm_count() * 8 : blocks);
    const dim3 grid((unsigned)blocks, (unsigned)n_entries, (unsigned)(n_inst > 1 ? n_inst : 1));
    if (is_c)
        k_leaf_grads<true><<<grid, 256, 0, s>>>(tab, n_entries);
    else
        k_leaf_grads<false><<<grid, 256, 0, s>>>(tab, n_entries);
    return cudaGetLastError();
}

// dst = src (or dst += src) for every entry of the table: blockIdx.y picks
// the entry, blockIdx.x a chunk.
__global__ void __launch_bounds__(256) k_copy_table(const CopyEntry* tab, int n_entries) {
    if ((int)blockIdx.y >= n_entries) return;
    const CopyEntry e = tab[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < e.nfloat; i += stride) {
        float v = e.src[i];
        for (int r = 1; r < e.n_sum; ++r) v += e.src[r * e.src_is + i];
        e.dst[i] = e.add ? e.dst[i] + v : v;
    }
}

cudaError_t launch_copy_table(const CopyEntry* tab, int n_entries, int64_t max_nfloat, cudaStream_t s) {
    int64_t blocks = (max_nfloat + 255) / 256;
    blocks = blocks < 1 ? 1 : (blocks > sm_count() * 4 ? sm_count() * 4 : blocks);
    for (int first = 0; first < n_entries; first += 65535) {  // grid y limit
        const int cnt = n_entries - first < 65535 ? n_entries - first : 65535;
        k_copy_table<<<dim3((unsigned)blocks, (unsigned)cnt), 256, 0, s>>>(tab + first, cnt);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// p[i * stride + j] = 0 for i < n, j < count.
__global__ void k_zero_strided(unsigned* p, int64_t count, int64_t stride, int n) {
    const int64_t total = count * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        p[(t / count) * stride + t % count] = 0u;
}

cudaError_t launch_zero_strided(unsigned* p, int64_t count, int64_t stride, int n, cudaStream_t s) {
    const int64_t total = count * n;
    if (total <= 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > sm_count() * 4) blocks = sm_count() * 4;
    k_zero_strided<<<(unsigned)blocks, 256, 0, s>>>(p, count, stride, n);
    return cudaGetLastError();
}

// The root adjoint in the form the sweep reads: largest |component| m of
// the FP64 adjoint, m = f * 2^e with f in [0.5, 1) (frexp), every component
// scaled by 2^-e (exact) and rounded to float into the root's layout; the
// root's scale slots get f and e plus the adjoint's own exponent.  One block.
__global__ void __launch_bounds__(1024) k_root_adjoint(RootAdjArgs a) {
    __shared__ double red[32];
    const int c = a.cplx ? 2 : 1;
    const int64_t nd = a.n_out * c;
    const int64_t inst = blockIdx.x;
    a.adj += inst * nd;
    a.dst += inst * a.dst_is;
    a.max_slot += inst * a.slot_is;
    a.exp_slot += inst * a.slot_is;
    if (a.exp_dev) a.exp_dev += inst;
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < nd; i += blockDim.x) m = fmax(m, fabs(a.adj[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    m = red[0];
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    for (int64_t i = threadIdx.x; i < nd; i += blockDim.x)
        a.dst[a.perm[i / c] * c + (i % c)] = (float)ldexp(a.adj[i], -e);
    if (threadIdx.x == 0) {
        const float f = m > 0.0 ? (float)ldexp(m, -e) : 0.f;
        *a.max_slot = __float_as_uint(f);
        *a.exp_slot = (int64_t)e + a.exp_host + (a.exp_dev ? *a.exp_dev : 0);
    }
}

cudaError_t launch_root_adjoint(const RootAdjArgs& a, int n_inst, cudaStream_t s) {
    k_root_adjoint<<<(unsigned)(n_inst > 1 ? n_inst : 1), 1024, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_batch_start(unsigned long long* t_start) { *t_start = global_ns(); }

cudaError_t launch_batch_start(unsigned long long* t_start, cudaStream_t s) {
    k_batch_start<<<1, 1, 0, s>>>(t_start);
    return cudaGetLastError();
}

__global__ void k_batch_finish(const BatchRoot* roots, int n, double* out, int64_t* out_exp,
                               const unsigned long long* t_start, const unsigned long long* t_done,
                               unsigned long long* latency) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BatchRoot r = roots[i];
    if (r.root == nullptr) {
        // a sliced network: its slice loop runs after this kernel and writes
        // its value, exponent and latency itself
        out[2 * i] = 0.0;
        out[2 * i + 1] = 0.0;
        out_exp[i] = 0;
        if (latency) latency[i] = 0;
        return;
    }
    const bool zero = !(__uint_as_float(*r.max) > 0.f);
    if (r.is_c) {
        const float2 v = *reinterpret_cast<const float2*>(r.root);
        out[2 * i] = v.x;
        out[2 * i + 1] = v.y;
    } else {
        out[2 * i] = *reinterpret_cast<const float*>(r.root);
        out[2 * i + 1] = 0.0;
    }
    out_exp[i] = zero ? 0 : *r.exp;
    if (latency) latency[i] = t_done[i] > *t_start ? t_done[i] - *t_start : 0;
}

__global__ void k_batch_mark(const unsigned long long* t_start, unsigned long long* latency) {
    const unsigned long long t = global_ns();
    *latency = t > *t_start ? t - *t_start : 0;
}

cudaError_t launch_batch_mark(const unsigned long long* t_start, unsigned long long* latency, cudaStream_t s) {
    k_batch_mark<<<1, 1, 0, s>>>(t_start, latency);
    return cudaGetLastError();
}

cudaError_t launch_batch_finish(const BatchRoot* roots, int n, double* out, int64_t* out_exp,
                                const unsigned long long* t_start, const unsigned long long* t_done,
                                unsigned long long* latency, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_batch_finish<<<(n + 127) / 128, 128, 0, s>>>(roots, n, out, out_exp, t_start, t_done, latency);
    return cudaGetLastError();
}

}  // namespace tn
